"""GPU parity of the fluid-predictor stand-in (prs_predict) against the FP64
oracle: both RK2 sub-steps, periodic and wall-bounded axes, points half a
cell off the walls and on them, the vector and scalar kernels, sizes that
leave ragged thread blocks."""
import numpy as np
import pytest

from oracle import fluid as F
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6}
STAG = [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]

CASES = [
    # (grid n, periodic, offsets, component); nx a multiple of 4 takes the
    # 16-byte vector kernel, other sizes the scalar one
    ((48, 13, 37), (1, 1, 1), None, 0),
    ((45, 13, 37), (1, 1, 0), STAG, 2),
    ((48, 13, 37), (1, 1, 0), STAG, 2),
    ((33, 20, 70), (0, 1, 0), STAG, 0),
    ((36, 20, 70), (0, 1, 0), STAG, 0),
    ((36, 20, 70), (0, 1, 0), STAG, 1),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_predict_rk2_parity(case, precision):
    import torch
    from paper_2108_01814_gb300 import binding as B
    n, per, off, comp = case
    h, nu, dt = 0.8, 0.05, 0.01
    ctx = B.Context(n, h, per, offset=off, precision=precision)
    rng = np.random.Generator(np.random.PCG64(17))
    u0 = rng.normal(size=(n[2], n[1], n[0]))
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    u0 = u0.astype(np.float32).astype(np.float64) if precision == "fp32" else u0
    cu = [torch.as_tensor(u0, dtype=dt_t, device="cuda"), torch.empty(u0.shape, dtype=dt_t,
                                                                      device="cuda")]
    H = torch.full(u0.shape, float("nan"), dtype=dt_t, device="cuda")  # not read at beta = 0
    o = (off[comp] if off else [0.5, 0.5, 0.5])
    ref_u, ref_H = u0, np.full(u0.shape, np.nan)
    for k, (al, be) in enumerate(((1.0, 0.0), (0.5, 0.5))):
        ctx.predict(comp, cu[k % 2], cu[(k + 1) % 2], H, nu, dt, al, be)
        ctx.sync()
        ref_u, ref_H = F.predict(ref_u, ref_H, nu, dt, al, be, h, per, o)
        got_u = cu[(k + 1) % 2].double().cpu().numpy()
        got_H = H.double().cpu().numpy()
        assert np.all(np.isfinite(got_u)) and np.all(np.isfinite(got_H))
        assert rel_err(got_u, ref_u) <= TOL[precision], k
        # H = nu lap_h(u) is a sum of seven terms of size up to
        # nu max|u| / h^2 each; its rounding error relative to max|H| grows
        # by sum|terms| / max|H| <= 14 max|u| / max|lap u| h^2 (about 5 for
        # this random field), and the second sub-step's H inherits the
        # first's error in u through the same factor: 10x the tolerance of u
        assert rel_err(got_H, ref_H) <= TOL[precision] * 10, k
        # the steps changed the field (the diffusion is not lost in the
        # tolerance; the second sub-step alone changes it by O(dt^2) only)
        assert rel_err(ref_u, u0) > 100 * TOL[precision]
    ctx.close()


def test_predict_argument_errors():
    import torch
    from paper_2108_01814_gb300 import binding as B
    ctx = B.Context((16, 8, 8), 1.0, (1, 1, 0), offset=[[0.5, 0.5, 0.25]] * 3,
                    precision="fp32")
    a, b, c = (torch.zeros((8, 8, 16), device="cuda") for _ in range(3))
    for args in ((0, a, a, c), (3, a, b, c)):
        with pytest.raises(B.PrsError) as e:
            ctx.predict(*args, 0.1, 0.01)
        assert e.value.status == -1          # PRS_ERR_ARG
    with pytest.raises(B.PrsError):          # offset 1/4 on the wall-bounded z axis
        ctx.predict(0, a, b, c, 0.1, 0.01)
    ctx.close()
