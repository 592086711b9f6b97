"""GPU parity of the paper's collision model options against the FP64
oracle (Sec. 2.1, text after Eq. 9-10): the adaptive collision time model
(a Hertzian spring whose stiffness and damping each contact takes from its
impact speed) and the two-parameter lubrication force, sphere-sphere and
sphere-wall, each alone and together, over 40 sub-steps with the history
carried. Contact sets bit for bit; states, forces and history within 1e-10
(FP64 form) and 1e-5 (FP32 form)."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_helpers import packing, rel_err

pytestmark = pytest.mark.gpu

OPTS = dict(e_n=0.9, e_t=0.39, mu=0.4, T_c=0.05)
TOL = {"fp64": 1e-10, "fp32": 1e-5}
MU_F = 0.05


def _case(seed=2, n=(20, 16, 24), per=(1, 1, 0), R=1.0, n_p=380):
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5, min_frac=0.985)
    # the six lowest spheres moving down onto the bottom wall: three inside
    # the wall's lubrication range, three touching it
    low = np.argsort(x[2])[:6]
    x[2, low] = R * (1.0 + np.array([0.004, 0.015, 0.035, -0.003, -0.008, -0.015]))
    u[2, low] = -0.2
    return n, per, R, L, x, u, om


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", ["actm", "lubrication", "actm+lubrication"])
def test_collision_model_parity(variant, precision):
    from paper_2108_01814_gb300 import binding as B
    n, per, R, L, x, u, om = _case()
    g = (0.0, 0.0, -0.5)
    actm = variant.startswith("actm")
    mu_f = MU_F if "lubrication" in variant else 0.0
    c = B.Context(n, 1.0, per, precision=precision)
    c.create_particles(x.shape[1], R, 2.65, 1.0)
    c.write_state(x, u, om)
    dt_p, k = 1e-3, 40
    c.dem_step(dt_p, k, g=g, model="actm" if actm else "linear", mu_f=mu_f, **OPTS)
    xg, ug, og = c.read_state()
    fg = c.read_forces()
    hg = c.read_history()
    c.close()
    d = O.dem_params(R, 2.65, 1.0, OPTS["e_n"], OPTS["e_t"], OPTS["mu"], OPTS["T_c"], g, L, per,
                     model="actm" if actm else "linear", mu_f=mu_f)
    z = np.zeros_like(x)
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_run(d, dt_p, k, x, u, om, z, z, O.History(x.shape[1]))
    assert not ov
    assert np.array_equal(hg["pid"], ho.pid) and np.array_equal(hg["cnt"], ho.cnt)
    assert np.array_equal(hg["wact"], ho.wact)
    tol = TOL[precision]
    for key, (a, b) in {"x": (xg - x, xo - x), "u": (ug, uo), "omega": (og, oo),
                        "F_c": (fg["F_c"], Fc), "T_c": (fg["T_c"], Tc),
                        "delta_t": (hg["dlt"], ho.dlt), "u_in": (hg["uin"], ho.uin)}.items():
        assert rel_err(a, b) <= tol, key
    # the option is in effect: the plain linear law without lubrication
    # ends elsewhere
    d0 = O.dem_params(R, 2.65, 1.0, OPTS["e_n"], OPTS["e_t"], OPTS["mu"], OPTS["T_c"], g, L, per)
    _, u0, _, _, _, _, _ = O.dem_run(d0, dt_p, k, x, u, om, z, z, O.History(x.shape[1]))
    assert rel_err(u0, uo) > 100 * tol


def test_lubrication_pairs_are_in_range():
    # the packing brings pairs and spheres near the bottom wall into the
    # lubrication range, so the tests above exercise both
    n, per, R, L, x, u, om = _case()
    wall_gap = x[2] - R
    assert np.sum((wall_gap >= 0) & (wall_gap < 0.05 * R)) == 3
    assert np.sum(wall_gap < 0) == 3
    d = O.dem_params(R, 2.65, 1.0, 0.9, 0.39, 0.4, 0.05, (0.0, 0.0, -0.5), L, per)
    pr = O.pairs(d, x, 2 * R * (1 + 0.025))
    gaps = []
    for p, q in pr:
        s = x[:, q] - x[:, p]
        for a in range(2):
            s[a] -= L[a] * np.round(s[a] / L[a])
        gaps.append(np.linalg.norm(s) - 2 * R)
    gaps = np.array(gaps)
    assert np.sum((gaps >= 0) & (gaps < 0.05 * R)) >= 5


def test_option_errors():
    from paper_2108_01814_gb300 import binding as B
    n, per, R, L, x, u, om = _case()
    c = B.Context(n, 1.0, per, precision="fp64")
    c.create_particles(x.shape[1], R, 2.65, 1.0)
    c.write_state(x, u, om)
    for kw in (dict(eps_d=(0.2, 0.0)), dict(mu_f=-1.0), dict(eps_s=0.06)):
        with pytest.raises(B.PrsError) as e:
            c.dem_step(1e-3, 1, **OPTS, **kw)
        assert e.value.status == B.PRS_ERR_ARG
    with pytest.raises(B.PrsError):
        c.dem_step(1e-3, 1, e_n=1.0, e_t=0.39, mu=0.4, T_c=0.05, model="actm")
    c.close()
