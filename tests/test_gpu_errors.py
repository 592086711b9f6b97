"""The library's error paths, each provoked on the host or by a bounded
wait that runs out, never by a fault: an allocator that refuses memory
(PRS_ERR_OOM), a non-finite particle state (PRS_ERR_NONFINITE), a slip
tolerance the forcing passes cannot reach (PRS_WARN_NOT_CONVERGED) and a
device-side wait that runs out (PRS_ERR_TIMEOUT)."""
import numpy as np
import pytest

from paper_2108_01814_gb300 import binding as B
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import gpu_context, to_device

pytestmark = pytest.mark.gpu

OPTS = dict(e_n=0.9, e_t=0.39, mu=0.4, T_c=0.05)


def test_allocator_refusal_is_reported_as_oom():
    # a caller's budget of 256 kB cannot hold the particle state of 20,000
    # spheres: the allocator returns NULL and the call reports it
    c = B.Context((32, 32, 32), 1.0, (1, 1, 1), precision="fp64", device_budget=256 << 10)
    with pytest.raises(B.PrsError) as e:
        c.create_particles(20000, 1.0, 2.65, 1.0)
    assert e.value.status == B.PRS_ERR_OOM
    c.close()
    # the same call under a budget that holds it succeeds
    c = B.Context((32, 32, 32), 1.0, (1, 1, 1), precision="fp64", device_budget=1 << 30)
    c.create_particles(20000, 1.0, 2.65, 1.0)
    assert 0 < c._alloc.used <= 1 << 30
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_non_finite_state_is_latched(precision):
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.uniform(2.0, 18.0, (3, 40))
    u = np.zeros_like(x)
    u[1, 7] = np.nan
    c = B.Context((20, 20, 20), 1.0, (1, 1, 1), precision=precision)
    c.create_particles(40, 0.5, 2.65, 1.0)
    c.write_state(x, u, np.zeros_like(x))
    c.dem_step(1e-3, 2, **OPTS)
    with pytest.raises(B.PrsError) as e:
        c.read_state()
    assert e.value.status == B.PRS_ERR_NONFINITE
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unreachable_tolerance_warns(precision):
    import torch
    w = W.tiny()
    c = gpu_context(w, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    flds = to_device(w.fluid_numpy(), dt)
    f = [torch.zeros_like(flds[0]) for _ in range(3)]
    st = c.ibm_step(*flds, *f, w.dt, 1.0, n_mdf_max=2, tol=1e-30)
    assert st == B.PRS_WARN_NOT_CONVERGED
    s = c.stats()
    assert s.mdf_passes == 2 and s.residual > 1e-30
    c.sync()  # a warning latches nothing
    c.close()


def test_wait_that_runs_out_is_reported_as_timeout():
    c = B.Context((16, 16, 16), 1.0, (1, 1, 1), precision="fp32")
    c.create_particles(4, 1.0, 2.65, 1.0)
    c.sync()
    c.probe_wait(1000)
    with pytest.raises(B.PrsError) as e:
        c.sync()
    assert e.value.status == B.PRS_ERR_TIMEOUT
    assert b"ran out" in c.lib.prs_last_error_string()
    with pytest.raises(B.PrsError) as e:
        c.probe_wait(0)
    assert e.value.status == B.PRS_ERR_ARG
    c.close()
