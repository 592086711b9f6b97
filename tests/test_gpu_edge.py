"""Edge cases through the C ABI against the FP64 oracle: a single sphere, a
sphere across the corner of two periodic faces, a sphere on a wall, and the
argument errors of an empty particle set."""
import numpy as np
import pytest

import oracle as O
from oracle import saltation as S
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import gpu_context, oracle_grid, oracle_template, rel_err, to_device

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _one(x, periodic=(1, 1, 1), n=(48, 40, 32), R=3.0, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.asarray(x, dtype=np.float64).reshape(3, -1)
    k = x.shape[1]
    return W.Workload(name="edge", n=n, h=1.0, periodic=periodic, R=R, rho_p=2.65, rho_f=1.0,
                      x=x, u=rng.uniform(-0.1, 0.1, (3, k)), om=rng.uniform(-0.05, 0.05, (3, k)),
                      dt=0.01, n_sub=50, e_n=0.9, e_t=0.39, mu=0.4, T_c=0.1,
                      g=(0.0, 0.0, -0.5), fluid_mean="none", fluid_std=0.1)


def _ibm_both(w, precision):
    import torch
    fl = w.fluid_numpy()
    z = [np.zeros_like(fl[0]) for _ in range(3)]
    t, dV = oracle_template(w)
    ref = O.ibm_step(oracle_grid(w), w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, *z, w.dt, 1.0,
                     n_mdf_max=2)
    c = gpu_context(w, precision)
    dev = to_device(fl + z, torch.float64 if precision == "fp64" else torch.float32)
    c.ibm_step(*dev, w.dt, 1.0, n_mdf_max=2)
    c.sync()
    got = {k: d.cpu().numpy() for k, d in zip(("u", "v", "w", "fx", "fy", "fz"), dev)}
    got.update(c.read_forces())
    c.close()
    return ref, got


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("where", ["middle", "corner", "wall"])
def test_single_sphere_ibm(where, precision):
    if where == "middle":
        w = _one([23.7, 19.2, 15.6])
    elif where == "corner":          # across the x and y faces at once
        w = _one([0.6, 39.3, 15.6])
    else:                            # on the bottom wall, markers beyond it
        w = _one([23.7, 19.2, 1.2], periodic=(1, 1, 0))
    ref, got = _ibm_both(w, precision)
    for k in ("u", "v", "w", "fx", "fy", "fz", "F_h", "T_h"):
        assert rel_err(got[k], ref[k]) <= TOL[precision], k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_sphere_dem_and_bed(precision):
    # no contact: gravity alone; resting on the wall: one wall contact
    for z0, bed in ((12.0, 0), (2.95, 1)):
        w = _one([23.7, 19.2, z0], periodic=(1, 1, 0))
        c = gpu_context(w, precision)
        dt_p = w.dt / w.n_sub
        assert list(c.bed_detect()) == [int(z0 < 2 * w.R)]
        c.dem_step(dt_p, 3, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
        xg, ug, og = c.read_state()
        hg = c.read_history()
        c.close()
        d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)
        zz = np.zeros((3, 1))
        xo, uo, oo, _, _, ho, _ = O.dem_run(d, dt_p, 3, w.x, w.u, w.om, zz, zz, O.History(1))
        assert int(hg["wact"].sum()) == int(ho.wact.sum()) == bed
        for a, b in ((xg, xo), (ug, uo), (og, oo)):
            assert rel_err(a, b) <= TOL[precision]
        assert list(S.bed_flags(d, w.x, w.R)) == [int(z0 < 2 * w.R)]


def test_empty_particle_set_is_rejected():
    from paper_2108_01814_gb300 import binding as B
    c = B.Context((16, 16, 16), 1.0, (1, 1, 1), precision="fp32")
    with pytest.raises(B.PrsError) as e:
        c.create_particles(0, 2.0, 2.65, 1.0)
    assert e.value.status == -1              # PRS_ERR_ARG
    with pytest.raises(B.PrsError) as e:     # nothing to step yet
        c.dem_step(1e-3, 1, e_n=0.9, e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0))
    assert e.value.status == -4              # PRS_ERR_STATE
    c.close()
