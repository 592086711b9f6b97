"""GPU parity of the coupled particle step against the FP64 oracle, through
the C ABI: one prs_ibm_step, whose per-particle hydrodynamic load F_h, T_h
(Eq. 7-8 in rigid-body form) is then held over the n_sub = 50 particle
sub-steps of one prs_dem_step (Sec. 2.1: dt_p = dt_f / 50), exactly as the
paper couples the fluid step to the DEM. Both forms: FP64 (<= 1e-10) and
FP32 grid and marker arithmetic with FP64 state (<= 1e-5), normwise
relative error per field; contact sets bit for bit.

The configuration-1 trajectory (the tiny triply periodic box, ten steps of
interpolation, forcing, spreading and 50 DEM sub-steps, each step's forced
fluid feeding the next) is gated in FP64 at 1e-10.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import gpu_context, oracle_grid, oracle_template, rel_err, to_device

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _dem_params(w):
    return O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)


def _oracle_step(w, g, t, dV, x, up, om, fl, hist, dt_p, n_sub):
    z = np.zeros_like(fl[0])
    r = O.ibm_step(g, w.R, w.rho_f, t, dV, x, up, om, *fl, z, z, z, w.dt, 1.0)
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_run(_dem_params(w), dt_p, n_sub, x, up, om,
                                           r["F_h"], r["T_h"], hist)
    return r, (xo, uo, oo, Fc, Tc, ho, ov)


def _gpu_step(ctx, w, dev, f_dev, dt_p, n_sub):
    for f in f_dev:
        f.zero_()
    ctx.ibm_step(*dev, *f_dev, w.dt, 1.0)
    ibm = ctx.read_forces()
    ctx.dem_step(dt_p, n_sub, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
    return ibm


def _small_bed_settled():
    # the channel bed lowered by 0.3 cells so that the bottom layer presses
    # on the wall: wall contacts and particle contacts both occur
    w = W.small_bed()
    w.x = w.x.copy()
    w.x[2] -= 0.3
    return w


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["tiny", "small_bed"])
def test_coupled_step_parity(name, precision):
    import torch
    w = W.tiny() if name == "tiny" else _small_bed_settled()
    dt_p, n_sub = w.dt / w.n_sub, w.n_sub
    tol = TOL[precision]
    fl = w.fluid_numpy()
    if precision == "fp32":
        # both sides start from the same FP32 fluid values
        fl = [a.astype(np.float32).astype(np.float64) for a in fl]
    g = oracle_grid(w)
    t, dV = oracle_template(w)
    ref, (xo, uo, oo, Fc, Tc, ho, ov) = _oracle_step(w, g, t, dV, w.x, w.u, w.om, fl,
                                                     O.History(w.n_p), dt_p, n_sub)
    assert not ov
    ctx = gpu_context(w, precision)
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    dev = to_device(fl, dt_t)
    f_dev = [torch.zeros_like(dev[0]) for _ in range(3)]
    ibm = _gpu_step(ctx, w, dev, f_dev, dt_p, n_sub)
    xg, ug, og = ctx.read_state()
    fg = ctx.read_forces()
    hg = ctx.read_history()
    ctx.close()
    # the load that drives the sub-steps is non-trivial: it changes the
    # velocities by more than the tolerance over the step
    m = (w.rho_p - w.rho_f) * 4.0 / 3.0 * np.pi * w.R ** 3
    assert np.max(np.abs(ref["F_h"])) * w.dt / m > 1e3 * tol * np.max(np.abs(uo))
    assert rel_err(ibm["F_h"], ref["F_h"]) <= tol
    assert rel_err(ibm["T_h"], ref["T_h"]) <= tol
    # contact sets after the 50 sub-steps: exact
    assert np.array_equal(hg["cnt"], ho.cnt)
    assert np.array_equal(hg["pid"], ho.pid)
    assert np.array_equal(hg["wact"], ho.wact)
    if name == "small_bed":
        assert ho.cnt.sum() > 0 and ho.wact.sum() > 0  # the settled bed touches
    for k, (a, b) in {"x": (xg, xo), "u": (ug, uo), "omega": (og, oo), "F_c": (fg["F_c"], Fc),
                      "T_c": (fg["T_c"], Tc), "delta_t": (hg["dlt"], ho.dlt)}.items():
        assert rel_err(a, b) <= tol, k
    # the displacement over the step, not only the position, within the
    # tolerance (positions are O(L); the step moves them by O(u dt))
    assert rel_err(xg - w.x, xo - w.x) <= tol


def test_config1_trajectory_fp64():
    # configuration 1: ten steps of interp + forcing + spread + 50 DEM
    # sub-steps; each step's forced velocity field is the next step's input
    # and f starts from zero each step
    import torch
    w = W.tiny()
    dt_p, n_sub = w.dt / w.n_sub, w.n_sub
    fl = w.fluid_numpy()
    g = oracle_grid(w)
    t, dV = oracle_template(w)
    ctx = gpu_context(w, "fp64")
    dev = to_device(fl, torch.float64)
    f_dev = [torch.zeros_like(dev[0]) for _ in range(3)]
    x, up, om, hist = w.x, w.u, w.om, O.History(w.n_p)
    for step in range(10):
        ref, (x, up, om, Fc, Tc, hist, ov) = _oracle_step(w, g, t, dV, x, up, om, fl, hist,
                                                          dt_p, n_sub)
        assert not ov
        fl = [ref["u"], ref["v"], ref["w"]]
        ibm = _gpu_step(ctx, w, dev, f_dev, dt_p, n_sub)
        assert rel_err(ibm["F_h"], ref["F_h"]) <= 1e-10, step
        assert rel_err(ibm["T_h"], ref["T_h"]) <= 1e-10, step
    xg, ug, og = ctx.read_state()
    hg = ctx.read_history()
    got_fl = [d.cpu().numpy() for d in dev]
    ctx.close()
    assert np.array_equal(hg["pid"], hist.pid) and np.array_equal(hg["cnt"], hist.cnt)
    for k, (a, b) in {"x": (xg, x), "u": (ug, up), "omega": (og, om),
                      "dx": (xg - w.x, x - w.x)}.items():
        assert rel_err(a, b) <= 1e-10, k
    for c in range(3):
        assert rel_err(got_fl[c], fl[c]) <= 1e-10
    # the spheres moved: the trajectory is not the initial state
    assert np.max(np.abs(x - w.x)) > 1e-3
