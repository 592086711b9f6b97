"""Measured error of every field of one coupled step (prs_ibm_step, then
prs_dem_step with the load it produced) against the FP64 oracle, for the
FP64 form and the FP32 form (FP32 grid and marker arithmetic, FP64 state),
normwise max|a - b| / max|b| per field (Sec. 2.1 and Eq. 7-10 for what
each field is). The test gates every field at the form's tolerance and,
when PRS_ERROR_TABLE names a file, writes the measured errors there as
JSON, one record per configuration and form.

Configurations: the tiny triply periodic box (50 sub-steps), a settled
channel bed with walls (600 + 20 spheres of D = 6h, 50 sub-steps) and the
8448-sphere channel bed of D = 10h (5 sub-steps: the oracle's brute-force
contact search is quadratic in the sphere count)."""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import (gpu_context, oracle_grid, oracle_template, record_errors,
                               rel_err, to_device)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _settled(w):
    w.x = w.x.copy()
    w.x[2] -= 0.3
    return w


CASES = {
    "tiny": (W.tiny, 50),
    "small_bed": (lambda: _settled(W.small_bed()), 50),
    "bed": (lambda: _settled(W.bed()), 5),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_field_errors(name, precision):
    import torch
    make, n_sub = CASES[name]
    w = make()
    dt_p = w.dt / w.n_sub
    fl = w.fluid_numpy()
    if precision == "fp32":
        fl = [a.astype(np.float32).astype(np.float64) for a in fl]
    z = np.zeros_like(fl[0])
    g = oracle_grid(w)
    t, dV = oracle_template(w)
    ref = O.ibm_step(g, w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, z, z, z, w.dt, 1.0,
                     want_marker_force=True)
    d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_run(d, dt_p, n_sub, w.x, w.u, w.om, ref["F_h"],
                                           ref["T_h"], O.History(w.n_p))
    assert not ov
    ctx = gpu_context(w, precision)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    dev = to_device(fl, tdt)
    f_dev = [torch.zeros_like(dev[0]) for _ in range(3)]
    ctx.ibm_step(*dev, *f_dev, w.dt, 1.0)
    ibm = ctx.read_forces()
    F_l = ctx.read_marker_forces().astype(np.float64)
    ctx.dem_step(dt_p, n_sub, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
    xg, ug, og = ctx.read_state()
    fg = ctx.read_forces()
    hg = ctx.read_history()
    got_fl = [a.double().cpu().numpy() for a in dev]
    got_f = [a.double().cpu().numpy() for a in f_dev]
    ctx.close()
    assert np.array_equal(hg["pid"], ho.pid) and np.array_equal(hg["wact"], ho.wact)
    err = {
        "x (displacement)": rel_err(xg - w.x, xo - w.x),
        "u": rel_err(ug, uo),
        "omega": rel_err(og, oo),
        "F_h": rel_err(ibm["F_h"], ref["F_h"]),
        "T_h": rel_err(ibm["T_h"], ref["T_h"]),
        "F_c": rel_err(fg["F_c"], Fc),
        "T_c": rel_err(fg["T_c"], Tc),
        "F_l": rel_err(F_l, ref["F_l"]),
        "f": max(rel_err(a, ref[k]) for a, k in zip(got_f, ("fx", "fy", "fz"))),
        "grid u increment": max(rel_err(a - b, ref[k] - b)
                                for a, b, k in zip(got_fl, fl, ("u", "v", "w"))),
    }
    record_errors({"config": name, "form": precision, "n_p": int(w.n_p), "n_sub": n_sub,
                   "contacts": int(ho.cnt.sum()), "wall_contacts": int(ho.wact.sum()),
                   "errors": err})
    for k, v in err.items():
        assert v <= TOL[precision], (k, v)
