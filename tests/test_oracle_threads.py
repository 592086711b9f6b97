"""The oracle on several host threads gives bit for bit what it gives on
one: its loops over particles and markers write disjoint outputs, and its
spreading (Sec. 3.3) hands each slab of z-planes to one thread that adds the
terms in ascending marker order. Checked on a periodic box and a walled
channel bed with contacts, with the 3-point and the 4-point kernel and with
multi-direct forcing (several spreads per step), at thread counts that do
and do not divide the plane count."""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W


def _settled_bed():
    w = W.small_bed()
    w.x = w.x.copy()
    w.x[2] -= 0.3
    return w


def _run(w, kernel, threads, n_mdf, n_sub, lub):
    used = O.set_threads(threads)
    try:
        g = O.make_grid(w.n, w.h, w.periodic, kernel=kernel)
        n_l = O.marker_count(w.R, w.h)
        t, dV = O.template(n_l), O.marker_volume(w.R, w.h, n_l)
        fl = w.fluid_numpy()
        z = np.zeros_like(fl[0])
        r = O.ibm_step(g, w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, z, z, z, w.dt, 1.0,
                       n_mdf_max=n_mdf, want_marker_force=True)
        d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L,
                         w.periodic, mu_f=lub)
        out = O.dem_run(d, w.dt / w.n_sub, n_sub, w.x, w.u, w.om, r["F_h"], r["T_h"],
                        O.History(w.n_p))
    finally:
        O.set_threads(1)
    return used, r, out


@pytest.mark.parametrize("name,kernel,n_mdf,lub", [
    ("tiny", 3, 3, 0.0),
    ("tiny", 4, 2, 0.0),
    ("small_bed", 3, 2, 1e-2),
])
def test_threads_bit_identical(name, kernel, n_mdf, lub):
    w = W.tiny() if name == "tiny" else _settled_bed()
    _, r1, o1 = _run(w, kernel, 1, n_mdf, 5, lub)
    assert r1["iterations"] == n_mdf
    # the case exercises what it claims: forcing changed the field and, for
    # the bed, contacts occurred
    assert np.max(np.abs(r1["fx"])) > 0
    if name == "small_bed":
        assert o1[5].cnt.sum() > 0 and o1[5].wact.sum() > 0
    for threads in (3, 8):
        used, r, o = _run(w, kernel, threads, n_mdf, 5, lub)
        if used == 1:
            pytest.skip("oracle built without OpenMP")
        for k in ("u", "v", "w", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
            assert np.array_equal(r[k], r1[k]), (k, threads)
        for a, b in zip(o1[:5], o[:5]):
            assert np.array_equal(a, b), threads
        for f in ("cnt", "pid", "uin", "dlt", "wact", "wuin", "wdlt"):
            assert np.array_equal(getattr(o[5], f), getattr(o1[5], f)), (f, threads)
        assert o[6] == o1[6] and r["residual"] == r1["residual"]


def test_set_threads_reports_the_count():
    try:
        n = O.set_threads(4)
        assert n in (1, 4)
        assert O.set_threads(0) == 1
    finally:
        O.set_threads(1)
