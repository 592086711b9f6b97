"""GPU parity of the IBM half (markers, interpolation, direct forcing,
spreading, per-particle sums) against the FP64 oracle, through the C ABI.

Tolerances (normwise relative error per field, max|a-b|/max|b|): FP64 form
<= 1e-10, FP32 form <= 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import gpu_context, oracle_grid, oracle_template, rel_err, to_device

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _run_both(w, precision, n_mdf=1, tol=0.0, off=None, final_residual=False, zero_f=True,
              kernel=3):
    import torch
    fl = w.fluid_numpy()
    if precision == "fp32":
        # both sides start from the same FP32 values, so that the forced
        # increment u - u_in is compared, not the rounding of the input
        fl = [a.astype(np.float32).astype(np.float64) for a in fl]
    shape = fl[0].shape
    f0 = [np.zeros(shape) for _ in range(3)]
    if not zero_f:
        rng = np.random.Generator(np.random.PCG64(99))
        f0 = [rng.normal(size=shape) for _ in range(3)]
    g = oracle_grid(w, off)
    g.kernel = kernel
    t, dV = oracle_template(w)
    ref = O.ibm_step(g, w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, *f0, w.dt, 1.0,
                     n_mdf_max=n_mdf, tol=tol, want_marker_force=True)
    ctx = gpu_context(w, precision, off)
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev = to_device(fl + f0, dt)
    ctx.ibm_step(*dev, w.dt, 1.0, n_mdf_max=n_mdf, tol=tol, final_residual=final_residual,
                 delta_kernel=kernel)
    ctx.sync()
    got = {k: d.cpu().numpy().astype(np.float64) for k, d in zip(("u", "v", "w", "fx", "fy", "fz"), dev)}
    got.update(ctx.read_forces())
    got["F_l"] = ctx.read_marker_forces().astype(np.float64)
    got["stats"] = ctx.stats()
    ctx.close()
    # the forced increments of the velocity field (Sec. 2.1: u += alpha dt f)
    for k, a in zip(("u", "v", "w"), fl):
        ref["d" + k] = ref[k] - a
        got["d" + k] = got[k] - a
    return ref, got


def test_template_matches_oracle():
    for wl in (W.tiny(), W.small_bed()):
        ctx = gpu_context(wl)
        t, dV, n_l = ctx.read_template()
        t_ref, dV_ref = oracle_template(wl)
        assert n_l == t_ref.shape[1]
        assert np.max(np.abs(t - t_ref)) < 1e-15
        assert dV == pytest.approx(dV_ref, rel=1e-15)
        ctx.close()
    assert t_ref.shape[1] == 114  # R = 3h (D = 6h)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ibm_tiny_parity(precision):
    w = W.tiny()
    ref, got = _run_both(w, precision)
    tol = TOL[precision]
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz"):
        assert rel_err(got[k], ref[k]) <= tol, k
    # the increment alone (f starts at zero, so f is the increment)
    assert rel_err(got["F_h"], ref["F_h"]) <= tol
    assert rel_err(got["T_h"], ref["T_h"]) <= tol
    assert rel_err(got["F_l"], ref["F_l"]) <= tol
    # cells the oracle leaves untouched stay untouched
    assert np.all(got["fx"][ref["fx"] == 0] == 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ibm_multidirect_forcing_parity(precision):
    w = W.tiny()
    ref, got = _run_both(w, precision, n_mdf=3, final_residual=True, zero_f=False)
    tol = TOL[precision]
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= tol, k
    assert got["stats"].mdf_passes == ref["iterations"] == 3
    assert got["stats"].residual == pytest.approx(ref["residual"], rel=10 * tol)


def test_ibm_tolerance_stops_like_oracle():
    w = W.tiny()
    probe, _ = _run_both(w, "fp64", n_mdf=4, final_residual=True)
    # a tolerance just above the residual after 2 passes stops after 2
    r2 = O.ibm_step(oracle_grid(w), w.R, w.rho_f, *oracle_template(w), w.x, w.u, w.om,
                    *w.fluid_numpy(), *[np.zeros((64, 64, 64))] * 3, w.dt, 1.0,
                    n_mdf_max=2)["residual"]
    ref, got = _run_both(w, "fp64", n_mdf=10, tol=r2 * (1 + 1e-6))
    assert ref["iterations"] == 2
    assert got["stats"].mdf_passes == 2
    assert rel_err(got["fx"], ref["fx"]) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ibm_walls_and_staggered_grid(precision):
    # channel with walls in z, staggered (MAC-like) component offsets
    w = W.small_bed()
    off = [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]
    ref, got = _run_both(w, precision, off=off)
    tol = TOL[precision]
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= tol, k


def test_ibm_bed_fp64_parity():
    # 8448 spheres of D = 10h (315 markers) in a 704 x 352 x 128 channel
    w = W.bed()
    ref, got = _run_both(w, "fp64")
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h"):
        assert rel_err(got[k], ref[k]) <= 1e-10, k


def test_ibm_is_bitwise_deterministic():
    import torch
    w = W.small_bed()
    outs = []
    for _ in range(2):
        ctx = gpu_context(w, "fp32")
        dev = w.fluid_torch(torch.float32, "cuda") + [torch.zeros((w.n[2], w.n[1], w.n[0]),
                                                                  device="cuda") for _ in range(3)]
        ctx.ibm_step(*dev, w.dt, 1.0)
        ctx.sync()
        outs.append([d.cpu().numpy() for d in dev] + [ctx.read_forces()["F_h"]])
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_ibm_host_buffers_match_device():
    import torch
    w = W.tiny()
    fl = [a.astype(np.float32) for a in w.fluid_numpy()]
    f0 = [np.zeros_like(fl[0]) for _ in range(3)]
    ctx = gpu_context(w, "fp32")
    host = [a.copy() for a in fl + f0]
    ctx.ibm_step(*host, w.dt, 1.0)
    Fh_host = ctx.read_forces()["F_h"]
    ctx.close()
    ctx = gpu_context(w, "fp32")
    dev = to_device(fl + f0, torch.float32)
    ctx.ibm_step(*dev, w.dt, 1.0)
    ctx.sync()
    Fh_dev = ctx.read_forces()["F_h"]
    ctx.close()
    for h, d in zip(host, dev):
        assert np.array_equal(h, d.cpu().numpy())
    assert np.array_equal(Fh_host, Fh_dev)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ibm_narrow_periodic_axis(precision):
    # two tiles along x (16-cell tiles): the spread takes the markers of the
    # neighbouring tiles from the binned (tile, class) ranges instead of
    # per-tile visit lists, with periodic images on both sides
    import torch
    rng = np.random.Generator(np.random.PCG64(21))
    n = (32, 40, 24)
    L = np.array(n, float)
    x = W.random_addition(12, L, 8.0, rng)
    w = W.Workload(name="narrow", n=n, h=1.0, periodic=(1, 1, 1), R=3.0, rho_p=2.65,
                   rho_f=1.0, x=x, u=rng.uniform(-0.1, 0.1, (3, 12)),
                   om=rng.uniform(-0.05, 0.05, (3, 12)), dt=0.01, n_sub=50, e_n=0.9,
                   e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none",
                   fluid_std=0.1)
    ref, got = _run_both(w, precision, n_mdf=2)
    tol = TOL[precision]
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= tol, k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,periodic", [
    ((45, 38, 30), (0, 0, 0)),   # rows of 45 values: the staging falls back to plain loads
    ((48, 40, 32), (0, 1, 0)),   # walls in x: tensor copies start left of the grid (zero fill)
])
def test_ibm_walls_and_odd_sizes(n, periodic, precision):
    # spheres touching and crossing the walls (markers beyond a wall are
    # binned to the wall cells, stencil points beyond it are dropped)
    rng = np.random.Generator(np.random.PCG64(31))
    L = np.array(n, float)
    x = W.random_addition(10, L, 7.0, rng, periodic=periodic)
    for a in range(3):
        if not periodic[a]:
            x[a, :3] = rng.uniform(0.5, 2.5, 3) if a == 0 else x[a, :3]
            x[a, 3:5] = L[a] - rng.uniform(0.5, 2.5, 2) if a == 2 else x[a, 3:5]
    w = W.Workload(name="walls", n=n, h=1.0, periodic=periodic, R=3.0, rho_p=2.65,
                   rho_f=1.0, x=x, u=rng.uniform(-0.1, 0.1, (3, 10)),
                   om=rng.uniform(-0.05, 0.05, (3, 10)), dt=0.01, n_sub=50, e_n=0.9,
                   e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none",
                   fluid_std=0.1)
    ref, got = _run_both(w, precision, n_mdf=2, zero_f=False)
    tol = TOL[precision]
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= tol, k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ibm_dense_tiles_take_the_fallback_paths(precision):
    # 9000 spheres of R = 0.8h (9 markers each), overlapping freely, in a
    # 48 x 32 x 32 box: about 1.6 markers per cell, so a tile's sphere list
    # holds more spheres than the spread stages in shared memory, more
    # markers reach a tile than its kept-marker list holds, and a tile bins
    # more markers than the interpolation copies with its fields; every
    # fallback path runs
    rng = np.random.Generator(np.random.PCG64(41))
    n = (48, 32, 32)
    k = 9000
    x = rng.uniform(0.0, 1.0, (3, k)) * np.array(n, float)[:, None]
    w = W.Workload(name="dense", n=n, h=1.0, periodic=(1, 1, 1), R=0.8, rho_p=2.65,
                   rho_f=1.0, x=x, u=rng.uniform(-0.1, 0.1, (3, k)),
                   om=rng.uniform(-0.05, 0.05, (3, k)), dt=0.01, n_sub=50, e_n=0.9,
                   e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none",
                   fluid_std=0.1)
    assert O.marker_count(w.R, w.h) == 9
    ref, got = _run_both(w, precision, n_mdf=2, zero_f=False)
    tol = TOL[precision]
    for key in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[key], ref[key]) <= tol, key


@pytest.mark.parametrize("opts,pinned", [
    (dict(n_mdf_max=1), True),
    (dict(n_mdf_max=1, host_async=True), True),
    (dict(n_mdf_max=2, final_residual=True), False),
    (dict(n_mdf_max=3, tol=1e-3, host_async=True), True),
])
def test_ibm_host_buffers_with_walls_match_device(opts, pinned):
    # walls in z: host fields are copied only over the z-slab the stencils
    # can reach, the last pass's spread runs in z-chunks whose planes are
    # copied out while the next chunk runs; two steps in a row must give
    # every cell as on the device path
    import torch
    w = W.small_bed()
    fl = [a.astype(np.float32) for a in w.fluid_numpy()]
    rng = np.random.Generator(np.random.PCG64(5))
    f0 = [rng.normal(size=fl[0].shape).astype(np.float32) for _ in range(3)]
    ctx = gpu_context(w, "fp32")
    if pinned:
        host = []
        for a in fl + f0:
            t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
            t.copy_(torch.from_numpy(a))
            host.append(t.numpy())
    else:
        host = [a.copy() for a in fl + f0]
    for _ in range(2):      # asynchronous steps: the second waits for the first's copies
        ctx.ibm_step(*host, w.dt, 1.0, **opts)
    st = ctx.stats()
    Fh_host = ctx.read_forces()["F_h"]      # synchronises
    ctx.close()
    ctx = gpu_context(w, "fp32")
    dev = to_device(fl + f0, torch.float32)
    dopts = {k: v for k, v in opts.items() if k != "host_async"}
    for _ in range(2):
        ctx.ibm_step(*dev, w.dt, 1.0, **dopts)
    ctx.sync()
    Fh_dev = ctx.read_forces()["F_h"]
    ctx.close()
    for h, d in zip(host, dev):
        assert np.array_equal(h, d.cpu().numpy())
    assert np.array_equal(Fh_host, Fh_dev)
    plane = 4 * w.n[0] * w.n[1]
    assert 0 < st.h2d_bytes == st.d2h_bytes < 6 * plane * w.n[2]
    assert st.h2d_bytes % (6 * plane) == 0


@pytest.mark.parametrize("precision,stag,asy", [("fp32", False, False), ("fp32", True, True),
                                                ("fp64", True, False)])
def test_ibm_host_pipeline_many_chunks(precision, stag, asy):
    # a tall channel whose z-slab spans more tile layers than the host path
    # has chunks (chunks of two and three layers, staggered halos of two
    # cells): the one-pass host step, pipelined over the chunks, against the
    # oracle through the device path, and bit for bit against the device path
    import torch
    w = W.channel("tall", (64, 32, 320), 6.0, 300, 30, 0.5, 0.1, 11)
    off = [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]] if stag else None
    ref, got = _run_both(w, precision, off=off, zero_f=False)
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h"):
        assert rel_err(got[k], ref[k]) <= TOL[precision], k
    tdt = torch.float64 if precision == "fp64" else torch.float32
    fl = w.fluid_numpy()
    rng = np.random.Generator(np.random.PCG64(99))
    f0 = [rng.normal(size=fl[0].shape) for _ in range(3)]
    host = []
    for a in fl + f0:
        t = torch.empty(a.shape, dtype=tdt, pin_memory=True)
        t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(tdt))
        host.append(t.numpy())
    ctx = gpu_context(w, precision, off)
    ctx.ibm_step(*host, w.dt, 1.0, host_async=asy)
    if asy:
        ctx.sync()
    st = ctx.stats()
    frc = ctx.read_forces()
    ctx.close()
    for k, h in zip(("u", "v", "w", "fx", "fy", "fz"), host):
        assert np.array_equal(h.astype(np.float64), got[k]), k
    assert np.array_equal(frc["F_h"], got["F_h"])
    assert np.array_equal(frc["T_h"], got["T_h"])
    plane = (8 if precision == "fp64" else 4) * w.n[0] * w.n[1]
    assert st.h2d_bytes == st.d2h_bytes > 6 * plane * 16 * 8   # more than 16 tile layers


# ----------------------------------------------------------------- 4-point kernel
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["tiny", "walls_staggered", "odd_mdf2", "large_spheres"])
def test_ibm_four_point_kernel_parity(case, precision):
    # Peskin's 4-point kernel (a variant of Sec. 3.3's regularised delta):
    # cell-centred and staggered offsets, walls, a periodic grid of odd
    # sizes, two forcing passes on accumulated forces
    tol = TOL[precision]
    if case == "tiny":
        ref, got = _run_both(W.tiny(), precision, kernel=4)
    elif case == "walls_staggered":
        off = [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]
        ref, got = _run_both(W.small_bed(), precision, off=off, kernel=4)
    elif case == "large_spheres":
        # three spheres of R = 8h (805 markers): beyond the 512 markers of
        # the FP32 form's 32-bit box and beyond the FP64 form's 48 KB box,
        # so both forms take the per-contribution spread
        rng = np.random.Generator(np.random.PCG64(9))
        n = (48, 48, 48)
        x = np.array([[12.0, 36.0, 24.0], [12.3, 12.7, 36.1], [24.0, 24.4, 11.8]])
        w = W.Workload(name="large", n=n, h=1.0, periodic=(1, 1, 1), R=8.0, rho_p=2.65,
                       rho_f=1.0, x=x, u=rng.uniform(-0.1, 0.1, (3, 3)),
                       om=rng.uniform(-0.05, 0.05, (3, 3)), dt=0.01, n_sub=50, e_n=0.9,
                       e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none",
                       fluid_std=0.1)
        assert O.marker_count(w.R, w.h) == 805
        ref, got = _run_both(w, precision, kernel=4)
    else:
        rng = np.random.Generator(np.random.PCG64(5))
        n = (45, 38, 30)
        L = np.array(n, float)
        x = W.random_addition(10, L, 7.0, rng)
        w = W.Workload(name="odd", n=n, h=1.0, periodic=(1, 1, 1), R=3.0, rho_p=2.65,
                       rho_f=1.0, x=x, u=rng.uniform(-0.1, 0.1, (3, 10)),
                       om=rng.uniform(-0.05, 0.05, (3, 10)), dt=0.01, n_sub=50, e_n=0.9,
                       e_t=0.39, mu=0.4, T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none",
                       fluid_std=0.1)
        ref, got = _run_both(w, precision, n_mdf=2, zero_f=False, kernel=4,
                             final_residual=True)
        assert got["stats"].residual == pytest.approx(ref["residual"], rel=10 * tol)
    for k in ("u", "v", "w", "du", "dv", "dw", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= tol, k
    if case == "tiny":
        # the kernel is in effect: the 3-point step gives other forces
        w = W.tiny()
        fl = w.fluid_numpy()
        if precision == "fp32":
            fl = [a.astype(np.float32).astype(np.float64) for a in fl]
        z = np.zeros_like(fl[0])
        ref3 = O.ibm_step(oracle_grid(w), w.R, w.rho_f, *oracle_template(w), w.x, w.u, w.om,
                          *fl, z, z, z, w.dt, 1.0)
        assert rel_err(got["F_h"], ref3["F_h"]) > 1e3 * tol


def test_ibm_four_point_kernel_rejects_host_fields():
    from paper_2108_01814_gb300 import binding as B
    w = W.tiny()
    ctx = gpu_context(w, "fp32")
    host = [np.zeros((64, 64, 64), np.float32) for _ in range(6)]
    with pytest.raises(B.PrsError) as e:
        ctx.ibm_step(*host, w.dt, 1.0, delta_kernel=4)
    assert e.value.status == B.PRS_ERR_ARG
    with pytest.raises(B.PrsError):
        ctx.ibm_step(*host, w.dt, 1.0, delta_kernel=5)
    ctx.close()
