"""GPU parity at full size: the million-sphere bed (1024 x 768 x 512 grid,
1,048,576 spheres of D = 6h), FP32 form, the launch configuration the bench
times. The FP64 oracle recomputes sampled outputs one by one on local blocks
of the same fields: the hydrodynamic load of sampled spheres, f and the
forced u at sampled cells, and one DEM sub-step of sampled spheres with
their neighbours (contact lists bit for bit). Tolerance: normwise 1e-5 over
the samples, as for the FP32 form everywhere."""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5
NS = 48


@pytest.fixture(scope="module")
def bed():
    return W.million()


def _block(flds, lo, B):
    """Copies of the fields on the block [lo, lo + B) (z, y, x order of the
    fields; x and y wrap, z must stay inside the grid)."""
    import torch
    nz, ny, nx = flds[0].shape
    assert 0 <= lo[2] and lo[2] + B <= nz
    iz = torch.arange(lo[2], lo[2] + B, device=flds[0].device)
    iy = torch.arange(lo[1], lo[1] + B, device=flds[0].device) % ny
    ix = torch.arange(lo[0], lo[0] + B, device=flds[0].device) % nx
    out = []
    for f in flds:
        b = f.index_select(0, iz).index_select(1, iy).index_select(2, ix)
        out.append(b.double().cpu().numpy())
    return out


def _local(x, lo, B, L, periodic):
    """Positions relative to a block origin, on the periodic image nearest
    the block's centre."""
    y = np.asarray(x, dtype=np.float64) - np.asarray(lo, dtype=np.float64)[:, None]
    for a in range(3):
        if periodic[a]:
            y[a] -= L[a] * np.round((y[a] - B / 2) / L[a])
    return y


def _near(w, p_or_pt, r):
    """Spheres whose centres lie within r of a point (minimum image in x, y)."""
    d = w.x - np.asarray(p_or_pt, dtype=np.float64)[:, None]
    for a in range(2):
        d[a] -= w.L[a] * np.round(d[a] / w.L[a])
    return np.nonzero((d * d).sum(0) < r * r)[0]


@pytest.mark.parametrize("kernel", [3, 4])
def test_million_ibm_sampled(bed, kernel):
    # the 3-point kernel (the bank-bucketed kernels) and Peskin's 4-point
    # kernel, whose stencils reach two cells: the blocks around the samples
    # hold every stencil point that matters for either
    import torch
    from paper_2108_01814_gb300 import binding as B
    w = bed
    dev = torch.device("cuda", 0)
    ctx = B.Context(w.n, w.h, w.periodic, precision="fp32", device=dev)
    ctx.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    ctx.write_state(w.x, w.u, w.om)
    flds = w.fluid_torch(torch.float32, dev)
    frc = [torch.zeros_like(flds[0]) for _ in range(3)]
    rng = np.random.Generator(np.random.PCG64(2024))
    inner = np.nonzero((w.x[2] > 12) & (w.x[2] < w.n[2] - 12))[0]
    ps = np.sort(rng.choice(inner, NS, replace=False))
    # the sampled cells: next to the surface of the sampled spheres
    dirs = rng.normal(size=(3, NS))
    dirs /= np.linalg.norm(dirs, axis=0)
    cells = np.floor(w.x[:, ps] + (w.R + 0.3) * dirs).astype(np.int64)
    cells[:2] %= np.array(w.n[:2])[:, None]
    B0 = 19
    before, around = {}, {}
    for k in range(NS):      # the fluid near each sampled cell and sphere before the step
        before[k] = _block(flds, cells[:, k] - 7, 15)
        around[k] = _block(flds, np.floor(w.x[:, ps[k]]).astype(np.int64) - B0 // 2, B0)
    ctx.ibm_step(*flds, *frc, w.dt, 1.0, delta_kernel=kernel)
    ctx.sync()
    got = ctx.read_forces()
    n_l = O.marker_count(w.R, w.h)
    t, dV = O.template(n_l), O.marker_volume(w.R, w.h, n_l)
    # hydrodynamic load of each sampled sphere, from the fluid before the
    # step (one forcing pass interpolates before it spreads)
    Fh, Th = np.zeros((3, NS)), np.zeros((3, NS))
    gl = O.make_grid((B0, B0, B0), w.h, (0, 0, 0), kernel=kernel)
    for k, p in enumerate(ps):
        lo = np.floor(w.x[:, p]).astype(np.int64) - B0 // 2
        u, v, wz = around[k]
        xl = _local(w.x[:, [p]], lo, B0, w.L, w.periodic)
        z = np.zeros_like(u)
        r = O.ibm_step(gl, w.R, w.rho_f, t, dV, xl, w.u[:, [p]], w.om[:, [p]], u, v, wz,
                       z, z, z, w.dt, 1.0)
        Fh[:, k], Th[:, k] = r["F_h"][:, 0], r["T_h"][:, 0]
    assert rel_err(got["F_h"][:, ps], Fh) <= TOL
    assert rel_err(got["T_h"][:, ps], Th) <= TOL
    # f and the forced u at the sampled cells: every sphere whose markers can
    # reach the cell, on a block around it
    gc = O.make_grid((15, 15, 15), w.h, (0, 0, 0), kernel=kernel)
    f_ref, f_got, du_ref, du_got = [], [], [], []
    for k in range(NS):
        c = cells[:, k]
        lo = c - 7
        u, v, wz = before[k]
        near = _near(w, c + 0.5, w.R + 4.0)
        xl = _local(w.x[:, near], lo, 15, w.L, w.periodic)
        z = np.zeros_like(u)
        r = O.ibm_step(gc, w.R, w.rho_f, t, dV, xl, w.u[:, near], w.om[:, near], u, v, wz,
                       z, z, z, w.dt, 1.0)
        f_ref.append([r[n][7, 7, 7] for n in ("fx", "fy", "fz")])
        du_ref.append([r[n][7, 7, 7] - b[7, 7, 7] for n, b in zip(("u", "v", "w"), (u, v, wz))])
        after = _block(flds + frc, lo, 15)
        f_got.append([after[3 + i][7, 7, 7] for i in range(3)])
        du_got.append([after[i][7, 7, 7] - before[k][i][7, 7, 7] for i in range(3)])
    ctx.close()
    f_ref, f_got = np.array(f_ref), np.array(f_got)
    assert np.count_nonzero(f_ref) > NS          # the sampled cells are forced
    assert rel_err(f_got, f_ref) <= TOL
    assert rel_err(np.array(du_got), np.array(du_ref)) <= TOL


@pytest.mark.parametrize("model,mu_f", [("linear", 0.0), ("actm", 0.0), ("linear", 0.02)])
def test_million_dem_substep_sampled(bed, model, mu_f):
    # the default contact law, the adaptive collision time model and the
    # two-parameter lubrication (Sec. 2.1), each at full size. The bed at
    # rest gives neither impact nor approach speeds, so the last two run
    # with seeded velocities and spins. Its contacts overlap and its other
    # neighbours stand 0.3 R off or more, and its bottom layer presses on
    # the wall: the lubrication case lifts the bed by 0.03 R, which puts
    # every bottom-layer sphere inside the wall's lubrication range, and
    # samples half its spheres there (sphere-sphere lubrication is checked
    # on the small beds)
    from paper_2108_01814_gb300 import binding as B
    w = bed
    x, u, om = w.x, w.u, w.om
    if model != "linear" or mu_f > 0:
        r = np.random.Generator(np.random.PCG64(11))
        u = r.normal(0.0, 0.05, w.u.shape)
        om = r.normal(0.0, 0.01, w.om.shape)
    if mu_f > 0:
        x = w.x.copy()
        x[2] += 0.03 * w.R
    ctx = B.Context(w.n, w.h, w.periodic, precision="fp32")
    ctx.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    ctx.write_state(x, u, om)
    dt_p = w.dt / w.n_sub
    ctx.dem_step(dt_p, 1, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g, model=model,
                 mu_f=mu_f)
    xg, ug, og = ctx.read_state()
    hg = ctx.read_history()
    ctx.close()
    d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic,
                     model=model, mu_f=mu_f)
    rng = np.random.Generator(np.random.PCG64(7))
    if mu_f > 0:
        bottom = np.nonzero(x[2] < 2 * w.R)[0]
        ps = np.sort(np.concatenate([rng.choice(w.n_p, NS // 2, replace=False),
                                     rng.choice(bottom, NS // 2, replace=False)]))
        ps = np.unique(ps)
        gap = x[2, ps] - w.R
        assert np.count_nonzero((gap > 0.001 * w.R) & (gap < 0.05 * w.R)) >= NS // 4
    else:
        ps = np.sort(rng.choice(w.n_p, NS, replace=False))
    ref = {"x": [], "u": [], "om": []}
    n_contacts = 0
    for p in ps:
        # the sphere and every sphere that can touch it, in ascending id
        d2 = x - x[:, p:p + 1]
        for a in range(2):
            d2[a] -= w.L[a] * np.round(d2[a] / w.L[a])
        sub = np.nonzero((d2 * d2).sum(0) < (2 * w.R + 0.5) ** 2)[0]
        i = int(np.searchsorted(sub, p))
        z = np.zeros((3, len(sub)))
        xo, uo, oo, _, _, ho, ov = O.dem_substep(d, dt_p, x[:, sub], u[:, sub],
                                                 om[:, sub], z, z, O.History(len(sub)))
        assert not ov
        # contacts p owns (higher ids), mapped back to sphere ids
        cnt = int(ho.cnt[i])
        assert hg["cnt"][p] == cnt
        assert np.array_equal(hg["pid"][p, :cnt], sub[ho.pid[i, :cnt]])
        n_contacts += cnt
        ref["x"].append(xo[:, i])
        ref["u"].append(uo[:, i])
        ref["om"].append(oo[:, i])
    assert n_contacts > len(ps)     # the bed's spheres touch their neighbours
    assert rel_err(xg[:, ps], np.array(ref["x"]).T) <= 1e-12    # positions barely move
    assert rel_err(ug[:, ps], np.array(ref["u"]).T) <= TOL
    assert rel_err(og[:, ps], np.array(ref["om"]).T) <= TOL


def test_million_coupled_substep_sampled(bed):
    # the coupling at full size in the FP32 form: one IBM step, then one
    # sub-step driven by the load it produced (the FP32 copies of F_h, T_h
    # enter the update). The oracle takes every sphere of a sampled
    # neighbourhood with the GPU's own F_h, T_h (compared above against the
    # oracle's) and runs the same sub-step in FP64.
    import torch
    from paper_2108_01814_gb300 import binding as B
    w = bed
    dev = torch.device("cuda", 0)
    ctx = B.Context(w.n, w.h, w.periodic, precision="fp32", device=dev)
    ctx.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    ctx.write_state(w.x, w.u, w.om)
    flds = w.fluid_torch(torch.float32, dev)
    frc = [torch.zeros_like(flds[0]) for _ in range(3)]
    ctx.ibm_step(*flds, *frc, w.dt, 1.0)
    load = ctx.read_forces()
    del flds, frc
    dt_p = w.dt / w.n_sub
    ctx.dem_step(dt_p, 1, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
    xg, ug, og = ctx.read_state()
    hg = ctx.read_history()
    ctx.close()
    Fh, Th = load["F_h"], load["T_h"]
    m = (w.rho_p - w.rho_f) * 4.0 / 3.0 * np.pi * w.R ** 3
    # the load moves the spheres by far more than the tolerance in one sub-step
    assert np.max(np.abs(Fh)) * dt_p / m > 1e3 * TOL * np.max(np.abs(w.u))
    d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)
    rng = np.random.Generator(np.random.PCG64(8))
    ps = np.sort(rng.choice(w.n_p, NS, replace=False))
    ref = {"u": [], "om": []}
    for p in ps:
        sub = np.sort(_near(w, w.x[:, p], 2 * w.R + 0.5))
        i = int(np.searchsorted(sub, p))
        xo, uo, oo, _, _, ho, ov = O.dem_substep(d, dt_p, w.x[:, sub], w.u[:, sub],
                                                 w.om[:, sub], Fh[:, sub], Th[:, sub],
                                                 O.History(len(sub)))
        assert not ov
        cnt = int(ho.cnt[i])
        assert hg["cnt"][p] == cnt
        assert np.array_equal(hg["pid"][p, :cnt], sub[ho.pid[i, :cnt]])
        ref["u"].append(uo[:, i])
        ref["om"].append(oo[:, i])
    ur, orf = np.array(ref["u"]).T, np.array(ref["om"]).T
    assert rel_err(ug[:, ps], ur) <= TOL
    assert rel_err(og[:, ps], orf) <= TOL
    # the velocity change of the sub-step, not only the velocity
    assert rel_err(ug[:, ps] - w.u[:, ps], ur - w.u[:, ps]) <= TOL
