"""CPU pins of the oracle's IBM half: delta kernel, marker template,
interpolation, spreading, direct forcing and per-particle summation.

Every check compares the oracle with something other than itself: values
the paper prints, identities of the Roma-Peskin-Berger kernel, exactness on
fields the kernel reproduces, conservation laws and closed forms.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.Generator(np.random.PCG64(7))


# ----------------------------------------------------------------- delta kernel
def test_phi_identities_random_shifts():
    # Roma et al. (1999) kernel: for every shift x, with the sum over all
    # integers j: sum phi(x-j) = 1, sum (x-j) phi(x-j) = 0,
    # sum phi(x-j)^2 = 1/2. A wrong branch or constant breaks one of them.
    xs = np.concatenate([rng.uniform(-3, 3, 4000), [0.0, 0.5, -0.5, 1.5, -1.5, 1.0, 2.0, 0.25]])
    js = np.arange(-6, 7)
    for x in xs:
        r = x - js
        w = O.phi(r)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs((r * w).sum()) < 1e-15
        assert abs((w * w).sum() - 0.5) < 1e-15


def test_phi_values_and_support():
    assert O.phi(0.0)[0] == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert O.phi(0.5)[0] == pytest.approx(0.5, abs=1e-16)
    assert O.phi(1.5)[0] == 0.0
    assert O.phi(1.5000001)[0] == 0.0
    r = rng.uniform(-2, 2, 200)
    assert np.all(O.phi(r) == O.phi(-r))
    assert np.all(O.phi(r) >= 0.0)
    # continuous at the branch point |r| = 0.5
    assert abs(O.phi(0.5 - 1e-12)[0] - O.phi(0.5 + 1e-12)[0]) < 1e-9


# ----------------------------------------------------------------- template
def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "marker_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()[:2]
                rows.append((float(a), int(b)))
    return rows


def test_marker_count_matches_paper():
    for r_over_h, n in _golden_counts():
        assert O.marker_count(r_over_h, 1.0) == n
    # scale invariance: the count depends on R/h only
    assert O.marker_count(10.0, 2.0) == 315


def test_marker_volume_is_shell_volume():
    for R in (3.0, 5.0, 8.0):
        n_l = O.marker_count(R, 1.0)
        shell = 4.0 / 3.0 * math.pi * ((R + 0.5) ** 3 - (R - 0.5) ** 3)
        assert n_l * O.marker_volume(R, 1.0, n_l) == pytest.approx(shell, rel=1e-14)


def test_template_points():
    for n_l in (114, 315):
        t = O.template(n_l)
        assert t.shape == (3, n_l)
        assert np.allclose(np.linalg.norm(t, axis=0), 1.0, atol=1e-15)
        # the spiral is symmetric in z and nearly balanced in x, y
        assert abs(t[2].sum()) < 1e-12
        assert np.linalg.norm(t.sum(axis=1)) < 2.0
        # second moment close to isotropic: sum t t^T ~ N/3 I
        M = t @ t.T
        assert np.allclose(M, n_l / 3.0 * np.eye(3), atol=0.02 * n_l)
        # markers spaced about one grid cell apart on a sphere of R = 5h / 3h
        R = 5.0 if n_l == 315 else 3.0
        P = R * t.T
        d = np.linalg.norm(P[:, None, :] - P[None, :, :], axis=2)
        np.fill_diagonal(d, np.inf)
        nn = d.min(axis=1)
        assert 0.8 < nn.mean() < 1.3


# ----------------------------------------------------------------- interp
def _grid_coords(g, c):
    nx, ny, nz = g.n[0], g.n[1], g.n[2]
    off = [g.off[c][a] for a in range(3)]
    xs = (np.arange(nx) + off[0]) * g.h
    ys = (np.arange(ny) + off[1]) * g.h
    zs = (np.arange(nz) + off[2]) * g.h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("off", [None, [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]])
def test_interp_reproduces_linear_fields(off):
    # the kernel's zeroth and first moments make interpolation exact on
    # linear fields (away from walls)
    g = O.make_grid((20, 18, 16), h=0.7, periodic=(0, 0, 0), off=off)
    n_m = 300
    L = np.array([20, 18, 16]) * 0.7
    Xm = np.stack([rng.uniform(2.5, L[a] - 2.5, n_m) for a in range(3)])
    for c in range(3):
        a0 = rng.normal()
        B = rng.normal(size=3)
        X, Y, Z = _grid_coords(g, c)
        field = a0 + B[0] * X + B[1] * Y + B[2] * Z
        U = O.interp(g, c, field, Xm)
        exact = a0 + B @ Xm
        assert np.max(np.abs(U - exact)) < 1e-12


def test_interp_constant_periodic():
    g = O.make_grid((12, 10, 14), periodic=(1, 1, 1))
    Xm = rng.uniform(-5, 20, size=(3, 500))
    U = O.interp(g, 1, np.full((14, 10, 12), 3.25), Xm)
    assert np.max(np.abs(U - 3.25)) < 1e-14


def test_interp_periodic_wrap_equals_shift():
    # a marker and its image one period away see the same values
    g = O.make_grid((12, 10, 14), periodic=(1, 1, 1))
    field = rng.normal(size=(14, 10, 12))
    Xm = rng.uniform(0, 10, size=(3, 50))
    U0 = O.interp(g, 0, field, Xm)
    U1 = O.interp(g, 0, field, Xm + np.array([[12.0], [-10.0], [28.0]]))
    assert np.max(np.abs(U0 - U1)) < 1e-13


def test_interp_wall_truncation():
    # bounded axis: stencil points outside the domain are dropped, so a
    # constant field is under-represented next to the wall by exactly the
    # dropped weight
    g = O.make_grid((10, 10, 10), periodic=(1, 1, 0))
    X = np.array([[5.0], [5.0], [0.2]])
    U = O.interp(g, 2, np.ones((10, 10, 10)), X)
    # nearest index 0 (centre 0.5): stencil -1, 0, 1 at -0.5, 0.5, 1.5, so
    # r = -0.7, 0.3, 1.3 and index -1 is dropped
    dropped = O.phi(-0.7)[0]
    assert U[0] == pytest.approx(1.0 - dropped, abs=1e-15)


# ----------------------------------------------------------------- spread
def test_spread_conserves_force_periodic():
    g = O.make_grid((16, 12, 10), h=0.5, periodic=(1, 1, 1))
    n_m = 400
    Xm = rng.uniform(-3, 12, size=(3, n_m))
    F = rng.normal(size=n_m)
    dV = 0.37
    f = O.spread(g, 1, np.zeros((10, 12, 16)), Xm, F, dV)
    assert f.sum() * 0.5 ** 3 == pytest.approx(F.sum() * dV, rel=1e-13)


def test_spread_conserves_first_moment():
    # sum x f h^3 = sum X F dV  (torque conservation), away from walls
    g = O.make_grid((20, 20, 20), periodic=(0, 0, 0))
    n_m = 200
    Xm = rng.uniform(3, 17, size=(3, n_m))
    F = rng.normal(size=n_m)
    dV = 1.3
    for c in range(3):
        f = O.spread(g, c, np.zeros((20, 20, 20)), Xm, F, dV)
        X, Y, Z = _grid_coords(g, c)
        for a, Q in enumerate((X, Y, Z)):
            assert (Q * f).sum() == pytest.approx((Xm[a] * F).sum() * dV, rel=1e-12)


def test_interp_spread_adjoint():
    # <interp(u), F> dV = <u, spread(F)> h^3
    g = O.make_grid((11, 13, 9), h=1.0, periodic=(1, 0, 1))
    n_m = 120
    Xm = np.stack([rng.uniform(0, 11, n_m), rng.uniform(-1, 14, n_m), rng.uniform(0, 9, n_m)])
    u = rng.normal(size=(9, 13, 11))
    F = rng.normal(size=n_m)
    dV = 0.9
    lhs = (O.interp(g, 2, u, Xm) * F).sum() * dV
    rhs = (u * O.spread(g, 2, np.zeros_like(u), Xm, F, dV)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-13)


# ----------------------------------------------------------------- forcing
def _fields(shape, val=0.0):
    return [np.full(shape, float(val)) for _ in range(6)]


def test_forcing_isolated_marker_closed_form():
    # one marker: after k forcing passes the slip U_d - U shrinks by
    # (1 - dV/(8 h^3))^k, because sum_j phi^2 = 1/2 on each axis
    g = O.make_grid((16, 16, 16), periodic=(1, 1, 1))
    t = np.array([[1.0], [0.0], [0.0]])
    x = np.array([[7.3], [8.1], [6.6]])
    up = np.array([[0.2], [-0.1], [0.05]])
    om = np.zeros((3, 1))
    u, v, w, fx, fy, fz = _fields((16, 16, 16))
    u[:] = rng.normal(scale=0.1, size=u.shape)
    R, dV, dt = 2.0, 1.0, 0.01
    X = x + R * t
    U0 = np.array([O.interp(g, c, f, X)[0] for c, f in enumerate((u, v, w))])
    slip0 = np.max(np.abs(up[:, 0] - U0))
    for k in (1, 2, 3):
        r = O.ibm_step(g, R, 1.0, t, dV, x, up, om, u, v, w, fx, fy, fz, dt, 1.0,
                       n_mdf_max=k)
        assert r["iterations"] == k
        assert r["residual"] == pytest.approx(slip0 * (7.0 / 8.0) ** k, rel=1e-12)


def test_forcing_uniform_flow_closed_form():
    # constant fluid velocity U0, particle translating at u_p: every marker
    # sees U = U0, so F_h = -rho_f N_L dV (u_p - U0)/(alpha dt) and
    # T_h = -rho_f dV R (sum_l t_l) x (u_p - U0)/(alpha dt)
    n = (24, 24, 24)
    g = O.make_grid(n, periodic=(1, 1, 1))
    R = 5.0
    n_l = O.marker_count(R)
    t = O.template(n_l)
    dV = O.marker_volume(R, 1.0, n_l)
    U0 = np.array([0.3, -0.2, 0.1])
    flds = _fields((24, 24, 24))
    for c in range(3):
        flds[c][:] = U0[c]
    x = np.array([[11.3], [12.2], [10.9]])
    up = np.array([[0.05], [0.02], [-0.04]])
    rho_f, dt, alpha = 1.3, 0.02, 0.5
    r = O.ibm_step(g, R, rho_f, t, dV, x, up, np.zeros((3, 1)), *flds, dt, alpha)
    slip = (up[:, 0] - U0) / (alpha * dt)
    assert np.allclose(r["F_h"][:, 0], -rho_f * n_l * dV * slip, rtol=1e-12, atol=1e-12)
    T = -rho_f * dV * R * np.cross(t.sum(axis=1), slip)
    assert np.allclose(r["T_h"][:, 0], T, atol=1e-10)


def test_forcing_spinning_sphere_torque_closed_form():
    # fluid at rest, sphere spinning at omega: U_d = omega x R t_l, so
    # T_h = -rho_f dV R^2 (N_L omega - (sum t t^T) omega)/(alpha dt)
    n = (24, 24, 24)
    g = O.make_grid(n, periodic=(1, 1, 1))
    R = 5.0
    n_l = O.marker_count(R)
    t = O.template(n_l)
    dV = O.marker_volume(R, 1.0, n_l)
    om = np.array([[0.03], [-0.02], [0.05]])
    x = np.array([[12.0], [12.4], [11.7]])
    dt, alpha, rho_f = 0.01, 1.0, 1.0
    r = O.ibm_step(g, R, rho_f, t, dV, x, np.zeros((3, 1)), om, *_fields(n[::-1]), dt, alpha)
    M = t @ t.T
    T = -rho_f * dV * R ** 2 * (n_l * om[:, 0] - M @ om[:, 0]) / (alpha * dt)
    assert np.allclose(r["T_h"][:, 0], T, rtol=1e-12, atol=1e-12)
    # and no net force beyond the template's imbalance
    F = -rho_f * dV * R * np.cross(om[:, 0], t.sum(axis=1)) / (alpha * dt)
    assert np.allclose(r["F_h"][:, 0], F, atol=1e-10)


def test_momentum_exchange_grid_vs_particles():
    # the force spread on the grid equals minus the particles' hydrodynamic
    # force over rho_f (spreading conserves force, summation negates it)
    n = (32, 32, 32)
    g = O.make_grid(n, periodic=(1, 1, 1))
    R = 4.0
    n_l = O.marker_count(R)
    t = O.template(n_l)
    dV = O.marker_volume(R, 1.0, n_l)
    x = np.array([[8.0, 22.0, 15.0], [9.0, 20.0, 25.0], [7.0, 16.0, 26.0]])
    up = rng.uniform(-0.1, 0.1, size=(3, 3))
    om = rng.uniform(-0.01, 0.01, size=(3, 3))
    flds = [rng.normal(scale=0.1, size=(32, 32, 32)) for _ in range(3)] + \
        [np.zeros((32, 32, 32)) for _ in range(3)]
    rho_f = 1.0
    for k in (1, 3):
        r = O.ibm_step(g, R, rho_f, t, dV, x, up, om, *flds, 0.01, 1.0, n_mdf_max=k)
        for c, key in enumerate(("fx", "fy", "fz")):
            assert r[key].sum() == pytest.approx(-r["F_h"][c].sum() / rho_f, rel=1e-11)
        # u changed by alpha dt f exactly where f was added
        du = r["u"] - flds[0]
        assert np.allclose(du, 0.01 * r["fx"], atol=1e-14)


def test_mdf_iterations_reduce_slip():
    n = (32, 32, 32)
    g = O.make_grid(n, periodic=(1, 1, 1))
    R = 5.0
    n_l = O.marker_count(R)
    t = O.template(n_l)
    dV = O.marker_volume(R, 1.0, n_l)
    x = np.array([[16.0], [15.5], [16.2]])
    up = np.array([[0.1], [0.0], [-0.05]])
    om = np.array([[0.0], [0.02], [0.0]])
    flds = [rng.normal(scale=0.1, size=(32, 32, 32)) for _ in range(3)] + \
        [np.zeros((32, 32, 32)) for _ in range(3)]
    res = [O.ibm_step(g, R, 1.0, t, dV, x, up, om, *flds, 0.01, 1.0, n_mdf_max=k)["residual"]
           for k in (1, 2, 4, 8)]
    assert all(b < a for a, b in zip(res, res[1:]))
    # tolerance stops the iteration early
    tol = res[2] * (1 + 1e-9)
    r = O.ibm_step(g, R, 1.0, t, dV, x, up, om, *flds, 0.01, 1.0, n_mdf_max=50, tol=tol)
    assert r["iterations"] == 4 and r["residual"] < tol


# ----------------------------------------------------------------- 4-point kernel
# Peskin's 4-point kernel, the wider variant of the regularised delta: the
# zeroth and first moments and the sum of squares 3/8 hold for every shift,
# which is what fixes its two branches; with them the interpolation is exact
# on linear fields, the spreading conserves force and first moment, and one
# forcing pass on an isolated marker leaves the slip times 1 - (3/8)^3 dV/h^3.

def test_phi4_identities_random_shifts():
    xs = np.concatenate([rng.uniform(-3, 3, 4000), [0.0, 0.5, 1.0, -1.0, 2.0, 1.5, 0.25]])
    js = np.arange(-7, 8)
    for x in xs:
        r = x - js
        w = O.phi4(r)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs((r * w).sum()) < 1e-14
        assert abs((w * w).sum() - 0.375) < 1e-15


def test_phi4_values_and_support():
    assert O.phi4(0.0)[0] == pytest.approx(0.5, abs=1e-16)
    assert O.phi4(1.0)[0] == pytest.approx(0.25, abs=1e-16)  # (1 - phi(0)) / 2
    assert O.phi4(2.0)[0] == 0.0 and O.phi4(2.0000001)[0] == 0.0
    r = rng.uniform(-3, 3, 200)
    assert np.all(O.phi4(r) == O.phi4(-r)) and np.all(O.phi4(r) >= 0.0)
    assert abs(O.phi4(1 - 1e-12)[0] - O.phi4(1 + 1e-12)[0]) < 1e-9


@pytest.mark.parametrize("off", [None, [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]])
def test_interp4_reproduces_linear_fields(off):
    g = O.make_grid((20, 18, 16), h=0.7, periodic=(0, 0, 0), off=off, kernel=4)
    n_m = 300
    L = np.array([20, 18, 16]) * 0.7
    Xm = np.stack([rng.uniform(3.0, L[a] - 3.0, n_m) for a in range(3)])
    for c in range(3):
        a0, B = rng.normal(), rng.normal(size=3)
        X, Y, Z = _grid_coords(g, c)
        U = O.interp(g, c, a0 + B[0] * X + B[1] * Y + B[2] * Z, Xm)
        assert np.max(np.abs(U - (a0 + B @ Xm))) < 1e-12


def test_spread4_conserves_force_and_first_moment():
    g = O.make_grid((20, 20, 20), periodic=(0, 0, 0), kernel=4)
    n_m = 200
    Xm = rng.uniform(4, 16, size=(3, n_m))
    F = rng.normal(size=n_m)
    dV = 1.3
    for c in range(3):
        f = O.spread(g, c, np.zeros((20, 20, 20)), Xm, F, dV)
        assert f.sum() == pytest.approx(F.sum() * dV, rel=1e-12)
        X, Y, Z = _grid_coords(g, c)
        for a, Q in enumerate((X, Y, Z)):
            assert (Q * f).sum() == pytest.approx((Xm[a] * F).sum() * dV, rel=1e-12)
    # periodic: the force is conserved across the wrap too
    gp = O.make_grid((12, 10, 14), periodic=(1, 1, 1), kernel=4)
    Xp = rng.uniform(-5, 20, size=(3, n_m))
    fp = O.spread(gp, 0, np.zeros((14, 10, 12)), Xp, F, dV)
    assert fp.sum() == pytest.approx(F.sum() * dV, rel=1e-12)


def test_forcing4_isolated_marker_closed_form():
    g = O.make_grid((16, 16, 16), periodic=(1, 1, 1), kernel=4)
    t = np.array([[1.0], [0.0], [0.0]])
    x = np.array([[7.3], [8.1], [6.6]])
    up = np.array([[0.2], [-0.1], [0.05]])
    om = np.zeros((3, 1))
    u, v, w, fx, fy, fz = _fields((16, 16, 16))
    u[:] = rng.normal(scale=0.1, size=u.shape)
    R, dV, dt = 2.0, 1.0, 0.01
    X = x + R * t
    U0 = np.array([O.interp(g, c, f, X)[0] for c, f in enumerate((u, v, w))])
    slip0 = np.max(np.abs(up[:, 0] - U0))
    for k in (1, 2):
        r = O.ibm_step(g, R, 1.0, t, dV, x, up, om, u, v, w, fx, fy, fz, dt, 1.0, n_mdf_max=k)
        assert r["residual"] == pytest.approx(slip0 * (1 - 0.375 ** 3) ** k, rel=1e-12)
