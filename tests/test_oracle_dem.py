"""CPU pins of the oracle's DEM half: contact sets (Appendix A, Eq. A.1-A.4),
the tangential displacement (A.9-A.11), the contact history events
(Sec. 3.4), the spring-dashpot collision (Sec. 2.1) and the Newton-Euler
update (Eq. 7-8).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.Generator(np.random.PCG64(11))


def _params(R=1.0, L=(10.0, 10.0, 10.0), periodic=(1, 1, 1), e_n=0.9, e_t=0.39, mu=0.4,
            T_c=0.1, g=(0.0, 0.0, 0.0), rho_p=2.65, rho_f=1.0, clip=False):
    return O.dem_params(R, rho_p, rho_f, e_n, e_t, mu, T_c, g, L, periodic, clip_normal=clip)


# ----------------------------------------------------------------- contact sets
def _read_contact_golden():
    P, Cs, Ns = {}, [], []
    with open(os.path.join(GOLDEN, "contact_pairs.txt")) as f:
        for line in f:
            s = line.split()
            if not s or s[0].startswith("#"):
                continue
            if s[0] == "P":
                P[int(s[1])] = [float(v) for v in s[2:5]]
            elif s[0] == "C":
                Cs.append((int(s[1]), int(s[2])))
            elif s[0] == "N":
                Ns.append((int(s[1]), int(s[2])))
    x = np.array([P[i] for i in sorted(P)]).T
    return x, sorted(Cs), sorted(Ns)


def test_contact_pairs_golden():
    x, Cs, Ns = _read_contact_golden()
    d = _params(R=1.0)
    got_c = [tuple(p) for p in O.pairs(d, x, 2.0)]
    got_n = [tuple(p) for p in O.pairs(d, x, 2.0 + 0.5)]
    assert got_c == Cs
    assert got_n == Ns


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_contact_pairs_match_kdtree(seed):
    # brute-force pair search equals scipy's k-d tree on random periodic and
    # bounded boxes (ties at exactly the cutoff have probability zero)
    from scipy.spatial import cKDTree
    r = np.random.Generator(np.random.PCG64(seed))
    L = np.array([9.0, 7.0, 8.0])
    n = 64
    x = r.uniform(0, 1, size=(3, n)) * L[:, None]
    for periodic in ((1, 1, 1), (1, 1, 0)):
        d = _params(R=0.6, L=L, periodic=periodic)
        for cut in (1.2, 1.7):
            got = {tuple(p) for p in O.pairs(d, x, cut)}
            box = np.where(np.array(periodic, bool), L, 3 * L)
            tree = cKDTree(np.mod(x.T, box), boxsize=box)
            ref = {tuple(sorted(p)) for p in tree.query_pairs(cut)}
            assert got == ref


# ----------------------------------------------------------------- collisions
def _collide(dt_frac, e_n=0.9, v=0.2, wall=False, rho_f=1.0, clip=False):
    """Head-on collision of two equal spheres (or one sphere on the bottom
    wall), no fluid force, no gravity. Returns restitution and contact time."""
    R, T_c = 1.0, 0.1
    dt_p = T_c * dt_frac
    if wall:
        d = _params(R=R, L=(20.0, 20.0, 20.0), periodic=(1, 1, 0), e_n=e_n, T_c=T_c, rho_f=rho_f,
                    clip=clip)
        x = np.array([[10.0], [10.0], [R + 0.5 * v * dt_p]])
        u = np.array([[0.0], [0.0], [-v]])
    else:
        d = _params(R=R, L=(20.0, 20.0, 20.0), e_n=e_n, T_c=T_c, rho_f=rho_f, clip=clip)
        x = np.array([[10.0 - R - 0.25 * v * dt_p, 10.0 + R + 0.25 * v * dt_p],
                      [10.0, 10.0], [10.0, 10.0]])
        u = np.array([[v / 2, -v / 2], [0.0, 0.0], [0.0, 0.0]])
    om = np.zeros_like(x)
    z = np.zeros_like(x)
    hist = O.History(x.shape[1])
    steps_in_contact = 0
    started = False
    for _ in range(int(5 / dt_frac)):
        x, u, om, Fc, Tc, hist, ov = O.dem_substep(d, dt_p, x, u, om, z, z, hist)
        touching = np.any(np.abs(Fc) > 0)
        if touching:
            started = True
            steps_in_contact += 1
        elif started:
            break
    if wall:
        e = u[2, 0] / v
    else:
        e = (u[0, 1] - u[0, 0]) / v
    return e, steps_in_contact * dt_p


def test_normal_restitution_closed_form():
    # linear spring-dashpot with k_n = m_eff (pi^2 + ln^2 e)/T_c^2 and
    # d_n = -2 m_eff ln e / T_c: the exact solution rebounds with e after T_c
    e1, t1 = _collide(1 / 500)
    assert abs(e1 - 0.9) <= 1e-3
    assert abs(t1 - 0.1) <= 2 * 0.1 / 500
    e2, _ = _collide(1 / 250)
    e3, _ = _collide(1 / 1000)
    # first-order (semi-implicit Euler) convergence towards 0.9
    assert abs(e3 - 0.9) < abs(e1 - 0.9) < abs(e2 - 0.9)
    assert 1.5 < abs(e2 - 0.9) / abs(e1 - 0.9) < 2.6


def _clipped_restitution(e_n, T_c=0.1):
    """Closed form of the damped linear oscillator xi'' + 2 z w xi' + w^2 xi = 0
    (xi the overlap, xi(0) = 0, xi'(0) = v) whose force w^2 xi + 2 z w xi'
    may not change sign: the contact ends when that force first reaches zero,
    at w_d t* = pi - atan(2 z sqrt(1 - z^2) / (1 - 2 z^2)), and the rebound is
    -xi'(t*)/v. With the constants calibrated on T_c and e_n, w_d = pi / T_c
    and z w = -ln(e_n) / T_c."""
    wd = math.pi / T_c
    zw = -math.log(e_n) / T_c
    w = math.hypot(wd, zw)
    z = zw / w
    t = (math.pi - math.atan2(2 * z * math.sqrt(1 - z * z), 1 - 2 * z * z)) / wd
    xdot = math.exp(-zw * t) * (math.cos(wd * t) - (zw / wd) * math.sin(wd * t))
    return -xdot, t


@pytest.mark.parametrize("wall", [False, True])
def test_clipped_normal_force_restitution_closed_form(wall):
    # the clipped variant rebounds faster than e_n and ends the contact
    # earlier than T_c; e_n = 0.5 makes the difference large (0.550 vs 0.5)
    e_ref, t_ref = _clipped_restitution(0.5)
    assert e_ref > 0.54 and t_ref < 0.09
    e, t = _collide(1 / 2000, e_n=0.5, wall=wall, clip=True)
    assert abs(e - e_ref) <= 2e-3
    assert abs(t - t_ref) <= 2 * 0.1 / 2000
    e_plain, t_plain = _collide(1 / 2000, e_n=0.5, wall=wall)
    assert abs(e_plain - 0.5) <= 2e-3 and abs(t_plain - 0.1) <= 2 * 0.1 / 2000


def test_wall_restitution_closed_form():
    e, t = _collide(1 / 500, wall=True)
    assert abs(e - 0.9) <= 1e-3
    assert abs(t - 0.1) <= 2 * 0.1 / 500


def test_restitution_independent_of_fluid_density():
    # the collision constants use the inertia of the rigid-body equation,
    # (rho_p - rho_f) V_p, so the rebound does not depend on rho_f
    e0, _ = _collide(1 / 500, rho_f=0.0)
    e1, _ = _collide(1 / 500, rho_f=1.5)
    assert e0 == pytest.approx(e1, abs=1e-12)


# ----------------------------------------------------------------- tangential
def _two_touching(dprev, om=None, u=None):
    R = 1.0
    d = _params(R=R)
    x = np.array([[4.0, 5.95], [5.0, 5.3], [5.0, 4.8]])
    om = np.zeros((3, 2)) if om is None else om
    u = np.zeros((3, 2)) if u is None else u
    hist = O.History(2)
    hist.cnt[:] = 1
    hist.pid[0, 0], hist.pid[1, 0] = 1, 0
    hist.dlt[0, 0] = dprev
    hist.dlt[1, 0] = dprev
    hist.uin[:, 0] = 0.05
    z = np.zeros((3, 2))
    return d, x, u, om, z, hist


def test_tangential_rotation_preserves_length():
    # A.9-A.10 project the stored displacement on the new tangent plane and
    # restore its length; with no sliding velocity A.11 adds nothing
    dprev = np.array([0.003, -0.002, 0.004])
    d, x, u, om, z, hist = _two_touching(dprev)
    _, _, _, Fc, Tc, neu, _ = O.dem_substep(d, 1e-4, x, u, om, z, z, hist)
    dn = neu.dlt[0, 0]
    nvec = (x[:, 1] - x[:, 0]) / np.linalg.norm(x[:, 1] - x[:, 0])
    assert np.linalg.norm(dn) == pytest.approx(np.linalg.norm(dprev), rel=1e-14)
    assert abs(dn @ nvec) < 1e-15
    # existing event: u_in inherited, both copies identical
    assert neu.uin[0, 0] == 0.05 and neu.uin[1, 0] == 0.05
    assert np.array_equal(neu.dlt[0, 0], neu.dlt[1, 0])
    # Newton's third law holds bit for bit
    assert np.array_equal(Fc[:, 0], -Fc[:, 1])
    assert np.array_equal(Tc[:, 0], Tc[:, 1])


def test_sliding_contact_is_capped_at_coulomb():
    # a fast tangential slip saturates |F_t| = mu |F_n| and resets the spring
    dprev = np.zeros(3)
    u = np.zeros((3, 2))
    u[2, 0] = 5.0
    d, x, u, om, z, hist = _two_touching(dprev, u=u)
    hist.cnt[:] = 0
    _, _, _, Fc, _, neu, _ = O.dem_substep(d, 1e-3, x, u, om, z, z, hist)
    nvec = (x[:, 1] - x[:, 0]) / np.linalg.norm(x[:, 1] - x[:, 0])
    F = Fc[:, 0]
    Fn = (F @ nvec) * nvec
    Ft = F - Fn
    assert np.linalg.norm(Ft) == pytest.approx(0.4 * np.linalg.norm(Fn), rel=1e-12)
    # new event: u_in is the approach speed u_cp . n, u_cp = u_p - u_q (A.5)
    assert neu.uin[0, 0] == pytest.approx((u[:, 0] - u[:, 1]) @ nvec, rel=1e-14)
    # ... and the spring was reset so that -k_t delta_t - d_t u_cp,t = F_t
    assert np.linalg.norm(neu.dlt[0, 0]) > 0


def test_contact_event_state_machine():
    # Sec. 3.4 example: particle p touches {a, b} at step n and {b, c} at
    # step n + 1: a is finished (dropped), b existing (u_in inherited),
    # c new (u_in recorded from the approach velocity)
    R = 1.0
    d = _params(R=R, L=(40.0, 40.0, 40.0))
    p = np.array([20.0, 20.0, 20.0])
    a = p + np.array([-1.99, 0.0, 0.0])
    b = p + np.array([0.0, 1.99, 0.0])
    c_far = p + np.array([0.0, 0.0, 2.5])
    c_near = p + np.array([0.0, 0.0, 1.99])
    a_far = p + np.array([-2.5, 0.0, 0.0])
    u = np.zeros((3, 4))
    u[2, 3] = -0.3  # c approaches p along z
    om = np.zeros((3, 4))
    z = np.zeros((3, 4))
    hist = O.History(4)
    x1 = np.stack([p, a, b, c_far], axis=1)
    _, _, _, _, _, h1, _ = O.dem_substep(d, 1e-5, x1, u, om, z, z, hist)
    assert list(h1.pid[0, :h1.cnt[0]]) == [1, 2]
    uin_b = h1.uin[0, 1]
    x2 = np.stack([p, a_far, b, c_near], axis=1)
    _, _, _, _, _, h2, _ = O.dem_substep(d, 1e-5, x2, u, om, z, z, h1)
    assert list(h2.pid[0, :h2.cnt[0]]) == [2, 3]
    assert h2.uin[0, 0] == uin_b                     # existing: inherited
    assert h2.uin[0, 1] == pytest.approx(0.3, abs=1e-15)  # new: approach speed
    assert h2.cnt[1] == 0                             # finished on a's side too


def test_slot_overflow_flagged():
    # 13 spheres pressed onto one: more than 12 contacts is reported
    R = 1.0
    d = _params(R=R, L=(40.0, 40.0, 40.0))
    dirs = rng.normal(size=(3, 13))
    dirs /= np.linalg.norm(dirs, axis=0)
    x = np.concatenate([np.full((3, 1), 20.0), 20.0 + 1.5 * dirs], axis=1)
    z = np.zeros_like(x)
    *_, neu, ov = O.dem_substep(d, 1e-5, x, z, z, z, z, O.History(14))
    assert ov and neu.cnt[0] == 12


# ----------------------------------------------------------------- integration
def test_free_flight_closed_form():
    # no contacts: semi-implicit Euler gives u_k = u_0 + k dt a and
    # x_k = x_0 + k dt u_0 + dt^2 a k (k + 1)/2, a = F_h/m + g,
    # omega_k = omega_0 + k dt T_h/J
    R = 0.5
    g = (0.0, 0.1, -0.98)
    d = _params(R=R, L=(50.0, 50.0, 50.0), periodic=(1, 1, 0), g=g)
    x = np.array([[3.0], [4.0], [25.0]])
    u = np.array([[0.1], [-0.2], [0.0]])
    om = np.array([[0.0], [0.1], [0.2]])
    Fh = np.array([[0.3], [0.0], [0.1]])
    Th = np.array([[0.01], [0.0], [-0.02]])
    k, dt = 40, 1e-3
    x1, u1, om1, *_ = O.dem_run(d, dt, k, x, u, om, Fh, Th, O.History(1))
    m = (2.65 - 1.0) * 4 / 3 * math.pi * R ** 3
    J = 0.4 * m * R ** 2
    a = Fh[:, 0] / m + np.array(g)
    assert np.allclose(u1[:, 0], u[:, 0] + k * dt * a, rtol=0, atol=1e-13)
    assert np.allclose(x1[:, 0], x[:, 0] + k * dt * u[:, 0] + dt * dt * a * k * (k + 1) / 2,
                       rtol=0, atol=1e-12)
    assert np.allclose(om1[:, 0], om[:, 0] + k * dt * Th[:, 0] / J, rtol=0, atol=1e-13)


def test_periodic_wrap():
    d = _params(R=0.5, L=(10.0, 10.0, 10.0))
    x = np.array([[9.99], [0.001], [5.0]])
    u = np.array([[1.0], [-1.0], [0.0]])
    z = np.zeros((3, 1))
    x1, *_ = O.dem_substep(d, 0.02, x, u, z, z, z, O.History(1))
    assert x1[0, 0] == pytest.approx(0.01, abs=1e-12)
    assert x1[1, 0] == pytest.approx(9.981, abs=1e-12)
    assert np.all((x1 >= 0) & (x1 < 10))


def test_momentum_conserved_without_walls():
    # pair forces are evaluated once per canonical pair and negated, so the
    # total momentum of a periodic packing is conserved to round-off
    R = 0.5
    L = (6.0, 6.0, 6.0)
    d = _params(R=R, L=L, T_c=0.05)
    n = 80
    r = np.random.Generator(np.random.PCG64(5))
    x = r.uniform(0, 6, size=(3, n))
    # push apart the worst overlaps so the run starts with moderate contacts
    for _ in range(200):
        pr = O.pairs(d, x, 0.9)
        if len(pr) == 0:
            break
        for p, q in pr:
            dv = x[:, q] - x[:, p]
            dv -= np.array(L)[:, None][:, 0] * np.round(dv / np.array(L))
            x[:, q] = np.mod(x[:, q] + 0.05 * dv, 6.0)
    u = r.normal(scale=0.3, size=(3, n))
    om = r.normal(scale=0.3, size=(3, n))
    z = np.zeros((3, n))
    P0 = u.sum(axis=1)
    hist = O.History(n)
    n_contacts = 0
    for _ in range(200):
        x, u, om, Fc, Tc, hist, _ = O.dem_substep(d, 5e-4, x, u, om, z, z, hist)
        n_contacts += int(hist.cnt.sum())
    assert n_contacts > 100
    assert np.max(np.abs(u.sum(axis=1) - P0)) < 1e-12 * max(1.0, np.abs(u).sum())


# ----------------------------------------------------------------- tangential law
# Appendix A (A.5-A.11) with the spring-dashpot of Eq. 9-10. For a solid
# sphere (J = 2/5 m R^2) a tangential force F_t at the contact point changes
# the contact point's tangential velocity w = u_t + R (omega x n)_t at the rate
# F_t (1/m + R^2/J) = 7 F_t / (2 m) against a wall, and 7 F_t / m for the
# relative velocity of two equal spheres. The tangential oscillator thus has
# the effective mass (2/7) m_eff, and with k_t, d_t scaled by 2/7 and built on
# e_t it has the damped half-period T_c, like the normal one. While nothing
# slides, the contact therefore ends at T_c with w = -e_t w0 and delta_t back
# at zero: the exact solution is delta_t = (w0/w_d) exp(-z w t) sin(w_d t),
# w_d = pi/T_c, z w = -ln(e_t)/T_c.

def _oblique(dt_frac, pair=False, w0=0.01, v=0.2, spin_only=False, e_n=0.9, e_t=0.39,
             mu=1e6):
    """Oblique impact of a sphere on the bottom wall (or of two equal spheres
    head-on with a small tangential relative velocity), no fluid, no gravity.
    Returns (w_end / w0, the contact time, |delta_t| at the last contact
    sub-step, the state before and after)."""
    R, T_c = 1.0, 0.1
    dt_p = T_c * dt_frac
    if pair:
        d = _params(R=R, L=(20.0, 20.0, 20.0), e_n=e_n, e_t=e_t, mu=mu, T_c=T_c)
        x = np.array([[10.0, 10.0], [10.0, 10.0],
                      [10.0 - R - 0.25 * v * dt_p, 10.0 + R + 0.25 * v * dt_p]])
        u = np.array([[w0 / 2, -w0 / 2], [0.0, 0.0], [v / 2, -v / 2]])
        om = np.zeros((3, 2))
        n = np.array([0.0, 0.0, 1.0])            # from the lower id to the higher
    else:
        d = _params(R=R, L=(20.0, 20.0, 20.0), periodic=(1, 1, 0), e_n=e_n, e_t=e_t, mu=mu,
                    T_c=T_c)
        x = np.array([[10.0], [10.0], [R + 0.5 * v * dt_p]])
        u = np.array([[w0], [0.0], [-v]])
        om = np.zeros((3, 1))
        n = np.array([0.0, 0.0, -1.0])           # from the sphere to the wall
        if spin_only:
            # the same contact-point velocity from spin alone: R omega x n = (w0, 0, 0)
            u[0, 0] = 0.0
            om[1, 0] = -w0 / R
    z = np.zeros_like(x)

    def wcp(x, u, om):
        # contact-point velocity (A.5-A.6), its part in the current tangent
        # plane, along x
        if pair:
            nn = (x[:, 1] - x[:, 0]) / np.linalg.norm(x[:, 1] - x[:, 0])
            c = R * np.cross(om[:, 0], nn) + R * np.cross(om[:, 1], nn)
            ucp = u[:, 0] - u[:, 1] + c
        else:
            nn = n
            ucp = u[:, 0] + R * np.cross(om[:, 0], nn)
        return (ucp - (ucp @ nn) * nn)[0]

    assert wcp(x, u, om) == pytest.approx(w0, rel=1e-15)
    start = (x.copy(), u.copy(), om.copy())
    hist = O.History(x.shape[1])
    steps, started, dlast = 0, False, None
    for _ in range(int(5 / dt_frac)):
        x, u, om, Fc, Tc, neu, _ = O.dem_substep(d, dt_p, x, u, om, z, z, hist)
        if np.any(np.abs(Fc) > 0):
            started = True
            steps += 1
            dlast = (neu.wdlt[0, 4] if not pair else neu.dlt[0, 0]).copy()
        elif started:
            break
        hist = neu
    return wcp(x, u, om) / w0, steps * dt_p, np.linalg.norm(dlast), start, (x, u, om), d


@pytest.mark.parametrize("pair", [False, True])
def test_tangential_rebound_closed_form(pair):
    # w_end = -e_t w0 after the contact time T_c, first order in dt_p; a
    # spring without the 2/7 factor, or built on e_n, misses both
    # (for the pair the normal approach is slow, v T_c/R = 5e-4, so that the
    # turn of n during the contact, which feeds a little of the normal
    # velocity into the tangent plane, stays well below the O(dt) error)
    T_c = 0.1
    kw = dict(pair=True, v=0.005, w0=1e-3) if pair else dict(pair=False, v=0.2, w0=1e-2)
    r1, t1, dl1, *_ = _oblique(1 / 500, **kw)
    assert abs(r1 + 0.39) <= 1.5e-3
    assert abs(t1 - T_c) <= 2 * T_c / 500
    # the spring has relaxed: |delta_t| at release is O(dt) of its peak w0 T_c/pi
    assert dl1 <= 0.05 * kw["w0"] * T_c / math.pi
    r2, *_ = _oblique(1 / 250, **kw)
    r3, *_ = _oblique(1 / 1000, **kw)
    assert abs(r3 + 0.39) < abs(r1 + 0.39) < abs(r2 + 0.39)
    assert 1.5 < abs(r2 + 0.39) / abs(r1 + 0.39) < 2.6


def test_tangential_rebound_depends_on_e_t_only():
    # the same impact with e_t = 0.7 gives -0.7; the normal e_n does not enter
    r, *_ = _oblique(1 / 1000, e_t=0.7)
    assert abs(r + 0.7) <= 3e-3
    r5, *_ = _oblique(1 / 1000, e_n=0.5)
    assert abs(r5 + 0.39) <= 3e-3


def test_spin_only_sphere_on_wall():
    # a spinning sphere dropped on the wall with no translation: the contact
    # point reverses to -e_t w0 as above, and the angular momentum about the
    # contact point, J omega - m R n x u, is unchanged (the friction force
    # acts at the contact point, the normal force through it and the centre;
    # gravity is along n), with J = 2/5 m R^2 for a solid sphere
    w0, R = 0.01, 1.0
    r, tc, _, (x0, u0, om0), (x1, u1, om1), d = _oblique(1 / 1000, w0=w0, spin_only=True)
    assert abs(r + 0.39) <= 3e-3
    assert abs(tc - 0.1) <= 2 * 0.1 / 1000
    m = (2.65 - 1.0) * 4.0 / 3.0 * math.pi * R ** 3
    J = 0.4 * m * R * R
    n = np.array([0.0, 0.0, -1.0])
    L0 = J * om0[:, 0] - m * R * np.cross(n, u0[:, 0])
    L1 = J * om1[:, 0] - m * R * np.cross(n, u1[:, 0])
    assert np.max(np.abs(L1 - L0)) <= 1e-14 * J * w0 / R * 10
    # the contact point slips along +x (omega_y < 0, R omega x n = +x), so
    # friction pushes the sphere along -x and slows the spin; with the
    # contact-point change -(1 + e_t) w0 and the invariant above, the
    # velocity takes 2/7 of that change and the spin term R omega 5/7:
    # u_x = -(1 + e_t) (2/7) w0
    assert u1[0, 0] == pytest.approx(-(1 + 0.39) * 2 / 7 * w0, rel=5e-3)
    assert om1[1, 0] - om0[1, 0] == pytest.approx((1 + 0.39) * 5 / 7 * w0 / R, rel=5e-3)


def test_pair_tangential_momentum_exact():
    # the pair's tangential force is equal and opposite on both spheres, and
    # the torques are equal (R n x F_t on the lower id, R (-n) x (-F_t) on
    # the higher one): linear momentum is conserved to round-off and the
    # spins stay equal
    _, _, _, (x0, u0, om0), (x1, u1, om1), _ = _oblique(1 / 500, pair=True, v=0.005, w0=1e-3)
    assert np.max(np.abs(u1.sum(axis=1) - u0.sum(axis=1))) <= 1e-15
    assert np.array_equal(om1[:, 0], om1[:, 1])
    assert abs(om1[1, 0]) > 0


# ----------------------------------------------------------------- lubrication
# The two-parameter lubrication model cited in Sec. 2.1 adds, below a gap of
# eps_d R, the small-gap Stokes resistance the grid no longer resolves. Its
# amplification factors are asymptotic expansions; the exact Stokes
# solutions in bispherical coordinates (Brenner 1961) pin them: a sphere
# approaching a no-slip wall, and a sphere approaching a free surface, which
# is the symmetry plane of two equal spheres approaching each other.

def _brenner(h_over_a, free=False):
    al = math.acosh(h_over_a)
    s = 0.0
    for n in range(1, 20000):
        c = n * (n + 1) / ((2 * n - 1) * (2 * n + 3))
        if not free:
            num = 2 * math.sinh((2 * n + 1) * al) + (2 * n + 1) * math.sinh(2 * al)
            den = 4 * math.sinh((n + 0.5) * al) ** 2 - (2 * n + 1) ** 2 * math.sinh(al) ** 2
        else:
            num = 4 * math.cosh((n + 0.5) * al) ** 2 + (2 * n + 1) ** 2 * math.sinh(al) ** 2
            den = 2 * math.sinh((2 * n + 1) * al) - (2 * n + 1) * math.sinh(2 * al)
        term = c * (num / den - 1.0)
        s += term
        if n > 50 and abs(term) < 1e-17 * abs(s):
            break
    return 4.0 / 3.0 * math.sinh(al) * s


def test_brenner_series_far_field():
    # the series reproduces the leading reflection 1 + 9a/8h (wall) and
    # 1 + 3a/4h (free surface) far away
    for h in (40.0, 80.0):
        assert _brenner(h) - 1 == pytest.approx(9 / (8 * h), rel=0.1)
        assert _brenner(h, free=True) - 1 == pytest.approx(3 / (4 * h), rel=0.1)


@pytest.mark.parametrize("eps", [0.05, 0.02, 0.01, 0.005, 0.002])
def test_lubrication_expansions_match_exact_stokes(eps):
    # wall: lambda(eps) vs the no-slip series at h/a = 1 + eps; two equal
    # spheres at gap eps R: lambda vs the free-surface series at 1 + eps/2;
    # the expansions drop terms of O(eps) against lambda ~ 1/eps
    w = O.lub_lambda(True, eps)
    assert abs(w - _brenner(1 + eps)) <= 0.4 * eps * eps * _brenner(1 + eps)
    p = O.lub_lambda(False, eps)
    pe = _brenner(1 + eps / 2, free=True)
    assert abs(p - pe) <= 0.4 * eps * eps * pe


def _lub_dem(mu_f=0.02, eps_d=(0.05, 0.05), eps_s=0.001, wall=False):
    R = 1.0
    if wall:
        return _params(R=R, L=(20.0, 20.0, 20.0), periodic=(1, 1, 0)), R
    return _params(R=R, L=(20.0, 20.0, 20.0)), R


def _with_lub(d, mu_f=0.02, eps_d=(0.05, 0.05), eps_s=0.001):
    d.mu_f, d.eps_d_pp, d.eps_d_pw, d.eps_s = mu_f, eps_d[0], eps_d[1], eps_s
    return d


@pytest.mark.parametrize("eps", [0.03, 0.01, 0.003])
def test_lubrication_force_against_exact_stokes(eps):
    # the force the sub-step applies: 6 pi mu R U times the amplification
    # minus its value at eps_d, for a sphere approaching the wall at speed U,
    # and for two spheres approaching each other at U each (per sphere);
    # the exact series stand in for the expansions within their error
    mu_f, U, R = 0.02, 0.3, 1.0
    dw = _with_lub(_params(R=R, L=(20.0, 20.0, 20.0), periodic=(1, 1, 0)), mu_f=mu_f)
    x = np.array([[10.0], [10.0], [R + eps * R]])
    u = np.array([[0.0], [0.0], [-U]])
    z = np.zeros_like(x)
    _, _, _, Fc, Tc, _, _ = O.dem_substep(dw, 1e-9, x, u, z, z, z, O.History(1))
    ref = 6 * math.pi * mu_f * R * U * (_brenner(1 + eps) - _brenner(1 + 0.05))
    assert Fc[2, 0] == pytest.approx(ref, rel=2e-3)
    assert np.all(Tc == 0) and Fc[0, 0] == 0 and Fc[1, 0] == 0
    dp = _with_lub(_params(R=R, L=(20.0, 20.0, 20.0)), mu_f=mu_f)
    x = np.array([[10.0 - R - eps * R / 2, 10.0 + R + eps * R / 2], [10.0, 10.0], [10.0, 10.0]])
    u = np.array([[U, -U], [0.0, 0.0], [0.0, 0.0]])
    z = np.zeros_like(x)
    _, _, _, Fc, _, _, _ = O.dem_substep(dp, 1e-9, x, u, z, z, z, O.History(2))
    ref = 6 * math.pi * mu_f * R * U * (_brenner(1 + eps / 2, True) - _brenner(1 + 0.025, True))
    assert -Fc[0, 0] == pytest.approx(ref, rel=2e-3)
    assert np.array_equal(Fc[:, 0], -Fc[:, 1])  # equal and opposite, bit for bit


def test_lubrication_range_and_saturation():
    # zero beyond eps_d R and in contact, continuous at eps_d, held at its
    # eps_s value below eps_s R
    d = _with_lub(_params(R=1.0, L=(20.0, 20.0, 20.0), periodic=(1, 1, 0)))

    def force(gap):
        x = np.array([[10.0], [10.0], [1.0 + gap]])
        u = np.array([[0.0], [0.0], [-0.3]])
        z = np.zeros_like(x)
        return O.dem_substep(d, 1e-12, x, u, z, z, z, O.History(1))[3][2, 0]

    assert force(0.0501) == 0.0
    assert 0 < force(0.0499) < 1e-3 * force(0.01)
    assert force(0.0005) == pytest.approx(force(0.001), rel=1e-12)
    assert force(0.0002) == pytest.approx(force(0.001), rel=1e-12)


# ----------------------------------------------------------------- adaptive collision time model
def test_actm_unit_collision_undamped_closed_form():
    # without damping the Hertzian contact x'' = -x^(3/2), x(0) = 0, x'(0) = 1
    # lasts 2 (5/4)^(2/5) sqrt(pi) Gamma(7/5) / Gamma(9/10) and rebounds
    # with the impact speed
    from scipy.special import gamma
    S, e = O.actm_unit(0.0)
    exact = 2 * (5 / 4) ** 0.4 * math.sqrt(math.pi) * gamma(1.4) / gamma(0.9)
    assert S == pytest.approx(exact, rel=1e-10)
    assert e == pytest.approx(1.0, abs=1e-12)


def test_actm_calibration_hits_restitution():
    for e_n in (0.97, 0.9, 0.5):
        b, S = O.actm_calibrate(e_n)
        S2, e2 = O.actm_unit(b)
        assert e2 == pytest.approx(e_n, abs=1e-12) and S2 == S
        assert b > 0 and S > 3.2180654597


def _actm_collide(v, wall, dt_frac, e_n=0.9):
    """Head-on impact at speed v under the adaptive model: restitution and
    contact time."""
    R, T_c = 1.0, 0.1
    dt_p = T_c * dt_frac
    L = (20.0, 20.0, 20.0)
    d = O.dem_params(R, 2.65, 1.0, e_n, 0.39, 0.4, T_c, (0.0, 0.0, 0.0), L,
                     (1, 1, 0) if wall else (1, 1, 1), model="actm", u_min=1e-6)
    if wall:
        x = np.array([[10.0], [10.0], [R + 0.5 * v * dt_p]])
        u = np.array([[0.0], [0.0], [-v]])
    else:
        x = np.array([[10.0 - R - 0.25 * v * dt_p, 10.0 + R + 0.25 * v * dt_p],
                      [10.0, 10.0], [10.0, 10.0]])
        u = np.array([[v / 2, -v / 2], [0.0, 0.0], [0.0, 0.0]])
    om, z = np.zeros_like(x), np.zeros_like(x)
    hist = O.History(x.shape[1])
    steps, started = 0, False
    for _ in range(int(5 / dt_frac)):
        x, u, om, Fc, Tc, hist, ov = O.dem_substep(d, dt_p, x, u, om, z, z, hist)
        if np.any(np.abs(Fc) > 0):
            started = True
            steps += 1
        elif started:
            break
    e = u[2, 0] / v if wall else (u[0, 1] - u[0, 0]) / v
    return e, steps * dt_p


@pytest.mark.parametrize("wall", [False, True])
def test_actm_duration_and_restitution_independent_of_impact_speed(wall):
    # the point of the adaptive model: whatever the impact speed, the contact
    # lasts T_c and rebounds with e_n (a fixed Hertzian stiffness would give
    # a duration falling as v^(-1/5)); first order in dt_p
    for v in (0.02, 0.2, 2.0):
        e1, t1 = _actm_collide(v, wall, 1 / 500)
        e2, t2 = _actm_collide(v, wall, 1 / 1000)
        assert abs(e2 - 0.9) < abs(e1 - 0.9) + 1e-12 and abs(e2 - 0.9) <= 2e-3, (v, e1, e2)
        assert abs(t2 - 0.1) <= 2 * 0.1 / 1000, (v, t2)
