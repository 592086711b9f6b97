"""CPU pins of the oracle's fluid-predictor stand-in (Sec. 2.1): discrete
eigenmodes of the 7-point Laplacian under each boundary rule, whose
eigenvalues are known in closed form, and the RK2 combination of H."""
import math

import numpy as np
import pytest

from oracle import fluid as F


def _lam(n, m, h, kind):
    """Eigenvalue of the second difference for mode m on n points:
    periodic sin(2 pi m i / n); mirrored walls sin(pi m (i + 1/2) / n);
    wall points sin(pi m i / n)."""
    th = 2 * math.pi * m / n if kind == "periodic" else math.pi * m / n
    return (2 * math.cos(th) - 2) / (h * h)


def _mode(n, m, kind):
    i = np.arange(n, dtype=np.float64)
    if kind == "periodic":
        return np.sin(2 * math.pi * m * i / n)
    if kind == "mirror":
        return np.sin(math.pi * m * (i + 0.5) / n)
    return np.sin(math.pi * m * i / n)


@pytest.mark.parametrize("zkind", ["periodic", "mirror", "node"])
def test_laplacian_eigenmodes(zkind):
    nx, ny, nz, h = 12, 10, 9, 0.7
    mx, my, mz = 2, 3, 4
    ux, uy, uz = _mode(nx, mx, "periodic"), _mode(ny, my, "periodic"), _mode(nz, mz, zkind)
    u = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    per = (1, 1, 1 if zkind == "periodic" else 0)
    off = (0.5, 0.5, 0.0 if zkind == "node" else 0.5)
    lap, held = F.laplacian(u, h, per, off)
    lam = _lam(nx, mx, h, "periodic") + _lam(ny, my, h, "periodic") + _lam(nz, mz, h, zkind)
    free = ~held
    assert np.max(np.abs(lap[free] - lam * u[free])) < 1e-12 * abs(lam)
    assert held.sum() == (nx * ny if zkind == "node" else 0)


def test_mirror_ghost_is_zero_on_the_wall():
    # a field linear across the lower wall, u = z with z measured from the
    # wall at the points (k + 1/2) h: its mirrored ghost continues the line,
    # so the second difference vanishes next to the wall as inside
    n, h = 8, 1.0
    z = (np.arange(n) + 0.5) * h
    u = np.broadcast_to(z[:, None, None], (n, 4, 4)).copy()
    lap, _ = F.laplacian(u, h, (1, 1, 0), (0.5, 0.5, 0.5))
    assert np.max(np.abs(lap[:-1])) < 1e-12      # not the top layer: its ghost is -u


def test_predictor_and_rk2_combination():
    rng = np.random.Generator(np.random.PCG64(4))
    nx, ny, nz, h, nu, dt = 16, 8, 6, 0.5, 0.3, 0.01
    u0 = np.broadcast_to(_mode(nx, 1, "periodic")[None, None, :], (nz, ny, nx)).copy()
    lam = _lam(nx, 1, h, "periodic")
    per, off = (1, 1, 1), (0.5, 0.5, 0.5)
    garbage = np.full_like(u0, np.nan)
    # sub-step 1 (alpha = 1, beta = 0): H_prev is not read
    u1, H1 = F.predict(u0, garbage, nu, dt, 1.0, 0.0, h, per, off)
    a1 = 1 + dt * nu * lam
    assert np.allclose(u1, a1 * u0, rtol=0, atol=1e-14)
    assert np.allclose(H1, nu * lam * u0, rtol=0, atol=1e-13)
    # sub-step 2 (alpha = beta = 1/2): H^{k-2} is the H of u0
    u2, H2 = F.predict(u1, H1, nu, dt, 0.5, 0.5, h, per, off)
    a2 = a1 + dt * (0.5 * nu * lam * a1 - 0.5 * nu * lam)
    assert np.allclose(u2, a2 * u0, rtol=0, atol=1e-14)
    assert np.allclose(H2, nu * lam * a1 * u0, rtol=0, atol=1e-13)
    # a random H_prev enters with -dt beta
    Hr = rng.normal(size=u0.shape)
    u3, _ = F.predict(u0, Hr, nu, dt, 0.0, 2.0, h, per, off)
    assert np.allclose(u3, u0 - 2 * dt * Hr, rtol=0, atol=1e-14)


def test_wall_points_are_held():
    rng = np.random.Generator(np.random.PCG64(5))
    u = rng.normal(size=(7, 5, 6))
    u_out, Hn = F.predict(u, np.zeros_like(u), 1.0, 0.1, 1.0, 0.0, 1.0, (1, 1, 0),
                          (0.5, 0.5, 0.0))
    assert np.array_equal(u_out[0], u[0]) and not Hn[0].any()
    assert not np.array_equal(u_out[1:], u[1:])
