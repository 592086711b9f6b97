"""FP64 oracle of the fluid sub-step predictor with an explicit viscous
stand-in (Sec. 2.1). Test infrastructure only: the tests, the smoke check
and the bench's baseline legs call it; the product path never does.

The paper's RK2 sub-step k forms hat-u^k = u^{k-1} + dt_f [alpha_k H^{k-1} -
beta_k (H^{k-2} - grad p^{k-2} / rho_f)], H = -div(uu) + nu lap(u), with
alpha_1 = 1, beta_1 = 0, alpha_2 = beta_2 = 1/2. The stand-in keeps the
viscous part of H and no pressure, H = nu lap_h(u) with the second-order
central difference the paper names for space, so

    u_out = u_in + dt (alpha nu lap_h(u_in) - beta H_prev),  H_new = nu lap_h(u_in).

Walls: on a non-periodic axis the walls sit at 0 and n h (no-slip). A
component whose points sit half a cell off the walls (offset 1/2) sees the
mirrored ghost -u beyond each wall (zero on the wall, linear across it); one
whose points sit on the walls (offset 0) holds its point 0 (on the lower
wall; H = 0 there, u_out = u_in) and sees the value 0 at the upper wall
point n. Fields are [nz][ny][nx] (x fastest).
"""
import numpy as np


def _shifted(u, axis, step, periodic, node):
    """u at index i + step along a field axis (0 = z, 1 = y, 2 = x), with the
    boundary rule of that axis."""
    if periodic:
        return np.roll(u, -step, axis=axis)
    n = u.shape[axis]
    out = np.empty_like(u)
    idx = np.arange(n) + step
    inside = (idx >= 0) & (idx < n)
    src = np.take(u, np.clip(idx, 0, n - 1), axis=axis)
    shape = [1, 1, 1]
    shape[axis] = n
    inside = inside.reshape(shape)
    if node:
        ghost = np.zeros_like(u)              # the wall point beyond n - 1 is 0
    else:
        ghost = -np.take(u, np.clip(np.arange(n), 0, n - 1), axis=axis)   # mirror: -u
    out[...] = np.where(inside, src, ghost)
    return out


def laplacian(u, h, periodic, off):
    """lap_h(u) and the mask of held wall points. periodic: (px, py, pz);
    off: the component's offsets (ox, oy, oz)."""
    u = np.asarray(u, dtype=np.float64)
    lap = -6.0 * u
    held = np.zeros(u.shape, dtype=bool)
    for a_xyz, axis in ((0, 2), (1, 1), (2, 0)):
        per = bool(periodic[a_xyz])
        node = (not per) and off[a_xyz] == 0.0
        lap = lap + _shifted(u, axis, -1, per, node) + _shifted(u, axis, +1, per, node)
        if node:
            sl = [slice(None)] * 3
            sl[axis] = 0
            held[tuple(sl)] = True
    return lap / (h * h), held


def predict(u_in, H, nu, dt, alpha, beta, h, periodic, off):
    """One predictor: returns (u_out, H_new)."""
    u_in = np.asarray(u_in, dtype=np.float64)
    lap, held = laplacian(u_in, h, periodic, off)
    Hn = np.where(held, 0.0, nu * lap)
    Hp = np.asarray(H, dtype=np.float64) if beta != 0.0 else 0.0
    u_out = np.where(held, u_in, u_in + dt * (alpha * Hn - beta * Hp))
    return u_out, Hn
