"""Seeded synthetic inputs shaped like the workloads of arXiv 2108.01814.

This module is shared by the tests, the benchmark and the smoke check. It
holds no arithmetic of the method itself (no markers, delta kernel, forcing
or contact model): only positions, velocities, fluid fields and physical
constants, drawn from numpy's PCG64 generator (host) or torch's generator
(device) with a fixed seed.

Workloads (paper: Sec. 3.5 scaling case, Sec. 4.1 erodible bed):
  tiny     64^3 triply periodic, 128 spheres D = 10h, random sequential
           addition (no overlap), u_p ~ U[-0.1, 0.1], omega ~ U[-0.01, 0.01],
           fluid N(0, 0.1^2), dt = 0.01.
  bed      8192 bed spheres D = 10h + 256 saltators with vertical velocity
           U(0, 0.5), channel periodic in x, y with walls in z. The grid is
           704 x 352 x 128: a 256 x 128 x 128 grid cannot hold 8192 spheres
           of D = 10h at solid fraction 0.58, so x and y are enlarged with
           L_x = 2 L_y to keep the bed in the lower part of the channel.
  fp32bed  131072 spheres D = 10h, 2 % lofted with vertical velocity U(0, 1),
           grid 1664 x 832 x 256 (enlarged for the same reason).
  million  1,048,576 spheres D = 6h (114 markers), grid 1024 x 768 x 512,
           bed over the lower ~260 cells; stands in for the paper's
           1,050,624-sphere case of Sec. 3.5.

Bed packing: triangular layers at solid fraction 0.58, the first resting on
the bottom wall and every later sphere resting on three spheres of the layer
below (touching them with a relative overlap of 1e-3, so the bed starts in
contact, about six contacts per sphere), the first layer jittered in the
plane. Fluid: a log law
u(z) = ln(1 + (z - z_b)/10)/0.4 above the bed top z_b (zero below) for the
streamwise component, plus i.i.d. Gaussian noise on all three components.
Gravity follows from a Shields number of 0.065 with u_tau = 1 (Sec. 4.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    n: tuple                    # cells (nx, ny, nz)
    h: float
    periodic: tuple             # (px, py, pz)
    R: float
    rho_p: float
    rho_f: float
    x: np.ndarray               # (3, n_p) positions
    u: np.ndarray               # (3, n_p) velocities
    om: np.ndarray              # (3, n_p) angular velocities
    dt: float                   # fluid step
    n_sub: int                  # particle sub-steps per fluid step (Sec. 2.1: 50)
    e_n: float
    e_t: float
    mu: float
    T_c: float
    g: tuple
    fluid_mean: str             # "none" or "loglaw"
    fluid_std: float
    bed_top: float = 0.0
    skin: float = 1.0
    seed: int = 12345
    info: dict = field(default_factory=dict)

    @property
    def n_p(self) -> int:
        return self.x.shape[1]

    @property
    def L(self) -> tuple:
        return tuple(self.n[a] * self.h for a in range(3))

    def fluid_numpy(self, seed_offset: int = 1):
        """Host fluid fields u, v, w as float64 arrays of shape (nz, ny, nx)."""
        rng = np.random.Generator(np.random.PCG64(self.seed + seed_offset))
        shape = (self.n[2], self.n[1], self.n[0])
        flds = [rng.normal(0.0, self.fluid_std, size=shape) for _ in range(3)]
        if self.fluid_mean == "loglaw":
            flds[0] += self._loglaw()[:, None, None]
        return flds

    def fluid_torch(self, dtype, device, seed_offset: int = 1):
        """Device fluid fields (torch), same recipe, torch's own generator."""
        import torch
        gen = torch.Generator(device=device)
        gen.manual_seed(self.seed + seed_offset)
        shape = (self.n[2], self.n[1], self.n[0])
        flds = []
        for _ in range(3):
            f = torch.empty(shape, dtype=dtype, device=device)
            f.normal_(0.0, self.fluid_std, generator=gen)
            flds.append(f)
        if self.fluid_mean == "loglaw":
            prof = torch.as_tensor(self._loglaw(), dtype=dtype, device=device)
            flds[0] += prof[:, None, None]
        return flds

    def _loglaw(self):
        z = (np.arange(self.n[2]) + 0.5) * self.h
        above = np.maximum(z - self.bed_top, 0.0)
        return np.log1p(above / 10.0) / 0.4

    def subset(self, idx) -> "Workload":
        """Same workload restricted to the particles idx."""
        import copy
        w = copy.copy(self)
        w.x = self.x[:, idx].copy()
        w.u = self.u[:, idx].copy()
        w.om = self.om[:, idx].copy()
        return w


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_addition(n_p, box, D, rng, margin=0.0, periodic=(1, 1, 1), zrange=None,
                    existing=None, max_tries=2_000_000):
    """Random sequential addition of n_p non-overlapping spheres (centre
    distance >= D + margin) in box, minimum image on periodic axes."""
    box = np.asarray(box, dtype=np.float64)
    pts = [] if existing is None else [tuple(p) for p in existing.T]
    placed = []
    lo = np.zeros(3)
    hi = box.copy()
    for a in range(3):
        if not periodic[a]:
            lo[a] = D / 2
            hi[a] = box[a] - D / 2
    if zrange is not None:
        lo[2], hi[2] = zrange
    # cell hash for neighbour queries
    cs = D + margin
    nc = np.maximum((box // cs).astype(int), 1)
    cells = {}

    def key(p):
        return tuple((np.floor(p / box * nc).astype(int)) % nc)

    for p in pts:
        cells.setdefault(key(np.asarray(p)), []).append(np.asarray(p))
    tries = 0
    while len(placed) < n_p:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_addition: could not place spheres")
        c = lo + (hi - lo) * rng.random(3)
        k = key(c)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % nc[0], (k[1] + dy) % nc[1], (k[2] + dz) % nc[2])
                    for q in cells.get(kk, ()):
                        d = c - q
                        for a in range(3):
                            if periodic[a]:
                                d[a] -= box[a] * np.round(d[a] / box[a])
                        if d @ d < (D + margin) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            placed.append(c)
            cells.setdefault(k, []).append(c)
    return np.array(placed).T.reshape(3, -1)


def stacked_bed(n_bed, Lx, Ly, D, phi, rng, overlap=1e-3, jitter=0.04):
    """Layered bed in mechanical contact, periodic in x and y.

    Each layer is a triangular lattice (in-plane spacing a, an even number of
    rows); the first rests on the wall z = 0, every later sphere rests on the
    three spheres of the triangle below it, at centre distance D (1 - overlap)
    from each (found by trilateration), so it touches its three supports.
    a is chosen for the solid fraction phi. The first layer is jittered in
    the plane by up to jitter * D, which makes every later layer irregular.
    Returns (x (3, n_bed), bed_top, info)."""
    Dp = D * (1.0 - overlap)
    target = (math.pi / 6 * D ** 3) / phi

    def vol(a):  # cell volume per sphere for in-plane spacing a
        return a * a * math.sqrt(3) / 2 * math.sqrt(max(Dp * Dp - a * a / 3, 0.0))

    lo, hi = D, math.sqrt(3) * Dp * 0.999
    amax = max(np.linspace(lo, hi, 2001), key=vol)
    if vol(amax) < target:
        raise ValueError("stacked_bed: solid fraction too low for touching layers")
    lo, hi = D, amax            # vol increases on [D, amax]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if vol(mid) < target:
            lo = mid
        else:
            hi = mid
    a = 0.5 * (lo + hi)
    nxc = max(int(round(Lx / a)), 3)
    nyr = max(int(round(Ly / (a * math.sqrt(3) / 2))), 4)
    nyr -= nyr % 2
    ax, ay = Lx / nxc, Ly / nyr
    per_layer = nxc * nyr
    n_layers = -(-n_bed // per_layer)
    L2 = np.array([Lx, Ly])
    row = np.repeat(np.arange(nyr), nxc)
    col = np.tile(np.arange(nxc), nyr)
    xy = np.stack([(col + 0.5 * (row % 2)) * ax, row * ay], axis=1)
    rad = jitter * D * np.sqrt(rng.random(per_layer))
    ang = 2 * math.pi * rng.random(per_layer)
    xy = xy + np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    layer = np.concatenate([np.mod(xy, L2), np.full((per_layer, 1), D / 2 - overlap * D)], axis=1)
    layers = [layer]
    # supports of site (r, c): (r, c), (r, c + 1), (r + 1, c + r % 2)
    i0 = row * nxc + col
    i1 = row * nxc + (col + 1) % nxc
    i2 = ((row + 1) % nyr) * nxc + (col + row % 2) % nxc
    for _ in range(1, n_layers):
        prev = layers[-1]
        p1, p2, p3 = prev[i0], prev[i1], prev[i2]

        def unwrap(q):
            d = q - p1
            d[:, :2] -= L2 * np.round(d[:, :2] / L2)
            return d
        v2, v3 = unwrap(p2), unwrap(p3)
        d = np.linalg.norm(v2, axis=1)
        ex = v2 / d[:, None]
        i = np.einsum("ij,ij->i", ex, v3)
        ey = v3 - i[:, None] * ex
        j = np.linalg.norm(ey, axis=1)
        ey /= j[:, None]
        ez = np.cross(ex, ey)
        xx = d / 2
        yy = (i * i + j * j) / (2 * j) - i / j * xx
        zz2 = Dp * Dp - xx * xx - yy * yy
        if np.any(zz2 <= 0):
            raise ValueError("stacked_bed: supports too far apart")
        zz = np.sqrt(zz2)
        ez *= np.sign(ez[:, 2])[:, None]
        new = p1 + xx[:, None] * ex + yy[:, None] * ey + zz[:, None] * ez
        new[:, :2] = np.mod(new[:, :2], L2)
        layers.append(new)
    x = np.concatenate(layers, axis=0)[:n_bed].T.copy()
    bed_top = float(x[2].max() + D / 2)
    c = float(np.mean(layers[-1][:, 2] - layers[-2][:, 2])) if n_layers > 1 else D
    return x, bed_top, dict(a=a, ax=ax, ay=ay, c=c, layers=int(n_layers), per_layer=int(per_layer),
                            overlap=overlap, packing="stacked")


def min_distance(x, L, periodic):
    """Smallest centre distance, minimum image on periodic axes (input check)."""
    from scipy.spatial import cKDTree
    L = np.asarray(L, dtype=np.float64)
    # cKDTree wraps every axis; a bounded axis gets a box three times its size
    box = np.where(np.asarray(periodic, bool), L, 3.0 * L + 10.0)
    pts = np.mod(x.T + np.where(np.asarray(periodic, bool), 0.0, L), box)
    d, _ = cKDTree(pts, boxsize=box).query(pts, k=2)
    return float(d[:, 1].min())


def tiny(seed: int = 12345) -> Workload:
    rng = _rng(seed)
    n = (64, 64, 64)
    D = 10.0
    x = random_addition(128, np.array(n, float), D, rng)
    u = rng.uniform(-0.1, 0.1, size=(3, 128))
    om = rng.uniform(-0.01, 0.01, size=(3, 128))
    dt = 0.01
    return Workload(name="tiny", n=n, h=1.0, periodic=(1, 1, 1), R=D / 2, rho_p=2.65,
                    rho_f=1.0, x=x, u=u, om=om, dt=dt, n_sub=50, e_n=0.9, e_t=0.39, mu=0.4,
                    T_c=10 * dt, g=(0.0, 0.0, 0.0), fluid_mean="none", fluid_std=0.1,
                    seed=seed)


def _shields_gravity(D, s=2.65, theta=0.065, u_tau=1.0):
    return u_tau ** 2 / (theta * (s - 1.0) * D)


def channel(name, n, D, n_bed, n_lofted, loft_vmax, fluid_std, seed, lofted_from_bed=False,
            dt=0.01) -> Workload:
    rng = _rng(seed)
    Lx, Ly, Lz = (float(v) for v in n)
    n_total = n_bed + (0 if lofted_from_bed else n_lofted)
    xb, bed_top, info = stacked_bed(n_bed, Lx, Ly, D, 0.58, rng)
    if bed_top > Lz - 2 * D:
        raise ValueError(f"{name}: bed top {bed_top} leaves no room in Lz={Lz}")
    u = np.zeros((3, n_total))
    om = np.zeros((3, n_total))
    if lofted_from_bed:
        x = xb
        # lift the chosen spheres above the bed, keep them non-overlapping
        pick = rng.choice(n_bed, size=n_lofted, replace=False)
        keep = np.setdiff1d(np.arange(n_bed), pick)
        above = random_addition(n_lofted, np.array([Lx, Ly, Lz]), D, rng, margin=0.1 * D,
                                periodic=(1, 1, 0), zrange=(bed_top + D / 2, Lz - D))
        x = np.concatenate([x[:, keep], above], axis=1)
        u[2, n_bed - n_lofted:] = rng.uniform(0.0, loft_vmax, size=n_lofted)
    else:
        above = random_addition(n_lofted, np.array([Lx, Ly, Lz]), D, rng, margin=0.1 * D,
                                periodic=(1, 1, 0), zrange=(bed_top + D / 2, Lz - D)) \
            if n_lofted else np.zeros((3, 0))
        x = np.concatenate([xb, above], axis=1)
        u[2, n_bed:] = rng.uniform(0.0, loft_vmax, size=n_lofted)
    info.update(n_bed=n_bed, n_lofted=n_lofted, bed_top=bed_top, phi=0.58)
    return Workload(name=name, n=tuple(n), h=1.0, periodic=(1, 1, 0), R=D / 2, rho_p=2.65,
                    rho_f=1.0, x=x, u=u, om=om, dt=dt, n_sub=50, e_n=0.9, e_t=0.39, mu=0.4,
                    T_c=10 * dt, g=(0.0, 0.0, -_shields_gravity(D)), fluid_mean="loglaw",
                    fluid_std=fluid_std, bed_top=bed_top, seed=seed, info=info)


def bed(seed: int = 12345) -> Workload:
    return channel("bed", (704, 352, 128), 10.0, 8192, 256, 0.5, 0.05, seed)


def fp32bed(seed: int = 12345) -> Workload:
    return channel("fp32bed", (1664, 832, 256), 10.0, 131072, 2621, 1.0, 0.05, seed,
                   lofted_from_bed=True)


def million(seed: int = 12345) -> Workload:
    return channel("million", (1024, 768, 512), 6.0, 1 << 20, 0, 0.0, 0.1, seed)


def slab(seed: int = 12345) -> Workload:
    """A 384 x 384 x 160 cut of the million-sphere recipe (75,000 spheres,
    D = 6h): fields of 0.28 GB per FP32 set, larger than L2, for profiling."""
    return channel("slab", (384, 384, 160), 6.0, 75000, 0, 0.0, 0.1, seed)


def small_bed(seed: int = 12345, n=(128, 64, 64), D=6.0, n_bed=600, n_lofted=20) -> Workload:
    """A bed small enough for the oracle, same recipe as `million`."""
    return channel("small_bed", n, D, n_bed, n_lofted, 0.5, 0.1, seed)


WORKLOADS = {"tiny": tiny, "bed": bed, "fp32bed": fp32bed, "million": million,
             "small_bed": small_bed, "slab": slab}


# ----------------------------------------------------------------- warm-start network
MLP_SHAPES = ((64, 9), (64,), (64, 64), (64,), (3, 64), (3,))


def mlp_init_params(seed: int = 2024) -> np.ndarray:
    """Initial parameters of the 9 -> 64 -> 64 -> 3 warm-start network as one
    float32 vector (W1, b1, W2, b2, W3, b3, row-major): weights drawn from
    N(0, 2 / fan_in), biases zero."""
    rng = _rng(seed)
    parts = []
    for shp in MLP_SHAPES:
        if len(shp) == 2:
            parts.append(rng.normal(0.0, math.sqrt(2.0 / shp[1]), size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts).astype(np.float32)
