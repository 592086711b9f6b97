"""FP64 reference of the learned warm start of the direct forcing.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The GPU product path never imports it.

The paper has no learned component. This module defines the warm start and
its training plainly, in numpy FP64:

- A per-marker network 9 -> 64 -> 64 -> 3 with ReLU:
  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3.
- Features x = [s, w, t]. s = U_d - U is the slip at the first
  interpolation of the step. w = omega_p x (X_l - x_p) is the rotational part
  of the surface velocity. t is the outward normal (Sec. 2.1, Sec. 3.3).
- Target y* = (F_K - F^(1)) alpha dt. It is the marker force after K plain
  forcing passes minus that of the first pass, in velocity units. The warm
  start adds y / (alpha dt) to the first forcing increment only.
- Loss: L = mean over markers and the 3 components of (y - y*)^2.
- Adam.

The flat parameter vector (4995 values) is W1 [64][9], b1 [64], W2 [64][64],
b2 [64], W3 [3][64], b3 [3].

With ``bf16=True`` the network rounds to bfloat16 (round to nearest even)
exactly where the tensor-core kernels round: the inputs, the weights and
biases, the hidden activations and the back-propagated errors, each before
it enters a product. Sums stay in FP64.

Parity: pinned. Central finite differences pin the gradient. Networks with
a closed-form output pin the forward. The closed form of the first Adam
step pins the optimiser. torch's bfloat16 conversion pins the rounding.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 9, 64, 3
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Views W1, b1, W2, b2, W3, b3 of the flat parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits), ties to even."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                 # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def features(R, t, x, up, om, U0):
    """x = [U_d - U, omega x r, t] per marker, markers ordered p * n_l + l.

    t: (3, n_l) template; x, up, om: (3, n_p); U0: (3, n_p * n_l) velocity
    interpolated at the markers. Returns (n_p * n_l, 9)."""
    t = np.asarray(t, dtype=np.float64)
    n_l = t.shape[1]
    n_p = np.asarray(x).shape[1]
    r = (R * t)[:, None, :] * np.ones((1, n_p, 1))          # (3, n_p, n_l)
    o = np.asarray(om, dtype=np.float64)[:, :, None]
    w = np.stack([o[1] * r[2] - o[2] * r[1],
                  o[2] * r[0] - o[0] * r[2],
                  o[0] * r[1] - o[1] * r[0]])
    Ud = np.asarray(up, dtype=np.float64)[:, :, None] + w
    s = Ud.reshape(3, -1) - np.asarray(U0, dtype=np.float64)
    tt = np.broadcast_to(t[:, None, :], (3, n_p, n_l)).reshape(3, -1)
    return np.concatenate([s, w.reshape(3, -1), tt]).T.copy()


def forward(theta, X, bf16_=False):
    """Network output (n, 3) and the intermediate values."""
    p = unpack(theta)
    rnd = bf16 if bf16_ else (lambda a: np.asarray(a, dtype=np.float64))
    X = rnd(X)
    W1, b1, W2, b2, W3, b3 = (rnd(p[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    Z1 = X @ W1.T + b1
    A1 = rnd(np.maximum(Z1, 0.0))
    Z2 = A1 @ W2.T + b2
    A2 = rnd(np.maximum(Z2, 0.0))
    Y = A2 @ W3.T + b3
    return Y, dict(X=X, W1=W1, W2=W2, W3=W3, Z1=Z1, A1=A1, Z2=Z2, A2=A2)


def loss_grad(theta, X, T, bf16_=False):
    """Loss L = mean (y - y*)^2 over the n x 3 outputs and its gradient."""
    rnd = bf16 if bf16_ else (lambda a: np.asarray(a, dtype=np.float64))
    T = np.asarray(T, dtype=np.float64)
    Y, c = forward(theta, X, bf16_)
    n = Y.shape[0]
    E = Y - T
    L = float(np.sum(E * E) / (3 * n))
    dY = rnd(2.0 * E / (3 * n))
    gW3 = dY.T @ c["A2"]
    gb3 = dY.sum(0)
    dZ2 = rnd((dY @ c["W3"]) * (c["Z2"] > 0))
    gW2 = dZ2.T @ c["A1"]
    gb2 = dZ2.sum(0)
    dZ1 = rnd((dZ2 @ c["W2"]) * (c["Z1"] > 0))
    gW1 = dZ1.T @ c["X"]
    gb1 = dZ1.sum(0)
    g = pack(dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2, W3=gW3, b3=gb3))
    return L, g


def adam_step(theta, g, m, v, k, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """Step k (k = 1, 2, ...) of Adam (Kingma & Ba 2015). Returns new
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** k)
    vh = v / (1.0 - beta2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def collect(grid, R, rho_f, t, dV, x, up, om, u, v, w, fx, fy, fz, dt, alpha, n_mdf):
    """Training pairs from the plain solver: features at the first
    interpolation and targets (F_K - F^(1)) alpha dt after K = n_mdf plain
    forcing passes. Returns (X (n_m, 9), T (n_m, 3), the step's result)."""
    from . import ibm_step, interp  # the plain oracle
    t = np.asarray(t, dtype=np.float64)
    n_l = t.shape[1]
    x = np.asarray(x, dtype=np.float64)
    Xm = (x[:, :, None] + R * t[:, None, :]).reshape(3, -1)
    U0 = np.stack([interp(grid, c, f, Xm) for c, f in enumerate((u, v, w))])
    feats = features(R, t, x, up, om, U0)
    res = ibm_step(grid, R, rho_f, t, dV, x, up, om, u, v, w, fx, fy, fz, dt, alpha,
                   n_mdf_max=n_mdf, want_marker_force=True)
    T = res["F_l"].T * (alpha * dt) - feats[:, 0:3]
    assert res["F_l"].shape[1] == x.shape[1] * n_l
    return feats, T, res


def warm_increment(theta, feats, dt, alpha, bf16_=False):
    """dF0 (3, n_m): the network's correction in force units."""
    Y, _ = forward(theta, feats, bf16_)
    return Y.T / (alpha * dt)
