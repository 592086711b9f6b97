"""CPU pins of the oracle's learned warm start: the network, its gradient,
the optimiser, the bfloat16 rounding and the warm-started forcing step.

Each check compares the oracle with something other than itself:
- central finite differences;
- networks whose output has a closed form;
- the closed form of Adam's first step;
- torch's bfloat16 conversion;
- the isolated-marker closed form of the forcing.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2108_01814_gb300 import workloads as W

rng = np.random.Generator(np.random.PCG64(11))


def _random_theta(scale=0.5):
    return rng.normal(0.0, scale, size=M.NPARAM)


def test_parameter_count_and_layout():
    assert M.NPARAM == 64 * 9 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 4995
    th = np.arange(M.NPARAM, dtype=np.float64)
    p = M.unpack(th)
    assert p["W1"][1, 0] == 9 and p["b1"][0] == 576 and p["W2"][0, 1] == 641
    assert p["b3"][-1] == M.NPARAM - 1
    assert np.array_equal(M.pack(p), th)
    assert W.mlp_init_params().shape == (M.NPARAM,)


def test_forward_closed_form_linear_network():
    # relu(x) - relu(-x) = x: with W1 = [I; -I], W2 passing both halves
    # through and W3 = [A, -A], the network is y = A x + b3 for any x. A is
    # 3 x 9, so a transposed operand or a swapped index would break it.
    A = rng.normal(size=(3, 9))
    b3 = rng.normal(size=3)
    p = {k: np.zeros(s) for k, s in M.SHAPES}
    p["W1"][:9, :] = np.eye(9)
    p["W1"][9:18, :] = -np.eye(9)
    p["W2"][:18, :18] = np.eye(18)
    p["W3"][:, :9] = A
    p["W3"][:, 9:18] = -A
    p["b3"] = b3
    X = rng.normal(size=(50, 9))
    Y, _ = M.forward(M.pack(p), X)
    assert np.max(np.abs(Y - (X @ A.T + b3))) < 1e-13


def test_forward_closed_form_biases():
    # zero weights: the output is b3 whatever the input; with W3 = 0 and
    # W2 = 0 but b2 > 0, it is still b3
    p = {k: np.zeros(s) for k, s in M.SHAPES}
    p["b2"][:] = 1.0
    p["b3"] = np.array([0.25, -1.5, 3.0])
    Y, _ = M.forward(M.pack(p), rng.normal(size=(7, 9)))
    assert np.array_equal(Y, np.tile(p["b3"], (7, 1)))


def test_gradient_matches_central_differences():
    # the loss is piecewise quadratic in the parameters (ReLU), so central
    # differences are exact up to rounding away from kinks
    th = _random_theta()
    X = rng.normal(size=(16, 9))
    T = rng.normal(size=(16, 3))
    L, g = M.loss_grad(th, X, T)
    h = 1e-6
    fd = np.empty(M.NPARAM)
    for i in range(M.NPARAM):
        e = np.zeros(M.NPARAM)
        e[i] = h
        fd[i] = (M.loss_grad(th + e, X, T)[0] - M.loss_grad(th - e, X, T)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) / np.max(np.abs(g)) < 1e-6
    assert L == pytest.approx(np.mean((M.forward(th, X)[0] - T) ** 2), rel=1e-14)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [0.0, 1.0, -1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 255.5, 1e-30]])
    a = a.astype(np.float32).astype(np.float64)  # values the GPU kernels hold
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(a), ref)
    assert M.bf16(1.0 + 2 ** -8) == 1.0                  # tie, to even
    assert M.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie, to even (up)


def test_bf16_network_stays_close_to_fp64():
    th = _random_theta(0.2)
    X = rng.normal(size=(64, 9))
    Y, _ = M.forward(th, X)
    Yb, _ = M.forward(th, X, bf16_=True)
    assert np.max(np.abs(Yb - Y)) / np.max(np.abs(Y)) < 2e-2
    T = rng.normal(size=(64, 3))
    _, g = M.loss_grad(th, X, T)
    _, gb = M.loss_grad(th, X, T, bf16_=True)
    assert np.max(np.abs(gb - g)) / np.max(np.abs(g)) < 3e-2


def test_adam_first_step_closed_form():
    # from zero moments the bias-corrected moments are g and g^2, so the
    # first step is -lr g / (|g| + eps)
    th = _random_theta()
    g = rng.normal(size=M.NPARAM)
    z = np.zeros(M.NPARAM)
    th1, m, v = M.adam_step(th, g, z, z, 1, lr=1e-2, eps=1e-8)
    assert np.max(np.abs((th1 - th) - (-1e-2 * g / (np.abs(g) + 1e-8)))) < 1e-15
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_reduces_a_regression_loss():
    th = M.pack({k: rng.normal(0, np.sqrt(2.0 / s[-1]) if len(s) == 2 else 0.0, size=s)
                 for k, s in M.SHAPES})
    X = rng.normal(size=(256, 9))
    T = np.stack([np.sin(X[:, 0]) + X[:, 1] * X[:, 2], np.abs(X[:, 3]), X[:, 4] - X[:, 5]], 1)
    m = v = np.zeros(M.NPARAM)
    L0 = M.loss_grad(th, X, T)[0]
    for k in range(1, 301):
        L, g = M.loss_grad(th, X, T)
        th, m, v = M.adam_step(th, g, m, v, k, lr=3e-3)
    assert L < 0.2 * L0


# ------------------------------------------------------------ warm-started forcing
def _isolated():
    g = O.make_grid((16, 16, 16), periodic=(1, 1, 1))
    t = np.array([[1.0], [0.0], [0.0]])
    x = np.array([[7.3], [8.1], [6.6]])
    up = np.array([[0.2], [-0.1], [0.05]])
    om = np.zeros((3, 1))
    shape = (16, 16, 16)
    u = rng.normal(scale=0.1, size=shape)
    z = [np.zeros(shape) for _ in range(5)]
    return g, t, x, up, om, [u] + z


def test_warm_start_zero_is_the_plain_step():
    w = W.tiny()
    g = O.make_grid(w.n, w.h, w.periodic)
    n_l = O.marker_count(w.R)
    t, dV = O.template(n_l), O.marker_volume(w.R, 1.0, n_l)
    fl = w.fluid_numpy()
    z = [np.zeros_like(fl[0]) for _ in range(3)]
    a = O.ibm_step(g, w.R, 1.0, t, dV, w.x, w.u, w.om, *fl, *z, w.dt, 1.0, n_mdf_max=2)
    b = O.ibm_step(g, w.R, 1.0, t, dV, w.x, w.u, w.om, *fl, *z, w.dt, 1.0, n_mdf_max=2,
                   dF0=np.zeros((3, w.n_p * n_l)))
    for k in ("u", "v", "w", "fx", "fy", "fz", "F_h", "T_h"):
        assert np.array_equal(a[k], b[k]), k


def test_warm_start_isolated_marker_closed_form():
    # one marker, first increment (1 + c) (U_d - U)/(alpha dt): the slip
    # after it is (1 - (1 + c) dV/(8 h^3)) times the initial slip; the
    # following plain passes shrink it by (1 - dV/(8 h^3)) each
    g, t, x, up, om, flds = _isolated()
    R, dV, dt = 2.0, 1.0, 0.01
    X = x + R * t
    U0 = np.array([O.interp(g, c, f, X)[0] for c, f in enumerate(flds[:3])])
    slip = up[:, 0] - U0
    for c in (0.5, 1.0, 3.0):
        dF0 = (c * slip / dt)[:, None]
        for k in (1, 2):
            r = O.ibm_step(g, R, 1.0, t, dV, x, up, om, *flds, dt, 1.0, n_mdf_max=k, dF0=dF0)
            fac = (1.0 - (1.0 + c) / 8.0) * (7.0 / 8.0) ** (k - 1)
            assert r["residual"] == pytest.approx(abs(fac) * np.max(np.abs(slip)), rel=1e-12)


def test_collect_targets_closed_forms():
    # K = 1: the target is zero; for an isolated marker and K = 2 it is the
    # second increment, (7/8) of the first slip
    g, t, x, up, om, flds = _isolated()
    R, dV, dt = 2.0, 1.0, 0.01
    X1, T1, _ = M.collect(g, R, 1.0, t, dV, x, up, om, *flds, dt, 1.0, 1)
    assert X1.shape == (1, 9) and np.max(np.abs(T1)) < 1e-15
    X2, T2, _ = M.collect(g, R, 1.0, t, dV, x, up, om, *flds, dt, 1.0, 2)
    assert np.allclose(T2[0], 7.0 / 8.0 * X2[0, :3], rtol=1e-12, atol=1e-15)
    assert np.array_equal(X2[0, 6:], t[:, 0])


def test_features_of_a_spinning_sphere():
    # w = omega x (R t) for each marker, s = U_d - U0
    R = 2.0
    t = O.template(20)
    x = rng.uniform(0, 10, size=(3, 2))
    up = rng.normal(size=(3, 2))
    om = rng.normal(size=(3, 2))
    U0 = rng.normal(size=(3, 40))
    f = M.features(R, t, x, up, om, U0)
    for p in range(2):
        for l in range(20):
            m = p * 20 + l
            w = np.cross(om[:, p], R * t[:, l])
            assert np.allclose(f[m, 3:6], w, rtol=1e-15, atol=1e-15)
            assert np.allclose(f[m, 0:3], up[:, p] + w - U0[:, m], rtol=1e-15, atol=1e-15)
            assert np.array_equal(f[m, 6:9], t[:, l])
