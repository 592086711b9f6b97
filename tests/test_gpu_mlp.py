"""GPU parity of the learned warm start (tensor-core network, its gradient,
Adam, the training pairs and the warm-started forcing step) against the FP64
oracle through the C ABI, and what the trained network gains over the plain
forcing.

Tolerances. The kernels round operands to BF16 and accumulate in FP32. The
oracle's bf16 mode rounds at the same places and sums in FP64, so the two
differ only where an FP32 partial sum falls on the other side of a BF16
rounding boundary. That is rare, and a flip moves one activation by one
BF16 ulp:
- against the bf16 oracle: normwise 5e-3;
- against the plain FP64 oracle (what the BF16 network approximates):
  normwise 3e-2.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import (gpu_context, oracle_grid, oracle_template, record_errors,
                               rel_err, to_device)

pytestmark = pytest.mark.gpu

TOL_BF16, TOL_FP64 = 5e-3, 3e-2


def _theta(seed=3):
    th = W.mlp_init_params(seed).astype(np.float64)
    r = np.random.Generator(np.random.PCG64(seed))
    p = M.unpack(th.copy())
    for b in ("b1", "b2", "b3"):
        p[b][:] = r.normal(0.0, 0.1, size=p[b].shape)
    return M.pack(p).astype(np.float32).astype(np.float64)


def _data(n, seed=5):
    r = np.random.Generator(np.random.PCG64(seed))
    X = np.concatenate([r.normal(0, 0.5, (n, 3)), r.normal(0, 0.05, (n, 3)),
                        r.normal(0, 1, (n, 3))], 1)
    X[:, 6:] /= np.linalg.norm(X[:, 6:], axis=1, keepdims=True)
    T = r.normal(0, 0.3, (n, 3))
    return X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)


def _ctx():
    return gpu_context(W.tiny(), "fp32")


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 50_000])
def test_forward_matches_oracle(n):
    th = _theta()
    X, _ = _data(n)
    c = _ctx()
    c.mlp_set_params(th)
    assert np.array_equal(c.mlp_get_params(), th.astype(np.float32))
    got = c.mlp_forward(_dev(X)).cpu().numpy().astype(np.float64)
    c.close()
    ref_b, _ = M.forward(th, X, bf16_=True)
    ref, _ = M.forward(th, X)
    assert rel_err(got, ref_b) <= TOL_BF16
    assert rel_err(got, ref) <= TOL_FP64
    # most rows agree to FP32 accumulation order
    assert np.median(np.abs(got - ref_b).max(1) / np.abs(ref_b).max()) < 1e-5


@pytest.mark.parametrize("n", [100, 4000, 33_333, 150_000])
def test_gradient_matches_oracle(n):
    # 150,000 rows: 1172 tiles, several per CTA (two CTAs per SM), so the
    # weight gradients accumulate across tiles in the tensor memory
    th = _theta()
    X, T = _data(n)
    c = _ctx()
    c.mlp_set_params(th)
    g, loss = c.mlp_grad(_dev(X), _dev(T))
    c.close()
    Lb, gb = M.loss_grad(th, X, T, bf16_=True)
    L, g64 = M.loss_grad(th, X, T)
    assert loss == pytest.approx(Lb, rel=1e-4)
    assert rel_err(g, gb) <= TOL_BF16
    assert rel_err(g, g64) <= TOL_FP64


def test_adam_steps_match_oracle():
    th0 = _theta()
    X, T = _data(3000)
    c = _ctx()
    c.mlp_set_params(th0)
    th, m, v = th0.copy(), np.zeros(M.NPARAM), np.zeros(M.NPARAM)
    for k in range(1, 4):
        loss = c.mlp_train_step(_dev(X), _dev(T), lr=1e-3)
        L, gb = M.loss_grad(th.astype(np.float32).astype(np.float64), X, T, bf16_=True)
        assert loss == pytest.approx(L, rel=1e-3)
        th, m, v = M.adam_step(th, gb, m, v, k, lr=1e-3)
    got = c.mlp_get_params().astype(np.float64)
    c.close()
    assert rel_err(got - th0, th - th0) <= 2e-2


def test_collect_matches_oracle():
    # training pairs of the plain solver: features at the first interpolation
    # and targets after K = 3 plain passes, FP64 context
    import torch
    w = W.tiny()
    K = 3
    fl = w.fluid_numpy()
    z = [np.zeros_like(fl[0]) for _ in range(3)]
    t, dV = oracle_template(w)
    Xo, To, _ = M.collect(oracle_grid(w), w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, *z, w.dt,
                          1.0, K)
    c = gpu_context(w, "fp64")
    dev = to_device(fl + z, torch.float64)
    feats, targets = c.mlp_collect(*dev, w.dt, 1.0, n_mdf_max=K)
    c.close()
    assert rel_err(feats.cpu().numpy(), Xo) <= 1e-6
    assert rel_err(targets.cpu().numpy(), To) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_step_matches_oracle(precision):
    import torch
    w = W.tiny()
    th = _theta(7) * 0.5
    fl = w.fluid_numpy()
    z = [np.zeros_like(fl[0]) for _ in range(3)]
    g = oracle_grid(w)
    t, dV = oracle_template(w)
    X0, _, _ = M.collect(g, w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, *z, w.dt, 1.0, 1)
    dF0 = M.warm_increment(th, X0, w.dt, 1.0, bf16_=True)
    ref = O.ibm_step(g, w.R, w.rho_f, t, dV, w.x, w.u, w.om, *fl, *z, w.dt, 1.0, n_mdf_max=2,
                     want_marker_force=True, dF0=dF0)
    c = gpu_context(w, precision)
    c.mlp_set_params(th)
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev = to_device(fl + z, dt)
    c.ibm_step(*dev, w.dt, 1.0, n_mdf_max=2, learned=True)
    c.sync()
    got = {k: d.cpu().numpy().astype(np.float64) for k, d in zip(("u", "v", "w", "fx", "fy", "fz"), dev)}
    got.update(c.read_forces())
    got["F_l"] = c.read_marker_forces().astype(np.float64)
    c.close()
    err = {k: rel_err(got[k], ref[k]) for k in ("F_h", "T_h", "F_l")}
    err["f"] = max(rel_err(got[k], ref[k]) for k in ("fx", "fy", "fz"))
    err["grid u increment"] = max(rel_err(got[k] - a, ref[k] - a)
                                  for k, a in zip(("u", "v", "w"), fl))
    record_errors({"config": "tiny", "form": precision + " + learned warm start (2 passes)",
                   "n_p": int(w.n_p), "n_sub": 0, "errors": err})
    for k in ("u", "v", "w", "fx", "fy", "fz", "F_h", "T_h", "F_l"):
        assert rel_err(got[k], ref[k]) <= 1e-3, k


def _collect_bed(seed, n_mdf):
    import torch
    w = W.small_bed(seed=seed)
    c = gpu_context(w, "fp32")
    fl = [torch.from_numpy(a.astype(np.float32)).cuda() for a in w.fluid_numpy()]
    z = [torch.zeros_like(fl[0]) for _ in range(3)]
    feats, targets = c.mlp_collect(*fl, *z, w.dt, 1.0, n_mdf_max=n_mdf)
    return w, c, feats, targets


def _residual(w, params, learned, passes):
    import torch
    c = gpu_context(w, "fp32")
    if params is not None:
        c.mlp_set_params(params)
    fl = [torch.from_numpy(a.astype(np.float32)).cuda() for a in w.fluid_numpy()]
    z = [torch.zeros_like(fl[0]) for _ in range(3)]
    c.ibm_step(*fl, *z, w.dt, 1.0, n_mdf_max=passes, final_residual=True, learned=learned)
    r = c.stats().residual
    c.close()
    return r


def test_trained_network_gains_over_plain_forcing():
    # train on one seeded bed (targets from 10 plain passes), evaluate on
    # another: the warm-started first pass must leave a smaller slip than
    # the plain first pass, and smaller than two plain passes
    from paper_2108_01814_gb300 import warmstart
    _, c, feats, targets = _collect_bed(12345, 10)
    L0, L = warmstart.train(c, feats, targets, steps=1500)
    params = c.mlp_get_params()
    c.close()
    assert L < 0.25 * L0
    wb = W.small_bed(seed=777)
    plain1 = _residual(wb, None, False, 1)
    plain2 = _residual(wb, None, False, 2)
    learned1 = _residual(wb, params, True, 1)
    learned2 = _residual(wb, params, True, 2)
    print(f"loss {L0:.4f} -> {L:.4f}; residual after 1 pass: plain {plain1:.4f}, "
          f"learned {learned1:.4f}; after 2: plain {plain2:.4f}, learned {learned2:.4f}")
    assert learned1 < 0.6 * plain1
    assert learned1 < plain2
    assert learned2 < plain2


def test_sampled_step_equals_the_gathered_batch():
    # a minibatch drawn as rows (start + i stride) mod n_total inside the
    # kernel is the same Adam step, bit for bit, as the explicit gather
    X, T = _data(5000)
    n, start, stride = 1000, 4321, 2347
    idx = (start + np.arange(n) * stride) % len(X)
    assert len(np.unique(idx)) == n
    got = []
    for sampled in (True, False):
        c = _ctx()
        c.mlp_set_params(_theta())
        if sampled:
            loss = c.mlp_train_step_sampled(_dev(X), _dev(T), n, start, stride, lr=1e-3)
        else:
            loss = c.mlp_train_step(_dev(X[idx]), _dev(T[idx]), lr=1e-3)
        got.append((loss, c.mlp_get_params()))
        c.close()
    assert got[0][0] == got[1][0]
    assert np.array_equal(got[0][1], got[1][1])


def test_sampled_step_rejects_bad_draws():
    from paper_2108_01814_gb300 import binding as B
    X, T = _data(5000)
    c = _ctx()
    c.mlp_set_params(_theta())
    for n, start, stride in ((1000, 0, 10), (6000, 0, 7), (1000, 5000, 7), (1000, 0, 0)):
        with pytest.raises(B.PrsError) as e:
            c.mlp_train_step_sampled(_dev(X), _dev(T), n, start, stride)
        assert e.value.status == B.PRS_ERR_ARG
    c.close()


def test_training_is_deterministic():
    X, T = _data(20_000)
    out = []
    for _ in range(2):
        c = _ctx()
        c.mlp_set_params(_theta())
        for _ in range(5):
            c.mlp_train_step(_dev(X), _dev(T), lr=1e-3, want_loss=False)
        out.append(c.mlp_get_params())
        c.close()
    assert np.array_equal(out[0], out[1])


def test_learned_needs_parameters():
    from paper_2108_01814_gb300 import binding as B
    import torch
    w = W.tiny()
    c = _ctx()
    fl = [torch.zeros(w.n[::-1], device="cuda") for _ in range(6)]
    with pytest.raises(B.PrsError) as e:
        c.ibm_step(*fl, w.dt, 1.0, learned=True)
    assert e.value.status == -4
    c.close()
