"""Training loop of the learned warm start of the direct forcing.

The paper has no learned component. The network, its features and targets
are defined by the C ABI (``prs_mlp_*`` in ``include/pr_sed.h``). This module
only sequences the calls:
- collect training pairs with the plain solver;
- initialise the parameters;
- run Adam on minibatches.

Every arithmetic step runs in the library's kernels. The pairs are ordered
by sphere and marker, so a contiguous slice is a patch of neighbouring
markers; each minibatch is instead drawn by the training kernel as the rows
(start + i stride) mod n of the pairs, with start and a stride coprime with
n drawn on the host from a seeded generator, which spreads every batch over
the whole set.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W


def collect(ctx, u, v, w, fx, fy, fz, dt, alpha=1.0, n_mdf=10):
    """One plain forcing step of n_mdf passes on the given fields (updated in
    place, like prs_ibm_step). Returns the training pairs (feats [n_m][9],
    targets [n_m][3]) as CUDA tensors."""
    return ctx.mlp_collect(u, v, w, fx, fy, fz, dt, alpha, n_mdf_max=n_mdf)


def sample_stride(rng, n, max_stride=1 << 22):
    """A random start in [0, n) and a random stride in [1, min(n, 2^22)]
    coprime with n (a stride of 1 when n is 1)."""
    start = int(rng.integers(0, n))
    hi = max(1, min(n - 1, max_stride))
    while True:
        stride = int(rng.integers(1, hi + 1))
        if math.gcd(stride, n) == 1:
            return start, stride


def train(ctx, feats, targets, steps=1500, batch=4096, lr=1e-3, seed=1, init_seed=2024,
          params=None):
    """Adam on minibatches of the pairs, starting from `params` (or the
    seeded initialisation). Returns the full-batch loss before and after."""
    ctx.mlp_set_params(W.mlp_init_params(init_seed) if params is None else params)
    n = int(feats.shape[0])
    bs = min(batch, n)
    _, loss0 = ctx.mlp_grad(feats, targets)
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(steps):
        start, stride = sample_stride(rng, n)
        ctx.mlp_train_step_sampled(feats, targets, bs, start, stride, lr=lr, want_loss=False)
    _, loss1 = ctx.mlp_grad(feats, targets)
    return loss0, loss1
