"""Training loop of the learned warm start of the direct forcing.

The paper has no learned component. The network, its features and targets
are defined by the C ABI (``prs_mlp_*`` in ``include/pr_sed.h``). This module
only sequences the calls:
- collect training pairs with the plain solver;
- initialise the parameters;
- run Adam on minibatches.

Every arithmetic step runs in the library's kernels. Minibatches are
contiguous slices of the collected pairs at host-drawn random offsets. The
pairs are ordered by sphere and marker, so a slice mixes many spheres and
needs no device-side shuffle.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def collect(ctx, u, v, w, fx, fy, fz, dt, alpha=1.0, n_mdf=10):
    """One plain forcing step of n_mdf passes on the given fields (updated in
    place, like prs_ibm_step). Returns the training pairs (feats [n_m][9],
    targets [n_m][3]) as CUDA tensors."""
    return ctx.mlp_collect(u, v, w, fx, fy, fz, dt, alpha, n_mdf_max=n_mdf)


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
        i0 = int(rng.integers(0, n - bs + 1))
        ctx.mlp_train_step(feats[i0:i0 + bs], targets[i0:i0 + bs], lr=lr, want_loss=False)
    _, loss1 = ctx.mlp_grad(feats, targets)
    return loss0, loss1
