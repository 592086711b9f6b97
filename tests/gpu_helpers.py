"""Shared helpers of the GPU parity tests (inputs and comparisons only)."""
import numpy as np

import oracle as O
from paper_2108_01814_gb300 import workloads as W


def rel_err(a, b):
    """Normwise relative error max|a - b| / max|b| of one field."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b)))


def oracle_grid(w: W.Workload, off=None):
    return O.make_grid(w.n, w.h, w.periodic, off)


def oracle_template(w: W.Workload):
    n_l = O.marker_count(w.R, w.h)
    return O.template(n_l), O.marker_volume(w.R, w.h, n_l)


def gpu_context(w: W.Workload, precision="fp64", off=None):
    from paper_2108_01814_gb300 import binding as B
    ctx = B.Context(w.n, w.h, w.periodic, offset=off, precision=precision)
    ctx.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    ctx.write_state(w.x, w.u, w.om)
    return ctx


def to_device(arrs, dtype):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda") for a in arrs]


def packing(n, L, R, seed, min_frac=0.97, periodic=(1, 1, 1), vel=0.1, spin=0.1, zrange=None):
    """Random sequential addition with centre distance >= 2 R min_frac, so
    that part of the pairs overlap slightly; random velocities and spins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = W.random_addition(n, np.asarray(L, float), 2 * R * min_frac, rng, periodic=periodic,
                          zrange=zrange)
    if not all(periodic):
        for a in range(3):
            if not periodic[a]:
                x[a] = np.clip(x[a], 0.8 * R, L[a] - 0.8 * R)
    u = rng.normal(scale=vel, size=x.shape)
    om = rng.normal(scale=spin, size=x.shape)
    return x, u, om


def record_errors(record):
    """Append one record of measured field errors to the JSON list in the
    file that PRS_ERROR_TABLE names (nothing when it is unset)."""
    import json
    import os
    path = os.environ.get("PRS_ERROR_TABLE")
    if not path:
        return
    rows = []
    if os.path.exists(path):
        with open(path) as f:
            rows = json.load(f)
    rows.append(record)
    with open(path, "w") as f:
        json.dump(rows, f, indent=1)
