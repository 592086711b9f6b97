#!/usr/bin/env python
"""Particle-steps/s of the GB300 particle-side hot path (IBM + DEM).

One step = prs_ibm_step (markers, interpolation, direct forcing, spreading,
per-particle sums; one forcing pass) + prs_dem_step with n_sub particle
sub-steps (cell-list contacts, 12-slot history, spring-dashpot forces,
Newton-Euler update). Default workload: the million-sphere bed
(1024 x 768 x 512 grid, 1,048,576 spheres of D = 6h with 114 markers each),
FP32 grid and marker arithmetic, FP64 particle state, n_sub = 50.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a
device synchronisation, timed with CUDA events on the library's stream, max
over ranks. The fluid fields (4.8 GB) are larger than L2, so no flush is
needed between steps. Prints one JSON line on rank 0.

--impl reference times the FP64 CPU oracle on all host cores instead, on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (IBM interp+spread+DEM) vs FP64 plain; % HBM roofline"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="million")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n-sub", type=int, default=50)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--dem-only", action="store_true",
                    help="time the DEM sub-steps alone on the workload's spheres (no fluid "
                         "fields on the device, F_h = T_h = 0): for profiling the DEM kernels "
                         "at full sphere count within a small device footprint")
    ap.add_argument("--variant", action="append", default=None,
                    choices=["n_sub=1", "forcing", "fp64", "bed_and_saltation",
                             "rk2_fluid_standin", "delta4"],
                    help="run only these variants (repeatable); default all")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def load_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("bf16_tflops", 1900.0)
    return 1900.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(w, target):
    """A bounded sample of the workload for the CPU oracle: the particles of
    a square column of the bed (all heights), on the matching sub-grid,
    bounded by walls so the cut does not wrap onto itself."""
    import numpy as np
    frac = min(1.0, target / w.n_p)
    side = max(16, int(round(((w.n[0] * w.n[1]) * frac) ** 0.5)))
    sx, sy = min(side, w.n[0]), min(side, w.n[1])
    keep = np.where((w.x[0] < sx) & (w.x[1] < sy))[0]
    s = w.subset(keep)
    s.n = (sx, sy, w.n[2])
    s.periodic = (0, 0, w.periodic[2])
    return s


def run_oracle_steps(s, n_sub, steps):
    """Times `steps` oracle steps (IBM + n_sub DEM sub-steps) on sample s."""
    import numpy as np
    import oracle as O
    g = O.make_grid(s.n, s.h, s.periodic)
    n_l = O.marker_count(s.R, s.h)
    t = O.template(n_l)
    dV = O.marker_volume(s.R, s.h, n_l)
    d = O.dem_params(s.R, s.rho_p, s.rho_f, s.e_n, s.e_t, s.mu, s.T_c, s.g, s.L, s.periodic)
    fl = s.fluid_numpy()
    zero = [np.zeros_like(fl[0]) for _ in range(3)]
    x, u, om = s.x, s.u, s.om
    hist = O.History(s.n_p)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        r = O.ibm_step(g, s.R, s.rho_f, t, dV, x, u, om, *fl, *zero, s.dt, 1.0)
        x, u, om, _, _, hist, _ = O.dem_run(d, s.dt / n_sub, n_sub, x, u, om, r["F_h"],
                                            r["T_h"], hist)
        times.append(time.perf_counter() - t0)
        fl = [r["u"], r["v"], r["w"]]
    return times


def host_cores():
    """Host cores this process may run on, and the machine's count."""
    try:
        avail = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        avail = os.cpu_count() or 1
    return avail, os.cpu_count() or avail


def timed_oracle(s, n_sub, steps, threads):
    """Mean seconds per oracle step on `threads` host threads (the oracle's
    results do not depend on the count); returns (seconds, threads used)."""
    import oracle as O
    used = O.set_threads(threads)
    try:
        times = run_oracle_steps(s, n_sub, steps)
    finally:
        O.set_threads(1)
    return sum(times) / len(times), used


def cpu_baseline(w, n_sub, target=2500, steps=2):
    """The FP64 oracle on the same bounded column, on one thread and on all
    host cores (OpenMP over particles, markers and grid slabs)."""
    s = oracle_sample(w, target)
    avail, nproc = host_cores()
    sec1, _ = timed_oracle(s, n_sub, 1, 1)
    secn, used = timed_oracle(s, n_sub, steps, avail)
    return {"value": s.n_p / secn, "unit": UNIT, "cores": used, "kind": "oracle",
            "nproc": nproc,
            "single_thread": {"value": s.n_p / sec1, "unit": UNIT, "cores": 1},
            "sample": f"{s.n_p} spheres of the {w.name} bed in a {s.n[0]}x{s.n[1]}x{s.n[2]} "
                      f"column (walls on the cut), IBM + {n_sub} DEM sub-steps per step, "
                      f"FP64; {steps} steps on {used} threads ({secn:.2f} s/step), "
                      f"1 step on 1 thread ({sec1:.2f} s/step)"}


def max_over_ranks(value, world, device="cpu"):
    """The largest of the ranks' values, on every rank (the value itself on
    one rank): a time for the whole job is that of its slowest replica."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- reference arm
def main_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2108_01814_gb300 import workloads as W
    import oracle as O
    w = W.WORKLOADS[a.workload]()
    s = oracle_sample(w, 1500)
    avail, nproc = host_cores()
    used = O.set_threads(avail)
    try:
        run_oracle_steps(s, a.n_sub, max(a.warmup, 0)) if a.warmup else None
        times = run_oracle_steps(s, a.n_sub, a.steps)
    finally:
        O.set_threads(1)
    sec = sum(times)
    value = s.n_p * a.steps / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000 * sec / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name} bed sample: {s.n_p} spheres, {s.n[0]}x{s.n[1]}x"
                               f"{s.n[2]} column, n_sub={a.n_sub}", "oracle": "plain C FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "nproc": nproc,
                         "kind": "oracle",
                         "sample": f"{s.n_p} spheres per step on {used} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def alg_bytes(kind, b, S, n_p, n_contacts, n_wall):
    """Algorithmic bytes per launch (what the method itself must move)."""
    if kind == "interp":
        return 3 * b * S + 72 * n_p          # u, v, w on S + particle state
    if kind == "spread":
        return 12 * b * S                    # read+write f and u on S
    if kind == "dem_contacts":
        # state in, slot counts in/out, per pair (each evaluated once, n_contacts
        # counts both spheres): history slot in and out (id, u_in, delta_t)
        return 72 * n_p + 8 * n_p + 72 * (n_contacts // 2)
    if kind == "dem_update":
        # state in/out, F_h/T_h in, F_c/T_c out, wall slots in/out (the pair
        # forces handed over by the contact kernel are not counted)
        return 240 * n_p + 66 * n_wall
    if kind == "dem_cells":
        return 24 * n_p + 16 * n_p            # positions in, cell keys and sorted ids out
    if kind == "ibm_bin":
        return 72 * n_p + 160 * n_p           # state in, per-particle records out
    return 0


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the IBM phases on the million-sphere FP32 workload (n_sub = 50), valid
# for the kernels as they were captured. Each is one ncu capture of one
# launch per kernel on the 384 x 384 x 160 slab of the same recipe (fields
# larger than L2), scaled to the million-sphere bed by the cells of the
# stencil support |S|: 204,392,806 / 14,982,573. The spread phase is the
# plan kernel and the bank-bucketed spread. The DEM kernels have no entry:
# at the slab's size their writes stay in L2 during the launch, so one
# launch's DRAM writes are not observable there.
_S_SCALE = 204392806 / 14982573
TRAFFIC = {
    ("million", "fp32", "interp"): (227.6544e6 + 106.664704e6) * _S_SCALE,
    ("million", "fp32", "spread"): (579.144448e6 + 318.7072e6 + 3.058432e6 + 256) * _S_SCALE,
}


def _time_steps(step, k, stream, dev):
    import torch
    step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / k


TRAIN_STEPS, TRAIN_BATCH = 6000, 16384


def forcing_variants(a, w, ctx, flds, dt_p, dem, stream, dev):
    """Plain multi-direct forcing against the learned warm start on the same
    bed: slip left after the passes (max |U_d - U|) and full-step throughput
    (IBM + n_sub DEM sub-steps). The network is trained first, on the GPU,
    with pairs from another seeded bed: for the million-sphere bed a
    75,000-sphere bed of the same recipe, pairs from 3 successive steps of a
    run (about 26M markers); for the 131,072-sphere FP32 bed the 8448-sphere
    channel bed, pairs from 8 successive steps of a run (about 21M markers).
    Minibatches are drawn across the whole set of pairs (strided sampling in
    the training kernel). The plain and learned forms are also run under the
    fallback rule: passes until the slip is below 1e-4 or 12 passes."""
    import numpy as np
    import torch
    from paper_2108_01814_gb300 import binding as B
    from paper_2108_01814_gb300 import warmstart
    from paper_2108_01814_gb300 import workloads as W
    snaps = 1
    if w.name in ("million", "slab"):
        # about 20M pairs: 3 successive steps of a 75,000-sphere bed
        wt, snaps = W.slab(seed=4242), 3
    elif w.name == "fp32bed":
        wt, snaps = W.bed(seed=4242), 8
    else:
        wt = W.small_bed(seed=4242, D=2 * w.R)
    with torch.cuda.stream(stream):
        tf = [torch.from_numpy(x.astype(np.float32)).to(dev) for x in wt.fluid_numpy()]
        tz = [torch.zeros_like(tf[0]) for _ in range(3)]
    tc = B.Context(wt.n, wt.h, wt.periodic, precision="fp32", device=dev, stream=stream)
    tc.create_particles(wt.n_p, wt.R, wt.rho_p, wt.rho_f)
    tc.write_state(wt.x, wt.u, wt.om)
    t0 = time.perf_counter()
    parts = []
    for k in range(snaps):
        if k:
            # one plain step of the run between snapshots
            tc.ibm_step(*tf, *tz, wt.dt, 1.0)
            tc.dem_step(wt.dt / wt.n_sub, wt.n_sub, e_n=wt.e_n, e_t=wt.e_t, mu=wt.mu,
                        T_c=wt.T_c, g=wt.g)
        parts.append(warmstart.collect(tc, *tf, *tz, wt.dt, 1.0, n_mdf=10))
    feats = torch.cat([f for f, _ in parts]) if snaps > 1 else parts[0][0]
    targets = torch.cat([t for _, t in parts]) if snaps > 1 else parts[0][1]
    del parts
    L0, L1 = warmstart.train(tc, feats, targets, steps=TRAIN_STEPS, batch=TRAIN_BATCH)
    stream.synchronize()
    t_train = time.perf_counter() - t0
    params = tc.mlp_get_params()
    tc.close()
    del tf, tz, feats, targets
    ctx.mlp_set_params(params)
    out = {"warm_start_training": {"pairs": int(snaps * wt.n_p * tc.n_l), "steps": TRAIN_STEPS,
                                   "batch": TRAIN_BATCH,
                                   "loss_before": L0, "loss_after": L1, "seconds": t_train,
                                   "bed": f"{wt.name} seed 4242, D={2 * wt.R:g}h, "
                                          f"{snaps} snapshot(s)"}}
    # the fluid as generated (the timed steps above have forced it)
    with torch.cuda.stream(stream):
        fresh = w.fluid_torch(torch.float32 if ctx.precision == B.PRS_FP32 else torch.float64,
                              dev)
    stream.synchronize()
    for name, learned, k in (("plain_mdf1", False, 1), ("plain_mdf2", False, 2),
                             ("plain_mdf3", False, 3), ("learned_mdf1", True, 1),
                             ("learned_mdf2", True, 2)):
        # the slip left on the bed as generated (spheres at rest, like the
        # training bed); the timed steps move it
        ctx.write_state(w.x, w.u, w.om)
        with torch.cuda.stream(stream):
            uc = [f.clone() for f in fresh]
            fc = [torch.zeros_like(fresh[0]) for _ in range(3)]
        ctx.ibm_step(*uc, *fc, w.dt, 1.0, n_mdf_max=k, final_residual=True, learned=learned)
        res = ctx.stats().residual

        def step():
            ctx.ibm_step(*uc, *fc, w.dt, 1.0, n_mdf_max=k, learned=learned)
            ctx.dem_step(dt_p, a.n_sub, **dem)
        ms = _time_steps(step, 2, stream, dev)
        out[name] = {"value": w.n_p / (ms / 1e3), "ms_per_step": ms, "residual": res}
        del uc, fc
    # the fallback rule: the learned (or plain) first pass, then plain passes
    # until the slip max |U_d - U| is below tol or n_mdf_max passes have run
    tol, kmax = 1e-4, 12
    for name, learned in (("plain_tol1e-4", False), ("learned_tol1e-4", True)):
        ctx.write_state(w.x, w.u, w.om)
        with torch.cuda.stream(stream):
            uc = [f.clone() for f in fresh]
            fc = [torch.zeros_like(fresh[0]) for _ in range(3)]
        st = ctx.ibm_step(*uc, *fc, w.dt, 1.0, n_mdf_max=kmax, tol=tol, learned=learned)
        s = ctx.stats()
        passes, res = s.mdf_passes, s.residual

        def step():
            ctx.ibm_step(*uc, *fc, w.dt, 1.0, n_mdf_max=kmax, tol=tol, learned=learned)
            ctx.dem_step(dt_p, a.n_sub, **dem)
        ms = _time_steps(step, 2, stream, dev)
        out[name] = {"value": w.n_p / (ms / 1e3), "ms_per_step": ms, "tol": tol,
                     "n_mdf_max": kmax, "passes": passes, "residual": res,
                     "converged": st == B.PRS_OK}
        del uc, fc
    # the network kernel alone, on the tensor cores
    ctx.set_profiling(True)
    with torch.cuda.stream(stream):
        uc = [f.clone() for f in fresh]
        fc = [torch.zeros_like(fresh[0]) for _ in range(3)]
    for _ in range(3):
        ctx.ibm_step(*uc, *fc, w.dt, 1.0, learned=True)
    prof = ctx.read_profile()
    ctx.set_profiling(False)
    del uc, fc
    del fresh
    ms_mlp, cnt = prof["mlp"]
    if cnt:
        n_m = w.n_p * ctx.n_l
        flop = 2.0 * (9 * 64 + 64 * 64 + 64 * 3) * n_m
        ach = flop / (ms_mlp / cnt * 1e-3) / 1e12
        peak = load_bf16_peak()
        out["roofline_mlp"] = {"bound": "tensor", "kernel": "k_mlp_forward (warm start)",
                               "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                               "frac": ach / peak, "ms_per_launch": ms_mlp / cnt,
                               "flop_per_launch": flop,
                               "peak_source": "measured bf16_tflops (burst)"}
    torch.cuda.empty_cache()
    return out


def bed_variant(w, ctx):
    """Bed / flying classification and saltation tracking of the current
    state (Sec. 4.3.1): wall time per call, which includes the contact-pair
    search and the copy of the results to the host."""
    ctx.bed_detect()
    t0 = time.perf_counter()
    k = 3
    for _ in range(k):
        f = ctx.bed_detect()
    t1 = time.perf_counter()
    ctx.reset_saltation()
    ctx.track_saltation(0.0, w.R, 5 * w.T_c)
    t2 = time.perf_counter()
    for i in range(k):
        ctx.track_saltation(0.1 * (i + 1), w.R, 5 * w.T_c)
    t3 = time.perf_counter()
    return {"bed_detect_ms": 1000 * (t1 - t0) / k, "track_saltation_ms": 1000 * (t3 - t2) / k,
            "bed_spheres": int(f.sum()), "spheres": int(w.n_p)}


def fluid_variant(a, w, ctx, flds, frc, dt_p, dem, stream, dev):
    """The RK2 fluid sub-steps of Sec. 2.1 around the particle path, with the
    explicit viscous stand-in for H (prs_predict: H = nu lap_h u, no
    convection, no pressure): per fluid step two sub-steps of (predictor of
    u, v, w; direct forcing with alpha_k), then the n_sub DEM sub-steps. The
    predictor kernel is reported against the HBM roofline (16 B per grid point
    and component: u and H read, u_out and H written)."""
    import torch
    nu = 0.05 * w.h * w.h / w.dt          # dt nu / h^2 = 0.05, inside explicit stability
    with torch.cuda.stream(stream):
        nxt = [torch.empty_like(f) for f in flds]
        H = [torch.zeros_like(f) for f in flds]
    cur = list(flds)
    torch.cuda.synchronize(dev)

    def predict(al, be):
        for c in range(3):
            ctx.predict(c, cur[c], nxt[c], H[c], nu, w.dt, al, be)
    ms_pred = _time_steps(lambda: predict(0.5, 0.5), 5, stream, dev) / 3
    cells = w.n[0] * w.n[1] * w.n[2]
    byt = 4 * flds[0].element_size() * cells
    hbm, src = load_peaks()

    def rk2_step():
        nonlocal cur, nxt
        for al, be in ((1.0, 0.0), (0.5, 0.5)):
            for c in range(3):
                ctx.predict(c, cur[c], nxt[c], H[c], nu, w.dt, al, be)
            cur, nxt = nxt, cur
            ctx.ibm_step(*cur, *frc, w.dt, al)
        ctx.dem_step(dt_p, a.n_sub, **dem)
    ms_step = _time_steps(rk2_step, 2, stream, dev)
    del nxt, H
    return {"predictor": {"kernel": "k_predict", "ms_per_launch": ms_pred,
                          "alg_bytes_per_launch": byt,
                          "achieved_GBps": byt / (ms_pred * 1e-3) / 1e9, "peak": hbm,
                          "frac": byt / (ms_pred * 1e-3) / 1e9 / hbm,
                          "peak_source": f"{src} hbm_gbs"},
            "rk2_step": {"value": w.n_p / (ms_step * 1e-3), "unit": UNIT, "ms_per_step": ms_step,
                         "what": "2 x (predictor of u, v, w + prs_ibm_step with alpha_k) + "
                                 f"{a.n_sub} DEM sub-steps"}}


def fp64_variant(a, w, dt_p, dem, dev):
    """The plain FP64 form on the same bed and GPU."""
    import torch
    from paper_2108_01814_gb300 import binding as B
    s = torch.cuda.Stream(device=dev)
    c = B.Context(w.n, w.h, w.periodic, precision="fp64", device=dev, stream=s)
    c.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    c.write_state(w.x, w.u, w.om)
    with torch.cuda.stream(s):
        f64 = w.fluid_torch(torch.float64, dev)
        z64 = [torch.zeros_like(f64[0]) for _ in range(3)]
    s.synchronize()

    def step():
        c.ibm_step(*f64, *z64, w.dt, 1.0)
        c.dem_step(dt_p, a.n_sub, **dem)
    ms = _time_steps(step, 2, s, dev)
    c.set_profiling(True)
    step()
    prof = c.read_profile()
    c.close()
    del f64, z64
    torch.cuda.empty_cache()
    # the GPU's FP64 rate, for the FP64 form's arithmetic roofline: a cuBLAS
    # DGEMM (the best FP64 throughput a library reaches on this part)
    with torch.cuda.stream(s):
        A = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        B_ = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        torch.matmul(A, B_)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(3):
            torch.matmul(A, B_)
        e1.record(s)
    s.synchronize()
    dgemm = 3 * 2.0 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    del A, B_
    torch.cuda.empty_cache()
    return {"value": w.n_p / (ms / 1e3), "ms_per_step": ms, "dtype": "f64",
            "n_sub": a.n_sub,
            "phases_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "fp64_dgemm_tflops": dgemm}


def dem_only(a, w, ctx, prec, dev, stream, world, barrier):
    """The DEM sub-steps alone (prs_dem_step with n_sub sub-steps per step) on
    the workload's spheres, with no hydrodynamic load: one JSON line with the
    sub-step phases."""
    import torch
    dt_p = w.dt / a.n_sub
    dem = dict(e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
    for _ in range(a.warmup):
        ctx.dem_step(dt_p, a.n_sub, **dem)
    ctx.sync()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        ctx.dem_step(dt_p, a.n_sub, **dem)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, world, dev)
    ctx.set_profiling(True)
    kp = max(2, min(a.steps, 5))
    for _ in range(kp):
        ctx.dem_step(dt_p, a.n_sub, **dem)
    prof = ctx.read_profile()
    ctx.set_profiling(False)
    phases = {k: {"ms_per_step": t / kp, "launches_per_step": c / kp}
              for k, (t, c) in prof.items() if c}
    line = {"metric": "particle-steps/s (DEM sub-steps only, no fluid)",
            "value": world * w.n_p / (ms / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.n_p} spheres D={2 * w.R:g}h, DEM only "
                                   f"(F_h = T_h = 0), n_sub={a.n_sub}",
                       "parallelism": f"replicas x{world}"},
            "phases": phases}
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    return 0


def main_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2108_01814_gb300 import binding as B
    from paper_2108_01814_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    dev = torch.device("cuda", local)
    w = W.WORKLOADS[a.workload]()
    prec = a.precision
    tdt = torch.float32 if prec == "fp32" else torch.float64
    b = 4 if prec == "fp32" else 8
    stream = torch.cuda.Stream(device=dev)
    ctx = B.Context(w.n, w.h, w.periodic, precision=prec, device=dev, stream=stream)
    ctx.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    ctx.write_state(w.x, w.u, w.om)
    if a.dem_only:
        rc = dem_only(a, w, ctx, prec, dev, stream, world, barrier)
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return rc
    with torch.cuda.stream(stream):
        flds = w.fluid_torch(tdt, dev)
        frc = [torch.zeros_like(flds[0]) for _ in range(3)]
    stream.synchronize()
    dt_p = w.dt / a.n_sub
    dem = dict(e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)

    # |S|: cells reached by some marker stencil, counted on a zeroed copy
    with torch.cuda.stream(stream):
        uc = [f.clone() for f in flds]
        fc = [torch.zeros_like(flds[0]) for _ in range(3)]
    ctx.ibm_step(*uc, *fc, w.dt, 1.0)
    stream.synchronize()
    S = int((fc[0] != 0).sum().item())
    del uc, fc
    torch.cuda.empty_cache()

    def step(n_sub=a.n_sub):
        ctx.ibm_step(*flds, *frc, w.dt, 1.0)
        ctx.dem_step(dt_p, n_sub, **dem)

    for _ in range(a.warmup):
        step()
    ctx.sync()

    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    l0 = ctx.stats().n_launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    launches = ctx.stats().n_launches - l0
    ctx.sync()
    ms_max = max_over_ranks(ms, world, dev)
    value = world * w.n_p / (ms_max / 1000.0)

    # per-phase timing with events on the library's stream
    ctx.set_profiling(True)
    kp = max(2, min(a.steps, 5))
    for _ in range(kp):
        step()
    prof = ctx.read_profile()
    ctx.set_profiling(False)
    st = ctx.stats()
    hbm, peak_src = load_peaks()
    phases = {}
    for name, (tms, cnt) in prof.items():
        if cnt:
            per = tms / cnt
            byts = alg_bytes(name, b, S, w.n_p, st.n_contacts, st.n_wall_contacts)
            phases[name] = {"ms_per_step": tms / kp, "launches_per_step": cnt / kp,
                            "ms_per_launch": per, "alg_bytes_per_launch": byts,
                            "alg_GBps": byts / (per * 1e-3) / 1e9 if per > 0 else None}
    dom = max(phases, key=lambda k: phases[k]["ms_per_step"])
    dp = phases[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dp["alg_GBps"], "peak": hbm,
                "unit": "GB/s", "frac": (dp["alg_GBps"] or 0) / hbm,
                "traffic": TRAFFIC.get((w.name, prec, dom)) if a.n_sub == 50 else None,
                "peak_source": f"{peak_src} hbm_gbs"}
    isp = ["interp", "spread"]
    t_is = sum(phases[k]["ms_per_launch"] for k in isp if k in phases)
    by_is = alg_bytes("interp", b, S, w.n_p, 0, 0) + alg_bytes("spread", b, S, w.n_p, 0, 0)
    roof_is = {"bound": "hbm", "kernels": "interp+spread", "achieved": by_is / (t_is * 1e-3) / 1e9,
               "peak": hbm, "unit": "GB/s", "frac": by_is / (t_is * 1e-3) / 1e9 / hbm,
               "alg_bytes": by_is, "S_cells": S}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"{w.name}: grid {w.n[0]}x{w.n[1]}x{w.n[2]}, {w.n_p} spheres "
                               f"D={2 * w.R:g}h ({ctx.n_l} markers), {prec} grid/markers, "
                               f"FP64 state, n_mdf=1, n_sub={a.n_sub}",
                   "l2": "inputs larger than L2 (fluid fields "
                         f"{3 * b * w.n[0] * w.n[1] * w.n[2] / 1e9:.1f} GB), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "roofline_interp_spread": roof_is,
        "phases": phases,
        "gpu_launches": launches,
        "clocks": ck,
    }

    # variants on the same GPU: the IBM-dominated step (n_sub = 1)
    if not a.no_variants:
        want = set(a.variant) if a.variant else None
        line["variants"] = {}
        if want is None or "n_sub=1" in want:
            for _ in range(2):
                step(1)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(a.steps):
                step(1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            line["variants"]["n_sub=1"] = {
                "value": w.n_p / (e0.elapsed_time(e1) / a.steps / 1e3),
                "ms_per_step": e0.elapsed_time(e1) / a.steps}
        if want is None or "delta4" in want:
            # Peskin's 4-point kernel for the IBM step (per-marker kernels,
            # 64-bit fixed-point scratch grid), the same DEM sub-steps
            def step4():
                ctx.ibm_step(*flds, *frc, w.dt, 1.0, delta_kernel=4)
                ctx.dem_step(dt_p, a.n_sub, **dem)
            ms4 = _time_steps(step4, max(2, min(a.steps, 5)), stream, dev)
            line["variants"]["delta4"] = {"value": w.n_p / (ms4 / 1e3), "ms_per_step": ms4}
        if want is None or "forcing" in want:
            line["variants"].update(forcing_variants(a, w, ctx, flds, dt_p, dem, stream, dev))
        if prec == "fp32" and (want is None or "fp64" in want):
            line["variants"]["fp64"] = fp64_variant(a, w, dt_p, dem, dev)
        if want is None or "bed_and_saltation" in want:
            line["variants"]["bed_and_saltation"] = bed_variant(w, ctx)
        if want is None or "rk2_fluid_standin" in want:
            line["variants"]["rk2_fluid_standin"] = fluid_variant(a, w, ctx, flds, frc, dt_p,
                                                                  dem, stream, dev)

    # end to end through the C ABI with host (pinned) grid buffers
    if not a.no_e2e:
        npdt = np.float32 if prec == "fp32" else np.float64
        host = []
        for f in flds + frc:
            hp = torch.empty(f.shape, dtype=tdt, pin_memory=True)
            hp.copy_(f)
            host.append(hp.numpy())
        # the step's results land in pinned host arrays too
        def pinned(shape):
            return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        xs = pinned((3, w.n_p))
        forces = [pinned((3, w.n_p)) for _ in range(4)]
        k2 = max(2, min(5, a.steps))

        def step_e2e():
            # the fields' copies out finish while the DEM sub-steps run; the
            # state read below waits for them
            ctx.ibm_step(*host, w.dt, 1.0, host_async=True)
            ctx.dem_step(dt_p, a.n_sub, **dem)
            ctx.lib.prs_read_state(ctx.ctx, xs.ctypes.data_as(B._vp), None, None, B.PRS_HOST)
            return ctx.read_forces(out=forces)

        step_e2e()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            step_e2e()
        t1 = time.perf_counter()
        barrier()
        # bytes of the last step: the library copies only the z-slab of the
        # host fields that the markers can reach, plus the state and forces read
        st = ctx.stats()
        sec = max_over_ranks(t1 - t0, world, dev)
        line["e2e"] = {"value": world * w.n_p * k2 / sec, "unit": UNIT,
                       "h2d_bytes_per_step": st.h2d_bytes,
                       "d2h_bytes_per_step": st.d2h_bytes + 24 * w.n_p + 4 * 24 * w.n_p,
                       "ms_per_step": 1000 * sec / k2,
                       "note": "pinned host fields, only the z-slab the stencils reach is "
                               "copied, by z-chunks in and out at once, overlapped with the "
                               "kernels; results read into pinned arrays"}
        del host, xs, forces

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, a.n_sub)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return main_reference(a)
    return main_ours(a)


if __name__ == "__main__":
    sys.exit(main())
