"""The benchmark's host side without a GPU: the CPU baseline (the FP64
oracle on one thread and on all host cores) and the reference arm's JSON
line, on the tiny box."""
import json
import os
import subprocess
import sys

import bench
from paper_2108_01814_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_baseline_records_cores():
    cb = bench.cpu_baseline(W.tiny(), 2, target=128, steps=1)
    avail, nproc = bench.host_cores()
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT
    assert cb["value"] > 0 and cb["single_thread"]["value"] > 0
    assert 1 <= cb["cores"] <= avail <= nproc == cb["nproc"]
    assert cb["single_thread"]["cores"] == 1
    assert f"{cb['cores']} threads" in cb["sample"]


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny",
                          "--steps", "1", "--warmup", "0", "--n-sub", "2"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def _ranks_max(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a slower rank 1: the job's time is its time, on every rank
        q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_ranks_max, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == {0: 15.0, 1: 15.0}
    assert bench.max_over_ranks(7.5, 1) == 7.5  # one rank: no collective


def test_reference_arm_other_ranks_do_nothing():
    # under torchrun the reference arm runs on rank 0 only; the others exit
    # 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "0", "--n-sub", "2", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
