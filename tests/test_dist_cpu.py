"""The multi-process paths of bench.py on the CPU (gloo, world size 2, 127.0.0.1).

The estimator runs as independent replicas, one per GPU, with no collective on the data path;
the only cross-rank step is the timing's max over ranks. These tests run that reduction over a
gloo process group, and the reference arm under torchrun (rank 0 alone prints its line).
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, local = bench.dist_setup()
        q.put((r, w, local, bench.max_over_ranks(10.0 + 3.0 * rank, w, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 13.0), (1, 2, 1, 13.0)]


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.5, 1, "cpu") == 4.5


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched like the N = 2 run: rank 0 times the oracle on the host
    cores and prints one JSON line; rank 1 exits 0 without work."""
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
