"""The multi-GPU path of bench.py, exercised on CPU with two gloo ranks.

With N GPUs every rank filters its own shard of the same size (weak
scaling): the only collectives are the barriers around the timed region and
the max-over-ranks reduction of its duration.  These tests check the shard
seeds, the reduction and the whole-job rate across two real processes, and
the launch contract of the reference arm under torchrun (rank 0 prints one
line, the other ranks exit 0 without work)."""
import hashlib
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.make_workload(0.0005, rank)
        digest = hashlib.sha256(w.reads.tobytes() + w.pair_read.tobytes() + w.pair_off.tobytes()).hexdigest()
        dist.barrier()
        slowest = bench.reduce_max(5.0 + 3.0 * rank, world, "cpu")
        rate = bench.whole_job_rate(w.n_pairs * len(bench.E_SWEEP), world, 4, slowest)
        got = [None] * world
        dist.all_gather_object(got, (digest, w.n_pairs, w.n_reads, slowest, rate))
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shards_and_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0] == results[1]  # every rank saw the same gathered view
    (d0, n0, r0, t0, v0), (d1, n1, r1, t1, v1) = results[0]
    assert d0 != d1, "the two ranks must filter different shards"
    assert (n0, r0) == (n1, r1) == (10_000, 2_500)  # same shard size: weak scaling
    assert t0 == t1 == 8.0  # the slower rank's time
    assert v0 == v1 == pytest.approx(10_000 * 11 * 2 * 4 / 8e-3 / 1e9)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--scale", "0.002"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env={**os.environ, "OMP_NUM_THREADS": "4"})
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
