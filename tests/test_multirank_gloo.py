"""The multi-rank host logic on CPU, as two gloo ranks (127.0.0.1): the
benchmark's whole-job timing reduction (slowest rank's time, every rank's
work) and the placement of independent lines on ranks (a partition of the
lines that every rank computes alike, balanced by particle count)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        import bench
        from paper_2609_17661_b300.shard import my_lines
        from paper_2609_17661_b300 import workloads as W
        # timing: rank r took (3 + 2r) ms for (10 + 5r) units
        ms, units = bench.reduce_over_ranks(3.0 + 2.0 * rank, 10.0 + 5.0 * rank, world, "cpu")
        # placement of the 256-line workload by particle count
        _, counts = W.ensemble_configs()
        mine = my_lines(counts, rank, world)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        q.put((rank, ms, units, shards, int(counts[mine].sum()), int(counts.sum()), int(counts.max())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ms, units, shards, load, total, biggest in res:
        assert ms == 5.0 and units == 25.0                     # max of 3, 5; sum of 10, 15
        assert shards == res[0][3]                             # every rank places alike
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(256))                        # a partition of the lines
    loads = [r[4] for r in res]
    assert sum(loads) == res[0][5]
    assert max(loads) - min(loads) <= res[0][6]               # balanced to within one line


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2609_17661_b300.shard import shard_lines
    assert bench.reduce_over_ranks(4.5, 7, 1, "cpu") == (4.5, 7.0)
    assert shard_lines([3, 1, 2], 1) == [[0, 1, 2]]
    assert shard_lines([5, 4, 3, 3], 2) == [[0, 3], [1, 2]]
    assert shard_lines([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard_lines([1.0], 0)


def test_reference_arm_under_torchrun_prints_one_line(tmp_path):
    """`bench.py --impl reference` launched as two ranks: rank 0 alone times
    the oracle and prints one JSON line, the other rank exits 0 without work."""
    import json
    import subprocess
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--ref-sample", "20000"]
    env = dict(os.environ, TMPDIR=str(tmp_path))          # torchrun's scratch stays in the test's directory
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["e2e"]["h2d_bytes_per_step"] == 0
