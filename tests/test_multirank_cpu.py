"""Multi-rank host logic on CPU (gloo, world size 2): channel sharding covers every channel
exactly once, the per-rank results reassemble into the single-process result, and the
whole-job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

from paper_2005_09481_gb300 import shard

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n_chan,world", [(1, 1), (7, 2), (16, 4), (3, 8), (1024, 8)])
def test_shards_cover_each_channel_once(n_chan, world):
    seen = []
    for r in range(world):
        mine = shard.channels_for_rank(n_chan, r, world)
        assert all(shard.owner_of(c, n_chan, world) == r for c in mine)
        seen += mine
    assert sorted(seen) == list(range(n_chan))
    sizes = [len(shard.channels_for_rank(n_chan, r, world)) for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_2005_09481_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, T, C = 24, 40, 5
    packed = synth.uniform(N, T, C, seed=77)
    mine = shard.channels_for_rank(C, rank, world)
    part = {c: oracle.correlate(packed[c], N, T, 1)[0] for c in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, part)
    slow = shard.slowest(0.5 + rank, None)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        full = oracle.correlate(packed, N, T, C)
        ok = sorted(merged) == list(range(C)) and all(np.array_equal(merged[c], full[c]) for c in range(C))
        q.put((ok, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharded_correlation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok, slow = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok
    assert slow == 1.5


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    # The oracle arm launched like the driver's N > 1 runs: rank 0 alone times the oracle on
    # every host core it may use (the launcher sets OMP_NUM_THREADS=1) and prints one JSON
    # line; the other rank exits 0 without work.
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"]["h2d_bytes_per_step"] == 0
