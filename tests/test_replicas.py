"""Replica (image-parallel) host logic with two gloo ranks on CPU: disjoint
shards that cover the job, barriers, and the max-over-ranks timing that
bench.py reports.  No GPU is involved."""
import os
import socket
import subprocess
import sys

import pytest

from paper_1904_09409_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_1904_09409_gb300 import replicas as r
    ws, rk, _ = r.env_world()
    r.init("gloo")
    idx = r.shard(rk, ws, 4)
    r.barrier()
    slowest = r.max_over_ranks(0.5 + rk)          # rank 1 is the slower one
    q.put((rk, list(idx), slowest))
    r.finish()


def test_shards_are_disjoint_and_cover():
    world, per = 4, 64
    seen = []
    for rk in range(world):
        seen += list(replicas.shard(rk, world, per))
    assert sorted(seen) == list(range(world * per))
    with pytest.raises(ValueError):
        replicas.shard(4, 4, 8)


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == [0, 1, 2, 3] and out[1][1] == [4, 5, 6, 7]
    assert out[0][2] == out[1][2] == 1.5


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
