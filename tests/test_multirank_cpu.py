"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would start
them (one process per GPU on a GPU machine).  The data path has no exchange:
each rank simulates its own batch; the only collective is the max over
ranks of the step time."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    slowest = bench.max_over_ranks(1.5 + rank, world, "cpu")
    w = bench.rank_workload(rank, 4)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, w["mesh"].theta.tolist(), w["mesh"].data.tolist(), list(w["c"][:8]), w["s"]))


def test_two_gloo_ranks_max_time_and_disjoint_batches():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time
    assert res[0][1] == res[1][1] == 2.5
    # same layer (input state, shapes), different seeded batches per rank
    assert res[0][5] == res[1][5]
    t0, t1 = np.array(res[0][2]), np.array(res[1][2])
    d0, d1 = np.array(res[0][3]), np.array(res[1][3])
    assert t0.shape == t1.shape and d0.shape == d1.shape
    assert not np.allclose(t0, t1) and not np.allclose(d0, d1)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--gpus", "2"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    w = bench.rank_workload(0, 2)
    assert w["mesh"].data.shape == (2, 16)
    json.dumps(w["s"])
