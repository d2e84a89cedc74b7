"""The multi-GPU path of bench.py is replicas only: each rank fixes its own configuration (generator seed
offset by the rank) and the only collective is the whole-job timing reduction (slowest rank's time,
summed site-iterations). These tests run that path on the CPU with gloo, world size 2."""
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t, w = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1), ws, "cpu")
    q.put((rank, t, w, bench.replica_seed(4, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w, seed in res:
        assert t == 11.0 and w == 300.0  # max of the times, sum of the work, on every rank
    assert [r[3] for r in res] == [4, 5]


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 1000, 1, "cpu") == (12.5, 1000)


def test_replicas_are_distinct_configurations():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    dims = (4, 4, 4, 4)
    U0 = synth.config(dims, bench.replica_seed(4, 0), 0.6)
    U1 = synth.config(dims, bench.replica_seed(4, 1), 0.6)
    assert not np.allclose(U0, U1)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
