"""bench.py's multi-GPU mode runs independent replicas (one problem per rank): the only host
logic across ranks is the max of the per-rank step times and the sum of the per-rank DOF counts.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.25][rank]
    dof = [1000.0, 3000.0][rank]
    q.put((rank, bench.max_over_ranks(ms, world), bench.sum_over_ranks(dof, world),
           bench.dist_env()))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, tot, env in res:
        assert mx == 20.25 and tot == 4000.0
        assert env[0] == rank and env[1] == 2
