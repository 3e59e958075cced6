"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks run independent
replicas (the problem does not shard: no data-path collective); the barrier
and the max-over-ranks time are the only collectives, and the whole-job value
is the units all ranks processed over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms_local = 10.0 * (rank + 1)                 # rank 1 is the slow one
    value, ms = bench.replica_value(world, 1000.0, ms_local)
    out[rank] = (value, ms)
    bench.barrier(world)
    dist.destroy_process_group()


def test_replicas_max_over_ranks_and_value():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # every rank sees the slowest time; value = 2 ranks x 1000 units / 20 ms
    for r in range(world):
        value, ms = out[r]
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1000.0 / 0.020)
