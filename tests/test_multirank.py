"""bench.py's multi-GPU bookkeeping on CPU: world_size-2 gloo ranks agree on
the slowest rank's time and the sum of the work (the data path shards by
process image with no exchange step: replicas only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, moved, recs = bench.across_ranks(100.0 + 50 * rank, 1000 * (rank + 1), 7 + rank, world)
    dist.barrier()
    out[rank] = (ms, moved, recs)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_max_and_work_sum():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (150.0, 3000, 15)


def test_single_rank_is_identity():
    import bench
    assert bench.across_ranks(12.5, 9, 4, 1) == (12.5, 9, 4)
