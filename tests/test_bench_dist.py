"""The N > 1 bench path on CPU: two gloo ranks (replicas) reduce to the slowest
rank's time and the sum of the flips."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, lr, pg = bench.dist_setup()
    assert (ws, r, lr) == (world, rank, rank)
    secs, flips = bench.aggregate(pg, 1.0 + rank, 1000.0 * (rank + 1))
    out[rank] = (secs, flips)
    pg.barrier()
    pg.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == out[1] == (2.0, 3000.0)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(None, 1.5, 42) == (1.5, 42)
