"""A solve split by island over ranks (Section IV-B) on CPU: two and three gloo
ranks, each running the batch searches of its own islands with the oracle as
its engine, exchange their results every generation and end with the pools,
global best and statistics of the same solve on one device.  Also the island
partition itself."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2207_03069_gb300 import islands, workloads as wl


def test_island_partition_covers_every_search_once():
    for P in (1, 2, 3, 4, 7, 12):
        for R in range(1, P + 1):
            ranges = [islands.island_range(P, R, r) for r in range(R)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert all(hi > lo for lo, hi in ranges)
            for S in (1, P, 3 * P + 1, 64):
                parts = [islands.search_slots(S, P, lo, hi) for lo, hi in ranges]
                allp = np.sort(np.concatenate(parts))
                assert np.array_equal(allp, np.arange(S))
                for (lo, hi), part in zip(ranges, parts):
                    assert ((part % P >= lo) & (part % P < hi)).all()
    with pytest.raises(ValueError):
        islands.island_range(2, 3, 0)


class OracleEngine:
    """The stages of a generation run by the oracle (test infrastructure),
    searches restricted to one rank's islands."""

    def __init__(self, W, params, lo, hi):
        from oracle import oracle as orc
        self.orc, self.W, self.params = orc, W, params
        self.S, self.P, self.n = params.searches, params.pools, W.shape[0]
        self.lo, self.hi = lo, hi

    def begin(self, seed, budget, target):
        self.seed, self.budget = seed, budget
        self.target = -(2**63) if target is None else target
        self.so = self.orc.Solver(self.W, self.params, seed)
        self.X, self.d, self.E = self.so.state()
        self.g, self.flips, self.done = 0, 0, False
        self.bX = np.zeros((self.S, self.n), np.uint8)
        self.bE = np.zeros(self.S, np.int64)
        self.f = np.zeros(self.S, np.uint32)

    def search(self):
        self.D, self.a, self.o = self.so.offspring(self.g)
        for s in islands.search_slots(self.S, self.P, self.lo, self.hi):
            r = self.orc.batch_search(self.W, self.params, self.seed, self.g, int(s), self.X[s],
                                      self.d[s], int(self.E[s]), self.D[s], int(self.a[s]))
            self.X[s], self.d[s], self.E[s] = r["X"], r["delta"], r["E"]
            self.bX[s], self.bE[s], self.f[s] = r["best_X"], r["best_E"], r["flips"]

    def results(self):
        return self.bX, self.bE, self.f, self.a, self.o

    def merge(self, bX, bE, f, a, o):
        self.so.merge(bX, bE, a, o)
        self.flips += int(f.sum())
        self.g += 1
        best = self.so.best()[1]
        self.done = self.flips >= self.budget or best <= self.target

    def status(self):
        return dict(done=self.done, flips=self.flips, generations=self.g, best_E=self.so.best()[1])

    def best(self):
        X, E, _, _ = self.so.best()
        return X, E


KW = dict(searches=14, pools=4, pool_cap=6, tabu=8, s=(1, 10), b=(2, 1), seed_mode=0)
GENS = 5


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
    import torch.distributed as dist
    from oracle import oracle as orc
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    W = wl.dense_qubo(40, -50, 50, seed=8)
    p = orc.make_params(**KW)
    lo, hi = islands.island_range(p.pools, world, rank)
    eng = OracleEngine(W, p, lo, hi)
    run = islands.IslandSolve(eng, rank, world, islands.torch_gather())
    run.begin(seed=21)
    for _ in range(GENS):
        run.generation()
    X, E = eng.best()
    pX, pE, pa, po = eng.so.pools()
    out[rank] = (X.tobytes(), E, eng.flips, pX.tobytes(), pE.tobytes(), pa.tobytes(),
                 po.tobytes(), [x.tobytes() for x in eng.so.stats()])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_island_split_equals_the_whole_solve(orc, world):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        got = [out[r] for r in range(world)]
    W = wl.dense_qubo(40, -50, 50, seed=8)
    so = orc.Solver(W, orc.make_params(**KW), 21)
    for _ in range(GENS):
        so.generation()
    X, E, flips, _ = so.best()
    pX, pE, pa, po = so.pools()
    want = (X.tobytes(), E, flips, pX.tobytes(), pE.tobytes(), pa.tobytes(), po.tobytes(),
            [x.tobytes() for x in so.stats()])
    for r in range(world):
        assert got[r] == want, f"rank {r}"
