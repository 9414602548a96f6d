"""A solve split by island on the GPU library: two (and four) ranks, each a
context that runs only its islands' searches (dabs_set_search_slots), driven
from one process with an in-process exchange (no collective and no kernel
waiting on another), give after every generation the pools, results and
global best of the same solve in one context, and the oracle's."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import islands, workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03069_gb300 import build, dabs
    build.build()
    return dabs


@pytest.mark.parametrize("ranks,seed_mode", [(2, 0), (4, 1), (3, 0)])
def test_island_split_equals_one_context(D, orc, ranks, seed_mode):
    n = 300
    W = wl.dense_qubo(n, -1000, 1000, seed=31)
    kw = dict(searches=96, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), seed_mode=seed_mode)
    whole = D.Context(W, **kw)
    whole.solve_begin(17)
    runs = []
    for r in range(ranks):
        lo, hi = islands.island_range(4, ranks, r)
        runs.append(islands.IslandSolve(islands.ContextEngine(D.Context(W, **kw), lo, hi), r, ranks,
                                        gather=None))
    for run in runs:
        run.begin(17)
    so = orc.Solver(W, orc.make_params(**kw), 17)
    for g in range(4):
        parts = [run.search_part() for run in runs]
        assert sum(len(p[1]) for p in parts) == kw["searches"]
        for run in runs:
            run.merge_part(parts)
        whole.solve_generations(1)
        so.generation(8)
        want = whole.read_pools()
        wantg = whole.read_generation()
        for run in runs:
            for x, y in zip(run.engine.ctx.read_pools(), want):
                assert np.array_equal(x, y), (g, run.rank)
            for x, y in zip(run.engine.ctx.read_generation()[3:], wantg[3:]):
                assert np.array_equal(x, y), (g, run.rank)
            assert run.engine.status() == whole.solve_status()
        oX, oE, oa, oo = so.pools()
        X, E, a, o = want
        assert np.array_equal(E, oE) and np.array_equal(wl.unpack_bits(X, n), oX)
    bx, be = runs[0].engine.best()
    ox, oe, of, og = so.best()
    assert be == oe and np.array_equal(bx, ox)
    for run in runs:
        run.engine.close()
