"""GPU parity on the five measured workloads, against the oracle element by
element (all work is integer, so equality is exact):

1. dense n = 64, W ~ U[-100, 100] (seed 0), 32 searches, 4 pools x 64, b = 1,
   s = 1/10, Straight seeding: all 200 generations;
2. sparse Max-Cut G(800, 0.06), w = +-1 (seed 1), 1024 searches, 4 x 100,
   b = 10: whole generations, so the searches' persistent X (Section III-B)
   and pool-bred targets are compared, not only generation 0;
3. TSP one-hot, 32 cities (1024 bits, seed 2, Section II-B), 2048 searches,
   b = 1: whole generations;
4. one instance of the batched workload at n = 4096 (dense, U[-1000, 1000]),
   256 searches, recompute seeding on the tensor cores: one generation, 16
   sampled searches re-run by the oracle;
5. the served workload's n = 16384 instance (512 MB of int16 W): one
   generation, sampled searches re-run by the oracle.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl

from test_gpu_parity import compare_generation

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03069_gb300 import build, dabs
    build.build()
    return dabs


def whole_generations(D, orc, W, kw, seed, gens, every=1):
    n = W.shape[0]
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), seed)
    ctx.solve_begin(seed)
    for g in range(gens):
        ctx.solve_generations(1)
        so.generation(THREADS)
        if (g + 1) % every == 0 or g + 1 == gens:
            compare_generation(ctx, so, n, f"generation {g}")
    st = ctx.solve_status()
    bx, be, bf, bg = so.best()
    assert (st["best_E"], st["flips"], st["generations"]) == (be, bf, bg)
    gx, ge = ctx.solve_best()
    assert ge == be and np.array_equal(gx, bx)
    for got, want in zip(ctx.stats(), so.stats()):
        assert np.array_equal(got, want)
    ctx.close()
    return be, bf


def test_config1_dense64_all_200_generations(D, orc):
    W = wl.dense_qubo(64, -100, 100, seed=0)
    kw = dict(searches=32, pools=4, pool_cap=64, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0)
    be, bf = whole_generations(D, orc, W, kw, seed=0, gens=200)
    assert bf >= 200 * 32 * 64  # at least b n flips per search and generation


def test_config1_twin_reaches_the_brute_force_optimum(D, orc):
    W = wl.dense_qubo(20, -100, 100, seed=0)
    opt = wl.brute_force_min(W)[0]
    kw = dict(searches=32, pools=4, pool_cap=64, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0,
              max_generations=200)
    ctx = D.Context(W, **kw)
    X, E, F = ctx.solve(10**12, seed=0, target=opt)
    ox, oe, of, og = orc.solve(W, orc.make_params(**kw), 10**12, 0, target=opt, threads=THREADS)
    assert E == oe == opt and F == of and np.array_equal(X, ox)
    ctx.close()


def test_config2_maxcut800_whole_generations(D, orc):
    W = wl.maxcut_qubo(800, 0.06, seed=1)
    kw = dict(searches=1024, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(10, 1), seed_mode=0)
    whole_generations(D, orc, W, kw, seed=1, gens=4)


def test_config3_tsp1024_whole_generations(D, orc):
    W, dist, p = wl.tsp_qubo(32, 1000, seed=2)
    assert W.shape == (1024, 1024)
    kw = dict(searches=2048, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0)
    whole_generations(D, orc, W, kw, seed=2, gens=3)


def sampled_generation(D, orc, W, kw, seed, samples, rng_seed=0):
    """One generation from the start on the GPU; the oracle breeds every
    target and re-runs `samples` searches from X = 0."""
    n = W.shape[0]
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), seed)
    ctx.solve_begin(seed)
    ctx.solve_generations(1)
    Dg, ag, og, bX, bE, fl = ctx.read_generation()
    sX, sd, sE = ctx.read_state()
    oD, oa, oo = so.offspring(0)
    assert np.array_equal(wl.unpack_bits(Dg, n), oD)
    assert np.array_equal(ag, oa) and np.array_equal(og, oo)
    p = orc.make_params(**kw)
    z = np.zeros(n, np.uint8)
    d0 = np.diag(W).astype(np.int32)
    S = kw["searches"]
    # every algorithm among the samples
    picks = []
    for a in range(5):
        idx = np.nonzero(oa == a)[0]
        if idx.size:
            picks.append(int(idx[0]))
    rest = np.random.default_rng(rng_seed).choice(S, samples, replace=False)
    picks = sorted(set(picks) | set(int(s) for s in rest))

    def one(s):
        return s, orc.batch_search(W, p, seed, 0, s, z, d0, 0, oD[s], int(oa[s]))

    gb = wl.unpack_bits(bX, n)
    gX = wl.unpack_bits(sX, n)
    with ThreadPoolExecutor(max_workers=min(THREADS, len(picks))) as ex:
        for s, r in ex.map(one, picks):
            tag = f"n={n} search={s} algo={oa[s]}"
            assert int(fl[s]) == r["flips"], tag
            assert int(bE[s]) == r["best_E"], tag
            assert np.array_equal(gb[s], r["best_X"]), tag
            assert np.array_equal(gX[s], r["X"]), tag
            assert int(sE[s]) == r["E"], tag
            assert np.array_equal(sd[s], r["delta"]), tag
    ctx.close()
    return picks


def test_config4_instance_n4096_recompute_seeding(D, orc):
    n = 4096
    W = wl.dense_qubo(n, -1000, 1000, seed=1000 + 17)
    kw = dict(searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1)
    picks = sampled_generation(D, orc, W, kw, seed=17, samples=16)
    assert len(picks) >= 16


def test_config5_instance_n16384_sampled(D, orc):
    n = 16384
    W = wl.dense_qubo(n, -1000, 1000, seed=9999)
    kw = dict(searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1)
    sampled_generation(D, orc, W, kw, seed=9999, samples=6)
