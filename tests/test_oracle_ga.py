"""Pins of the oracle's genetic layer (Section IV): operation statistics,
5%/95% adaptive choice, island neighbour for Xrossover, pool insertion as
top-C of the union without duplicates, determinism, and solution quality
against brute force on the n = 20 twin of the small dense workload."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl


def fixed_pools(orc, n, P, C, algo=3, op=None, xs=None):
    X = np.zeros((P, C, n), np.uint8)
    for p in range(P):
        X[p, :, :] = xs[p] if xs is not None else 0
    E = np.tile(np.arange(C, dtype=np.int64), (P, 1))
    a = np.full((P, C), algo, np.int32)
    o = np.full((P, C), 0 if op is None else op, np.int32)
    return X, E, a, o


def offspring_stats(orc, n, op, xs, gens=40, S=64, P=2):
    W = wl.dense_qubo(n, -5, 5, 1)
    so = orc.Solver(W, orc.make_params(searches=S, pools=P, pool_cap=16), seed=99)
    so.set_pools(*fixed_pools(orc, n, P, 16, op=op, xs=xs))
    out = []
    for g in range(gens):
        D, a, o = so.offspring(g)
        keep = o == op
        out.append((D[keep], np.arange(S)[keep] % P, a[keep]))
    return out


def test_mutation_zero_one_rates(orc):
    n = 256
    rng = np.random.default_rng(3)
    xs = [rng.integers(0, 2, n).astype(np.uint8) for _ in range(2)]
    for op, name in ((0, "mut"), (3, "zero"), (4, "one")):
        changed, base = 0, 0
        for D, pool, _ in offspring_stats(orc, n, op, xs):
            for d, p in zip(D, pool):
                x = xs[p]
                if name == "mut":
                    changed += int((d != x).sum()); base += n
                elif name == "zero":
                    assert not ((x == 0) & (d == 1)).any()
                    changed += int(((x == 1) & (d == 0)).sum()); base += int((x == 1).sum())
                else:
                    assert not ((x == 1) & (d == 0)).any()
                    changed += int(((x == 0) & (d == 1)).sum()); base += int((x == 0).sum())
        rate = changed / base
        assert abs(rate - 1 / 8) < 0.01, (name, rate)


def test_crossover_xrossover_best_random_intervalzero(orc):
    n = 200
    rng = np.random.default_rng(4)
    xs = [rng.integers(0, 2, n).astype(np.uint8) for _ in range(2)]
    # Crossover within one pool of identical vectors reproduces the vector
    for D, pool, _ in offspring_stats(orc, n, 1, xs):
        for d, p in zip(D, pool):
            assert np.array_equal(d, xs[p])
    # Xrossover mixes own pool p with pool (p+1) mod P about half/half
    frac = []
    for D, pool, _ in offspring_stats(orc, n, 2, xs):
        for d, p in zip(D, pool):
            a, b = xs[p], xs[(p + 1) % 2]
            diff = a != b
            assert np.all((d == a) | (d == b))
            frac.append((d[diff] == b[diff]).mean())
    assert abs(np.mean(frac) - 0.5) < 0.03
    for D, pool, _ in offspring_stats(orc, n, 6, xs):  # Best
        for d, p in zip(D, pool):
            assert np.array_equal(d, xs[p])
    ones = [d.mean() for D, _, _ in offspring_stats(orc, n, 7, xs) for d in D]  # Random
    assert abs(np.mean(ones) - 0.5) < 0.02
    ones_x = [np.ones(n, np.uint8), np.ones(n, np.uint8)]
    for D, pool, _ in offspring_stats(orc, n, 5, ones_x):  # IntervalZero
        for d in D:
            z = np.nonzero(d == 0)[0]
            assert 32 <= len(z) <= n // 2
            # one cyclic segment: at most one 1->0 boundary going around
            edges = int(((d == 1) & (np.roll(d, -1) == 0)).sum())
            assert edges == 1


def test_best_takes_the_first_pool_entry(orc):
    n, S, P, C = 40, 32, 2, 8
    W = wl.dense_qubo(n, -5, 5, 1)
    rng = np.random.default_rng(12)
    so = orc.Solver(W, orc.make_params(searches=S, pools=P, pool_cap=C), seed=7)
    pX = rng.integers(0, 2, (P, C, n)).astype(np.uint8)
    so.set_pools(pX, np.tile(np.arange(C, dtype=np.int64), (P, 1)),
                 np.zeros((P, C), np.int32), np.full((P, C), 6, np.int32))
    hits = 0
    for g in range(10):
        D, _, o = so.offspring(g)
        for s in np.nonzero(o == 6)[0]:
            assert np.array_equal(D[s], pX[s % P, 0])
            hits += 1
    assert hits > 100


def test_adaptive_choice_five_percent(orc):
    n, S = 64, 256
    W = wl.dense_qubo(n, -5, 5, 1)
    so = orc.Solver(W, orc.make_params(searches=S, pools=4, pool_cap=16), seed=5)
    so.set_pools(*fixed_pools(orc, n, 4, 16, algo=3, op=5))
    oth_a = oth_o = tot = 0
    for g in range(60):
        _, a, o = so.offspring(g)
        oth_a += int((a != 3).sum())
        oth_o += int((o != 5).sum())
        tot += S
    # 5% uniform choice lands on another value with probability 4/5 resp. 7/8
    assert abs(oth_a / tot - 0.05 * 4 / 5) < 0.006
    assert abs(oth_o / tot - 0.05 * 7 / 8) < 0.006


def reference_merge(pX, pE, pa, po, rX, rE, ra, ro, P):
    """Top-C of (pool entries, then results in search order) by energy,
    earlier first on ties, dropping a later copy of an equal (E, X)."""
    P_, C, n = pX.shape
    out = []
    for p in range(P):
        items = [(pE[p, k], 0, k, pX[p, k], pa[p, k], po[p, k]) for k in range(C)]
        items += [(rE[s], 1, s, rX[s], ra[s], ro[s]) for s in range(len(rE)) if s % P == p]
        seen, uniq = set(), []
        for it in items:
            key = (int(it[0]), it[3].tobytes())
            if key in seen:
                continue
            seen.add(key)
            uniq.append(it)
        uniq.sort(key=lambda it: (it[0], it[1], it[2]))
        out.append(uniq[:C])
    return out


def test_pool_merge_is_top_c_of_union(orc):
    n, S, P, C = 16, 48, 3, 8
    W = wl.dense_qubo(n, -5, 5, 1)
    rng = np.random.default_rng(8)
    so = orc.Solver(W, orc.make_params(searches=S, pools=P, pool_cap=C), seed=1)
    pX = rng.integers(0, 2, (P, C, n)).astype(np.uint8)
    pE = np.sort(rng.integers(-20, 20, (P, C)), axis=1).astype(np.int64)
    pa = rng.integers(0, 5, (P, C)).astype(np.int32)
    po = rng.integers(0, 8, (P, C)).astype(np.int32)
    pE[2, 0] = -90
    so.set_pools(pX, pE, pa, po)
    rX = rng.integers(0, 2, (S, n)).astype(np.uint8)
    rE = rng.integers(-25, 25, S).astype(np.int64)
    rX[5] = pX[2, 0]; rE[5] = -90                         # duplicate of a pool entry
    rE[4] = -100
    rX[7] = rX[4]; rE[7] = rE[4]; rX[10] = rX[4]; rE[10] = rE[4]  # duplicate results
    rE[13] = -100                                          # equal energy, other vector
    ra = rng.integers(0, 5, S).astype(np.int32)
    ro = rng.integers(0, 8, S).astype(np.int32)
    so.merge(rX, rE, ra, ro)
    X, E, a, o = so.pools()
    ref = reference_merge(pX, pE, pa, po, rX, rE, ra, ro, P)
    for p in range(P):
        assert list(E[p]) == [int(it[0]) for it in ref[p]]
        for k, it in enumerate(ref[p]):
            assert np.array_equal(X[p, k], it[3]) and a[p, k] == it[4] and o[p, k] == it[5]


def test_pool_init_random_with_infinite_energy(orc):
    n = 300
    W = wl.dense_qubo(n, -5, 5, 1)
    so = orc.Solver(W, orc.make_params(searches=8, pools=4, pool_cap=32), seed=3)
    X, E, a, o = so.pools()
    assert (E == orc.INT64_MAX).all()
    assert abs(X.mean() - 0.5) < 0.01
    assert set(np.unique(a)) == set(range(5)) and set(np.unique(o)) == set(range(8))


def test_solver_threads_do_not_change_results(orc):
    W = wl.dense_qubo(64, -100, 100, 0)
    p = orc.make_params(searches=32, pools=4, pool_cap=64, max_generations=6)
    r1 = orc.solve(W, p, budget=2**63, seed=1, threads=1)
    r4 = orc.solve(W, p, budget=2**63, seed=1, threads=4)
    assert r1[1] == r4[1] and r1[2] == r4[2] and np.array_equal(r1[0], r4[0])
    assert r1[1] == orc.energy(W, r1[0])


def test_solver_reaches_brute_force_optimum_n20(orc):
    """Quality sanity on the n = 20 twin of the small dense workload
    (weights uniform in [-100, 100], seed 0)."""
    W = wl.dense_qubo(20, -100, 100, 0)
    emin, _, _ = wl.brute_force_min(W)
    p = orc.make_params(searches=32, pools=4, pool_cap=64, max_generations=50)
    X, E, flips, gens = orc.solve(W, p, budget=2**63, seed=0, target=emin)
    assert E == emin and orc.energy(W, X) == emin
    assert gens <= 50


def test_solver_budget_and_target_stop(orc):
    W = wl.dense_qubo(64, -100, 100, 0)
    p = orc.make_params(searches=32, pools=4, pool_cap=64)
    X, E, flips, gens = orc.solve(W, p, budget=10000, seed=4)
    assert flips >= 10000 and gens >= 1
    so = orc.Solver(W, p, seed=4)
    f = 0
    for _ in range(gens - 1):
        f += so.generation()
    assert f < 10000
    X2, E2, _, g2 = orc.solve(W, p, budget=2**63, seed=4, target=E)
    assert E2 <= E and g2 <= gens


def test_statistics_count_every_search_and_each_new_best(orc):
    """Tables V/VI counters: one algorithm and one operation count per search
    per generation; first-finder credits only on improvements of the best."""
    W = wl.dense_qubo(48, -100, 100, 3)
    S, G = 24, 7
    so = orc.Solver(W, orc.make_params(searches=S, pools=3, pool_cap=8), seed=2)
    bests, improvements = [], 0
    for g in range(G):
        so.generation()
        X, E, f, a, o = so.results()
        bests.append(so.best()[1])
    improvements = sum(1 for g in range(G) if g == 0 or bests[g] < bests[g - 1])
    ac, oc, ba, bo = so.stats()
    assert ac.sum() == S * G and oc.sum() == S * G
    assert ba.sum() == improvements and bo.sum() == improvements


def hamming_to(pX, x):
    return (pX.reshape(-1, x.size) != x[None, :]).sum(axis=1)


@pytest.mark.parametrize("P,C,h", [(6, 1, 1), (3, 2, 6)])
def test_restart_fires_exactly_when_every_pool_entry_is_near_the_best(orc, P, C, h):
    """Section IV-B, last paragraph (reading R23): a twin without restarts
    shows the pools after each merge; the restarting solver must leave them
    untouched until the first generation where every entry lies within
    Hamming distance h of the global best, then redraw them and reset the
    searches while keeping the global best."""
    n = 14
    W = wl.dense_qubo(n, -20, 20, seed=5)
    kw = dict(searches=8, pools=P, pool_cap=C, b=(2, 1))
    on = orc.Solver(W, orc.make_params(restart=1, restart_dist=h, **kw), seed=3)
    off = orc.Solver(W, orc.make_params(**kw), seed=3)
    fired = None
    for g in range(60):
        on.generation(); off.generation()
        bx, be, _, _ = off.best()
        merged = (hamming_to(off.pools()[0], bx) <= h).all()
        if not merged:
            assert on.restarts() == 0
            for a, b in zip(on.pools(), off.pools()):
                assert np.array_equal(a, b)
            continue
        fired = g
        assert on.restarts() == 1
        X, E, a, o = on.pools()
        assert (E == np.iinfo(np.int64).max).all()
        assert not np.array_equal(X, off.pools()[0])
        sX, sd, sE = on.state()
        assert not sX.any() and (sE == 0).all()
        assert np.array_equal(sd, np.tile(np.diag(W).astype(np.int32), (8, 1)))
        assert on.best()[1] == be and np.array_equal(on.best()[0], bx)
        break
    assert fired is not None, "the pools never merged on this easy instance"


def test_restart_disabled_by_negative_radius_changes_nothing(orc):
    W = wl.dense_qubo(24, -20, 20, seed=6)
    kw = dict(searches=16, pools=2, pool_cap=4)
    a = orc.solve(W, orc.make_params(restart=1, restart_dist=-1, max_generations=20, **kw), 10**9, 4)
    b = orc.solve(W, orc.make_params(max_generations=20, **kw), 10**9, 4)
    assert a[1:] == b[1:] and np.array_equal(a[0], b[0])


def test_restart_every_generation_keeps_the_best_monotone(orc):
    W = wl.dense_qubo(40, -50, 50, seed=7)
    so = orc.Solver(W, orc.make_params(searches=16, pools=2, pool_cap=4, restart=1,
                                       restart_dist=40), seed=1)
    prev = None
    for g in range(6):
        so.generation()
        assert so.restarts() == g + 1
        be = so.best()[1]
        assert prev is None or be <= prev
        prev = be
    # each restart draws pools of its own
    X1 = so.pools()[0]
    so.generation()
    assert not np.array_equal(so.pools()[0], X1)


def test_abs_mode_is_cyclicmin_with_mutation_after_crossover(orc):
    """Section I (reading R24): the earlier ABS runs CyclicMin only and breeds
    every target as a crossover of two pool parents followed by a mutation.
    With parents all-zero (rank 0) and all-one (rank 1), a target's density
    of ones is 1/8 (both zero), 7/8 (both one) or 1/2 (mixed: independent
    coin, then 1/8 inversions) -- a coin correlated with the mutation mask
    would give 3/8 or 5/8."""
    n, S = 4096, 64
    W = np.zeros((n, n), np.int16)
    so = orc.Solver(W, orc.make_params(searches=S, pools=1, pool_cap=2, abs_mode=1), seed=8)
    X = np.zeros((1, 2, n), np.uint8)
    X[0, 1] = 1
    so.set_pools(X, np.array([[0, 1]], np.int64), np.full((1, 2), 0, np.int32),
                 np.full((1, 2), 6, np.int32))
    seen = set()
    for g in range(4):
        D, a, o = so.offspring(g)
        assert (a == 1).all() and (o == 1).all()
        for dens in D.mean(axis=1):
            near = [c for c in (1 / 8, 1 / 2, 7 / 8) if abs(dens - c) < 0.035]
            assert near, dens
            seen.add(near[0])
    assert seen == {1 / 8, 1 / 2, 7 / 8}
