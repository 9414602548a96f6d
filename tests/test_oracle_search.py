"""Pins of the oracle's incremental search (Section III) against invariants the
paper states: Delta/E maintained incrementally equal a from-scratch
recomputation, Greedy ends in a local minimum, Straight reaches D after exactly
Hamming(X, D) flips, the TwoNeighbor walk of the n = 6 example, every 2-bit
neighbour reachable by TwoNeighbor, the flip-budget arithmetic of
Section III-B, and the selection rule of every main search algorithm checked
on a replay of its trace with an independently computed Delta."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl


def delta_def(W, X):
    """Delta_k = E(f_k X) - E(X) computed from Eq. (2) directly."""
    W = np.asarray(W, np.int64)
    X = np.asarray(X, np.int64)
    Wu = np.triu(W, 1)
    dg = np.diag(W)
    e = lambda v: int(v @ dg + v @ Wu @ v)
    e0 = e(X)
    out = np.empty(len(X), np.int64)
    for k in range(len(X)):
        v = X.copy()
        v[k] ^= 1
        out[k] = e(v) - e0
    return out


def run(orc, W, algo, seed_mode=0, seed=5, g=3, s=7, X0=None, D=None, b=(2, 1), s_f=(1, 4),
        tabu=8, trace=100000, check=True):
    n = W.shape[0]
    p = orc.make_params(searches=1, pools=1, pool_cap=4, tabu=tabu, s=s_f, b=b,
                        seed_mode=seed_mode)
    rng = np.random.default_rng(seed)
    X0 = rng.integers(0, 2, n).astype(np.uint8) if X0 is None else X0
    D = rng.integers(0, 2, n).astype(np.uint8) if D is None else D
    d0 = orc.delta(W, X0)
    E0 = orc.energy(W, X0)
    r = orc.batch_search(W, p, seed, g, s, X0, d0, E0, D, algo, trace_cap=trace, check=check)
    return p, X0, D, r


@pytest.mark.parametrize("algo", range(5))
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64])
@pytest.mark.parametrize("seed_mode", [0, 1])
def test_incremental_state_equals_recomputation(orc, algo, n, seed_mode):
    W = wl.dense_qubo(n, -100, 100, seed=n)
    _, _, _, r = run(orc, W, algo, seed_mode=seed_mode)
    assert r["ok"], "Delta/E diverged from a from-scratch recomputation"
    assert np.array_equal(r["delta"], orc.delta(W, r["X"]))
    assert r["E"] == orc.energy(W, r["X"])
    assert r["best_E"] == orc.energy(W, r["best_X"])
    assert r["best_E"] <= r["E"]


@pytest.mark.parametrize("algo", range(5))
def test_batch_search_ends_in_greedy_local_minimum(orc, algo):
    W = wl.dense_qubo(40, -100, 100, seed=11)
    _, _, _, r = run(orc, W, algo)
    assert (r["delta"] >= 0).all()  # Section III-A Greedy: Delta_k >= 0 for all k
    assert r["phases"][-1] in (orc.PH_GREEDY, orc.PH_MAIN)


def replay(W, X0, trace):
    X = X0.astype(np.int64).copy()
    for i in trace:
        yield X.copy(), delta_def(W, X), i
        X[i] ^= 1


def test_straight_walks_to_target_and_greedy_is_argmin(orc):
    n = 48
    W = wl.dense_qubo(n, -100, 100, seed=3)
    p, X0, D, r = run(orc, W, orc.CYCLICMIN)
    ph = r["phases"]
    nst = int((ph == orc.PH_STRAIGHT).sum())
    assert nst == int((X0 != D).sum())  # exactly Hamming(X, D) flips
    assert set(r["trace"][:nst]) == set(np.nonzero(X0 != D)[0])
    for step, (X, dl, i) in enumerate(replay(W, X0, r["trace"])):
        if ph[step] == orc.PH_STRAIGHT:
            mask = X != D
            assert mask[i] and dl[i] == dl[mask].min()
            assert i == np.nonzero(mask & (dl == dl[mask].min()))[0][0]
        elif ph[step] == orc.PH_GREEDY:
            assert dl[i] < 0 and i == int(np.argmin(dl))


def test_two_neighbor_worked_example(orc):
    """Section III-A TwoNeighbor, n = 6 from X = 000000: the eleven states."""
    n = 6
    W = np.diag(np.arange(1, 7)).astype(np.int16)  # X = 0 is a local minimum
    z = np.zeros(n, np.uint8)
    _, _, _, r = run(orc, W, orc.TWONEIGHBOR, X0=z, D=z)
    main = r["trace"][r["phases"] == orc.PH_MAIN]
    assert list(main) == [0, 1, 0, 2, 1, 3, 2, 4, 3, 5, 4]
    states, X = [], z.copy()
    for i in main:
        X[i] ^= 1
        states.append("".join(map(str, X)))
    assert states == ["100000", "110000", "010000", "011000", "001000", "001100", "000100",
                      "000110", "000010", "000011", "000001"]


@pytest.mark.parametrize("a,b", [(0, 5), (2, 3), (4, 9), (8, 9)])
def test_two_neighbor_finds_every_two_bit_neighbour(orc, a, b):
    """Step 1 during TwoNeighbor examines all 2-bit neighbours of X: a pair
    whose joint flip is the unique improvement must become BEST although
    every single flip is uphill (Greedy alone cannot find it)."""
    n = 10
    W = np.diag(np.full(n, 5)).astype(np.int16)
    W[a, b] = W[b, a] = -30
    z = np.zeros(n, np.uint8)
    _, _, _, r = run(orc, W, orc.TWONEIGHBOR, X0=z, D=z)
    want = z.copy()
    want[[a, b]] = 1
    assert r["best_E"] == -20 and np.array_equal(r["best_X"], want)


def test_ties_go_to_the_lowest_index(orc):
    """Tie rules of Step 1, Greedy and Straight (lowest index first)."""
    n = 8
    W = np.diag([3, -5, 2, -5, -5, 4, 1, 1]).astype(np.int16)
    z = np.zeros(n, np.uint8)
    _, _, _, r = run(orc, W, orc.CYCLICMIN, X0=z, D=z, b=(1, 8))
    assert list(r["trace"][:3]) == [1, 3, 4]  # Greedy: equal Delta = -5, ascending
    assert r["best_E"] == -15
    D = np.array([0, 0, 1, 0, 0, 1, 1, 1], np.uint8)
    _, _, _, r = run(orc, W, orc.CYCLICMIN, X0=z, D=D, b=(1, 8))
    assert list(r["trace"][:4]) == [6, 7, 2, 5]  # Straight: Delta 1, 1, 2, 4
    # Step 1 on the first Straight step sees neighbours -5 at bits 1, 3, 4:
    # BEST must be the lowest one, later replaced only on strict improvement
    Wb = np.diag([0, -5, 0, 0, 0, 0, 0, 0]).astype(np.int16)
    D2 = np.array([0, 0, 0, 0, 0, 0, 1, 0], np.uint8)
    _, _, _, r = run(orc, Wb, orc.TWONEIGHBOR, X0=z, D=D2, b=(1, 8), check=False)
    assert list(r["trace"]) == [6, 1]
    # first Step 1 (X = 0) records bit 1; the equal-energy neighbours seen at
    # X = e6 and X = e1 + e6 must not replace it
    assert r["best_E"] == -5 and list(np.nonzero(r["best_X"])[0]) == [1]


def test_flip_budget_worked_example(orc):
    """Section III-B: Straight 300, Greedy 50, main 600 and b n = 2000 give
    300+50+600+50+600+50+600+50 = 2300 flips and three main searches."""
    total, runs = 300 + 50, 0
    while orc.batch_continue(total, 2000, runs, orc.MAXMIN):
        total += 600 + 50
        runs += 1
    assert (total, runs) == (2300, 3)
    assert not orc.batch_continue(350, 2000, 1, orc.TWONEIGHBOR)  # TwoNeighbor once


@pytest.mark.parametrize("algo", [0, 1, 2, 3])
def test_batch_schedule_and_tabu(orc, algo):
    n = 40
    W = wl.dense_qubo(n, -100, 100, seed=21)
    p, X0, D, r = run(orc, W, algo, b=(3, 1), s_f=(1, 4), tabu=8)
    ph, tr = r["phases"], r["trace"]
    T = max(1, n * p.s_num // p.s_den)
    B = -(-n * p.b_num // p.b_den)
    assert r["flips"] >= B
    # main runs are exactly T flips; each main run is followed by Greedy
    runs = np.split(np.arange(len(ph)), np.nonzero(np.diff(ph))[0] + 1)
    mains = [x for x in runs if ph[x[0]] == orc.PH_MAIN]
    assert all(len(x) == T for x in mains)
    # tabu: within a main run no bit repeats inside tau+1 consecutive flips
    tau = min(8, n - 1)
    for x in mains:
        seq = list(tr[x])
        for t in range(len(seq)):
            assert seq[t] not in seq[max(0, t - tau):t]


def _tabu_sets(seq, tau):
    return [set(seq[max(0, t - tau):t]) for t in range(len(seq))]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_selector_rules_on_replay(orc, seed):
    """Each main algorithm's pick obeys its definition at every iteration
    (Section III-A), with Delta recomputed from Eq. (2)."""
    n = 36
    W = wl.dense_qubo(n, -50, 50, seed=seed)
    tau = 8
    for algo in range(4):
        p, X0, D, r = run(orc, W, algo, seed=seed, b=(3, 1), s_f=(1, 2), tabu=tau)
        T = n * p.s_num // p.s_den
        ph, tr = r["phases"], r["trace"]
        states = list(replay(W, X0, tr))
        t_in_run, seq, win = 0, [], 0
        for step, (X, dl, i) in enumerate(states):
            if ph[step] != orc.PH_MAIN:
                t_in_run, seq, win = 0, [], 0
                continue
            t_in_run += 1
            tabu = set(seq[max(0, len(seq) - tau):])
            free = np.array([k not in tabu for k in range(n)])
            assert free[i]
            if algo == orc.MAXMIN:
                if t_in_run == T:  # D(T) = min Delta: the pick is a minimiser
                    assert dl[i] == dl[free].min()
            elif algo == orc.CYCLICMIN:
                w = min(n, max(32, (orc.cube21(t_in_run, T) * n) >> 32))
                window = [(win + r_) % n for r_ in range(w)]
                cand = [k for k in window if free[k]]
                assert i in cand and dl[i] == min(dl[k] for k in cand)
                assert i == next(k for k in cand if dl[k] == dl[i])
                win = (win + w) % n
                if t_in_run == T:
                    assert w == n
            elif algo == orc.RANDOMMIN:
                if t_in_run == T:  # p(T) = 1: every free bit is a candidate
                    assert i == np.nonzero(free & (dl == dl[free].min()))[0][0]
            else:  # PositiveMin
                pos = dl[free & (dl > 0)]
                if pos.size:
                    assert dl[i] <= pos.min()
            seq.append(i)


def test_positive_min_pick_is_uniform_over_candidates(orc):
    """PositiveMin picks one candidate at random (Section III-A): over many
    iterations the pick's rank among the candidates is uniform."""
    n, tau = 40, 8
    ranks = []
    for seed in range(6):
        W = wl.dense_qubo(n, -20, 20, seed=seed + 40)
        p, X0, D, r = run(orc, W, orc.POSITIVEMIN, seed=seed, b=(4, 1), s_f=(1, 1), tabu=tau,
                          check=False)
        ph, tr = r["phases"], r["trace"]
        seq = []
        for step, (X, dl, i) in enumerate(replay(W, X0, tr)):
            if ph[step] != orc.PH_MAIN:
                seq = []
                continue
            tabu = set(seq[max(0, len(seq) - tau):])
            free = np.array([k not in tabu for k in range(n)])
            pos = dl[free & (dl > 0)]
            cand = np.nonzero(free & (dl <= pos.min()))[0] if pos.size else np.nonzero(free)[0]
            assert i in cand
            if len(cand) > 1:
                ranks.append(list(cand).index(i) / (len(cand) - 1))
            seq.append(i)
    assert len(ranks) > 200 and abs(np.mean(ranks) - 0.5) < 0.06


def test_cube21_endpoints_and_monotone(orc):
    for T in (1, 3, 6, 80, 1000):
        vals = [orc.cube21(a, T) for a in range(T + 1)]
        assert vals[0] == 0 and vals[-1] == 1 << 32
        assert all(x <= y for x, y in zip(vals, vals[1:]))
        for a in range(T + 1):
            assert abs(vals[a] / 2**32 - (a / T) ** 3) < 2e-6


def test_parent_rank_first_probability(orc):
    """Section IV-A: the best packet is taken with probability m^(-1/3)."""
    rng = np.random.default_rng(0)
    us = rng.integers(0, 2**32, 60000, dtype=np.uint64)
    for m in (8, 64, 100):
        ranks = np.array([orc.parent_rank(int(u), m) for u in us])
        assert ranks.min() == 0 and ranks.max() <= m - 1
        p0 = (ranks == 0).mean()
        assert abs(p0 - m ** (-1 / 3)) < 4 * np.sqrt(p0 * (1 - p0) / len(us)) + 1e-3
    assert orc.parent_rank(0, 100) == 0 and orc.parent_rank(2**32 - 1, 100) == 99


def test_search_is_deterministic(orc):
    W = wl.dense_qubo(50, -100, 100, seed=2)
    a = run(orc, W, orc.RANDOMMIN, check=False)[3]
    b = run(orc, W, orc.RANDOMMIN, check=False)[3]
    assert np.array_equal(a["trace"], b["trace"]) and a["best_E"] == b["best_E"]
    c = run(orc, W, orc.RANDOMMIN, check=False, seed=6)[3]
    assert not np.array_equal(a["trace"], c["trace"])
