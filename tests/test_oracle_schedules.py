"""Pins of the oracle's iteration-dependent selectors (Section III-A) at every
iteration t, not only at t = T: RandomMin's candidate probability
p(t) = max((t/T)^3, 32/n) and its per-bit draws, MaxMin's threshold d drawn
uniformly from [min Delta, D(t)] with D(t) decreasing from max Delta to
min Delta, and PositiveMin's bound.  The expected values are computed here in
floating point from the paper's formulas; Delta is recomputed from Eq. (2) on
a replay of the search, independently of the oracle's incremental state."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl

from test_oracle_search import delta_def


def p_of(t, T, n):
    """Section III-A RandomMin: p(t) = max((t/T)^3, c) with c = 32/n (capped at 1)."""
    return min(1.0, max((t / T) ** 3, 32.0 / n))


@pytest.mark.parametrize("n", [1, 5, 20, 32, 33, 64, 800, 1000, 1024, 4096, 5627, 8192, 16384,
                               65536])
@pytest.mark.parametrize("T", [1, 6, 80, 102, 1638])
def test_randmin_threshold_is_the_schedule(orc, n, T):
    ts = sorted(set(np.linspace(1, T, min(T, 200)).astype(int)))
    for t in ts:
        thr = orc.randmin_threshold(t, T, n)
        p = p_of(t, T, n)
        # 16-bit units: the floor is 32/n rounded up to the next 2^-16, the
        # cube is truncated to 2^-16 after a 21-bit ratio (error < 2e-6)
        assert abs(thr / 65536 - p) <= 2 ** -16 + 2e-6, (t, T, n, thr, p)
        assert thr / 65536 >= min(1.0, 32.0 / n)  # never below the paper's c
        assert thr <= 65536
    assert orc.randmin_threshold(T, T, n) == 65536  # p(T) = 1


def test_randmin_draws_are_uniform_16_bit_values(orc):
    n = 4096
    u = np.concatenate([orc.randmin_draws(9, f, 2, 5, n) for f in range(40)]).astype(np.int64)
    assert u.min() >= 0 and u.max() <= 65535
    N = u.size
    assert abs(u.mean() - 32767.5) < 5 * 18918 / np.sqrt(N)  # sd of U{0..65535}
    for part in (u >> 8, u & 0xFF):  # both bytes of every draw are uniform
        h = np.bincount(part, minlength=256)
        chi2 = ((h - N / 256) ** 2 / (N / 256)).sum()
        assert chi2 < 255 + 6 * np.sqrt(2 * 255)
    # a different flip, search or generation gives different draws
    a = orc.randmin_draws(9, 3, 2, 5, 64)
    for other in (orc.randmin_draws(9, 4, 2, 5, 64), orc.randmin_draws(9, 3, 2, 6, 64),
                  orc.randmin_draws(9, 3, 3, 5, 64), orc.randmin_draws(10, 3, 2, 5, 64)):
        assert not np.array_equal(a, other)


@pytest.mark.parametrize("n,T", [(16384, 1638), (800, 80), (5627, 562)])
def test_randmin_candidate_count_at_the_floor(orc, n, T):
    """Early iterations sit at the floor c = 32/n: about 32 candidates each,
    for every n (Section III-A: "expected n p(t) bits are selected")."""
    thr = orc.randmin_threshold(1, T, n)
    K = 120 if n > 4000 else 400
    counts = np.array([(orc.randmin_draws(3, f, 1, 7, n) < thr).sum() for f in range(K)])
    p = 32.0 / n
    mean_expected = n * p
    sd = np.sqrt(n * p * (1 - p) / K)
    assert abs(counts.mean() - mean_expected) < 5 * sd + 0.5 * 2 ** -16 * n, counts.mean()


def _main_iterations(orc, r, W, X0, tau, T):
    """(flip index, t within its main run, replayed X and Delta, free mask, pick);
    a main run is T flips, and a Greedy of no flips may join two runs"""
    ph, tr = r["phases"], r["trace"]
    n = W.shape[0]
    X = X0.astype(np.int64).copy()
    t, seq = 0, []
    for step, i in enumerate(tr):
        if ph[step] == orc.PH_MAIN:
            if t == T:
                t, seq = 0, []
            t += 1
            tabu = set(seq[max(0, len(seq) - tau):])
            free = np.array([k not in tabu for k in range(n)])
            yield step, t, X.copy(), delta_def(W, X), free, int(i)
            seq.append(int(i))
        else:
            t, seq = 0, []
        X[i] ^= 1


def _search(orc, W, algo, seed, tau, s_f, b):
    n = W.shape[0]
    p = orc.make_params(searches=1, pools=1, pool_cap=4, tabu=tau, s=s_f, b=b, seed_mode=0)
    rng = np.random.default_rng(seed)
    X0 = rng.integers(0, 2, n).astype(np.uint8)
    D = rng.integers(0, 2, n).astype(np.uint8)
    r = orc.batch_search(W, p, seed, 4, 11, X0, orc.delta(W, X0), orc.energy(W, X0), D, algo,
                         trace_cap=200000, sel=True)
    T = max(1, n * s_f[0] // s_f[1])
    return r, X0, T


def test_maxmin_threshold_lies_in_min_to_D_t_and_bounds_the_pick(orc):
    n, tau = 48, 8
    frac = []
    for seed in range(3):
        W = wl.dense_qubo(n, -60, 60, seed=100 + seed)
        r, X0, T = _search(orc, W, orc.MAXMIN, seed, tau, (1, 2), (6, 1))
        seen = 0
        for step, t, X, dl, free, i in _main_iterations(orc, r, W, X0, tau, T):
            d, R, cnt = int(r["sel_a"][step]), int(r["sel_r"][step]), int(r["sel_count"][step])
            mn, mx = int(dl[free].min()), int(dl[free].max())
            q = ((T - t) / T) ** 3
            D_t = mn + q * (mx - mn)  # the paper's D(t), real-valued
            assert mn <= d <= D_t + 1e-5 * (mx - mn) + 1e-9, (t, d, mn, D_t)
            assert mn <= d <= mx
            assert abs(R - q * (mx - mn)) <= 1 + 2e-6 * (mx - mn)
            assert cnt == int((free & (dl <= d)).sum()) >= 1
            assert free[i] and dl[i] <= d  # Step 2 picks a bit with Delta_i <= d
            if t == T:
                assert d == mn
            if R >= 8:
                frac.append((d - mn) / (R + 1))
            seen += 1
        assert seen >= 3 * T
    # d is uniform on [min Delta, min Delta + R]
    frac = np.array(frac)
    assert len(frac) > 300
    assert abs(frac.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(frac))
    assert (frac < 0.25).mean() > 0.15 and (frac > 0.75).mean() > 0.15


def test_maxmin_threshold_function(orc):
    """D(t) decreases from max Delta (t = 0) to min Delta (t = T), and d covers
    [min Delta, D(t)] uniformly (Section III-A, MaxMin)."""
    rng = np.random.default_rng(4)
    for _ in range(60):
        mn = int(rng.integers(-30000, 30000))
        mx = mn + int(rng.integers(0, 60000))
        T = int(rng.integers(1, 2000))
        last = None
        for t in sorted(set(np.linspace(1, T, min(T, 50)).astype(int))):
            d_lo, R = orc.maxmin_threshold(mn, mx, t, T, 0)
            d_hi, _ = orc.maxmin_threshold(mn, mx, t, T, 2 ** 32 - 1)
            D_t = mn + ((T - t) / T) ** 3 * (mx - mn)
            assert d_lo == mn and mn <= d_hi <= D_t + 1e-5 * (mx - mn) + 1e-9
            assert d_hi >= D_t - 1 - 2e-6 * (mx - mn)  # the top of [mn, D(t)] is reached
            if last is not None:
                assert R <= last  # non-increasing in t
            last = R
        assert orc.maxmin_threshold(mn, mx, T, T, 2 ** 32 - 1)[0] == mn


def test_randmin_candidate_rate_follows_p_of_t(orc):
    """Over many iterations, the candidate count per t-bin averages free * p(t)
    within a binomial bound, and the pick is the arg-min of Delta over the
    candidates (Section III-A, RandomMin)."""
    n, tau, s_f = 96, 8, (1, 2)
    T = n * s_f[0] // s_f[1]
    nb = 6
    obs, exp, var = np.zeros(nb), np.zeros(nb), np.zeros(nb)
    for seed in range(4):
        W = wl.dense_qubo(n, -40, 40, seed=200 + seed)
        r, X0, _ = _search(orc, W, orc.RANDOMMIN, seed, tau, s_f, (8, 1))
        for step, t, X, dl, free, i in _main_iterations(orc, r, W, X0, tau, T):
            thr = int(r["sel_a"][step])
            cnt, nf = int(r["sel_count"][step]), int(r["sel_free"][step])
            assert nf == int(free.sum())
            p = p_of(t, T, n)
            b = min(nb - 1, (t - 1) * nb // T)
            obs[b] += cnt
            exp[b] += nf * p
            var[b] += nf * p * (1 - p)
            # the pick: arg-min over the free bits whose draw is below thr
            u = orc.randmin_draws(seed, step, 4, 11, n)
            cand = free & (u < thr)
            assert int(cand.sum()) == cnt
            pool = cand if cand.any() else free
            assert i == int(np.nonzero(pool & (dl == dl[pool].min()))[0][0])
    for b in range(nb):
        assert abs(obs[b] - exp[b]) <= 5 * np.sqrt(var[b]) + 2 ** -16 * exp[b] * n, (b, obs, exp)


def test_positivemin_bound_is_the_smallest_positive_delta(orc):
    n, tau = 40, 8
    W = wl.dense_qubo(n, -30, 30, seed=300)
    r, X0, T = _search(orc, W, orc.POSITIVEMIN, 1, tau, (1, 2), (4, 1))
    seen = 0
    for step, t, X, dl, free, i in _main_iterations(orc, r, W, X0, tau, T):
        pm, cnt = int(r["sel_a"][step]), int(r["sel_count"][step])
        pos = dl[free & (dl > 0)]
        if pos.size:
            assert pm == int(pos.min()) and cnt == int((free & (dl <= pm)).sum())
        else:
            assert pm == np.iinfo(np.int64).max and cnt == int(free.sum())
        seen += 1
    assert seen >= 2 * T
