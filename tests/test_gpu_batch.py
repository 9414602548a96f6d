"""Batched and served forms: every instance's result equals its solve alone
(and the oracle's), whatever the mix, kernel variants and arrival order;
the server never exceeds its HBM budget."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03069_gb300 import build, dabs
    build.build()
    return dabs


SIZES = [64, 200, 300, 700, 1100, 2100]


def instance(n, k):
    return wl.dense_qubo(n, -1000, 1000, seed=100 + k)


@pytest.mark.parametrize("seed_mode,extra", [(0, {}), (1, {}),
                                             (0, dict(restart=1, restart_dist=100, abs_mode=1))])
def test_batch_solve_equals_alone(D, orc, seed_mode, extra):
    kw = dict(searches=48, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), seed_mode=seed_mode,
              max_generations=5, **extra)
    Ws = [instance(n, k) for k, n in enumerate(SIZES)]
    ctxs = [D.Context(W, **kw) for W in Ws]
    budgets = [10**9, 10**9, 40000, 10**9, 10**9, 10**9]  # one stops early on its budget
    seeds = [11 + k for k in range(len(Ws))]
    out = D.batch_solve(ctxs, budgets, seeds)
    variants = {(c.info()["warps"], c.info()["chunks"]) for c in ctxs}
    assert len(variants) >= 3  # several multi-instance search launches
    for k, (W, c) in enumerate(zip(Ws, ctxs)):
        alone = D.Context(W, **kw).solve(budgets[k], seeds[k])
        assert out[k][1] == alone[1] and out[k][2] == alone[2], k
        assert np.array_equal(out[k][0], alone[0]), k
        if W.shape[0] <= 300:
            ox, oe, of, _ = orc.solve(W, orc.make_params(**kw), budgets[k], seeds[k], threads=8)
            assert (out[k][1], out[k][2]) == (oe, of) and np.array_equal(out[k][0], ox)


def test_server_equals_alone_and_respects_budget(D):
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1,
              max_generations=4)
    sizes = [512, 1024, 128, 2048, 256, 768, 1500, 96]
    Ws = [instance(n, k) for k, n in enumerate(sizes)]
    params = D.default_params(**kw)
    # a budget that holds about two of the larger contexts at once
    srv = D.Server(hbm_budget_bytes=48 << 20)
    srv.set_limits(0)  # HBM budget only
    tickets = []
    for k, W in enumerate(Ws[:4]):
        tickets.append(srv.submit(W, params, 10**9, 7 + k))
    max_running, max_used, rounds = 0, 0, 0
    while True:
        if rounds == 1:  # requests arriving while others run
            for k, W in enumerate(Ws[4:], start=4):
                tickets.append(srv.submit(W, params, 10**9, 7 + k))
        pending = srv.step(1)
        used, q, r = srv.info()
        max_running, max_used = max(max_running, r), max(max_used, used)
        rounds += 1
        if pending == 0 and rounds > 1:
            break
        assert rounds < 200
    assert max_used <= 48 << 20 and max_running >= 2
    for k, (t, W) in enumerate(zip(tickets, Ws)):
        st, X, E, F, lat = srv.poll(t)
        assert st == 2 and lat > 0
        aX, aE, aF = D.Context(W, **kw).solve(10**9, 7 + k)
        assert (E, F) == (aE, aF) and np.array_equal(X, aX), k
    too_big = np.zeros((8192, 8192), np.int16)
    with pytest.raises(D.DabsError):
        srv.submit(too_big, params, 10, 1)


def test_server_warp_cap_serves_in_arrival_order(D):
    kw = dict(searches=128, pools=2, pool_cap=8, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0,
              max_generations=3)
    params = D.default_params(**kw)
    Ws = [instance(300, k) for k in range(6)]
    srv = D.Server(hbm_budget_bytes=8 << 30)
    srv.set_limits(2 * 128)  # two one-warp requests at a time
    tickets = [srv.submit(W, params, 10**9, 40 + k) for k, W in enumerate(Ws)]
    order = []
    while True:
        pending = srv.step(1)
        assert srv.info()[2] <= 2
        for t in tickets:
            if t not in order and srv.poll(t)[0] == 2:
                order.append(t)
        if pending == 0:
            break
    assert order == tickets  # equal requests finish in arrival order
    for k, (t, W) in enumerate(zip(tickets, Ws)):
        st, X, E, F, _ = srv.poll(t)
        aX, aE, aF = D.Context(W, **kw).solve(10**9, 40 + k)
        assert (E, F) == (aE, aF) and np.array_equal(X, aX)


def test_batch_with_row_formats_equals_alone(D):
    """Contexts set to sparse rows (shared or global) or to W in shared memory
    join a batched solve (whose launches read dense rows) with the results each
    gets alone in its own format."""
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), max_generations=3)
    Ws = [wl.maxcut_qubo(300, 0.05, seed=1), wl.maxcut_qubo(700, 0.03, seed=2),
          wl.dense_qubo(200, -100, 100, seed=3)]
    modes = [D.ROWS_SPARSE_SMEM, D.ROWS_SPARSE_GLOBAL, D.ROWS_DENSE_SMEM]
    ctxs = []
    for W, m in zip(Ws, modes):
        c = D.Context(W, **kw)
        c.set_rows(m)
        ctxs.append(c)
    out = D.batch_solve(ctxs, [10**9] * 3, [5, 6, 7])
    for k, (W, m) in enumerate(zip(Ws, modes)):
        alone = D.Context(W, **kw)
        alone.set_rows(m)
        a = alone.solve(10**9, 5 + k)
        assert out[k][1] == a[1] and out[k][2] == a[2] and np.array_equal(out[k][0], a[0])


def test_stepwise_batch_generations_equal_alone(D, orc):
    """dabs_batch_* one generation at a time: after every generation each
    instance's pools, results and per-search state equal its generations
    alone (and, for the small instances, the oracle's)."""
    from test_gpu_parity import compare_generation
    kw = dict(searches=40, pools=4, pool_cap=12, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1)
    sizes = [96, 700, 1500, 300]
    Ws = [instance(n, 30 + k) for k, n in enumerate(sizes)]
    ctxs = [D.Context(W, **kw) for W in Ws]
    alone = [D.Context(W, **kw) for W in Ws]
    small = [orc.Solver(W, orc.make_params(**kw), 70 + k) if W.shape[0] <= 300 else None
             for k, W in enumerate(Ws)]
    b = D.Batch(ctxs)
    budgets = [10**12, 10**12, 10**12, 3 * 40 * 300]  # the last stops on its budget
    b.begin(budgets, [70 + k for k in range(len(Ws))])
    for k, a in enumerate(alone):
        a.solve_begin(70 + k, budget=budgets[k])
    running = len(Ws)
    for g in range(5):
        running = b.generations(1)
        for k, (c, a) in enumerate(zip(ctxs, alone)):
            a.solve_generations(1)
            assert c.solve_status() == a.solve_status(), (g, k)
            for x, y in zip(c.read_pools(), a.read_pools()):
                assert np.array_equal(x, y), (g, k)
            for x, y in zip(c.read_generation(), a.read_generation()):
                assert np.array_equal(x, y), (g, k)
            if small[k] is not None and g < 3:
                small[k].generation(8)
                compare_generation(c, small[k], Ws[k].shape[0], f"gen {g} instance {k}")
    assert running == len(Ws) - 1  # the budget-limited instance retired
    b.close()
    # the contexts work on their own again afterwards (two generations' budget)
    X, E, F = ctxs[0].solve(2 * 40 * 96, seed=3)
    assert (E, F) == alone[0].solve(2 * 40 * 96, seed=3)[1:]
