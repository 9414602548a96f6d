"""GPU parity: the CUDA library against the oracle, bit for bit (all integer
work).  Covers energy/Delta (Eqs. (2)-(3)), the batch-search kernel for every
main algorithm and both seeding modes on ragged sizes and every kernel
variant, offspring and merge in isolation, whole generations and whole solves.
"""
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


def ctx_for(D, W, **kw):
    base = dict(searches=8, pools=2, pool_cap=16, tabu=8, s=(1, 4), b=(2, 1), seed_mode=0)
    base.update(kw)
    return D.Context(W, **base)


@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 257, 800, 1000, 2048, 4100, 8192])
def test_energy_delta(D, orc, n):
    W = wl.dense_qubo(n, -32767, 32767, seed=n)
    ctx = ctx_for(D, W, searches=1, pools=1, pool_cap=1)
    rng = np.random.default_rng(n)
    for dens in (0.0, 0.5, 1.0, 0.1):
        X = (rng.random(n) < dens).astype(np.uint8)
        assert ctx.energy(X) == orc.energy(W, X)
        assert np.array_equal(ctx.delta(X), orc.delta(W, X))
    # batched device form
    cnt = 5
    Xs = (rng.random((cnt, n)) < 0.5).astype(np.uint8)
    Xd = torch.from_numpy(wl.pack_bits(Xs).view(np.int32)).cuda()
    Ed = torch.zeros(cnt, dtype=torch.int64, device="cuda")
    dd = torch.zeros((cnt, n + 3), dtype=torch.int32, device="cuda")
    ctx.energy_delta_dev(Xd, Ed, dd)
    torch.cuda.synchronize()
    for v in range(cnt):
        assert int(Ed[v]) == orc.energy(W, Xs[v])
        assert np.array_equal(dd[v, :n].cpu().numpy(), orc.delta(W, Xs[v]))


def test_host_arguments_are_validated(D):
    W = wl.dense_qubo(8, -5, 5, 0)
    ctx = ctx_for(D, W)
    with pytest.raises(D.DabsError):
        ctx.energy(np.array([0, 1, 2, 0, 0, 0, 0, 0], np.uint8))
    Wm = W.copy()
    Wm[2, 3] = Wm[3, 2] = -32768
    with pytest.raises(D.DabsError) as e:
        D.Context(Wm, searches=4, pools=1)
    assert e.value.code == D.E_INVALID_ARG
    Wa = W.copy()
    Wa[0, 1] += 1
    with pytest.raises(D.DabsError) as e:
        D.Context(Wa, searches=4, pools=1)
    assert e.value.code == D.E_NOT_SYMMETRIC


def bulk_case(D, orc, W, algos, variant=None, seed=11, g=5, seed_mode=0, s=(1, 4), b=(2, 1),
              tabu=8, S=None, dflip=None, rows=None, keyed=None):
    n = W.shape[0]
    S = S or len(algos)
    ctx = ctx_for(D, W, searches=S, pools=1, pool_cap=4, s=s, b=b, tabu=tabu, seed_mode=seed_mode)
    if variant:
        ctx.set_variant(*variant)
    if keyed is not None:  # True: the instance must allow the keyed form
        ctx.set_keyed(keyed)
        assert not keyed or ctx.keyed()[1] > 0
    if rows is not None:
        ctx.set_rows(rows)
        assert ctx.rows()[0] == rows
    rng = np.random.default_rng(seed + n)
    X0 = (rng.random((S, n)) < 0.5).astype(np.uint8)
    Dt = (rng.random((S, n)) < 0.5).astype(np.uint8)
    if dflip is not None:  # targets near the start: short Straight walks
        Dt = X0 ^ (rng.random((S, n)) < dflip).astype(np.uint8)
    if seed_mode == 1:
        X0 = Dt.copy()
    d0 = np.stack([orc.delta(W, x) for x in X0])
    E0 = np.array([orc.energy(W, x) for x in X0], np.int64)
    dpad = np.zeros((S, ctx.ld), np.int32)
    dpad[:, :n] = d0
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()
    Xd = t(wl.pack_bits(X0), np.int32)
    Dd = t(wl.pack_bits(Dt), np.int32)
    dd = t(dpad, np.int32)
    Ed = t(E0, np.int64)
    ad = t(np.asarray(algos, np.uint8), np.uint8)
    bX = torch.zeros((S, ctx.words), dtype=torch.int32, device="cuda")
    bE = torch.zeros(S, dtype=torch.int64, device="cuda")
    fl = torch.zeros(S, dtype=torch.int32, device="cuda")
    ctx.bulk_search_dev(seed, g, Xd, dd, Ed, Dd, ad, bX, bE, fl)
    torch.cuda.synchronize()
    p = orc.make_params(searches=1, pools=1, pool_cap=4, tabu=tabu, s=s, b=b, seed_mode=seed_mode)
    gX = wl.unpack_bits(Xd.cpu().numpy().view(np.uint32), n)
    gb = wl.unpack_bits(bX.cpu().numpy().view(np.uint32), n)
    for si in range(S):
        r = orc.batch_search(W, p, seed, g, si, X0[si], d0[si], int(E0[si]), Dt[si], int(algos[si]))
        ctx_msg = f"n={n} slot={si} algo={algos[si]} variant={ctx.variant_name()}"
        assert int(fl[si]) == r["flips"], ctx_msg
        assert int(bE[si]) == r["best_E"], ctx_msg
        assert np.array_equal(gb[si], r["best_X"]), ctx_msg
        assert np.array_equal(gX[si], r["X"]), ctx_msg
        assert int(Ed[si]) == r["E"], ctx_msg
        assert np.array_equal(dd[si, :n].cpu().numpy(), r["delta"]), ctx_msg
    return ctx


ALGOS = [0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 2, 3]


@pytest.mark.parametrize("keyed", [True, False])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 100, 257, 800])
def test_bulk_search_matches_oracle(D, orc, n, keyed):
    W = wl.dense_qubo(n, -100, 100, seed=3 * n)
    bulk_case(D, orc, W, ALGOS, keyed=keyed)


@pytest.mark.parametrize("variant", [(1, 1), (1, 2), (1, 4), (2, 1), (2, 2), (2, 4), (4, 1),
                                     (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (16, 1), (16, 2),
                                     (16, 4)])
def test_every_variant_matches_oracle(D, orc, variant):
    """Both forms of the flip loop on every variant: wide weights (plain
    Delta) and weights small enough for the keyed form at the same n."""
    nw, ch = variant
    cap = 256 * nw * ch
    for n in sorted({max(1, cap // 3 + 5), cap - 7}):
        W = wl.dense_qubo(n, -1000, 1000, seed=n + 1)
        bulk_case(D, orc, W, [0, 1, 2, 3, 4], variant=variant, s=(1, 32), b=(1, 4), dflip=0.02,
                  keyed=False)
        W = wl.dense_qubo(n, -2, 2, seed=n + 1)
        bulk_case(D, orc, W, [0, 1, 2, 3, 4], variant=variant, s=(1, 32), b=(1, 4), dflip=0.02,
                  keyed=True)


@pytest.mark.parametrize("n", [33, 300])
def test_bulk_search_recompute_seeding(D, orc, n):
    W = wl.dense_qubo(n, -100, 100, seed=n)
    for keyed in (True, False):
        bulk_case(D, orc, W, ALGOS, seed_mode=1, keyed=keyed)


@pytest.mark.parametrize("tabu,s,b", [(0, (1, 4), (2, 1)), (31, (1, 2), (3, 1)),
                                      (8, (0, 1), (1, 1)), (8, (1, 4), (0, 1))])
def test_bulk_search_parameter_edges(D, orc, tabu, s, b):
    W = wl.dense_qubo(70, -100, 100, seed=9)
    for keyed in (True, False):
        bulk_case(D, orc, W, ALGOS, tabu=tabu, s=s, b=b, keyed=keyed)


def test_bulk_search_extreme_weights(D, orc):
    n = 512
    W = wl.dense_qubo(n, -32767, 32767, seed=1)
    bulk_case(D, orc, W, ALGOS, s=(1, 8), b=(1, 1))
    Z = np.zeros((n, n), np.int16)  # all Delta zero: ties everywhere
    bulk_case(D, orc, Z, ALGOS, s=(1, 8), b=(1, 1), keyed=True)
    bulk_case(D, orc, Z, ALGOS, s=(1, 8), b=(1, 1), keyed=False)
    # +-32767 at n = 64 still fits the keyed form (|Delta| < 2^21 = 2^31 / 2^7 / 2^3)
    W64 = wl.dense_qubo(64, -32767, 32767, seed=2)
    bulk_case(D, orc, W64, ALGOS, s=(1, 8), b=(1, 1), keyed=True)


def compare_generation(ctx, so, n, tag):
    X, E, a, o = ctx.read_pools()
    oX, oE, oa, oo = so.pools()
    assert np.array_equal(E, oE), tag
    assert np.array_equal(wl.unpack_bits(X, n), oX), tag
    assert np.array_equal(a, oa) and np.array_equal(o, oo), tag
    Dg, ag, og, bX, bE, fl = ctx.read_generation()
    rX, rE, rf, ra, ro = so.results()
    assert np.array_equal(ag, ra) and np.array_equal(og, ro), tag
    assert np.array_equal(bE, rE) and np.array_equal(fl, rf), tag
    assert np.array_equal(wl.unpack_bits(bX, n), rX), tag
    sX, sd, sE = ctx.read_state()
    oX2, od2, oE2 = so.state()
    assert np.array_equal(wl.unpack_bits(sX, n), oX2) and np.array_equal(sd, od2), tag
    assert np.array_equal(sE, oE2), tag


@pytest.mark.parametrize("n,S,P,C,seed_mode", [(64, 32, 4, 64, 0), (20, 32, 4, 64, 0),
                                               (97, 48, 3, 10, 1), (200, 64, 64, 1, 0),
                                               (33, 16, 1, 8, 0)])
def test_generations_match_oracle(D, orc, n, S, P, C, seed_mode):
    W = wl.dense_qubo(n, -100, 100, seed=0)
    kw = dict(searches=S, pools=P, pool_cap=C, tabu=8, s=(1, 10), b=(1, 1), seed_mode=seed_mode)
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), 5)
    ctx.solve_begin(5)
    X, E, a, o = ctx.read_pools()
    oX, oE, oa, oo = so.pools()
    assert np.array_equal(wl.unpack_bits(X, n), oX) and np.array_equal(a, oa)
    for g in range(6):
        ctx.solve_generations(1)
        so.generation()
        compare_generation(ctx, so, n, f"generation {g}")
    st = ctx.solve_status()
    bx, be, bf, bg = so.best()
    assert (st["best_E"], st["flips"], st["generations"]) == (be, bf, bg)
    gx, ge = ctx.solve_best()
    assert ge == be and np.array_equal(gx, bx)
    # Tables V/VI counters
    for got, want in zip(ctx.stats(), so.stats()):
        assert np.array_equal(got, want)


def test_graph_generations_equal_kernel_by_kernel(D):
    """Generations replayed from the captured CUDA graph equal generations
    launched kernel by kernel, across a variant change (re-capture) and the
    stop condition (replays after it are no-ops)."""
    n = 300
    W = wl.dense_qubo(n, -100, 100, seed=12)
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), max_generations=9)
    outs = []
    for graphs in (True, False):
        ctx = D.Context(W, **kw)
        ctx.set_graphs(graphs)
        ctx.solve_begin(21)
        ctx.solve_generations(3)
        ctx.set_variant(2, 4)
        ctx.solve_generations(3)
        ctx.set_variant(1, 2)
        ctx.solve_generations(6)  # stops after 9
        outs.append((ctx.read_pools(), ctx.read_state(), ctx.solve_status(), ctx.solve_best()))
    assert outs[0][2] == outs[1][2] and outs[0][2]["generations"] == 9 and outs[0][2]["done"]
    for a, b in zip(outs[0][0] + outs[0][1] + outs[0][3], outs[1][0] + outs[1][1] + outs[1][3]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_graph_survives_new_weights_of_the_same_shape(D):
    """dabs_load_weights keeps the captured generation when no launch argument
    changes (same key bits, no sparse rows): the replay must read the new W."""
    n = 200
    W1, W2 = wl.dense_qubo(n, -100, 100, seed=41), wl.dense_qubo(n, -100, 100, seed=42)
    kw = dict(searches=32, pools=4, pool_cap=8, tabu=8, s=(1, 10), b=(1, 1), max_generations=4)
    ctx = D.Context(W1, **kw)
    ctx.solve(10**9, seed=1)
    ctx.load_weights(W2)
    got = ctx.solve(10**9, seed=2)
    ref = D.Context(W2, **kw)
    ref.set_graphs(False)
    want = ref.solve(10**9, seed=2)
    assert got[1:] == want[1:] and np.array_equal(got[0], want[0])


def test_checkpoint_restore_continues_exactly(D, orc):
    n, S = 90, 48
    W = wl.dense_qubo(n, -100, 100, seed=6)
    kw = dict(searches=S, pools=3, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0)
    a = D.Context(W, **kw)
    a.solve_begin(4)
    a.solve_generations(3)
    blob = a.checkpoint()
    a.solve_generations(4)
    want = (a.read_pools(), a.read_state(), a.solve_status(), a.solve_best(), a.stats())
    b = D.Context(W, **kw)
    b.solve_begin(99)  # a different solve in flight; the restore replaces all of it
    b.solve_generations(1)
    b.restore(blob)
    b.solve_generations(4)
    got = (b.read_pools(), b.read_state(), b.solve_status(), b.solve_best(), b.stats())
    assert got[2] == want[2]
    for g, w in zip(got[0] + got[1] + got[3] + got[4], want[0] + want[1] + want[3] + want[4]):
        assert np.array_equal(np.asarray(g), np.asarray(w))
    # the oracle, run straight through, agrees with the restored continuation
    so = orc.Solver(W, orc.make_params(**kw), 4)
    for _ in range(7):
        so.generation()
    bx, be, bf, bg = so.best()
    assert (got[2]["best_E"], got[2]["flips"], got[2]["generations"]) == (be, bf, bg)
    # a checkpoint only restores into a context of the same instance and parameters
    with pytest.raises(D.DabsError):
        D.Context(W, **dict(kw, tabu=9)).restore(blob)
    W2 = W.copy(); W2[0, 1] += 1; W2[1, 0] += 1
    with pytest.raises(D.DabsError):
        D.Context(W2, **kw).restore(blob)
    with pytest.raises(D.DabsError):
        b.restore(blob[:-1])


def test_offspring_and_merge_on_crafted_pools(D, orc):
    n, S, P, C = 150, 40, 4, 12
    W = wl.dense_qubo(n, -50, 50, seed=2)
    kw = dict(searches=S, pools=P, pool_cap=C)
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), 9)
    rng = np.random.default_rng(1)
    pX = rng.integers(0, 2, (P, C, n)).astype(np.uint8)
    pE = np.sort(rng.integers(-30, 30, (P, C)), axis=1).astype(np.int64)
    pa = rng.integers(0, 5, (P, C)).astype(np.int32)
    po = rng.integers(0, 8, (P, C)).astype(np.int32)
    ctx.solve_begin(9)
    ctx.write_pools(wl.pack_bits(pX), pE, pa, po)
    so.set_pools(pX, pE, pa, po)
    ctx.run_stage(D.STAGE_OFFSPRING)
    Dg, ag, og, _, _, _ = ctx.read_generation()
    oD, oa, oo = so.offspring(0)
    assert np.array_equal(wl.unpack_bits(Dg, n), oD)
    assert np.array_equal(ag, oa) and np.array_equal(og, oo)
    # merge crafted results (duplicates, equal energies, pool copies)
    rX = rng.integers(0, 2, (S, n)).astype(np.uint8)
    rE = rng.integers(-40, 40, S).astype(np.int64)
    rE[4] = -100
    rX[8] = rX[4]; rE[8] = -100
    rX[12] = rX[4]; rE[12] = -100
    rE[16] = -100
    rX[5] = pX[1, 0]; rE[5] = pE[1, 0]
    ra = rng.integers(0, 5, S).astype(np.int32)
    ro = rng.integers(0, 8, S).astype(np.int32)
    ctx.write_results(wl.pack_bits(rX), rE, np.ones(S, np.uint32), ra, ro)
    ctx.run_stage(D.STAGE_MERGE)
    ctx.run_stage(D.STAGE_FINALIZE)
    so.merge(rX, rE, ra, ro)
    X, E, a, o = ctx.read_pools()
    oX, oE, oa, oo = so.pools()
    assert np.array_equal(E, oE)
    assert np.array_equal(wl.unpack_bits(X, n), oX)
    assert np.array_equal(a, oa) and np.array_equal(o, oo)
    st = ctx.solve_status()
    assert st["best_E"] == -100 and st["flips"] == S and st["generations"] == 1


@pytest.mark.parametrize("n,budget,maxg,target", [(64, 10**9, 12, None), (20, 10**9, 60, "opt"),
                                                  (128, 30000, 0, None)])
def test_solve_matches_oracle(D, orc, n, budget, maxg, target):
    W = wl.dense_qubo(n, -100, 100, seed=0)
    tgt = wl.brute_force_min(W)[0] if target == "opt" else None
    kw = dict(searches=32, pools=4, pool_cap=64, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0,
              max_generations=maxg)
    ctx = D.Context(W, **kw)
    gx, ge, gf = ctx.solve(budget, seed=3, target=tgt)
    ox, oe, of, og = orc.solve(W, orc.make_params(**kw), budget, 3, target=tgt, threads=4)
    assert (ge, gf) == (oe, of) and np.array_equal(gx, ox)
    if tgt is not None:
        assert ge == tgt


def test_maxcut_workload_sampled_at_full_size(D, orc):
    """Sparse Max-Cut n=800, 1024 searches, P=4, C=100, b=10, s=1/10: one full
    generation on the GPU; 48 sampled searches re-run by the oracle."""
    n = 800
    W = wl.maxcut_qubo(n, 0.06, seed=1)
    kw = dict(searches=1024, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(10, 1), seed_mode=0)
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), 1)
    ctx.solve_begin(1)
    ctx.solve_generations(1)
    Dg, ag, og, bX, bE, fl = ctx.read_generation()
    oD, oa, oo = so.offspring(0)
    assert np.array_equal(wl.unpack_bits(Dg, n), oD) and np.array_equal(ag, oa)
    p = orc.make_params(**kw)
    gb = wl.unpack_bits(bX, n)
    z = np.zeros(n, np.uint8)
    for s in np.random.default_rng(0).choice(1024, 48, replace=False):
        r = orc.batch_search(W, p, 1, 0, int(s), z, np.diag(W).astype(np.int32), 0, oD[s], int(oa[s]))
        assert int(fl[s]) == r["flips"] and int(bE[s]) == r["best_E"]
        assert np.array_equal(gb[s], r["best_X"])
    # b*n = 8000 flips, except TwoNeighbor, which runs once (Section III-B)
    assert (fl[ag != 4] >= 8000).all() and (fl[ag == 4] >= 2 * n - 1).all()


def test_autotune_keeps_results(D, orc):
    n = 300
    W = wl.dense_qubo(n, -100, 100, seed=4)
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(2, 1), seed_mode=0,
              max_generations=3)
    ctx = D.Context(W, **kw)
    w, c, ns, table = ctx.autotune(1)
    assert 256 * w * c >= n and ns > 0 and table[ctx.variant_name()] == min(table.values())
    gx, ge, gf = ctx.solve(10**9, seed=2)
    ox, oe, of, _ = orc.solve(W, orc.make_params(**kw), 10**9, 2, threads=4)
    assert (ge, gf) == (oe, of) and np.array_equal(gx, ox)


@pytest.mark.parametrize("P,C,h,abs_mode", [(6, 1, 1, 0), (3, 2, 6, 0), (2, 4, 10, 1),
                                            (1, 4, 6, 1)])
def test_restart_and_abs_modes_match_oracle(D, orc, P, C, h, abs_mode):
    """Restart on merged pools (Section IV-B) and the ABS ablation (Section I)
    generation by generation against the oracle, restarts included."""
    n = 14
    W = wl.dense_qubo(n, -20, 20, seed=5)
    kw = dict(searches=8, pools=P, pool_cap=C, b=(2, 1), restart=1, restart_dist=h,
              abs_mode=abs_mode)
    ctx = D.Context(W, **kw)
    so = orc.Solver(W, orc.make_params(**kw), 3)
    ctx.solve_begin(3)
    for g in range(25):
        ctx.solve_generations(1)
        so.generation()
        compare_generation(ctx, so, n, f"generation {g}")
        assert ctx.restarts() == so.restarts()
    assert so.restarts() > 0
    st = ctx.solve_status()
    bx, be, bf, bg = so.best()
    assert (st["best_E"], st["flips"], st["generations"]) == (be, bf, bg)
    for got, want in zip(ctx.stats(), so.stats()):
        assert np.array_equal(got, want)


def test_abs_mode_solve_at_size_matches_oracle(D, orc):
    n = 300
    W = wl.dense_qubo(n, -100, 100, seed=8)
    kw = dict(searches=64, pools=2, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), abs_mode=1,
              restart=1, restart_dist=60, max_generations=6)
    ctx = D.Context(W, **kw)
    gx, ge, gf = ctx.solve(10**9, seed=5)
    ox, oe, of, og = orc.solve(W, orc.make_params(**kw), 10**9, 5, threads=4)
    assert (ge, gf) == (oe, of) and np.array_equal(gx, ox)


# ---------------------------------------------------------------- sparse rows
SPARSE = [1, 2]  # ROWS_SPARSE_SMEM, ROWS_SPARSE_GLOBAL


@pytest.mark.parametrize("rows", SPARSE)
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 100, 257, 800])
def test_sparse_rows_bulk_search_matches_oracle(D, orc, n, rows):
    """Step 3 from sparse rows (shared-memory copy or global memory, scattered
    into a scratch row) gives the oracle's trajectories: Max-Cut rows (+-2)
    and a resolution-256 Ising model (weights up to 1024, diagonal larger)."""
    bulk_case(D, orc, wl.maxcut_qubo(n, 0.06 if n > 50 else 0.15, seed=n), ALGOS, rows=rows)
    if n >= 5:
        m = min(2 * n, n * (n - 1) // 2)
        bulk_case(D, orc, wl.sparse_ising_qubo(n, m, 256, seed=n), ALGOS, rows=rows, seed=12)


@pytest.mark.parametrize("rows", SPARSE)
@pytest.mark.parametrize("variant", [(1, 1), (1, 2), (1, 4), (2, 1), (2, 2), (2, 4), (4, 1),
                                     (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (16, 1), (16, 2),
                                     (16, 4)])
def test_sparse_rows_every_variant_matches_oracle(D, orc, variant, rows):
    nw, ch = variant
    cap = 256 * nw * ch
    for n in sorted({max(5, cap // 3 + 5), cap - 7}):
        W = wl.sparse_ising_qubo(n, 2 * n, 256, seed=n + 2)
        ctx = ctx_for(D, W, searches=5, pools=1, pool_cap=4)
        ctx.set_variant(nw, ch)
        try:
            ctx.set_rows(rows)
        except D.DabsError as e:  # the shared-memory copy of a large instance does not fit
            assert rows == 1 and e.code == D.E_TOO_LARGE and n > 4000
            continue
        bulk_case(D, orc, W, [0, 1, 2, 3, 4], variant=variant, s=(1, 32), b=(1, 4), dflip=0.02,
                  rows=rows)


def test_sparse_rows_extreme_and_dense_weights(D, orc):
    """+-32767 weights through the scatter (both signs of sigma(x_i)), and a
    fully dense W held as sparse rows (every entry non-zero)."""
    n = 300
    W = wl.sparse_ising_qubo(n, 500, 1, seed=3).astype(np.int32)
    W[W != 0] = np.where(W[W != 0] > 0, 32767, -32767)
    W = W.astype(np.int16)
    for rows in SPARSE:
        bulk_case(D, orc, W, ALGOS, rows=rows, s=(1, 8), b=(1, 1))
    # n^2/4 off-diagonal non-zeros: the most that is stored; dense rows by default
    Wd = wl.sparse_ising_qubo(120, 1800, 256, seed=1)
    ctx = ctx_for(D, Wd, searches=4, pools=1)
    assert ctx.rows() == (0, 120 * 120 // 4)
    for rows in SPARSE:
        bulk_case(D, orc, Wd, ALGOS, rows=rows, s=(1, 8), b=(1, 1))


@pytest.mark.parametrize("keyed", [True, False])
@pytest.mark.parametrize("variant,n", [((1, 1), 1), ((1, 1), 5), ((1, 1), 64), ((1, 2), 257),
                                       ((1, 4), 300), ((1, 2), 320)])
def test_w_in_shared_memory_matches_oracle(D, orc, variant, n, keyed):
    """Rows of W from the shared-memory copy (negated for x_i = 0) give the
    oracle's trajectories, keyed and plain."""
    W = wl.dense_qubo(n, -100, 100, seed=n + 40) if keyed else wl.dense_qubo(n, -32767, 32767, seed=n)
    bulk_case(D, orc, W, ALGOS, variant=variant, rows=3, keyed=keyed)


def test_row_format_defaults_and_limits(D):
    kw = dict(searches=64, pools=4, pool_cap=16)
    mc = D.Context(wl.maxcut_qubo(800, 0.06, seed=1), **kw)
    assert mc.rows()[0] == D.ROWS_DENSE
    mc.set_rows(D.ROWS_SPARSE_SMEM)
    qa = D.Context(wl.sparse_ising_qubo(5627, 40279, 256, seed=6), **kw)
    assert qa.rows() == (D.ROWS_DENSE, 80558)
    qa.set_rows(D.ROWS_SPARSE_GLOBAL)  # 322 KB of entries: not in shared memory
    with pytest.raises(D.DabsError) as e:
        qa.set_rows(D.ROWS_SPARSE_SMEM)
    assert e.value.code == D.E_TOO_LARGE
    dn = D.Context(wl.dense_qubo(2000, -100, 100, seed=1), **kw)
    assert dn.rows() == (D.ROWS_DENSE, -1)  # more than n^2/4 non-zeros: not stored
    with pytest.raises(D.DabsError):
        dn.set_rows(D.ROWS_DENSE_SMEM)  # 8 MB of W
    sm = D.Context(wl.dense_qubo(330, -100, 100, seed=1), **kw)
    with pytest.raises(D.DabsError):
        sm.set_rows(D.ROWS_DENSE_SMEM)  # ld = 384: 253 KB
    sm = D.Context(wl.dense_qubo(320, -100, 100, seed=1), **kw)
    sm.set_rows(D.ROWS_DENSE_SMEM)  # 200 KB
    sm.set_variant(2, 2)  # one-warp variants only: falls back to dense rows
    assert sm.rows()[0] == D.ROWS_DENSE
    for mode in SPARSE:
        with pytest.raises(D.DabsError):
            dn.set_rows(mode)
    with pytest.raises(D.DabsError):
        mc.set_rows(4)
    # new weights of the same size: a format that no longer applies falls back
    mc.load_weights(wl.dense_qubo(800, -100, 100, seed=2))
    assert mc.rows() == (D.ROWS_DENSE, -1)
    mc.load_weights(wl.maxcut_qubo(800, 0.06, seed=1))
    mc.set_rows(D.ROWS_SPARSE_GLOBAL)
    assert mc.rows()[0] == D.ROWS_SPARSE_GLOBAL


@pytest.mark.parametrize("n,gen", [(800, "maxcut"), (2000, "ising")])
def test_sparse_rows_solve_equals_dense_and_oracle(D, orc, n, gen):
    """Whole generations (pools, state, global best) do not depend on the row
    format; the oracle agrees on sampled searches."""
    W = (wl.maxcut_qubo(n, 0.06, seed=1) if gen == "maxcut"
         else wl.sparse_ising_qubo(n, 6 * n, 16, seed=2))
    kw = dict(searches=256, pools=4, pool_cap=32, tabu=8, s=(1, 10), b=(2, 1), seed_mode=0)
    outs = []
    for mode in (0, 1, 2):
        ctx = D.Context(W, **kw)
        try:
            ctx.set_rows(mode)
        except D.DabsError:
            assert mode == 1
            continue
        ctx.solve_begin(7)
        ctx.solve_generations(3)
        outs.append((ctx.read_pools(), ctx.read_state(), ctx.solve_status(), ctx.solve_best(),
                     ctx.read_generation()))
    for o in outs[1:]:
        assert o[2] == outs[0][2]
        for a, b in zip(o[0] + o[1] + o[3] + o[4], outs[0][0] + outs[0][1] + outs[0][3] + outs[0][4]):
            assert np.array_equal(np.asarray(a), np.asarray(b))
    so = orc.Solver(W, orc.make_params(**kw), 7)
    for _ in range(2):
        so.generation(threads=16)
    oD, oa, oo = so.offspring(2)
    Dg, ag, og, bX, bE, fl = outs[-1][4]
    assert np.array_equal(wl.unpack_bits(Dg, n), oD) and np.array_equal(ag, oa)
    X2, d2, E2 = so.state()
    p = orc.make_params(**kw)
    gb = wl.unpack_bits(bX, n)
    for s in np.random.default_rng(0).choice(256, 12, replace=False):
        r = orc.batch_search(W, p, 7, 2, int(s), X2[s], d2[s], int(E2[s]), oD[s], int(oa[s]))
        assert int(fl[s]) == r["flips"] and int(bE[s]) == r["best_E"]
        assert np.array_equal(gb[s], r["best_X"])


# ---------------------------------------------------------------- Delta in shared memory
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 100, 257, 800, 1025, 2047, 3001])
def test_smem_delta_variant_matches_oracle(D, orc, n):
    """Variant (1, 0): one warp per search with the stored Delta (tabu bits
    offset by 2^30) in shared memory and rows fetched by bulk copies."""
    W = wl.dense_qubo(n, -1000, 1000, seed=n + 7)
    bulk_case(D, orc, W, ALGOS, variant=(1, 0), s=(1, 4), b=(2, 1))


@pytest.mark.parametrize("n", [8192, 16384])
def test_smem_delta_variant_at_large_n(D, orc, n):
    W = wl.dense_qubo(n, -100, 100, seed=n)
    bulk_case(D, orc, W, [0, 1, 2, 3, 4], variant=(1, 0), s=(1, 64), b=(1, 16), dflip=0.005)


def test_smem_delta_variant_generations_and_batch(D, orc):
    n = 1500
    W = wl.sparse_ising_qubo(n, 6 * n, 16, seed=3)
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0)
    ctx = D.Context(W, **kw)
    ctx.set_variant(1, 0)
    so = orc.Solver(W, orc.make_params(**kw), 5)
    ctx.solve_begin(5)
    for g in range(3):
        ctx.solve_generations(1)
        so.generation(threads=16)
        compare_generation(ctx, so, n, f"generation {g}")
    ctx.kernel_status()
    # batched with instances of other sizes on the same variant
    kw2 = dict(kw, max_generations=3)
    Ws = [W, wl.dense_qubo(700, -500, 500, seed=1), wl.dense_qubo(2100, -50, 50, seed=2)]
    ctxs = [D.Context(Wi, **kw2) for Wi in Ws]
    for c in ctxs:
        c.set_variant(1, 0)
    out = D.batch_solve(ctxs, [10**9] * 3, [1, 2, 3])
    for k, Wi in enumerate(Ws):
        alone = D.Context(Wi, **kw2)
        alone.set_variant(1, 0)
        a = alone.solve(10**9, k + 1)
        assert out[k][1] == a[1] and out[k][2] == a[2] and np.array_equal(out[k][0], a[0])
        plain = D.Context(Wi, **kw2).solve(10**9, k + 1)  # register variant, same result
        assert plain[1] == a[1] and plain[2] == a[2] and np.array_equal(plain[0], a[0])


def test_smem_delta_variant_at_the_delta_range_limit(D, orc):
    """int16 weights and n <= 16384 bound every Delta by 16384 * 32767 < 2^29,
    so the variant accepts every instance; at n = 16384 with weights near
    32767 the stored values (tabu offset 2^30 included) come within 2^14 of
    that bound and must still match the oracle."""
    n = 16384
    W = wl.dense_qubo(n, 32000, 32767, seed=5)
    bulk_case(D, orc, W, [0, 1, 2, 3, 4], variant=(1, 0), s=(1, 256), b=(1, 256), dflip=0.001, S=5)


def test_bounded_wait_runs_out_and_the_context_stays_usable(D, orc):
    """Variant (1, 0) waits for each row copy with a bounded mbarrier wait.
    The test hook withholds one copy: the wait runs out, the kernel sets the
    flag and returns, dabs_kernel_status reports DABS_E_TIMEOUT, and the same
    context then runs a batch search that matches the oracle."""
    n, S = 300, 2
    W = wl.dense_qubo(n, -100, 100, seed=31)
    ctx = ctx_for(D, W, searches=S, pools=1, pool_cap=4)
    ctx.set_variant(1, 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()
    X0 = np.zeros((S, n), np.uint8)
    dpad = np.zeros((S, ctx.ld), np.int32)
    dpad[:, :n] = np.diag(W)
    args = [t(wl.pack_bits(X0), np.int32), t(dpad, np.int32), t(np.zeros(S, np.int64), np.int64),
            t(wl.pack_bits(X0), np.int32), t(np.array([1, 2], np.uint8), np.uint8),
            torch.zeros((S, ctx.words), dtype=torch.int32, device="cuda"),
            torch.zeros(S, dtype=torch.int64, device="cuda"),
            torch.zeros(S, dtype=torch.int32, device="cuda")]
    ctx.test_stall_next_search()
    ctx.bulk_search_dev(3, 0, *args)
    with pytest.raises(D.DabsError) as e:
        ctx.kernel_status()
    assert e.value.code == D.E_TIMEOUT
    ctx.kernel_status()  # the flag was cleared
    ctx.bulk_search_dev(3, 0, *args)  # the same context, no hook: a normal batch search
    ctx.kernel_status()
    p = orc.make_params(searches=1, pools=1, pool_cap=4, tabu=8, s=(1, 4), b=(2, 1))
    for s in range(S):
        r = orc.batch_search(W, p, 3, 0, s, X0[s], np.diag(W).astype(np.int32), 0, X0[s], [1, 2][s])
        assert int(args[7][s]) == r["flips"] and int(args[6][s]) == r["best_E"]
    with pytest.raises(D.DabsError):
        D.Context(W, searches=4, pools=1).test_stall_next_search()  # register variants: no hook
