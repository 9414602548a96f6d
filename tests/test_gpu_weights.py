"""GPU: residency of an instance (W of Eq. (1) in global memory, Section V-A).
W is checked and measured on the device after one DMA.  The measurements are
compared with their definitions computed here in numpy: the stored sparse-row
count (off-diagonal non-zeros, kept while at most max(n^2/4, 64)) and the key
width of the keyed Delta form (needs (2R + 2) * 2^kb < 2^31 with R the largest
row sum of |W|).  W, -W and the diagonal are compared through Eq. (2)/(3)
against the oracle.  A rejected W must leave the context as it was, and a
checkpoint is tied to the W loaded at the time it is taken and restored.
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


KW = dict(searches=8, pools=2, pool_cap=4, tabu=8, s=(1, 4), b=(2, 1))


def expected_nnz(W):
    n = W.shape[0]
    off = int(np.count_nonzero(W)) - int(np.count_nonzero(np.diag(W)))
    return off if off <= max(n * n // 4, 64) else -1


def expected_key_bits(W):
    n = W.shape[0]
    R = int(np.abs(W.astype(np.int64)).sum(axis=1).max())
    kb = (n - 1).bit_length() + 1
    return kb if ((2 * R + 2) << kb) < 2**31 - 1 else 0


def check_instance(D, orc, ctx, W, seed):
    n = W.shape[0]
    assert ctx.rows()[1] == expected_nnz(W)
    assert ctx.keyed()[1] == expected_key_bits(W)
    rng = np.random.default_rng(seed)
    for X in [np.zeros(n, np.uint8), np.ones(n, np.uint8),
              (rng.random(n) < 0.5).astype(np.uint8)]:
        assert ctx.energy(X) == orc.energy(W, X)
        assert np.array_equal(ctx.delta(X), orc.delta(W, X))


def instances(n):
    """Dense, sparse and extreme-weight instances of one size."""
    out = [wl.dense_qubo(n, -100, 100, seed=n), wl.dense_qubo(n, -32767, 32767, seed=n + 1)]
    if n >= 8:
        out.append(wl.maxcut_qubo(n, 0.06, seed=n + 2))
    one = np.zeros((n, n), np.int16)
    one[n - 1, n - 1] = 7
    out.append(one)
    return out


@pytest.mark.parametrize("n", [1, 2, 31, 33, 77, 100, 200, 800, 2000, 4100])
def test_measurements_match_their_definitions(D, orc, n):
    Ws = instances(n)
    ctx = D.Context(Ws[0], **KW)
    check_instance(D, orc, ctx, Ws[0], 1)
    for q, W in enumerate(Ws[1:] + Ws[:1]):  # reload every instance, then the first again
        ctx.load_weights(W)
        check_instance(D, orc, ctx, W, 2 + q)
        fresh = D.Context(W, **KW)
        assert fresh.rows()[1] == ctx.rows()[1] and fresh.keyed()[1] == ctx.keyed()[1]


def test_sparse_ising_measurements(D, orc):
    W = wl.sparse_ising_qubo(5627, 40279, 256, seed=6)
    ctx = D.Context(wl.dense_qubo(5627, -100, 100, seed=1), **KW)
    assert ctx.rows()[1] == -1
    ctx.load_weights(W)
    check_instance(D, orc, ctx, W, 3)


def test_rejected_weights_leave_the_context_unchanged(D, orc):
    n = 77
    W = wl.dense_qubo(n, -100, 100, seed=9)
    kw = dict(KW, max_generations=3)
    ctx = D.Context(W, **kw)
    before = ctx.solve(10**9, seed=5)
    state = (ctx.rows(), ctx.keyed())
    Wa = W.copy()
    Wa[76, 3] += 1  # the last row's tile against the first column's
    with pytest.raises(D.DabsError) as e:
        ctx.load_weights(Wa)
    assert e.value.code == D.E_NOT_SYMMETRIC and "W[3][76] != W[76][3]" in str(e.value)
    Wd = W.copy()
    Wd[40, 40] = -32768
    with pytest.raises(D.DabsError) as e:
        ctx.load_weights(Wd)
    assert e.value.code == D.E_INVALID_ARG and "W[40][40] = -32768" in str(e.value)
    Wo = W.copy()
    Wo[5, 70] = Wo[70, 5] = -32768
    with pytest.raises(D.DabsError) as e:
        ctx.load_weights(Wo)
    assert e.value.code == D.E_INVALID_ARG and "W[5][70] = -32768" in str(e.value)
    Wl = W.copy()
    Wl[70, 5] = -32768  # only below the diagonal: an asymmetric pair first
    with pytest.raises(D.DabsError) as e:
        ctx.load_weights(Wl)
    assert e.value.code == D.E_NOT_SYMMETRIC
    assert (ctx.rows(), ctx.keyed()) == state
    check_instance(D, orc, ctx, W, 4)
    after = ctx.solve(10**9, seed=5)
    assert after[1:] == before[1:] and np.array_equal(after[0], before[0])
    # the same solve on a context that never saw a rejected W
    ref = D.Context(W, **kw).solve(10**9, seed=5)
    assert ref[1:] == before[1:] and np.array_equal(ref[0], before[0])


def test_reloaded_sparse_rows_equal_a_fresh_context(D):
    n = 800
    Wm = wl.maxcut_qubo(n, 0.06, seed=1)
    kw = dict(searches=64, pools=4, pool_cap=16, tabu=8, s=(1, 10), b=(1, 1), max_generations=3)
    fresh = D.Context(Wm, **kw)
    reloaded = D.Context(wl.dense_qubo(n, -100, 100, seed=2), **kw)
    assert reloaded.rows()[1] == -1
    reloaded.load_weights(Wm)
    for mode in (D.ROWS_SPARSE_SMEM, D.ROWS_SPARSE_GLOBAL):
        fresh.set_rows(mode)
        reloaded.set_rows(mode)
        a, b = fresh.solve(10**9, seed=8), reloaded.solve(10**9, seed=8)
        assert a[1:] == b[1:] and np.array_equal(a[0], b[0])
    fresh.set_rows(D.ROWS_DENSE)
    dense = fresh.solve(10**9, seed=8)
    assert dense[1:] == a[1:] and np.array_equal(dense[0], a[0])


def test_checkpoint_follows_the_loaded_weights(D):
    n = 90
    W1, W2 = wl.dense_qubo(n, -100, 100, seed=6), wl.dense_qubo(n, -100, 100, seed=7)
    kw = dict(searches=32, pools=2, pool_cap=8, tabu=8, s=(1, 10), b=(1, 1))
    a = D.Context(W1, **kw)
    a.solve_begin(3)
    a.solve_generations(2)
    blob = a.checkpoint()
    a.solve_generations(2)
    want = (a.solve_status(), a.solve_best())
    a.load_weights(W2)
    with pytest.raises(D.DabsError):
        a.restore(blob)
    a.load_weights(W1)
    a.restore(blob)
    a.solve_generations(2)
    got = (a.solve_status(), a.solve_best())
    assert got[0] == want[0] and got[1][1] == want[1][1] and np.array_equal(got[1][0], want[1][0])
    b = D.Context(W2, **kw)
    b.load_weights(W1)
    b.restore(blob)
    b.solve_generations(2)
    assert b.solve_status() == want[0]
