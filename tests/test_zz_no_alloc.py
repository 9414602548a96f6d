"""The allocation-free batch search (dabs_bulk_search_noalloc) against the
context-based one (dabs_bulk_search_dev): identical outputs on two calls in a
row, through the C ABI.  Kept in a file of its own that runs last."""
import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_bulk_search_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03069_gb300 import build, dabs
    build.build()
    n, S = 300, 40
    W = wl.dense_qubo(n, -1000, 1000, seed=12)
    kw = dict(searches=S, pools=1, pool_cap=4, tabu=8, s=(1, 8), b=(2, 1), seed_mode=0)
    ctx = dabs.Context(W, **kw)
    ld = ctx.ld
    Wp = np.zeros((n, ld), np.int16)
    Wp[:, :n] = W
    Wd = torch.from_numpy(Wp).cuda()
    rng = np.random.default_rng(3)
    algo = torch.from_numpy(np.arange(S, dtype=np.uint8) % 5).cuda()

    def state(X0):
        from oracle import oracle as orc
        d = np.zeros((S, ld), np.int32)
        d[:, :n] = np.stack([orc.delta(W, x) for x in X0])
        E = np.array([orc.energy(W, x) for x in X0], np.int64)
        return [torch.from_numpy(wl.pack_bits(X0).view(np.int32)).cuda(),
                torch.from_numpy(d).cuda(), torch.from_numpy(E).cuda()]

    X0 = (rng.random((S, n)) < 0.5).astype(np.uint8)
    ref, new = state(X0), state(X0)
    for call, (seed, g) in enumerate([(21, 3), (22, 4)]):
        Dt = torch.from_numpy(wl.pack_bits((rng.random((S, n)) < 0.5).astype(np.uint8))
                              .view(np.int32)).cuda()
        outs = []
        for st, use_noalloc in ((ref, False), (new, True)):
            bX = torch.zeros((S, ctx.words), dtype=torch.int32, device="cuda")
            bE = torch.zeros(S, dtype=torch.int64, device="cuda")
            fl = torch.zeros(S, dtype=torch.int32, device="cuda")
            if use_noalloc:
                dabs.bulk_search_noalloc(Wd, n, ld, ctx.params, seed, g, st[0], st[1], st[2], Dt,
                                         algo, bX, bE, fl, torch.cuda.current_stream())
            else:
                ctx.bulk_search_dev(seed, g, st[0], st[1], st[2], Dt, algo, bX, bE, fl)
            torch.cuda.synchronize()
            outs.append((bX.cpu(), bE.cpu(), fl.cpu()))
        for a, b in zip(outs[0], outs[1]):
            assert torch.equal(a, b), f"call {call}"
        for a, b in zip(ref, new):
            assert torch.equal(a.cpu(), b.cpu()), f"call {call}"
        assert (outs[1][2] > 0).all()
    # sizes beyond the static scratch are refused with a clear error
    big = torch.zeros((2048, 2048), dtype=torch.int16, device="cuda")
    with pytest.raises(dabs.DabsError) as e:
        dabs.bulk_search_noalloc(big, 2048, 2048, ctx.params, 1, 0, ref[0], ref[1], ref[2], Dt,
                                 algo, bX, bE, fl)
    assert e.value.code == dabs.E_TOO_LARGE
