"""The allocation-free batch search (dabs_bulk_search_noalloc) against the
context-based one (dabs_bulk_search_dev): identical outputs on two calls in a
row, through the C ABI, one slot also against the oracle directly; the calls
leave the device's free memory unchanged; sizes beyond the static scratch and
a W entry of -32768 are refused.  Kept in a file of its own that runs last."""
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
    # a first call loads the library's module with the static array; the
    # calls compared below must then leave the device's free memory as it is
    warm = state(X0)
    wb = [torch.zeros((S, ctx.words), dtype=torch.int32, device="cuda"),
          torch.zeros(S, dtype=torch.int64, device="cuda"),
          torch.zeros(S, dtype=torch.int32, device="cuda")]
    dabs.bulk_search_noalloc(Wd, n, ld, ctx.params, 1, 0, warm[0], warm[1], warm[2], warm[0],
                             algo, *wb, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for call, (seed, g) in enumerate([(21, 3), (22, 4)]):
        Dh = (rng.random((S, n)) < 0.5).astype(np.uint8)
        Dt = torch.from_numpy(wl.pack_bits(Dh).view(np.int32)).cuda()
        Xh = wl.unpack_bits(new[0].cpu().numpy().view(np.uint32), n)
        dh = new[1].cpu().numpy()[:, :n]
        Eh = new[2].cpu().numpy()
        outs = []
        for st, use_noalloc in ((ref, False), (new, True)):
            bX = torch.zeros((S, ctx.words), dtype=torch.int32, device="cuda")
            bE = torch.zeros(S, dtype=torch.int64, device="cuda")
            fl = torch.zeros(S, dtype=torch.int32, device="cuda")
            if use_noalloc:
                torch.cuda.synchronize()
                free_before = torch.cuda.mem_get_info()[0]
                dabs.bulk_search_noalloc(Wd, n, ld, ctx.params, seed, g, st[0], st[1], st[2], Dt,
                                         algo, bX, bE, fl, torch.cuda.current_stream())
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free_before, "the call allocated"
            else:
                ctx.bulk_search_dev(seed, g, st[0], st[1], st[2], Dt, algo, bX, bE, fl)
            torch.cuda.synchronize()
            outs.append((bX.cpu(), bE.cpu(), fl.cpu()))
        for a, b in zip(outs[0], outs[1]):
            assert torch.equal(a, b), f"call {call}"
        for a, b in zip(ref, new):
            assert torch.equal(a.cpu(), b.cpu()), f"call {call}"
        assert (outs[1][2] > 0).all()
        # one slot of each algorithm against the oracle directly
        from oracle import oracle as orc
        p = orc.make_params(**kw)
        gb = wl.unpack_bits(outs[1][0].numpy().view(np.uint32), n)
        for si in range(5):
            r = orc.batch_search(W, p, seed, g, si, Xh[si], dh[si], int(Eh[si]), Dh[si], si % 5)
            assert int(outs[1][1][si]) == r["best_E"] and int(outs[1][2][si]) == r["flips"]
            assert np.array_equal(gb[si], r["best_X"])
    # sizes beyond the static scratch are refused with a clear error
    big = torch.zeros((2048, 2048), dtype=torch.int16, device="cuda")
    with pytest.raises(dabs.DabsError) as e:
        dabs.bulk_search_noalloc(big, 2048, 2048, ctx.params, 1, 0, ref[0], ref[1], ref[2], Dt,
                                 algo, bX, bE, fl)
    assert e.value.code == dabs.E_TOO_LARGE
    many = 16385
    with pytest.raises(dabs.DabsError) as e:
        dabs.bulk_search_noalloc(Wd, n, ld, ctx.params, 1, 0,
                                 torch.zeros((many, ctx.words), dtype=torch.int32, device="cuda"),
                                 torch.zeros((many, ld), dtype=torch.int32, device="cuda"),
                                 torch.zeros(many, dtype=torch.int64, device="cuda"),
                                 torch.zeros((many, ctx.words), dtype=torch.int32, device="cuda"),
                                 torch.zeros(many, dtype=torch.uint8, device="cuda"),
                                 torch.zeros((many, ctx.words), dtype=torch.int32, device="cuda"),
                                 torch.zeros(many, dtype=torch.int64, device="cuda"),
                                 torch.zeros(many, dtype=torch.int32, device="cuda"))
    assert e.value.code == dabs.E_TOO_LARGE
    # an entry of -32768 is refused on the device: no slot is searched
    Wbad = Wp.copy()
    Wbad[7, 9] = Wbad[9, 7] = -32768
    Wbd = torch.from_numpy(Wbad).cuda()
    fl.fill_(7)
    bE.fill_(0)
    dabs.bulk_search_noalloc(Wbd, n, ld, ctx.params, 5, 1, ref[0], ref[1], ref[2], Dt, algo, bX,
                             bE, fl, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert (fl.cpu() == 0).all() and (bE.cpu() == np.iinfo(np.int64).max).all()
