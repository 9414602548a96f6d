"""Tensor-core (tcgen05) recompute of Delta and E against the CUDA-core kernel
and the oracle: bit-exact on ragged sizes (several 128-wide tiles plus a
ragged tail), extreme weights, and inside whole solves with recompute
seeding."""
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


# wmax 32767: two bf16 limbs; 2048 and 1000: W itself as one fp16 operand
# (exact for |W| <= 2048 with n |W| < 2^24); 2049 just past that bound
@pytest.mark.parametrize("n,count,wmax", [(64, 1, 32767), (100, 5, 32767), (128, 128, 32767),
                                          (129, 130, 32767), (800, 256, 32767),
                                          (1000, 77, 32767), (2048, 256, 32767),
                                          (4100, 200, 32767), (8192, 64, 32767),
                                          (300, 300, 1000), (4096, 256, 1000), (8191, 260, 2048),
                                          (700, 129, 2049), (16384, 40, 1000)])
def test_recompute_matches_cuda_cores_and_oracle(D, orc, n, count, wmax):
    W = wl.dense_qubo(n, -wmax, wmax, seed=n + 7)
    W[0, 0] = wmax  # the bound itself occurs
    ctx = D.Context(W, searches=max(count, 1), pools=1, pool_cap=1)
    rng = np.random.default_rng(n)
    dens = rng.random((count, 1))
    Xs = (rng.random((count, n)) < dens).astype(np.uint8)
    Xs[0] = 1  # all-ones row: largest partial sums
    Xd = torch.from_numpy(wl.pack_bits(Xs).view(np.int32)).cuda()
    Etc = torch.zeros(count, dtype=torch.int64, device="cuda")
    dtc = torch.zeros((count, n + 5), dtype=torch.int32, device="cuda")
    ctx.recompute_dev(Xd, Etc, dtc)
    ctx.kernel_status()
    Ecc = torch.zeros(count, dtype=torch.int64, device="cuda")
    dcc = torch.zeros((count, n + 5), dtype=torch.int32, device="cuda")
    ctx.energy_delta_dev(Xd, Ecc, dcc)
    torch.cuda.synchronize()
    assert torch.equal(Etc, Ecc) and torch.equal(dtc[:, :n], dcc[:, :n])
    for v in sorted(set([0, count - 1, count // 2])):
        assert int(Etc[v]) == orc.energy(W, Xs[v])
        assert np.array_equal(dtc[v, :n].cpu().numpy(), orc.delta(W, Xs[v]))
    # a row stride that is a multiple of 4 takes the 16-byte-store epilogue
    ld4 = (n + 3) // 4 * 4 + 4
    dv = torch.full((count, ld4), -7, dtype=torch.int32, device="cuda")
    Ev = torch.zeros(count, dtype=torch.int64, device="cuda")
    ctx.recompute_dev(Xd, Ev, dv)
    ctx.kernel_status()
    torch.cuda.synchronize()
    assert torch.equal(Ev, Ecc) and torch.equal(dv[:, :n], dcc[:, :n])
    assert bool((dv[:, n:] == -7).all())  # nothing written past n


def test_solve_with_tensor_core_seeding_matches_oracle(D, orc):
    n = 300
    W = wl.dense_qubo(n, -1000, 1000, seed=5)
    kw = dict(searches=256, pools=4, pool_cap=32, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1,
              max_generations=4)
    ctx = D.Context(W, **kw)
    gx, ge, gf = ctx.solve(10**9, seed=6)
    ctx.kernel_status()
    ox, oe, of, _ = orc.solve(W, orc.make_params(**kw), 10**9, 6, threads=8)
    assert (ge, gf) == (oe, of) and np.array_equal(gx, ox)
    ctx.set_recompute(0)
    gx2, ge2, gf2 = ctx.solve(10**9, seed=6)
    assert (ge2, gf2) == (ge, gf) and np.array_equal(gx2, gx)
