"""Pins of the oracle's definitions against facts fixed by the paper and by
mathematics (no GPU): the worked Ising/QUBO example of Section I-A, the
Ising<->QUBO identity, Eq. (2) against brute-force definitions, Eq. (3)
against E(f_k X) - E(X), Philox known answers, and the problem reductions of
Section II."""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2207_03069_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def ising_H(J, h, S):
    """Eq. (1): sum over undirected edges (i<j) of J_ij s_i s_j + sum h_i s_i."""
    S = np.asarray(S, np.int64)
    return int(np.triu(J, 1).dot(S).dot(S) + h.dot(S))


def energy_def(W, X):
    """Eq. (2) written as a sum over pairs i<=j (independent of the oracle)."""
    W = np.asarray(W, np.int64)
    X = np.asarray(X, np.int64)
    return int(sum(W[i, j] * X[i] * X[j] for i in range(len(X)) for j in range(i, len(X))))


def fig1():
    g = json.load(open(os.path.join(GOLD, "fig1_reconstruction.json")))
    n = g["n"]
    J = np.zeros((n, n), np.int64)
    for i, j, v in g["J_edges"]:
        J[i, j] = J[j, i] = v
    return g, J, np.asarray(g["h"], np.int64)


def test_fig1_worked_example(orc):
    g, J, h = fig1()
    n = g["n"]
    W, offset = wl.ising_to_qubo(J, h)
    assert offset == g["offset"] == 6
    Hs, Es = {}, {}
    for bits in itertools.product([0, 1], repeat=n):
        X = np.asarray(bits, np.uint8)
        S = 2 * X.astype(np.int64) - 1
        Hs[bits] = ising_H(J, h, S)
        Es[bits] = orc.energy(W, X)
        assert Es[bits] == Hs[bits] + 6  # E(X) = H(S) + 6 for every pair
    xo = tuple(g["X_opt"])
    assert min(Es.values()) == Es[xo] == g["E_opt"] == -8
    assert min(Hs.values()) == Hs[xo] == g["H_opt"] == -14
    assert sum(1 for v in Es.values() if v == -8) == 1
    assert tuple(2 * np.asarray(xo) - 1) == tuple(g["S_opt"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ising_qubo_identity(orc, seed):
    J, h = wl.random_ising(10, r=3, density=0.5, seed=seed)
    W, offset = wl.ising_to_qubo(J, h)
    W16 = W.astype(np.int16)
    for bits in itertools.product([0, 1], repeat=10):
        X = np.asarray(bits, np.uint8)
        assert orc.energy(W16, X) == ising_H(J, h, 2 * X.astype(np.int64) - 1) + offset


@pytest.mark.parametrize("r", [1, 16, 256])
def test_sparse_ising_generator(orc, r):
    """Section II-C resolution-r model on random edges: value sets, the edge
    count, and E(X) = H(S) + offset over all 2^10 vectors."""
    n, m = 10, 17
    I, Jx, J, h = wl.sparse_ising(n, m, r, seed=r)
    assert len(set(zip(I.tolist(), Jx.tolist()))) == m and (I < Jx).all()
    assert (np.abs(J) >= 1).all() and (np.abs(J) <= r).all()
    assert (np.abs(h) >= 1).all() and (np.abs(h) <= 4 * r).all()
    Jd = np.zeros((n, n), np.int64)
    Jd[I, Jx] = J
    Jd = Jd + Jd.T
    W = wl.sparse_ising_qubo(n, m, r, seed=r)
    W2, offset = wl.ising_to_qubo(Jd, h)
    assert np.array_equal(W, W2.astype(np.int16))
    for bits in itertools.product([0, 1], repeat=n):
        X = np.asarray(bits, np.uint8)
        assert orc.energy(W, X) == ising_H(Jd, h, 2 * X.astype(np.int64) - 1) + offset


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (33, 3)])
def test_energy_matches_definition(orc, n, seed):
    W = wl.dense_qubo(n, -1000, 1000, seed)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        X = rng.integers(0, 2, n).astype(np.uint8)
        assert orc.energy(W, X) == energy_def(W, X)


@pytest.mark.parametrize("n,seed", [(1, 0), (5, 1), (37, 2), (64, 3)])
def test_delta_closed_form_is_energy_difference(orc, n, seed):
    """Eq. (3) against the definition Delta_k = E(f_k X) - E(X)."""
    W = wl.dense_qubo(n, -30000, 30000, seed)
    rng = np.random.default_rng(seed + 100)
    for _ in range(10):
        X = rng.integers(0, 2, n).astype(np.uint8)
        d = orc.delta(W, X)
        e0 = energy_def(W, X)
        for k in range(n):
            Xf = X.copy()
            Xf[k] ^= 1
            assert d[k] == energy_def(W, Xf) - e0


def test_zero_vector_delta_is_diagonal(orc):
    """Section III-A: at X = 0, E = 0 and Delta_k = W_kk."""
    W = wl.dense_qubo(50, -100, 100, 9)
    X = np.zeros(50, np.uint8)
    assert orc.energy(W, X) == 0
    assert np.array_equal(orc.delta(W, X), np.diag(W).astype(np.int32))


def test_philox_known_answers(orc):
    g = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for v in g["vectors"]:
        out = orc.philox([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert ["%08x" % x for x in out] == v["out"]


def test_brute_force_helper_agrees_with_oracle_energy(orc):
    W = wl.dense_qubo(12, -100, 100, 5)
    emin, xmin, _ = wl.brute_force_min(W)
    assert orc.energy(W, xmin) == emin
    allE = [orc.energy(W, np.asarray(b, np.uint8)) for b in itertools.product([0, 1], repeat=12)]
    assert min(allE) == emin


def test_maxcut_reduction(orc):
    """Section II-A: E(X) = -cut(X) for every X."""
    n = 12
    edges, w = wl.maxcut_graph(n, 0.4, seed=7)
    W = wl.maxcut_qubo(n, 0.4, seed=7)
    for bits in itertools.product([0, 1], repeat=n):
        X = np.asarray(bits, np.uint8)
        assert orc.energy(W, X) == -wl.cut_value(edges, w, X)


def test_tsp_qap_reduction(orc):
    """Section II-B: E = C(g) - n p for feasible one-hot X, E >= -(n-1) p else."""
    nc = 4
    W, dist, p = wl.tsp_qubo(nc, 1000, seed=2)
    N = nc * nc
    tours = {}
    for perm in itertools.permutations(range(nc)):
        # facility = tour position t, location = city perm[t]
        tours[perm] = sum(dist[perm[t], perm[(t + 1) % nc]] for t in range(nc))
    feasible = {}
    for perm, cost in tours.items():
        X = np.zeros(N, np.uint8)
        for t in range(nc):
            X[t * nc + perm[t]] = 1
        feasible[X.tobytes()] = cost
        assert orc.energy(W, X) == cost - nc * p
    allE = []
    for bits in itertools.product([0, 1], repeat=N):
        X = np.asarray(bits, np.uint8)
        if X.tobytes() in feasible:
            continue
        allE.append(orc.energy(W, X))
    assert min(allE) >= -(nc - 1) * p
    assert min(tours.values()) - nc * p < min(allE)
