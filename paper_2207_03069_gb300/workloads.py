"""Seeded synthetic QUBO instances and bit-layout helpers.

This module is shared by the tests, the benchmark and the oracle checks.  It
only builds problem instances (weight matrices) and converts bit layouts; it
holds none of the search method's arithmetic.  Every generator draws from
``numpy.random.default_rng(seed)`` so an instance is fixed by its arguments.

Weight convention (Section I-A, Eq. (2), each pair once): W is symmetric int16
and E(X) = sum_i W_ii x_i + sum_{i<j} W_ij x_i x_j.
"""
from __future__ import annotations

import math

import numpy as np


def symmetric_from_upper(U: np.ndarray) -> np.ndarray:
    """Mirror the upper triangle (diagonal included) of U into a symmetric matrix."""
    up = np.triu(U).astype(np.int16, copy=False)
    return up + np.triu(up, 1).T


def dense_qubo(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Dense symmetric W with i.i.d. integer weights uniform in [lo, hi]
    (upper triangle incl. diagonal drawn, then mirrored)."""
    if not (-32768 <= lo <= hi <= 32767):
        raise ValueError("weights must fit int16")
    rng = np.random.default_rng(seed)
    U = rng.integers(lo, hi + 1, size=(n, n), dtype=np.int32)
    return symmetric_from_upper(U)


def maxcut_graph(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p) with edge weights +-1 equiprobable.
    Returns (edges [m,2] with i<j, weights [m])."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    w = np.where(rng.random(iu.size) < 0.5, -1, 1)[keep]
    return np.stack([iu[keep], ju[keep]], 1), w.astype(np.int64)


def maxcut_qubo(n: int, p: float, seed: int) -> np.ndarray:
    """Section II-A: each edge contributes w (2 x_i x_j - x_i - x_j), so the
    minimum energy is minus the maximum cut.  Per-pair-once form:
    W_ij = 2 w_ij, W_ii = -sum_j w_ij."""
    edges, w = maxcut_graph(n, p, seed)
    W = np.zeros((n, n), np.int64)
    W[edges[:, 0], edges[:, 1]] = 2 * w
    W[edges[:, 1], edges[:, 0]] = 2 * w
    np.add.at(W, (edges[:, 0], edges[:, 0]), -w)
    np.add.at(W, (edges[:, 1], edges[:, 1]), -w)
    return W.astype(np.int16)


def cut_value(edges: np.ndarray, w: np.ndarray, X: np.ndarray) -> int:
    X = np.asarray(X).astype(np.int64)
    return int(np.sum(w * (X[edges[:, 0]] != X[edges[:, 1]])))


def tsp_cities(ncity: int, grid: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, grid, size=(ncity, 2), dtype=np.int64)


def tsp_distances(xy: np.ndarray) -> np.ndarray:
    """Integer Euclidean distances, rounded half up (TSPLIB 'nint')."""
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    d = np.floor(np.sqrt(d2.astype(np.float64)) + 0.5).astype(np.int64)
    return d


def qap_qubo(flow: np.ndarray, dist: np.ndarray, penalty: int) -> np.ndarray:
    """Section II-B one-hot QAP encoding with N = n^2 bits, bit <i,j> = i*n + j
    meaning facility i at location j.  The paper's matrix counts every ordered
    pair; folded into the per-pair-once symmetric form (W'_uv = W_uv + W_vu)
    so that E = C(g) - n p holds for every feasible X."""
    n = flow.shape[0]
    N = n * n
    i = np.repeat(np.arange(n), n)
    j = np.tile(np.arange(n), n)
    same_i = i[:, None] == i[None, :]
    same_j = j[:, None] == j[None, :]
    Wo = np.where(~same_i & ~same_j, flow[i][:, i] * dist[j][:, j], 0).astype(np.int64)
    Wo = np.where(same_i ^ same_j, penalty, Wo)
    Wo = np.where(same_i & same_j, -penalty, Wo)
    W = Wo + Wo.T
    W[np.arange(N), np.arange(N)] = -penalty
    if np.abs(W).max() > 32767:
        raise ValueError("QAP weights exceed int16")
    return W.astype(np.int16)


def tsp_qubo(ncity: int, grid: int, seed: int):
    """TSP as a QAP with a circular flow l(t, t+1 mod n) = 1 (Section II-B):
    facility = tour position, location = city.  Penalty p = 2 * max distance.
    Returns (W, dist, penalty)."""
    xy = tsp_cities(ncity, grid, seed)
    dist = tsp_distances(xy)
    flow = np.zeros((ncity, ncity), np.int64)
    flow[np.arange(ncity), (np.arange(ncity) + 1) % ncity] = 1
    p = 2 * int(dist.max())
    return qap_qubo(flow, dist, p), dist, p


def ising_to_qubo(J: np.ndarray, h: np.ndarray):
    """Ising (Section I-A, Eq. (1)) to QUBO with s = 2x - 1.
    J is symmetric with zero diagonal (each edge stored twice), h the biases.
    Returns (W, offset) with E(X) = H(S) + offset."""
    J = np.asarray(J, np.int64)
    h = np.asarray(h, np.int64)
    n = h.size
    W = 4 * J.copy()
    W[np.arange(n), np.arange(n)] = 2 * h - 2 * J.sum(1)
    offset = int(h.sum() - np.triu(J, 1).sum())
    return W, offset


def random_ising(n: int, r: int, density: float, seed: int):
    """Sparse random Ising model of resolution r (Section II-C): non-zero
    interactions in +-{1..r}, non-zero biases in +-{1..4r}, uniform."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < density
    vals = rng.integers(1, r + 1, size=keep.sum()) * np.where(rng.random(keep.sum()) < 0.5, -1, 1)
    J = np.zeros((n, n), np.int64)
    J[iu[keep], ju[keep]] = vals
    J = J + J.T
    h = rng.integers(1, 4 * r + 1, size=n) * np.where(rng.random(n) < 0.5, -1, 1)
    return J, h


def sparse_ising(n: int, edges: int, r: int, seed: int):
    """Sparse random Ising model of resolution r on `edges` distinct random
    edges (Section II-C; the quantum-annealer simulation problems use 5,627
    nodes and 40,279 edges): interactions uniform over the non-zero integers
    in [-r, r], biases over the non-zero integers in [-4r, 4r].
    Returns (i, j, J, h) with i < j per edge."""
    rng = np.random.default_rng(seed)
    if edges > n * (n - 1) // 2:
        raise ValueError("more edges than pairs")
    seen: set = set()
    I, Jx = [], []
    while len(I) < edges:
        a = rng.integers(0, n, size=2 * (edges - len(I)) + 16)
        b = rng.integers(0, n, size=a.size)
        for x, y in zip(a.tolist(), b.tolist()):
            k = (min(x, y), max(x, y))
            if x == y or k in seen:
                continue
            seen.add(k)
            I.append(k[0]); Jx.append(k[1])
            if len(I) == edges:
                break
    J = rng.integers(1, r + 1, size=edges) * np.where(rng.random(edges) < 0.5, -1, 1)
    h = rng.integers(1, 4 * r + 1, size=n) * np.where(rng.random(n) < 0.5, -1, 1)
    return np.asarray(I, np.int64), np.asarray(Jx, np.int64), J.astype(np.int64), h.astype(np.int64)


def sparse_ising_qubo(n: int, edges: int, r: int, seed: int) -> np.ndarray:
    """QUBO of sparse_ising(n, edges, r, seed), converted as in ising_to_qubo
    (W_ij = 4 J_ij, W_ii = 2 h_i - 2 sum_j J_ij) without forming the dense J."""
    I, Jx, J, h = sparse_ising(n, edges, r, seed)
    W = np.zeros((n, n), np.int32)
    W[I, Jx] = 4 * J
    W[Jx, I] = 4 * J
    rowJ = np.zeros(n, np.int64)
    np.add.at(rowJ, I, J)
    np.add.at(rowJ, Jx, J)
    W[np.arange(n), np.arange(n)] = 2 * h - 2 * rowJ
    if np.abs(W).max() > 32767:
        raise ValueError("weights exceed int16")
    return W.astype(np.int16)


def batched_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n drawn log-uniform in [lo, hi]: n = floor(lo * (hi/lo)^u), u ~ U[0,1)."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    return np.floor(lo * (hi / lo) ** u).astype(np.int64)


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(out)
        out.append(t)


# ---------------------------------------------------------------- bit layout
def words(n: int) -> int:
    return (n + 31) // 32


def pack_bits(X: np.ndarray) -> np.ndarray:
    """[..., n] 0/1 bytes -> [..., ceil(n/32)] uint32, bit k in word k//32 at k%32."""
    X = np.asarray(X, np.uint8)
    n = X.shape[-1]
    pad = words(n) * 32 - n
    Xp = np.concatenate([X, np.zeros(X.shape[:-1] + (pad,), np.uint8)], -1) if pad else X
    b = np.packbits(Xp, axis=-1, bitorder="little")
    return np.ascontiguousarray(b).view(np.uint32).reshape(X.shape[:-1] + (words(n),))


def unpack_bits(P: np.ndarray, n: int) -> np.ndarray:
    P = np.ascontiguousarray(P, np.uint32)
    b = P.view(np.uint8)
    return np.unpackbits(b, axis=-1, bitorder="little")[..., :n]


def brute_force_min(W: np.ndarray, chunk: int = 1 << 16):
    """Exhaustive minimum of Eq. (2) over all 2^n vectors (n <= 24), by
    vectorised evaluation of the definition.  Returns (E_min, X_argmin, count)."""
    W = np.asarray(W, np.int64)
    n = W.shape[0]
    Wu = np.triu(W, 1)
    dg = np.diag(W)
    best, arg, cnt = None, None, 0
    bits = np.arange(n, dtype=np.int64)
    for base in range(0, 1 << n, chunk):
        idx = np.arange(base, min(base + chunk, 1 << n), dtype=np.int64)
        X = ((idx[:, None] >> bits[None, :]) & 1).astype(np.int64)
        E = X @ dg + np.einsum("bi,ij,bj->b", X, Wu, X)
        m = E.min()
        if best is None or m < best:
            best, arg, cnt = int(m), X[np.argmin(E)].astype(np.uint8), int((E == m).sum())
        elif m == best:
            cnt += int((E == m).sum())
    return best, arg, cnt
