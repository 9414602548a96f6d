"""ctypes binding of the plain C oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import this module.  It builds ``liboracle.so`` from ``dabs_oracle.c`` with gcc
on first use (or via :func:`build`) and exposes numpy-friendly wrappers.  It
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dabs_oracle.c")
_HDR = os.path.join(_HERE, "dabs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXMIN, CYCLICMIN, RANDOMMIN, POSITIVEMIN, TWONEIGHBOR = range(5)
ALGOS = ("MaxMin", "CyclicMin", "RandomMin", "PositiveMin", "TwoNeighbor")
OPS = ("Mutation", "Crossover", "Xrossover", "Zero", "One", "IntervalZero", "Best", "Random")
PH_STRAIGHT, PH_GREEDY, PH_MAIN = 0, 1, 2
INT64_MAX = np.iinfo(np.int64).max


class Params(C.Structure):
    _fields_ = [(k, C.c_int32) for k in (
        "searches", "pools", "pool_cap", "tabu", "s_num", "s_den", "b_num", "b_den",
        "seed_mode", "max_generations", "restart", "restart_dist", "abs_mode")]


class SelTrace(C.Structure):
    _fields_ = [("a", C.POINTER(C.c_int64)), ("r", C.POINTER(C.c_int64)),
                ("count", C.POINTER(C.c_int32)), ("free", C.POINTER(C.c_int32)),
                ("cap", C.c_int64)]


def make_params(searches=32, pools=4, pool_cap=64, tabu=8, s=(1, 10), b=(1, 1),
                seed_mode=0, max_generations=0, restart=0, restart_dist=0,
                abs_mode=0) -> Params:
    return Params(searches, pools, pool_cap, tabu, s[0], s[1], b[0], b[1], seed_mode,
                  max_generations, restart, restart_dist, abs_mode)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no vector intrinsics)."""
    with _lock:
        fresh = os.path.exists(_LIB) and all(
            os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in (_SRC, _HDR))
        if force or not fresh:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        i16p, u8p, i32p, i64p, u32p, u64p = (P(C.c_int16), P(C.c_uint8), P(C.c_int32),
                                             P(C.c_int64), P(C.c_uint32), P(C.c_uint64))
        L.orc_energy.restype = C.c_int64
        L.orc_energy.argtypes = [i16p, C.c_int32, u8p]
        L.orc_delta.argtypes = [i16p, C.c_int32, u8p, i32p]
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_parent_rank.restype = C.c_uint32
        L.orc_parent_rank.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_cube21.restype = C.c_uint64
        L.orc_cube21.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_batch_continue.restype = C.c_int
        L.orc_batch_continue.argtypes = [C.c_uint64, C.c_uint64, C.c_int32, C.c_int32]
        L.orc_randmin_threshold.restype = C.c_uint32
        L.orc_randmin_threshold.argtypes = [C.c_uint64, C.c_uint64, C.c_int32]
        L.orc_randmin_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.c_int32, P(C.c_uint16)]
        L.orc_maxmin_threshold.restype = C.c_int64
        L.orc_maxmin_threshold.argtypes = [C.c_int32, C.c_int32, C.c_uint64, C.c_uint64,
                                           C.c_uint32, u64p]
        L.orc_batch_search_sel.restype = C.c_int
        L.orc_batch_search_sel.argtypes = [i16p, C.c_int32, P(Params), C.c_uint64, C.c_uint32,
                                           C.c_uint32, u8p, i32p, i64p, u8p, C.c_int32, u8p,
                                           i64p, u64p, i32p, i32p, C.c_int64, C.c_int32,
                                           P(SelTrace)]
        L.orc_batch_search.restype = C.c_int
        L.orc_batch_search.argtypes = [i16p, C.c_int32, P(Params), C.c_uint64, C.c_uint32,
                                       C.c_uint32, u8p, i32p, i64p, u8p, C.c_int32, u8p, i64p,
                                       u64p, i32p, i32p, C.c_int64, C.c_int32]
        L.orc_solver_create.restype = C.c_void_p
        L.orc_solver_create.argtypes = [i16p, C.c_int32, P(Params), C.c_uint64]
        L.orc_solver_destroy.argtypes = [C.c_void_p]
        L.orc_solver_generation.restype = C.c_uint64
        L.orc_solver_generation.argtypes = [C.c_void_p, C.c_int32]
        L.orc_solver_offspring.argtypes = [C.c_void_p, C.c_uint32, u8p, i32p, i32p]
        L.orc_solver_get_pools.argtypes = [C.c_void_p, u8p, i64p, i32p, i32p]
        L.orc_solver_set_pools.argtypes = [C.c_void_p, u8p, i64p, i32p, i32p]
        L.orc_solver_get_state.argtypes = [C.c_void_p, u8p, i32p, i64p]
        L.orc_solver_get_results.argtypes = [C.c_void_p, u8p, i64p, u64p, i32p, i32p]
        L.orc_solver_get_best.argtypes = [C.c_void_p, u8p, i64p, u64p, u32p]
        L.orc_pool_merge.argtypes = [C.c_void_p, u8p, i64p, i32p, i32p]
        L.orc_solver_get_stats.argtypes = [C.c_void_p, u64p, u64p, u64p, u64p]
        L.orc_solver_get_restarts.restype = C.c_uint32
        L.orc_solver_get_restarts.argtypes = [C.c_void_p]
        L.orc_solve.restype = C.c_int
        L.orc_solve.argtypes = [i16p, C.c_int32, P(Params), C.c_uint64, C.c_uint64, C.c_int64,
                                C.c_int32, u8p, i64p, u64p, u32p]
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _W(W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.int16)
    assert W.ndim == 2 and W.shape[0] == W.shape[1]
    return W


def energy(W, X) -> int:
    W = _W(W)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    return int(lib().orc_energy(_p(W, C.c_int16), W.shape[0], _p(X, C.c_uint8)))


def delta(W, X) -> np.ndarray:
    W = _W(W)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    out = np.zeros(W.shape[0], np.int32)
    lib().orc_delta(_p(W, C.c_int16), W.shape[0], _p(X, C.c_uint8), _p(out, C.c_int32))
    return out


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def parent_rank(u: int, m: int) -> int:
    return int(lib().orc_parent_rank(u, m))


def cube21(a: int, T: int) -> int:
    return int(lib().orc_cube21(a, T))


def batch_continue(total, B, main_runs, algo) -> bool:
    return bool(lib().orc_batch_continue(total, B, main_runs, algo))


def randmin_threshold(t: int, T: int, n: int) -> int:
    """RandomMin's p(t) in units of 2^-16."""
    return int(lib().orc_randmin_threshold(t, T, n))


def randmin_draws(seed: int, flip: int, g: int, s: int, n: int) -> np.ndarray:
    """The 16-bit uniform of every bit for one RandomMin iteration."""
    out = np.zeros(max(n, 1), np.uint16)
    lib().orc_randmin_draws(seed, flip, g, s, n, _p(out, C.c_uint16))
    return out[:n]


def maxmin_threshold(mn: int, mx: int, t: int, T: int, u0: int):
    """MaxMin's threshold d and the interval width R."""
    R = C.c_uint64(0)
    d = lib().orc_maxmin_threshold(mn, mx, t, T, u0, C.byref(R))
    return int(d), int(R.value)


def batch_search(W, params: Params, seed: int, g: int, s: int, X, dlt, E: int, D, algo: int,
                 trace_cap: int = 0, check: bool = False, sel: bool = False):
    """One batch search.  Returns dict(X, delta, E, best_X, best_E, flips, trace, phases, ok),
    plus sel_a, sel_r, sel_count, sel_free (per flip, see orc_sel_trace) when sel is set."""
    W = _W(W)
    n = W.shape[0]
    X = np.array(X, dtype=np.uint8, copy=True)
    dlt = np.array(dlt, dtype=np.int32, copy=True)
    D = np.ascontiguousarray(D, dtype=np.uint8)
    Ec = C.c_int64(E)
    bX = np.zeros(n, np.uint8)
    bE = C.c_int64(0)
    fl = C.c_uint64(0)
    tr = np.zeros(max(trace_cap, 1), np.int32)
    ph = np.zeros(max(trace_cap, 1), np.int32)
    cap = max(trace_cap, 1)
    sa, sr = np.zeros(cap, np.int64), np.zeros(cap, np.int64)
    sc, sf = np.full(cap, -1, np.int32), np.full(cap, -1, np.int32)
    st = SelTrace(_p(sa, C.c_int64), _p(sr, C.c_int64), _p(sc, C.c_int32), _p(sf, C.c_int32),
                  trace_cap if sel else 0)
    rc = lib().orc_batch_search_sel(_p(W, C.c_int16), n, C.byref(params), seed, g, s,
                                    _p(X, C.c_uint8), _p(dlt, C.c_int32), C.byref(Ec),
                                    _p(D, C.c_uint8), algo, _p(bX, C.c_uint8), C.byref(bE),
                                    C.byref(fl), _p(tr, C.c_int32) if trace_cap else None,
                                    _p(ph, C.c_int32) if trace_cap else None, trace_cap,
                                    1 if check else 0, C.byref(st) if sel else None)
    f = int(fl.value)
    m = min(f, trace_cap)
    out = dict(X=X, delta=dlt, E=int(Ec.value), best_X=bX, best_E=int(bE.value), flips=f,
               trace=tr[:m], phases=ph[:m], ok=(rc == 0))
    if sel:
        out.update(sel_a=sa[:m], sel_r=sr[:m], sel_count=sc[:m], sel_free=sf[:m])
    return out


class Solver:
    """The oracle's generational solver (pools + per-search persistent state)."""

    def __init__(self, W, params: Params, seed: int):
        self.W = _W(W)
        self.n = self.W.shape[0]
        self.params = params
        self.S, self.P, self.C = params.searches, params.pools, params.pool_cap
        self._h = lib().orc_solver_create(_p(self.W, C.c_int16), self.n, C.byref(params), seed)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_solver_destroy(h)
            self._h = None

    def generation(self, threads: int = 1) -> int:
        return int(lib().orc_solver_generation(self._h, threads))

    def offspring(self, g: int):
        D = np.zeros((self.S, self.n), np.uint8)
        a = np.zeros(self.S, np.int32)
        o = np.zeros(self.S, np.int32)
        lib().orc_solver_offspring(self._h, g, _p(D, C.c_uint8), _p(a, C.c_int32), _p(o, C.c_int32))
        return D, a, o

    def pools(self):
        PC = self.P * self.C
        X = np.zeros((self.P, self.C, self.n), np.uint8)
        E = np.zeros((self.P, self.C), np.int64)
        a = np.zeros((self.P, self.C), np.int32)
        o = np.zeros((self.P, self.C), np.int32)
        assert X.size == PC * self.n
        lib().orc_solver_get_pools(self._h, _p(X, C.c_uint8), _p(E, C.c_int64), _p(a, C.c_int32),
                                   _p(o, C.c_int32))
        return X, E, a, o

    def set_pools(self, X, E, a, o):
        X = np.ascontiguousarray(X, np.uint8)
        E = np.ascontiguousarray(E, np.int64)
        a = np.ascontiguousarray(a, np.int32)
        o = np.ascontiguousarray(o, np.int32)
        lib().orc_solver_set_pools(self._h, _p(X, C.c_uint8), _p(E, C.c_int64), _p(a, C.c_int32),
                                   _p(o, C.c_int32))

    def state(self):
        X = np.zeros((self.S, self.n), np.uint8)
        d = np.zeros((self.S, self.n), np.int32)
        E = np.zeros(self.S, np.int64)
        lib().orc_solver_get_state(self._h, _p(X, C.c_uint8), _p(d, C.c_int32), _p(E, C.c_int64))
        return X, d, E

    def results(self):
        X = np.zeros((self.S, self.n), np.uint8)
        E = np.zeros(self.S, np.int64)
        f = np.zeros(self.S, np.uint64)
        a = np.zeros(self.S, np.int32)
        o = np.zeros(self.S, np.int32)
        lib().orc_solver_get_results(self._h, _p(X, C.c_uint8), _p(E, C.c_int64),
                                     _p(f, C.c_uint64), _p(a, C.c_int32), _p(o, C.c_int32))
        return X, E, f, a, o

    def merge(self, best_X, best_E, algo, op):
        bX = np.ascontiguousarray(best_X, np.uint8)
        bE = np.ascontiguousarray(best_E, np.int64)
        a = np.ascontiguousarray(algo, np.int32)
        o = np.ascontiguousarray(op, np.int32)
        lib().orc_pool_merge(self._h, _p(bX, C.c_uint8), _p(bE, C.c_int64), _p(a, C.c_int32),
                             _p(o, C.c_int32))

    def stats(self):
        """(algo counts [5], op counts [8], first-finder algo [5], first-finder op [8])"""
        a, o, ba, bo = (np.zeros(5, np.uint64), np.zeros(8, np.uint64), np.zeros(5, np.uint64),
                        np.zeros(8, np.uint64))
        lib().orc_solver_get_stats(self._h, _p(a, C.c_uint64), _p(o, C.c_uint64),
                                   _p(ba, C.c_uint64), _p(bo, C.c_uint64))
        return a, o, ba, bo

    def restarts(self) -> int:
        return int(lib().orc_solver_get_restarts(self._h))

    def best(self):
        X = np.zeros(self.n, np.uint8)
        E = C.c_int64(0)
        f = C.c_uint64(0)
        g = C.c_uint32(0)
        lib().orc_solver_get_best(self._h, _p(X, C.c_uint8), C.byref(E), C.byref(f), C.byref(g))
        return X, int(E.value), int(f.value), int(g.value)


def solve(W, params: Params, budget: int, seed: int, target: int = None, threads: int = 1):
    W = _W(W)
    n = W.shape[0]
    tgt = np.iinfo(np.int64).min if target is None else int(target)
    bX = np.zeros(n, np.uint8)
    bE = C.c_int64(0)
    fl = C.c_uint64(0)
    gens = C.c_uint32(0)
    lib().orc_solve(_p(W, C.c_int16), n, C.byref(params), min(int(budget), 2**64 - 1), seed, tgt,
                    threads, _p(bX, C.c_uint8), C.byref(bE), C.byref(fl), C.byref(gens))
    return bX, int(bE.value), int(fl.value), int(gens.value)
