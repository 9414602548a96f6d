"""Thin ctypes binding of libdabs.so (include/dabs.h).

Argument marshalling only: every step of the search runs in the CUDA library.
There is no CPU fallback -- if the library is missing or no sm_103 device is
present, the calls raise.  Device buffers are passed as torch CUDA tensors
(their data pointers); host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdabs.so")
_lock = threading.Lock()
_lib = None

OK, E_INVALID_ARG, E_NOT_SYMMETRIC, E_TOO_LARGE, E_OOM, E_TIMEOUT, E_CUDA, E_BUSY, E_NO_DEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
N_MAX = 16384
INT64_MAX = np.iinfo(np.int64).max
INT64_MIN = np.iinfo(np.int64).min
STAGE_OFFSPRING, STAGE_SEARCH, STAGE_MERGE, STAGE_FINALIZE = range(4)
# row formats of the batch search (dabs_set_rows) and their variant-name suffixes
ROWS_DENSE, ROWS_SPARSE_SMEM, ROWS_SPARSE_GLOBAL, ROWS_DENSE_SMEM = range(4)
ROW_SUFFIX = ("", "s", "g", "w")


class Params(C.Structure):
    _fields_ = [(k, C.c_int32) for k in (
        "searches", "pools", "pool_cap", "tabu", "s_num", "s_den", "b_num", "b_den",
        "seed_mode", "max_generations", "restart", "restart_dist", "abs_mode")]


class DabsError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{code} ({strerror(code)}){': ' + msg if msg else ''}")
        self.code = code


EXPORTS = {
    "dabs_params_default": (C.c_int, [C.c_void_p]),
    "dabs_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "dabs_destroy": (None, [C.c_void_p]),
    "dabs_strerror": (C.c_char_p, [C.c_int]),
    "dabs_last_error": (C.c_char_p, [C.c_void_p]),
    "dabs_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dabs_load_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dabs_energy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dabs_delta": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dabs_energy_delta_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                        C.c_void_p, C.c_int32]),
    "dabs_solve": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p,
                             C.c_void_p, C.c_void_p]),
    "dabs_solve_begin": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64]),
    "dabs_solve_generations": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_solve_status": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "dabs_solve_best": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dabs_bulk_search_dev": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32]
                             + [C.c_void_p] * 8),
    "dabs_info": (C.c_int, [C.c_void_p] + [C.c_void_p] * 8),
    "dabs_set_variant": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "dabs_autotune": (C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 4),
    "dabs_read_pools": (C.c_int, [C.c_void_p] * 5),
    "dabs_write_pools": (C.c_int, [C.c_void_p] * 5),
    "dabs_read_state": (C.c_int, [C.c_void_p] * 4),
    "dabs_read_generation": (C.c_int, [C.c_void_p] * 7),
    "dabs_write_results": (C.c_int, [C.c_void_p] * 6),
    "dabs_run_stage": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_read_stats": (C.c_int, [C.c_void_p] * 5),
    "dabs_set_rows": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_set_keyed": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_set_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_test_stall_next_search": (C.c_int, [C.c_void_p]),
    "dabs_get_keyed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dabs_get_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dabs_solve_restarts": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dabs_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dabs_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "dabs_recompute_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_int32]),
    "dabs_set_recompute": (C.c_int, [C.c_void_p, C.c_int32]),
    "dabs_kernel_status": (C.c_int, [C.c_void_p]),
    "dabs_batch_solve": (C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 6),
    "dabs_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "dabs_batch_begin": (C.c_int, [C.c_void_p] * 4),
    "dabs_batch_generations": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "dabs_batch_destroy": (None, [C.c_void_p]),
    "dabs_batch_info": (C.c_int, [C.c_void_p] * 5),
    "dabs_set_search_slots": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "dabs_measure_read_gbs": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int32, C.c_void_p,
                                        C.c_void_p]),
    "dabs_server_create": (C.c_int, [C.c_size_t, C.c_void_p]),
    "dabs_server_destroy": (None, [C.c_void_p]),
    "dabs_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_uint64,
                                     C.c_uint64, C.c_int64, C.c_void_p]),
    "dabs_server_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "dabs_server_poll": (C.c_int, [C.c_void_p, C.c_uint64] + [C.c_void_p] * 5),
    "dabs_server_info": (C.c_int, [C.c_void_p] * 4),
    "dabs_server_set_limits": (C.c_int, [C.c_void_p, C.c_int64]),
    "dabs_bulk_search_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                           C.c_uint64, C.c_uint32, C.c_int32] + [C.c_void_p] * 9),
}


def lib(path: str = LIB_PATH):
    """Loads libdabs.so (built by build.py / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libdabs.so not built ({path}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().dabs_strerror(code).decode()
    except Exception:
        return "?"


def _ptr(a):
    """numpy array or torch tensor -> void*"""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    rc = lib().dabs_params_default(C.byref(p))
    assert rc == OK
    for k, v in kw.items():
        if k in ("s", "b"):
            setattr(p, k + "_num", v[0])
            setattr(p, k + "_den", v[1])
        else:
            setattr(p, k, v)
    return p


def batch_solve(ctxs, budgets, seeds, targets=None):
    """dabs_batch_solve: returns [(X, E, flips)] per context."""
    k = len(ctxs)
    hs = (C.c_void_p * k)(*[c._h.value for c in ctxs])
    bud = np.asarray([min(int(b), 2**64 - 1) for b in budgets], np.uint64)
    sd = np.asarray(seeds, np.uint64)
    tg = None if targets is None else np.asarray(
        [INT64_MIN if t is None else int(t) for t in targets], np.int64)
    Xs = [np.zeros(c.n, np.uint8) for c in ctxs]
    xp = (C.c_void_p * k)(*[x.ctypes.data for x in Xs])
    E = np.zeros(k, np.int64)
    F = np.zeros(k, np.uint64)
    rc = lib().dabs_batch_solve(hs, k, _ptr(bud), _ptr(sd), _ptr(tg), xp, _ptr(E), _ptr(F))
    if rc != OK:
        raise DabsError(rc, lib().dabs_last_error(ctxs[0]._h).decode() if k else "")
    return [(Xs[i], int(E[i]), int(F[i])) for i in range(k)]


def measure_read_gbs(buf, reps: int = 100, stream=None) -> float:
    """dabs_measure_read_gbs on a device tensor: its read bandwidth in GB/s."""
    handle = None if stream is None else getattr(stream, "cuda_stream", stream)
    g = C.c_double()
    rc = lib().dabs_measure_read_gbs(_ptr(buf), buf.numel() * buf.element_size(), reps,
                                     C.c_void_p(handle) if handle else None, C.byref(g))
    if rc != OK:
        raise DabsError(rc)
    return float(g.value)


class Batch:
    """dabs_batch_*: contexts advanced together, one call per group of generations."""

    def __init__(self, ctxs, stream=None):
        self.ctxs = list(ctxs)
        k = len(self.ctxs)
        hs = (C.c_void_p * k)(*[c._h.value for c in self.ctxs])
        handle = None if stream is None else getattr(stream, "cuda_stream", stream)
        self._h = C.c_void_p()
        rc = lib().dabs_batch_create(hs, k, C.c_void_p(handle) if handle else None,
                                     C.byref(self._h))
        if rc != OK:
            raise DabsError(rc)

    def close(self):
        if self._h:
            lib().dabs_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def begin(self, budgets, seeds, targets=None):
        bud = np.asarray([min(int(b), 2**64 - 1) for b in budgets], np.uint64)
        sd = np.asarray(seeds, np.uint64)
        tg = None if targets is None else np.asarray(
            [INT64_MIN if t is None else int(t) for t in targets], np.int64)
        rc = lib().dabs_batch_begin(self._h, _ptr(bud), _ptr(sd), _ptr(tg))
        if rc != OK:
            raise DabsError(rc)

    def generations(self, count: int = 1) -> int:
        r = C.c_int32(0)
        rc = lib().dabs_batch_generations(self._h, count, C.byref(r))
        if rc != OK:
            raise DabsError(rc)
        return int(r.value)

    def info(self) -> dict:
        r, g, l, ms = C.c_int32(), C.c_int32(), C.c_uint64(), C.c_double()
        rc = lib().dabs_batch_info(self._h, C.byref(r), C.byref(g), C.byref(l), C.byref(ms))
        if rc != OK:
            raise DabsError(rc)
        return dict(running=int(r.value), search_groups=int(g.value), launches=int(l.value),
                    search_ms=float(ms.value))


class Server:
    """Request server (continuous batching under an HBM budget)."""

    def __init__(self, hbm_budget_bytes: int):
        h = C.c_void_p()
        rc = lib().dabs_server_create(int(hbm_budget_bytes), C.byref(h))
        if rc != OK:
            raise DabsError(rc)
        self._h = h
        self.n_of = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().dabs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, W, params: Params, budget: int, seed: int, target=None) -> int:
        W = np.ascontiguousarray(W, dtype=np.int16)
        t = C.c_uint64()
        rc = lib().dabs_server_submit(self._h, _ptr(W), W.shape[0], C.byref(params),
                                      min(int(budget), 2**64 - 1), seed,
                                      INT64_MIN if target is None else int(target), C.byref(t))
        if rc != OK:
            raise DabsError(rc)
        self.n_of[t.value] = W.shape[0]
        return int(t.value)

    def step(self, generations: int = 1) -> int:
        p = C.c_int32()
        rc = lib().dabs_server_step(self._h, generations, C.byref(p))
        if rc != OK:
            raise DabsError(rc)
        return int(p.value)

    def poll(self, ticket: int):
        """(status, X, E, flips, latency_s); status 2 = done."""
        X = np.zeros(self.n_of[ticket], np.uint8)
        e, f, lat, st = C.c_int64(), C.c_uint64(), C.c_double(), C.c_int32()
        rc = lib().dabs_server_poll(self._h, ticket, _ptr(X), C.byref(e), C.byref(f),
                                    C.byref(lat), C.byref(st))
        if rc != OK:
            raise DabsError(rc)
        return int(st.value), X, int(e.value), int(f.value), float(lat.value)

    def set_limits(self, max_warps: int):
        rc = lib().dabs_server_set_limits(self._h, int(max_warps))
        if rc != OK:
            raise DabsError(rc)

    def info(self):
        u, q, r = C.c_size_t(), C.c_int32(), C.c_int32()
        rc = lib().dabs_server_info(self._h, C.byref(u), C.byref(q), C.byref(r))
        if rc != OK:
            raise DabsError(rc)
        return int(u.value), int(q.value), int(r.value)


def bulk_search_noalloc(W, n, ld, params, seed, g, X, delta, E, D, algo, best_X, best_E, flips,
                        stream=None):
    """dabs_bulk_search_noalloc on caller tensors (W: device int16 [n][ld])."""
    handle = None if stream is None else getattr(stream, "cuda_stream", stream)
    rc = lib().dabs_bulk_search_noalloc(
        _ptr(W), n, ld, C.byref(params), seed, g, X.shape[0], _ptr(X), _ptr(delta), _ptr(E),
        _ptr(D), _ptr(algo), _ptr(best_X), _ptr(best_E), _ptr(flips),
        C.c_void_p(handle) if handle else None)
    if rc != OK:
        raise DabsError(rc)


class Context:
    """One solver context: device-resident W, pools and search state."""

    def __init__(self, W: np.ndarray, params: Params | None = None, **kw):
        W = np.ascontiguousarray(W, dtype=np.int16)
        if W.ndim != 2 or W.shape[0] != W.shape[1]:
            raise ValueError("W must be square")
        self.n = W.shape[0]
        self.params = params if params is not None else default_params(**kw)
        h = C.c_void_p()
        rc = lib().dabs_create(_ptr(W), self.n, C.byref(self.params), C.byref(h))
        if rc != OK:
            raise DabsError(rc)
        self._h = h
        info = self.info()
        self.ld, self.words = info["ld"], info["words"]
        self.S, self.P, self.C = info["searches"], info["pools"], info["pool_cap"]

    def close(self):
        if getattr(self, "_h", None):
            lib().dabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != OK:
            raise DabsError(rc, lib().dabs_last_error(self._h).decode())

    # ---------------------------------------------------------------- basics
    def info(self) -> dict:
        v = [C.c_int32() for _ in range(8)]
        self._ck(lib().dabs_info(self._h, *[C.byref(x) for x in v]))
        keys = ("n", "ld", "words", "searches", "pools", "pool_cap", "warps", "chunks")
        return {k: x.value for k, x in zip(keys, v)}

    def set_variant(self, warps: int, chunks: int):
        self._ck(lib().dabs_set_variant(self._h, warps, chunks))

    # (warps, chunks); (1, 0) is one warp per search with Delta in shared memory
    VARIANTS = ((1, 1), (1, 2), (1, 4), (2, 1), (2, 2), (2, 4), (4, 1), (4, 2), (4, 4), (8, 1),
                (8, 2), (8, 4), (16, 1), (16, 2), (16, 4), (1, 0))

    def set_rows(self, mode: int):
        """Row format of the batch search: ROWS_DENSE, ROWS_SPARSE_SMEM,
        ROWS_SPARSE_GLOBAL or ROWS_DENSE_SMEM."""
        self._ck(lib().dabs_set_rows(self._h, int(mode)))

    def rows(self):
        """(row format, stored off-diagonal non-zeros or -1)"""
        md, nnz = C.c_int32(), C.c_int32()
        self._ck(lib().dabs_get_rows(self._h, C.byref(md), C.byref(nnz)))
        return int(md.value), int(nnz.value)

    def set_keyed(self, enable: bool):
        """Keyed Delta form of the batch search (used when the instance allows it)."""
        self._ck(lib().dabs_set_keyed(self._h, int(bool(enable))))

    def set_graphs(self, enable: bool):
        """Generations as CUDA graph launches (default) or kernel by kernel."""
        self._ck(lib().dabs_set_graphs(self._h, int(bool(enable))))

    def keyed(self):
        """(enabled, key bits; 0 when the instance does not allow the keyed form)"""
        en, kb = C.c_int32(), C.c_int32()
        self._ck(lib().dabs_get_keyed(self._h, C.byref(en), C.byref(kb)))
        return bool(en.value), int(kb.value)

    def variant_name(self) -> str:
        i = self.info()
        return "%dx%d%s" % (i["warps"], i["chunks"], ROW_SUFFIX[self.rows()[0]])

    def set_variant_name(self, name: str):
        """'WxC' (dense rows), 'WxCs' (sparse rows in shared memory), 'WxCg'
        (sparse rows in global memory) or 'WxCw' (W in shared memory)"""
        mode = ROW_SUFFIX.index(name[-1]) if name[-1] in "sgw" else ROWS_DENSE
        w, c = (int(x) for x in name.rstrip("sgw").split("x"))
        self.set_variant(w, c)
        self.set_rows(mode)

    def autotune(self, generations: int = 2):
        """Picks the fastest batch-search variant and row format; resets the
        solve state.  Returns (warps, chunks, ns_per_flip, {name: ns_per_flip})
        with names as in variant_name()."""
        w, c, ns = C.c_int32(), C.c_int32(), C.c_float()
        names = ["%dx%d%s" % (v + (sfx,)) for sfx in ROW_SUFFIX for v in self.VARIANTS]
        table = np.zeros(len(names), np.float32)
        self._ck(lib().dabs_autotune(self._h, generations, C.byref(w), C.byref(c), C.byref(ns),
                                     _ptr(table)))
        per = {k: round(float(x), 4) for k, x in zip(names, table) if x > 0}
        return int(w.value), int(c.value), float(ns.value), per

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (own stream)."""
        handle = None if stream is None else getattr(stream, "cuda_stream", stream)
        self._ck(lib().dabs_set_stream(self._h, C.c_void_p(handle) if handle else None))

    def load_weights(self, W: np.ndarray):
        W = np.ascontiguousarray(W, dtype=np.int16)
        assert W.shape == (self.n, self.n)
        self._ck(lib().dabs_load_weights(self._h, _ptr(W)))

    def energy(self, X) -> int:
        X = np.ascontiguousarray(X, dtype=np.uint8)
        e = C.c_int64()
        self._ck(lib().dabs_energy(self._h, _ptr(X), C.byref(e)))
        return int(e.value)

    def delta(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.uint8)
        out = np.zeros(self.n, np.int32)
        self._ck(lib().dabs_delta(self._h, _ptr(X), _ptr(out)))
        return out

    def energy_delta_dev(self, X, E, delta=None, ld_delta: int | None = None):
        count = X.shape[0]
        ldd = ld_delta if ld_delta is not None else (delta.shape[-1] if delta is not None else 0)
        self._ck(lib().dabs_energy_delta_dev(self._h, _ptr(X), count, _ptr(E), _ptr(delta), ldd))

    def recompute_dev(self, X, E, delta=None, ld_delta: int | None = None):
        """Tensor-core Eq. (2)/(3) of X (device, packed) into E (and delta)."""
        count = X.shape[0]
        ldd = ld_delta if ld_delta is not None else (delta.shape[-1] if delta is not None else 0)
        self._ck(lib().dabs_recompute_dev(self._h, _ptr(X), count, _ptr(E), _ptr(delta), ldd))

    def set_recompute(self, mode: int):
        self._ck(lib().dabs_set_recompute(self._h, mode))

    def kernel_status(self):
        self._ck(lib().dabs_kernel_status(self._h))

    def test_stall_next_search(self):
        """Test hook: the next bulk_search_dev on variant (1, 0) lets a bounded
        device wait run out (reported by kernel_status)."""
        self._ck(lib().dabs_test_stall_next_search(self._h))

    # ---------------------------------------------------------------- solve
    def solve(self, budget: int, seed: int, target: int | None = None):
        X = np.zeros(self.n, np.uint8)
        e = C.c_int64()
        f = C.c_uint64()
        tgt = INT64_MIN if target is None else int(target)
        self._ck(lib().dabs_solve(self._h, min(int(budget), 2**64 - 1), seed, tgt, _ptr(X),
                                  C.byref(e), C.byref(f)))
        return X, int(e.value), int(f.value)

    def solve_begin(self, seed: int, budget: int = 2**64 - 1, target: int | None = None):
        tgt = INT64_MIN if target is None else int(target)
        self._ck(lib().dabs_solve_begin(self._h, seed, min(int(budget), 2**64 - 1), tgt))

    def solve_generations(self, count: int):
        self._ck(lib().dabs_solve_generations(self._h, count))

    def solve_status(self) -> dict:
        f, g, e, d = C.c_uint64(), C.c_uint32(), C.c_int64(), C.c_int32()
        self._ck(lib().dabs_solve_status(self._h, C.byref(f), C.byref(g), C.byref(e), C.byref(d)))
        return dict(flips=int(f.value), generations=int(g.value), best_E=int(e.value),
                    done=bool(d.value))

    def restarts(self) -> int:
        r = C.c_uint32()
        self._ck(lib().dabs_solve_restarts(self._h, C.byref(r)))
        return int(r.value)

    def solve_best(self):
        X = np.zeros(self.n, np.uint8)
        e = C.c_int64()
        self._ck(lib().dabs_solve_best(self._h, _ptr(X), C.byref(e)))
        return X, int(e.value)

    def run_stage(self, stage: int):
        self._ck(lib().dabs_run_stage(self._h, stage))

    def set_search_slots(self, modulus: int, lo: int = 0, hi: int = 0):
        """Stage 1 runs only the searches s with lo <= s mod modulus < hi (0: all)."""
        self._ck(lib().dabs_set_search_slots(self._h, modulus, lo, hi))

    # ---------------------------------------------------------------- bulk search
    def bulk_search_dev(self, seed, g, X, delta, E, D, algo, best_X, best_E, flips):
        self._ck(lib().dabs_bulk_search_dev(self._h, seed, g, X.shape[0], _ptr(X), _ptr(delta),
                                            _ptr(E), _ptr(D), _ptr(algo), _ptr(best_X),
                                            _ptr(best_E), _ptr(flips)))

    # ---------------------------------------------------------------- inspection
    def read_pools(self):
        X = np.zeros((self.P, self.C, self.words), np.uint32)
        E = np.zeros((self.P, self.C), np.int64)
        a = np.zeros((self.P, self.C), np.uint8)
        o = np.zeros((self.P, self.C), np.uint8)
        self._ck(lib().dabs_read_pools(self._h, _ptr(X), _ptr(E), _ptr(a), _ptr(o)))
        return X, E, a, o

    def write_pools(self, X, E, a, o):
        X = np.ascontiguousarray(X, np.uint32)
        E = np.ascontiguousarray(E, np.int64)
        a = np.ascontiguousarray(a, np.uint8)
        o = np.ascontiguousarray(o, np.uint8)
        self._ck(lib().dabs_write_pools(self._h, _ptr(X), _ptr(E), _ptr(a), _ptr(o)))

    def read_state(self):
        X = np.zeros((self.S, self.words), np.uint32)
        d = np.zeros((self.S, self.ld), np.int32)
        E = np.zeros(self.S, np.int64)
        self._ck(lib().dabs_read_state(self._h, _ptr(X), _ptr(d), _ptr(E)))
        return X, d[:, :self.n], E

    def read_generation(self):
        S, w = self.S, self.words
        D = np.zeros((S, w), np.uint32)
        a = np.zeros(S, np.uint8)
        o = np.zeros(S, np.uint8)
        bX = np.zeros((S, w), np.uint32)
        bE = np.zeros(S, np.int64)
        f = np.zeros(S, np.uint32)
        self._ck(lib().dabs_read_generation(self._h, _ptr(D), _ptr(a), _ptr(o), _ptr(bX),
                                            _ptr(bE), _ptr(f)))
        return D, a, o, bX, bE, f

    def stats(self):
        """(algo counts [5], op counts [8], first-finder algo [5], first-finder op [8])"""
        a, o, ba, bo = (np.zeros(5, np.uint64), np.zeros(8, np.uint64), np.zeros(5, np.uint64),
                        np.zeros(8, np.uint64))
        self._ck(lib().dabs_read_stats(self._h, _ptr(a), _ptr(o), _ptr(ba), _ptr(bo)))
        return a, o, ba, bo

    def checkpoint(self) -> bytes:
        size = C.c_size_t()
        self._ck(lib().dabs_checkpoint(self._h, None, 0, C.byref(size)))
        buf = np.zeros(size.value, np.uint8)
        self._ck(lib().dabs_checkpoint(self._h, _ptr(buf), size.value, C.byref(size)))
        return buf.tobytes()

    def restore(self, blob: bytes):
        buf = np.frombuffer(blob, np.uint8).copy()
        self._ck(lib().dabs_restore(self._h, _ptr(buf), buf.size))

    def write_results(self, best_X, best_E, flips, algo, op):
        args = [np.ascontiguousarray(best_X, np.uint32), np.ascontiguousarray(best_E, np.int64),
                np.ascontiguousarray(flips, np.uint32), np.ascontiguousarray(algo, np.uint8),
                np.ascontiguousarray(op, np.uint8)]
        self._ck(lib().dabs_write_results(self._h, *[_ptr(x) for x in args]))
