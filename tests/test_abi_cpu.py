"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/dabs.h declares, reports parameter defaults and
error strings, and refuses to create a context without an sm_103 device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2207_03069_gb300 import build, dabs
    build.build()
    return dabs.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "dabs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dabs_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    from paper_2207_03069_gb300 import dabs
    assert set(names) == set(dabs.EXPORTS)


def test_params_default_and_strerror(L):
    from paper_2207_03069_gb300 import dabs
    p = dabs.default_params()
    assert (p.searches, p.pools, p.pool_cap, p.tabu) == (32, 4, 100, 8)
    assert (p.s_num, p.s_den, p.b_num, p.b_den, p.seed_mode) == (1, 10, 1, 1, 0)
    assert L.dabs_params_default(None) == dabs.E_INVALID_ARG
    for code in range(0, -9, -1):
        assert dabs.strerror(code) not in ("", "unknown error")


def test_create_rejects_bad_arguments_before_touching_a_device(L):
    from paper_2207_03069_gb300 import dabs
    W = np.zeros((4, 4), np.int16)
    h = C.c_void_p()
    p = dabs.default_params()
    assert L.dabs_create(None, 4, C.byref(p), C.byref(h)) == dabs.E_INVALID_ARG
    assert L.dabs_create(W.ctypes.data_as(C.c_void_p), 0, C.byref(p), C.byref(h)) == dabs.E_INVALID_ARG
    bad = dabs.default_params(tabu=32)
    assert L.dabs_create(W.ctypes.data_as(C.c_void_p), 4, C.byref(bad), C.byref(h)) == dabs.E_INVALID_ARG
    big = np.zeros((1, 1), np.int16)
    assert L.dabs_create(big.ctypes.data_as(C.c_void_p), dabs.N_MAX + 1, C.byref(p),
                         C.byref(h)) == dabs.E_TOO_LARGE
    assert h.value is None


def test_create_without_gpu_reports_no_device(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2207_03069_gb300 import dabs
    W = np.zeros((4, 4), np.int16)
    h = C.c_void_p()
    p = dabs.default_params(searches=4, pools=1)
    assert L.dabs_create(W.ctypes.data_as(C.c_void_p), 4, C.byref(p), C.byref(h)) == dabs.E_NO_DEVICE


def test_header_is_plain_c_and_links(L, tmp_path):
    """include/dabs.h is a C ABI: a C99 program using its types and calls
    compiles with gcc and links against libdabs.so (it is not run: no GPU)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "use_dabs.c"
    src.write_text(r"""
#include <stdint.h>
#include <stdio.h>
#include "dabs.h"
int main(void) {
    dabs_params p;
    int16_t W[4] = {1, -2, -2, 3};
    dabs_ctx* ctx = NULL;
    uint8_t x[2];
    int64_t e = 0;
    uint64_t flips = 0;
    if (dabs_params_default(&p) != DABS_OK) return 1;
    int rc = dabs_create(W, 2, &p, &ctx);
    if (rc != DABS_OK) { printf("%s\n", dabs_strerror(rc)); return 0; }
    rc = dabs_solve(ctx, 1000, 1, INT64_MIN, x, &e, &flips);
    dabs_destroy(ctx);
    return rc == DABS_OK ? 0 : 2;
}
""")
    lib = os.path.join(ROOT, "paper_2207_03069_gb300")
    out = tmp_path / "use_dabs"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", lib, "-ldabs", "-Wl,-rpath," + lib, "-o", str(out)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def header_constants():
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dabs.h")).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define (DABS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)}
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for k, v in re.findall(r"(DABS_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[k] = int(v)
    fields = re.search(r"typedef struct dabs_params \{(.*?)\} dabs_params;", src, re.S).group(1)
    names = [n for decl in re.findall(r"int32_t\s+([^;]+);", fields)
             for n in (x.strip() for x in decl.split(","))]
    return consts, names


def test_binding_constants_and_params_match_the_header():
    """The ctypes binding mirrors the header: error codes, row formats, the
    autotuner's table size, and dabs_params field by field (all int32_t)."""
    from paper_2207_03069_gb300 import dabs
    consts, names = header_constants()
    for k in ("OK", "E_INVALID_ARG", "E_NOT_SYMMETRIC", "E_TOO_LARGE", "E_OOM", "E_TIMEOUT",
              "E_CUDA", "E_BUSY", "E_NO_DEVICE", "ROWS_DENSE", "ROWS_SPARSE_SMEM",
              "ROWS_SPARSE_GLOBAL", "ROWS_DENSE_SMEM"):
        assert getattr(dabs, k) == consts["DABS_" + k], k
    assert len(dabs.Context.VARIANTS) * len(dabs.ROW_SUFFIX) == consts["DABS_N_VARIANTS"]
    assert [f for f, _ in dabs.Params._fields_] == names
    assert all(t is C.c_int32 for _, t in dabs.Params._fields_)
    assert C.sizeof(dabs.Params) == 4 * len(names)


def test_binding_argument_counts_match_the_header():
    """Every call the binding declares takes as many arguments as its
    prototype in include/dabs.h (ctypes would not notice a mismatch)."""
    from paper_2207_03069_gb300 import dabs
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dabs.h")).read(), flags=re.S)
    protos = {}
    for name, args in re.findall(r"\b(dabs_[a-z_]+)\s*\(([^()]*)\)\s*;", src):
        a = " ".join(args.split())
        protos[name] = 0 if a in ("", "void") else a.count(",") + 1
    assert len(protos) >= 20
    for name, (_, argtypes) in dabs.EXPORTS.items():
        assert name in protos, name
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])
