"""GPU: the device Philox4x32-10 (Salmon et al., SC'11) that every random draw
of the batch search and the genetic operations goes through, against three
things it does not share code with: CUDA's own curand_Philox4x32_10 (called
from its header), the published known-answer vectors, and the oracle's C
implementation.  A small probe kernel is compiled here against the library's
common.cuh; it reads only its input arrays and writes only its outputs."""
import json
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")

PROBE = r"""
#include <curand_philox4x32_x.h>
#include "common.cuh"
__global__ void k_philox_pair(const uint4* c, const uint2* k, uint4* ours, uint4* ref, int m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < m) {
    ours[q] = dabs::philox(c[q], k[q]);
    ref[q] = curand_Philox4x32_10(c[q], k[q]);
  }
}
extern "C" int philox_pair(const void* c, const void* k, void* ours, void* ref, int m) {
  if (m <= 0) return 0;
  k_philox_pair<<<(m + 255) / 256, 256>>>(static_cast<const uint4*>(c), static_cast<const uint2*>(k),
                                         static_cast<uint4*>(ours), static_cast<uint4*>(ref), m);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03069_gb300 import build
    d = tmp_path_factory.mktemp("philox")
    src, so = d / "probe.cu", d / "probe.so"
    src.write_text(PROBE)
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", build.CSRC, "-o", str(so), str(src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    import ctypes
    lib = ctypes.CDLL(str(so))
    lib.philox_pair.restype = ctypes.c_int
    lib.philox_pair.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int]

    def run(ctr, key):
        c = torch.from_numpy(np.ascontiguousarray(ctr, np.uint32).view(np.int32)).cuda()
        k = torch.from_numpy(np.ascontiguousarray(key, np.uint32).view(np.int32)).cuda()
        m = ctr.shape[0]
        ours = torch.zeros((m, 4), dtype=torch.int32, device="cuda")
        ref = torch.zeros((m, 4), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert lib.philox_pair(c.data_ptr(), k.data_ptr(), ours.data_ptr(), ref.data_ptr(), m) == 0
        return (ours.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    return run


def counters(m, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2**32, size=(m, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(m, 2), dtype=np.uint64).astype(np.uint32)
    # edges: all zero, all ones, and the layouts the solver uses (small words)
    ctr[0], key[0] = 0, 0
    ctr[1], key[1] = 0xFFFFFFFF, 0xFFFFFFFF
    ctr[2:66] = np.stack([np.arange(64), np.full(64, 7), np.full(64, 3), np.arange(64) << 12], 1)
    return ctr, key


def test_device_philox_equals_curand(probe):
    ctr, key = counters(4096, 1)
    ours, ref = probe(ctr, key)
    assert np.array_equal(ours, ref)


def test_device_philox_known_answers(probe):
    g = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    ctr = np.array([[int(x, 16) for x in v["ctr"]] for v in g["vectors"]], np.uint32)
    key = np.array([[int(x, 16) for x in v["key"]] for v in g["vectors"]], np.uint32)
    ours, ref = probe(ctr, key)
    want = np.array([[int(x, 16) for x in v["out"]] for v in g["vectors"]], np.uint32)
    assert np.array_equal(ours, want) and np.array_equal(ref, want)


def test_device_philox_equals_oracle(probe, orc):
    ctr, key = counters(256, 2)
    ours, _ = probe(ctr, key)
    for q in range(ctr.shape[0]):
        assert np.array_equal(ours[q], orc.philox(ctr[q], key[q]))
