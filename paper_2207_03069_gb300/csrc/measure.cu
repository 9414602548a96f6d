// measure.cu -- read bandwidth of the device for a buffer of a given size:
// the denominator of the flip kernel's roofline when its rows come from the
// L2 (a buffer well under the L2's 129 MB stays resident across repetitions).
#include <algorithm>

#include "dabs.h"
#include "kernels.cuh"

namespace {

// every thread XOR-folds its 16-byte words, `passes` times over the buffer
// (eight independent loads in flight per thread); a block stores its fold
// only when it equals a value that the caller never supplies, so the loads
// stay live
__global__ void __launch_bounds__(256) k_read(const uint4* p, size_t words, int passes,
                                              uint32_t never, uint32_t* sink) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (int r = 0; r < passes; ++r) {
    size_t q = t;
    for (; q + 7 * stride < words; q += 8 * stride) {
      uint4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldcg(p + q + j * stride);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc ^= v[j].x ^ v[j].y ^ v[j].z ^ v[j].w;
    }
    for (; q < words; q += stride) {
      const uint4 v = __ldcg(p + q);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  acc = __reduce_xor_sync(0xffffffffu, acc);
  if (acc == never && (threadIdx.x & 31) == 0) *sink = acc;
}

}  // namespace

extern "C" int dabs_measure_read_gbs(const void* buf, size_t bytes, int32_t reps, void* stream,
                                     double* gbs) {
  if (!buf || bytes < 16 || reps < 1 || !gbs || (reinterpret_cast<uintptr_t>(buf) & 15) != 0)
    return DABS_E_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DABS_E_CUDA;
  const size_t words = bytes / 16;
  const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>((size_t)sms * 4, (words + 255) / 256));
  // passes per launch: about 256 MB of reads per launch, so that launches
  // are long against their overhead
  const int passes = (int)std::max<size_t>(1, ((size_t)256 << 20) / std::max<size_t>(bytes, 1));
  uint32_t* sink = nullptr;  // the 4-byte slot the folds would be stored to
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DABS_OK;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) return DABS_E_OOM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = DABS_E_CUDA;
  const uint4* p = static_cast<const uint4*>(buf);
  for (int w = 0; w < 3 && !rc; ++w) {
    k_read<<<grid, 256, 0, st>>>(p, words, passes, 0x9E3779B9u, sink);
    if (cudaGetLastError() != cudaSuccess) rc = DABS_E_CUDA;
  }
  if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = DABS_E_CUDA;
  for (int r = 0; r < reps && !rc; ++r) {
    k_read<<<grid, 256, 0, st>>>(p, words, passes, 0x9E3779B9u, sink);
    if (cudaGetLastError() != cudaSuccess) rc = DABS_E_CUDA;
  }
  if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = DABS_E_CUDA;
  float ms = 0;
  if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = DABS_E_CUDA;
  if (!rc) *gbs = (double)words * 16.0 * passes * reps / (ms * 1e-3) / 1e9;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}
