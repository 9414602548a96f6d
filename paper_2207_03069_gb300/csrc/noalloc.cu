// noalloc.cu -- dabs_bulk_search_noalloc: the batch search of
// dabs_bulk_search_dev for callers that cannot allocate device memory.  Its
// scratch (the negated weight copy, the slot launch order and the control
// block) lives in one file-scope device array of fixed size instead of
// cudaMalloc'd buffers; no call here allocates or frees device memory.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call rewrites all of it that it reads: the control block is
// cleared and the negated copy and order are rebuilt.  Calls whose GPU work
// overlaps (different streams, no ordering between them) race on the array.
#include <cstdio>
#include <mutex>

#include "dabs.h"
#include "kernels.cuh"

using namespace dabs;

namespace {

constexpr size_t kWeightsMax = (size_t)1 << 20;  // n * ld int16 entries (2 MiB)
constexpr int kCountMax = 16384;                 // search slots per call
constexpr size_t kOffOrder = kWeightsMax * sizeof(int16_t);
constexpr size_t kOffCtrl = kOffOrder + (size_t)kCountMax * sizeof(int32_t);
constexpr size_t kScratchBytes = kOffCtrl + 256;

// the scratch: [-W (n*ld int16)] [slot order (count int32)] [control block]
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_lock;

// device address of g_scratch for the current device (looked up once per device)
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DABS_E_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_setup_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DABS_E_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DABS_OK;
}

__global__ void k_negate_clear(const int16_t* W, int16_t* Wneg, size_t count, DevCtrl* ctrl,
                               uint64_t seed, uint32_t g) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x)
    Wneg[q] = (int16_t)-W[q];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevCtrl c{};
    c.seed = seed;
    c.g = g;
    c.done = 0;
    *ctrl = c;
  }
}

}  // namespace

extern "C" int dabs_bulk_search_noalloc(const int16_t* W, int32_t n, int32_t ld,
                                        const dabs_params* p, uint64_t seed, uint32_t g,
                                        int32_t count, uint32_t* X, int32_t* delta, int64_t* E,
                                        const uint32_t* D, const uint8_t* algo, uint32_t* best_X,
                                        int64_t* best_E, uint32_t* flips, void* stream) {
  if (!W || !p || n < 1 || ld < n || (ld & 7) != 0 || count < 0 ||
      (reinterpret_cast<uintptr_t>(W) & 15) != 0 || (reinterpret_cast<uintptr_t>(delta) & 15) != 0)
    return DABS_E_INVALID_ARG;
  if (count > 0 && (!X || !delta || !E || !D || !algo || !best_X || !best_E || !flips))
    return DABS_E_INVALID_ARG;
  if (p->tabu < 0 || p->tabu > 31 || p->s_num < 0 || p->s_den < 1 || p->b_num < 0 ||
      p->b_den < 1 || (p->seed_mode != 0 && p->seed_mode != 1))
    return DABS_E_INVALID_ARG;
  if ((size_t)n * (size_t)ld > kWeightsMax || count > kCountMax || n > DABS_N_MAX)
    return DABS_E_TOO_LARGE;
  if (count == 0) return DABS_OK;
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != DABS_OK) return rc;
  int16_t* Wneg = reinterpret_cast<int16_t*>(base);
  int32_t* order = reinterpret_cast<int32_t*>(base + kOffOrder);
  DevCtrl* ctrl = reinterpret_cast<DevCtrl*>(base + kOffCtrl);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  static const int pick[][2] = {{1, 1}, {1, 2}, {1, 4}, {4, 2}, {4, 4}, {8, 4}, {16, 4}};
  SearchVariant var{};
  bool ok = false;
  for (auto& o : pick)
    if (launch_search(o[0], o[1], nullptr, nullptr, &var) && var.cap >= n) { ok = true; break; }
  if (!ok) return DABS_E_TOO_LARGE;

  const size_t entries = (size_t)n * ld;
  k_negate_clear<<<(unsigned)((entries + 255) / 256 < 1024 ? (entries + 255) / 256 : 1024), 256, 0, st>>>(
      W, Wneg, entries, ctrl, seed, g);
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;
  k_order_by_algo<<<1, 1024, 0, st>>>(algo, count, order, ctrl);
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;

  SearchArgs a{};
  a.W = W;
  a.Wneg = Wneg;
  a.n = n;
  a.ld = ld;
  a.nw = (n + 31) / 32;
  a.S = count;
  const uint64_t T = (uint64_t)n * (uint64_t)p->s_num / (uint64_t)p->s_den;
  a.T = (int)(T < 1 ? 1 : (T > (1u << 30) ? (1u << 30) : T));
  a.tau = p->tabu < n - 1 ? p->tabu : n - 1;
  a.B = (uint32_t)(((uint64_t)n * p->b_num + p->b_den - 1) / p->b_den);
  a.seed_mode = p->seed_mode;
  a.ctrl = ctrl;
  a.X = X; a.delta = delta; a.E = E; a.D = D; a.algo = algo;
  a.best_X = best_X; a.best_E = best_E; a.flips = flips;
  a.order = order;
  if (!launch_search(var.nw, var.ch, &a, st, nullptr)) return DABS_E_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;
  return DABS_OK;
}
