// noalloc.cu -- dabs_bulk_search_noalloc: the batch search of
// dabs_bulk_search_dev for callers that cannot allocate device memory.  Its
// scratch (the negated weight copy, the diagonal, the slot launch order and
// the control block) lives in one file-scope device array of fixed size
// instead of cudaMalloc'd buffers; no call here allocates or frees device
// memory.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call rewrites all of it that it reads: the control block is
// cleared and the negated copy, diagonal and order are rebuilt.  Calls whose
// GPU work overlaps (different streams, no ordering between them) race on
// the array.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "dabs.h"
#include "kernels.cuh"

using namespace dabs;

namespace {

constexpr size_t kWeightsMax = (size_t)1 << 20;  // n * ld int16 entries (2 MiB)
constexpr int kCountMax = 16384;                 // search slots per call
constexpr size_t kOffOrder = kWeightsMax * sizeof(int16_t);
constexpr size_t kOffDiag = kOffOrder + (size_t)kCountMax * sizeof(int32_t);
constexpr size_t kOffCtrl = kOffDiag + (size_t)DABS_N_MAX * sizeof(int32_t);
constexpr size_t kScratchBytes = kOffCtrl + 256;

// the scratch: [-W (n*ld int16)] [slot order (count int32)] [W_kk (n int32)]
// [control block]
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// device address of g_scratch per device, and the context it was looked up in
// (a cudaDeviceReset makes a new primary context, whose module has its own
// copy of the array: the address is looked up again then)
unsigned char* g_scratch_ptr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};
std::mutex g_setup_lock;

typedef int (*CtxGetCurrentFn)(void**);

// the current CUDA context of the calling thread (driver API, through the
// runtime's entry-point lookup so that no driver library is linked)
void* current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
    looked = true;
  }
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}

// device address of g_scratch for the current device: looked up once per
// device and context, with that device current
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DABS_E_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_setup_lock);
  void* cx = current_context();  // null before the runtime made one current
  if (!g_scratch_ptr[dev] || !cx || cx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DABS_E_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    g_scratch_ctx[dev] = current_context();
  }
  *out = g_scratch_ptr[dev];
  return DABS_OK;
}

// -W of the caller's W, and the control block's seed and generation; an
// entry of -32768 (whose negation does not fit int16) stops the call: the
// control block is marked done, so no search runs
__global__ void k_negate_clear(const int16_t* W, int16_t* Wneg, int32_t* diag, int n, int ld,
                               DevCtrl* ctrl, uint64_t seed, uint32_t g) {
  bool low = false;
  const size_t count = (size_t)n * ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x) {
    const int16_t w = W[q];
    low |= w == INT16_MIN;
    Wneg[q] = (int16_t)-w;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    diag[k] = W[(size_t)k * ld + k];
  if (low) atomicExch(&ctrl->done, 1u);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->seed = seed;
    ctrl->g = g;
  }
}

// a refused call reports every slot as not searched: best_E = INT64_MAX and
// flips = 0 (a search that ran has best_E < INT64_MAX: Step 1 always sets BEST)
__global__ void k_refused(const DevCtrl* ctrl, int count, int64_t* best_E, uint32_t* flips) {
  if (!ctrl->done) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
    best_E[s] = INT64_MAX;
    flips[s] = 0;
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
  int32_t* diag = reinterpret_cast<int32_t*>(base + kOffDiag);
  DevCtrl* ctrl = reinterpret_cast<DevCtrl*>(base + kOffCtrl);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  static const int pick[][2] = {{1, 1}, {1, 2}, {1, 4}, {4, 2}, {4, 4}, {8, 4}, {16, 4}};
  SearchVariant var{};
  bool ok = false;
  for (auto& o : pick)
    if (launch_search(o[0], o[1], nullptr, nullptr, &var) && var.cap >= n) { ok = true; break; }
  if (!ok) return DABS_E_TOO_LARGE;

  const size_t entries = (size_t)n * ld;
  if (cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), st) != cudaSuccess) return DABS_E_CUDA;
  k_negate_clear<<<(unsigned)((entries + 255) / 256 < 1024 ? (entries + 255) / 256 : 1024), 256, 0, st>>>(
      W, Wneg, diag, n, ld, ctrl, seed, g);
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;
  k_order_by_algo<<<1, 1024, 0, st>>>(algo, count, order, ctrl, 0, 0, 0);
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;

  SearchArgs a{};
  a.W = W;
  a.Wneg = Wneg;
  a.diag = diag;
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
  k_refused<<<(count + 255) / 256, 256, 0, st>>>(ctrl, count, best_E, flips);
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;
  if (!launch_search(var.nw, var.ch, &a, st, nullptr)) return DABS_E_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return DABS_E_CUDA;
  return DABS_OK;
}
