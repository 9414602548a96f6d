// ctx.cuh -- the solver context behind the C ABI's opaque dabs_ctx, and the
// internal helpers shared by the single-instance calls (abi.cu), the batched
// solve and the request server (batch.cu).
#pragma once
#include <cuda.h>

#include <string>
#include <vector>

#include "dabs.h"
#include "kernels.cuh"
#include "umma.cuh"

using namespace dabs;

struct dabs_ctx {
  int dev = 0;
  int n = 0, ld = 0, nw = 0;
  dabs_params p{};
  uint64_t w_hash = 0;      // FNV-1a-style hash of W (ties checkpoints to their instance)
  bool w_hash_ok = false;   // w_hash is that of the current W (computed on demand)
  int T = 1, tau = 0;
  uint32_t B = 1;
  int S = 0, P = 0, C = 0, Mmax = 1;
  size_t merge_smem = 0;
  cudaStream_t own = nullptr, stream = nullptr;
  int16_t* W = nullptr;
  int16_t* Wneg = nullptr;  // -W: lets the flip kernel read row i of sigma(x_i) W
  int32_t* diag = nullptr;
  uint32_t* wrow = nullptr;   // [2n] row sums of |W| and row non-zero counts of a staged W
  uint32_t* wptr = nullptr;   // [4 * sparse_row16(n)] their prefix sums (sparse row starts)
  WCheck* wchk = nullptr;     // checks of a staged W, and a pinned host copy
  WCheck* h_wchk = nullptr;
  DevCtrl* ctrl = nullptr;
  DevCtrl* bulk_ctrl = nullptr;
  DevCtrl* h_ctrl = nullptr;  // pinned staging
  uint32_t* poolX[2] = {nullptr, nullptr};
  int64_t* poolE[2] = {nullptr, nullptr};
  uint8_t* poolA[2] = {nullptr, nullptr};
  uint8_t* poolO[2] = {nullptr, nullptr};
  uint32_t* X = nullptr;
  int32_t* delta = nullptr;
  int64_t* E = nullptr;
  uint32_t* D = nullptr;
  uint8_t* algo = nullptr;
  uint8_t* op = nullptr;
  uint32_t* bestX = nullptr;
  int64_t* bestE = nullptr;
  uint32_t* flips = nullptr;
  int32_t* order = nullptr;   // slot launch order grouped by algorithm
  uint32_t* gbestX = nullptr;
  unsigned long long* stats = nullptr;  // [kStats] Tables V/VI counters
  uint32_t* rflag = nullptr;            // restart flag of the running generation
  uint32_t* one_X = nullptr;   // single-vector scratch for dabs_energy / dabs_delta
  int32_t* one_d = nullptr;
  int64_t* one_E = nullptr;
  SearchVariant var{};
  bool var_set = false;       // var chosen by dabs_set_variant or dabs_autotune
  // sparse rows of the batch search (Max-Cut- and QASP-like instances)
  int rows_mode = 0;          // RowFormat the batch search reads
  int key_bits = 0;           // keyed Delta bits when the instance allows it (0: not)
  int keyed = 1;              // 1: use the keyed form when key_bits > 0
  bool smem_ok = false;       // the shared-memory Delta variant (1, 0) can run this instance
  int* serr = nullptr;        // error flag of the batch-search kernels with bounded waits
  int stall_test = 0;         // test hook for the bounded waits (dabs_test_stall_next_search)
  // one generation captured as a CUDA graph and replayed per generation
  int graphs = 1;             // 1: dabs_solve_generations replays the graph
  bool graph_ok = false;      // gexec matches the current launch configuration
  cudaGraphExec_t gexec = nullptr;
  int sp_nnz = -1;            // stored off-diagonal non-zeros; -1 when not stored (> n^2/4)
  size_t sp_cap = 0;          // capacity of sp_ent in entries
  int smem_optin = 0;         // opt-in shared memory per block of the device
  uint32_t* sp_row = nullptr; // [4 * sparse_row16(n)]
  uint32_t* sp_ent = nullptr; // [sp_cap], owned here (not in allocs: it is resized)
  // tensor-core recompute (tcgen05): W limbs, bf16 copy of the vectors, maps
  int recompute_mode = 0;     // 0 = CUDA cores, 1 = tensor cores
  bool tc_ready = false;
  int tc_limbs_n = 2;         // tensor-core operand form: 1 fp16 W, 2 bf16 limbs
  int max_abs = 32767;        // max_ij |W_ij| of the loaded W
  int n_pad = 0, rows_pad = 0;
  uint16_t* Whi = nullptr;
  uint16_t* Wlo = nullptr;
  uint16_t* Abf = nullptr;
  int64_t* E2 = nullptr;
  int* kerr = nullptr;
  CUtensorMap mapA{}, mapHi{}, mapLo{};
  std::vector<void*> allocs;
  std::string err;
  uint64_t launches = 0;      // kernels launched by stage() (counted for the batched form)
  // the searches this context runs when a solve is split over devices by
  // island: slots s with slot_lo <= s mod slot_mod < slot_hi (slot_mod 0: all)
  int slot_mod = 0, slot_lo = 0, slot_hi = 0, slot_count = 0;
};


#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? DABS_E_OOM : DABS_E_CUDA,         \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);    \
  } while (0)

#define CKLAUNCH() CK(cudaGetLastError())
// a kernel launch of a generation's stages: checked and counted
#define CKSTAGE()        \
  do {                   \
    CKLAUNCH();          \
    ++ctx->launches;     \
  } while (0)


namespace dabs_internal {
int fail(dabs_ctx* c, int code, const char* fmt, ...);
SearchArgs solve_search_args(dabs_ctx* ctx);
// 0 offspring (+ recompute), 1 launch order + batch search, 2 merge,
// 3 finalise, 4 launch order only
int stage(dabs_ctx* ctx, int which);
int read_ctrl(dabs_ctx* ctx, DevCtrl* out);
// the captured generation no longer matches (variant, rows, stream, ...)
inline void graph_stale(dabs_ctx* ctx) { ctx->graph_ok = false; }
bool default_variant(int n, SearchVariant* v, bool many);
// the variant a context's batch searches use in the batched and served
// forms: its own when the caller or the autotuner chose it, else the default
// for many instances in flight
inline SearchVariant batch_variant(const dabs_ctx* ctx) {
  SearchVariant v = ctx->var;
  if (!ctx->var_set && !default_variant(ctx->n, &v, true)) v = ctx->var;
  return v;
}
}  // namespace dabs_internal
