// kernels.cuh -- argument blocks and launch entry points of the DABS device
// kernels (batch search, genetic layer, bookkeeping, energy/Delta).
#pragma once
#include "common.cuh"

namespace dabs {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int kMergeThreads = 512;

// bits of word w that hold bits k < n
__host__ __device__ __forceinline__ uint32_t valid_mask(int w, int n) {
  const int rem = n - 32 * w;
  return rem >= 32 ? 0xffffffffu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
}

struct PoolArgs {
  int n, nw, P, C;
  const DevCtrl* ctrl;
  const uint32_t* cond;  // restart flag: draw only where it reads 0 (NULL: always, epoch 0)
  uint32_t* pool_X[2];
  int64_t* pool_E[2];
  uint8_t* pool_algo[2];
  uint8_t* pool_op[2];
};

struct StateArgs {
  int n, ld, nw, S;
  const int32_t* diag;
  uint32_t* X;
  int32_t* delta;
  int64_t* E;
  uint32_t* gbest_X;     // cleared unless NULL
  const uint32_t* cond;  // restart flag: reset only where it reads 0 (NULL: always)
  DevCtrl* bump;         // restarts += 1 here after a restart (NULL: none)
};

struct RestartArgs {
  int nw, P, C, h;
  const DevCtrl* ctrl;
  const uint32_t* pool_X[2];
  const uint32_t* gbest_X;
  uint32_t* flag;  // 0 after k_finalize ran; set to 1 when some entry is farther than h
};

struct OffArgs {
  int n, nw, S, P, C;
  const DevCtrl* ctrl;
  const uint32_t* pool_X[2];
  const uint8_t* pool_algo[2];
  const uint8_t* pool_op[2];
  uint32_t* D;
  uint8_t* algo;
  uint8_t* op;
  int abs_mode;  // 1: CyclicMin and mutation after crossover for every search
};

struct MergeArgs {
  int nw, S, P, C, Mmax;
  const DevCtrl* ctrl;
  uint32_t* pool_X[2];
  int64_t* pool_E[2];
  uint8_t* pool_algo[2];
  uint8_t* pool_op[2];
  const uint32_t* best_X;
  const int64_t* best_E;
  const uint8_t* algo;
  const uint8_t* op;
};

// statistics counters (Tables V and VI): [0,5) algorithm runs, [5,13) operation
// uses, [13,18) algorithm of each new global best, [18,26) its operation
constexpr int kStats = 26;

struct FinArgs {
  int nw, S;
  DevCtrl* ctrl;
  const uint32_t* best_X;
  const int64_t* best_E;
  const uint32_t* flips;
  uint32_t* gbest_X;
  const uint8_t* algo;
  const uint8_t* op;
  unsigned long long* stats;  // [kStats]
  uint32_t* rflag;            // restart flag armed (0) here when restarts are on
};

struct EDArgs {
  const int16_t* W;
  int n, ld, nw;
  const uint32_t* X;   // [count][nw]
  int32_t* delta;      // [count][ld_delta] or null
  int ld_delta;
  int64_t* E;          // [count], zeroed before the launch
  const DevCtrl* ctrl; // optional: skip when a solve has stopped
};

// residency of W (weights.cu): outcome of the checks on a staged W
struct WCheck {
  unsigned long long bad;  // lowest i * n + j with W_ij != W_ji (all ones: none)
  unsigned long long low;  // lowest i * n + j with W_ij = -32768 (all ones: none)
  unsigned long long R;    // max_i sum_j |W_ij|
  unsigned long long nnz;  // off-diagonal non-zeros
  unsigned long long nmax; // ~max_ij |W_ij| (all ones: W = 0)
};

struct WeightsArgs {
  const int16_t* Ws;  // staged rows [n][ld] (columns >= n unspecified)
  int16_t* W;         // committed W [n][ld]
  int16_t* Wneg;      // committed -W [n][ld] (may be the staging buffer)
  int32_t* diag;      // [n]
  int n, ld;
  uint32_t* rowsum;   // [n] sums of |W_ij|, zeroed before k_weights_tiles
  uint32_t* rowcnt;   // [n] off-diagonal non-zeros, zeroed before k_weights_tiles
  uint32_t* rowptr;   // [rowptr_len] exclusive prefix sums of rowcnt, total, zeros
  int rowptr_len;
  WCheck* chk;        // bad and low set to all ones before k_weights_tiles
  uint32_t* ent;      // sparse entries written by k_sparse_fill
};

// ---- the batched form's fused generation (ga.cu): one entry per instance
struct BatchInst {
  OffArgs off;          // offspring (its ctrl is the instance's control block)
  MergeArgs merge;      // pool merge
  FinArgs fin;          // finalise
  int32_t* order;       // [S] launch order grouped by algorithm
  int seed_mode;        // 1: X = D, Delta and E recomputed on the tensor cores
  uint32_t* X;          // [S][nw]
  uint16_t* A;          // [rows_pad][n_pad] 16-bit 0/1 operand of the recompute
  int rows_pad, n_pad;
  uint32_t one;         // 1.0 in the operand's encoding
  int64_t* E2;          // [rows_pad] 2 E accumulated by the recompute
  uint32_t* merged;     // merge CTAs of this instance done in this generation
};
// offspring + launch order (+ X = D, the recompute operand, E2 = 0): one CTA
// of 1024 threads per instance
__global__ void k_gen_pre(const BatchInst* insts);
// pool merge, one CTA per pool (kMergeThreads threads); the last CTA of an
// instance to finish runs its finalisation.  prefix[i]: first CTA of instance i
__global__ void k_gen_post(const BatchInst* insts, const int32_t* prefix, int ninst);

__global__ void k_weights_tiles(const WeightsArgs a);
__global__ void k_weights_rows(const WeightsArgs a);
__global__ void k_weights_commit(const WeightsArgs a);
__global__ void k_sparse_fill(const WeightsArgs a);
__global__ void k_negate(const int16_t* W, int16_t* Wneg, size_t count);
__global__ void k_pool_init(const PoolArgs a);
__global__ void k_state_init(const StateArgs a);
__global__ void k_offspring(const OffArgs a);
__global__ void k_merge(const MergeArgs a);
__global__ void k_finalize(const FinArgs a);
__device__ void offspring_one(const OffArgs& a, int s, int lane);
__device__ void merge_pool(const MergeArgs& a, int p, unsigned char* smraw);
__device__ void finalize_one(const FinArgs& a);
__global__ void k_restart_check(const RestartArgs a);
__global__ void k_energy_delta(const EDArgs a);
__global__ void k_order_by_algo(const uint8_t* algo, int S, int32_t* order, const DevCtrl* ctrl,
                                int mod, int lo, int hi);
__global__ void k_copy_targets(const uint32_t* D, uint32_t* X, int64_t* E, size_t words, int S,
                               const DevCtrl* ctrl);

// searches per CTA: spread `slots` searches over the SMs (at most `maxspc` per CTA)
int spc_for(int slots, int maxspc);

// Batch-search variants: NW warps per search, CH chunks of 8 bits per thread.
struct SearchVariant {
  int nw, ch, cap, cta, spc;
};
// launches k_batch_search<NW, CH>; returns false if (nw, ch) is not built
bool launch_search(int nw, int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                   const MultiArgs* m = nullptr);
bool launch_search_w1(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m = nullptr);
bool launch_search_w2(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m = nullptr);
bool launch_search_w4(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m = nullptr);
bool launch_search_w8(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m = nullptr);
bool launch_search_w16(int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                       const MultiArgs* m = nullptr);
// variant (1, 0): one warp per search with Delta in shared memory (search_smem.cu)
bool launch_search_smem(const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                        const MultiArgs* m = nullptr);
size_t smem_search_bytes(int n);  // its shared memory per search

}  // namespace dabs
