// common.cuh -- device-side building blocks shared by the DABS kernels:
// the counter-based random stream, integer helpers for the iteration-dependent
// schedules, and the argument structs the C ABI hands to the kernels.
//
// All arithmetic is integer.  The random stream is Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, SC'11), keyed by the solve seed; the counter layout is
// fixed per purpose below so that every draw of a solve is reproducible.
#pragma once
#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace dabs {

// Main search algorithms (Section III-A) and genetic operations (Section IV-A).
enum Algo : int { MAXMIN = 0, CYCLICMIN = 1, RANDOMMIN = 2, POSITIVEMIN = 3, TWONEIGHBOR = 4,
                  N_ALGOS = 5 };
enum Op : int { MUTATION = 0, CROSSOVER = 1, XROSSOVER = 2, ZERO = 3, ONE = 4,
                INTERVALZERO = 5, BEST = 6, RANDOM = 7, N_OPS = 8 };

// Random-stream purposes: the high byte of the fourth counter word.
enum Purpose : uint32_t { RNG_MAXMIN = 1u << 24, RNG_POSMIN = 2u << 24, RNG_RANDMIN = 3u << 24,
                          RNG_CHOICE = 4u << 24, RNG_PARENT = 5u << 24, RNG_BITS = 6u << 24,
                          RNG_INIT_BITS = 7u << 24, RNG_INIT_TAGS = 8u << 24 };

constexpr uint32_t kMixThreshold = 214748364u;  // floor(0.05 * 2^32): 5% uniform choice

// Philox4x32-10: ten rounds; round r multiplies words 0 and 2 by the two
// Philox constants, mixes the high halves with words 1/3 and the key, and the
// key advances by the Weyl increments between rounds.
__host__ __device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t x, uint32_t y, uint32_t z,
                                               uint32_t w) {
  return philox(make_uint4(x, y, z, w), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// uniform integer in [0, m) by multiply-shift
__host__ __device__ __forceinline__ uint32_t uniform_below(uint32_t u, uint32_t m) {
  return (uint32_t)(((uint64_t)u * m) >> 32);
}

// (a / T)^3 in units of 2^-32, from a 21-bit fixed-point ratio (a <= T).
__host__ __device__ __forceinline__ uint64_t cube21(uint64_t a, uint64_t T) {
  const uint64_t f = (a << 21) / T;
  return (f * f * f) >> 31;
}

// Section IV-A parent rank: floor(r^3 m) for r = u / 2^32, as
// ((u^3 >> 32) * m) >> 64 in exact integer arithmetic.
__host__ __device__ __forceinline__ uint32_t parent_rank(uint32_t u, uint32_t m) {
  const uint64_t sq = (uint64_t)u * u;
#ifdef __CUDA_ARCH__
  const uint64_t hi = __umul64hi(sq, (uint64_t)u);
#else
  const uint64_t hi = (uint64_t)(((unsigned __int128)sq * u) >> 64);
#endif
  const uint64_t lo = sq * (uint64_t)u;
  const uint64_t t = (hi << 32) | (lo >> 32);  // floor(u^3 / 2^32)
#ifdef __CUDA_ARCH__
  return (uint32_t)__umul64hi(t, (uint64_t)m);
#else
  return (uint32_t)(((unsigned __int128)t * m) >> 64);
#endif
}

// Device-resident control block of a solve (read by every kernel of a
// generation, so that a captured generation can be replayed unchanged).
struct DevCtrl {
  uint64_t seed;
  uint32_t g;           // generation index
  uint32_t done;        // set when a stop condition holds; kernels then return at once
  uint64_t flips_total;
  uint64_t budget;
  int64_t target;
  uint32_t max_generations;  // 0 = unlimited
  uint32_t restarts;         // pool restarts so far (the epoch of the pool draws)
  int64_t best_E;
};

// Arguments of the batch-search kernel (one launch = one batch search per search slot).
struct SearchArgs {
  const int16_t* W;     // [n][ld] row-major, zero padded
  const int16_t* Wneg;  // -W, same layout
  const int32_t* diag;  // [n] W_kk
  int32_t n, ld, nw; // nw = 32-bit words of a bit vector
  int32_t S;         // search slots in this launch
  int32_t T;         // flips per main search
  int32_t tau;       // tabu period
  uint32_t B;        // batch flip budget b*n
  int32_t seed_mode; // 0 = Straight walk to D; 1 = X already set to D
  const DevCtrl* ctrl;
  uint32_t* X;       // [S][nw]  persistent state
  int32_t* delta;    // [S][ld]
  int64_t* E;        // [S]
  const int64_t* E2;  // [S] or null: 2 E from the batched recompute (E = E2 / 2 at the start)
  const uint32_t* D; // [S][nw]  targets
  const uint8_t* algo; // [S]
  uint32_t* best_X;  // [S][nw]
  int64_t* best_E;   // [S]
  uint32_t* flips;   // [S]
  const int32_t* order; // launch order of the slots (grouped by algorithm), or null
  int32_t spc;          // searches per CTA actually used (<= the variant's maximum; 0 = maximum)
  // row format (single-instance launches only): 0 dense rows of W; 3 the same
  // rows from a shared-memory copy of W (one-warp variants, small n); sparse
  // rows, where row i holds the entries sp_ent[sp_row[i] .. sp_row[i+1]), each
  // (k << 16) | (uint16) W_ik for k != i with W_ik != 0, k ascending, both
  // arrays padded with zeros to a multiple of four entries, read from a
  // shared-memory copy (1) or from global memory (2)
  int32_t sp_mode;
  const uint32_t* sp_row;
  const uint32_t* sp_ent;
  int32_t sp_nnz;
  // keyed Delta (single-instance dense-row launches): 0 = off; else the bits
  // of (k << 1 | x_k) below the Delta part of a key, bitlen(n - 1) + 1, valid
  // when (2 R + 2) 2^key_bits < 2^31 for R = max_k sum_j |W_kj|
  int32_t key_bits;
  int* serr;  // error flag of the kernels with bounded waits (may be null)
  int32_t stall_test;  // 1: the shared-memory variant's first row wait gets no copy (test hook)
};

enum RowFormat : int { ROWS_DENSE = 0, ROWS_SPARSE_SMEM = 1, ROWS_SPARSE_GLOBAL = 2,
                       ROWS_DENSE_SMEM = 3 };

// Dynamic shared memory of the sparse-row batch search: with the shared-memory
// copy, the row offsets and the entries (each section padded to 16 bytes);
// then one scratch row of ld int16 per search of the CTA.
__host__ __device__ inline int sparse_row16(int n) { return (n + 1 + 3) / 4; }
__host__ __device__ inline int sparse_ent16(int nnz) { return (nnz + 3) / 4; }
__host__ __device__ inline size_t sparse_smem_bytes(int mode, int n, int nnz, int ld, int spc) {
  if (mode == ROWS_DENSE_SMEM) return (size_t)n * ld * 2;  // W itself, no scratch rows
  const size_t copy = mode == ROWS_SPARSE_SMEM ? 16 * ((size_t)sparse_row16(n) + sparse_ent16(nnz)) : 0;
  return copy + (size_t)spc * ld * 2;
}

// Several instances in one batch-search launch: slot q belongs to the
// instance i with prefix[i] <= q < prefix[i+1] and is its (q - prefix[i])-th slot.
struct MultiArgs {
  const SearchArgs* insts;  // [ninst] in device memory
  const int32_t* prefix;    // [ninst + 1] slot offsets
  int32_t ninst;
  int32_t total;            // prefix[ninst]
  int32_t max_n;            // largest n among the instances
};

}  // namespace dabs
