// umma.cu -- from-scratch Delta and energy of a batch of vectors on the
// tensor cores (5th-generation, tcgen05): F = D * W for D in {0,1}^{S x n},
// then Eq. (3) Delta_k = -sigma(d_k) F_k + W_kk (1 - d_k) and Eq. (2)
// E = (sum_k d_k F_k + sum_k d_k W_kk) / 2.
//
// Exactness.  Every product is an integer and the fp32 accumulator is exact
// while every partial sum stays below 2^24 in magnitude.  Two operand forms:
//  - one limb: W itself as fp16, exact for |W_ij| <= 2048 (11 significant
//    bits), used when also n * max|W_ij| < 2^24 (all the benchmark
//    workloads: |W| <= 1000, n <= 16384);
//  - two limbs: W = 256 hi + lo with lo in [0, 255], hi in [-128, 127],
//    both exact in bf16; n * 255 < 2^24 holds for n <= 65,793, and
//    F = 256 F_hi + F_lo is exact in int32.
// D's 0/1 entries are exact in either type (A and B of one MMA share it).
// The int8 MMA (tcgen05.mma .kind::i8) that would keep D and the limbs in
// 8 bits is not available on sm_103a (ptxas rejects the form for this
// target), so the limbs are 16-bit floats.
//
// Kernel: one CTA per 256 x 64 output tile (256 vectors as two M = 128
// accumulators, so each column tile of W is streamed once for 256 vectors),
// 6 warps with fixed roles: warp 0 streams K-blocks of 64 (128 bytes) of D
// and of W's limb(s) into a 4-stage shared-memory ring with TMA (128-byte
// swizzle); warp 1 issues tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16)
// into the TMEM accumulators and releases each stage by tcgen05.commit;
// warps 2-5 then read their TMEM lane quarters with tcgen05.ld and write
// Delta and the energy partial sums.  Every mbarrier wait is bounded; on
// expiry the kernel records an error code and returns after releasing its
// TMEM.
#include <cuda.h>
#include <cuda_fp16.h>

#include "kernels.cuh"
#include "umma.cuh"

namespace dabs {
namespace {

constexpr int BM = 256, HM = 128, BN = 64, BK = 64, STAGES = 4;
constexpr uint32_t A_BYTES = BM * BK * 2;        // 32 KiB: D tile (two 16 KiB halves)
constexpr uint32_t B_BYTES = BN * BK * 2;        // 8 KiB: one limb tile
constexpr uint32_t STAGE_MAX = A_BYTES + 2 * B_BYTES;
constexpr uint64_t WAIT_NS = 2000000000ull;      // 2 s per wait
constexpr int kThreads = 192;                    // 6 warps

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false on timeout or abort
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if ((it & 63) == 63) {
      if (global_ns() - t0 > WAIT_NS) return false;
      __nanosleep(128);
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// of 1024 bytes (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}
// instruction descriptor of kind::f16: D fp32, A and B both fp16 (type 0) or
// both bf16 (type 1), K-major, N = BN, M = 128
template <int LIMBS>
__host__ __device__ constexpr uint32_t idesc() {
  constexpr uint32_t ty = LIMBS == 2 ? 1u : 0u;
  return (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(HM >> 4) << 24);
}

template <int LIMBS>
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc<LIMBS>()), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

// D bits [count][nw] -> 0/1 matrix [rows_pad][n_pad] of 16-bit floats (zero
// padding); `one` is the encoding of 1.0 (0x3C00 fp16, 0x3F80 bf16)
__global__ void k_bits_to_bf16(const uint32_t* D, int count, int n, int nw, int rows_pad,
                               int n_pad, uint16_t* A, uint32_t one, const DevCtrl* ctrl) {
  if (ctrl && ctrl->done) return;
  const size_t total = (size_t)rows_pad * (n_pad / 2);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / (n_pad / 2)), k = 2 * (int)(q % (n_pad / 2));
    uint32_t v = 0;
    if (r < count && k < n) {
      const uint32_t w = D[(size_t)r * nw + (k >> 5)];
      const uint32_t b0 = (w >> (k & 31)) & 1u, b1 = (k + 1 < n) ? ((w >> ((k + 1) & 31)) & 1u) : 0u;
      v = (b0 ? one : 0u) | ((b1 ? one : 0u) << 16);
    }
    reinterpret_cast<uint32_t*>(A)[q] = v;
  }
}

// W [n][ld] int16 -> [n_pad][n_pad] operand(s): one limb, W as fp16 in Whi;
// or two limbs, hi = W >> 8 (arithmetic) in Whi and lo = W & 255 in Wlo, bf16
__global__ void k_limbs(const int16_t* W, int n, int ld, int n_pad, int limbs, uint16_t* Whi,
                        uint16_t* Wlo) {
  const size_t total = (size_t)n_pad * n_pad;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n_pad), c = (int)(q % n_pad);
    const int w = (r < n && c < n) ? (int)W[(size_t)r * ld + c] : 0;
    if (limbs == 1) {
      Whi[q] = __half_as_ushort(__int2half_rn(w));  // exact: |w| <= 2048
    } else {
      // |limb| <= 255 needs at most 8 significant bits, so the upper half of
      // the fp32 encoding is the exact bf16 encoding
      Whi[q] = (uint16_t)(__float_as_uint((float)(w >> 8)) >> 16);
      Wlo[q] = (uint16_t)(__float_as_uint((float)(w & 255)) >> 16);
    }
  }
}

// F of one accumulator element (fp32 holding an exact integer)
__device__ __forceinline__ int fint(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }

// one 256 x 64 output tile (n_tile, m_tile) of one instance; the tensor maps
// may live in kernel parameters or in global memory
template <int LIMBS>
__device__ __forceinline__ void recompute_tile(const CUtensorMap* pA, const CUtensorMap* pHi,
                                               const CUtensorMap* pLo, const UmmaArgs& a,
                                               int n_tile, int m_tile, unsigned char* smraw) {
  constexpr uint32_t STAGE_BYTES = A_BYTES + LIMBS * B_BYTES;
  constexpr uint32_t TMEM_COLS = LIMBS * 2 * BN;  // accumulator (limb l, half h) at (2l + h) BN
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int sdiag[BN];  // W_kk of the tile's columns (0 past n)
  if (a.ctrl && a.ctrl->done) return;
  // 1024-byte aligned operand ring
  const uint32_t base = (smem_u32(smraw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = n_tile * BN, m0 = m_tile * BM;
  const int KB = a.n_pad / BK;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x < BN) sdiag[threadIdx.x] = n0 + (int)threadIdx.x < a.n ? a.diag[n0 + threadIdx.x] : 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // producer: TMA, up to STAGES K-blocks ahead of the MMAs
      int issued = 0;
      for (int kb = 0; kb < KB && !abort_flag; ++kb) {
        const int st = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[st], (uint32_t)((kb / STAGES) - 1) & 1u, &abort_flag)) {
          abort_flag = 1;
          break;
        }
        const uint32_t s0 = base + st * STAGE_BYTES;
        mbar_expect_tx(&full[st], STAGE_BYTES);
        tma_load_2d(s0, pA, kb * BK, m0, &full[st]);
        tma_load_2d(s0 + A_BYTES, pHi, kb * BK, n0, &full[st]);
        if constexpr (LIMBS == 2) tma_load_2d(s0 + A_BYTES + B_BYTES, pLo, kb * BK, n0, &full[st]);
        ++issued;
      }
      if (abort_flag) {  // let the copies in flight land before the CTA leaves (bounded)
        const int zero = 0;
        for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
          mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issue
      bool ok = true;
      for (int kb = 0; kb < KB && ok && !abort_flag; ++kb) {
        const int st = kb % STAGES;
        if (!mbar_wait(&full[st], (uint32_t)(kb / STAGES) & 1u, &abort_flag)) {
          abort_flag = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t s0 = base + st * STAGE_BYTES;
        const uint64_t da0 = sdesc(s0), da1 = sdesc(s0 + A_BYTES / 2);
        const uint64_t db0 = sdesc(s0 + A_BYTES), db1 = sdesc(s0 + A_BYTES + B_BYTES);
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
          // +32 bytes per K step of 16 elements inside the 128-byte swizzled row
          mma_f16<LIMBS>(tm, da0 + 2 * ks, db0 + 2 * ks, acc);
          mma_f16<LIMBS>(tm + BN, da1 + 2 * ks, db0 + 2 * ks, acc);
          if constexpr (LIMBS == 2) {
            mma_f16<LIMBS>(tm + 2 * BN, da0 + 2 * ks, db1 + 2 * ks, acc);
            mma_f16<LIMBS>(tm + 3 * BN, da1 + 2 * ks, db1 + 2 * ks, acc);
          }
        }
        mma_commit(&empty[st]);
      }
      mma_commit(&done);  // also after an abort: the MMAs issued complete before TMEM is freed
      if (!ok || abort_flag) {
        const int zero = 0;
        mbar_wait(&done, 0, (volatile int*)&zero);
      }
    }
  } else {
    // epilogue warps 2-5: warp w reads TMEM lane quarter w % 4, i.e. rows
    // 32 (w % 4) + lane of both halves; their D words are fetched while the
    // MMAs run
    const int q = warp & 3;
    uint32_t dwords[2][BN / 32];
    bool row_ok[2];
    int row[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      row[h] = m0 + HM * h + 32 * q + lane;
      row_ok[h] = row[h] < a.count;
#pragma unroll
      for (int c = 0; c < BN / 32; ++c) {
        const int kb0 = n0 + 32 * c;
        dwords[h][c] = (row_ok[h] && kb0 < a.n) ? a.D[(size_t)row[h] * a.nw + (kb0 >> 5)] : 0u;
      }
    }
    bool ok = mbar_wait(&done, 0, &abort_flag);
    __syncwarp();
    if (!ok || abort_flag) {
      if (a.err && lane == 0) atomicExch(a.err, DABS_KERNEL_TIMEOUT);
      abort_flag = 1;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t lane_off = (uint32_t)(32 * q) << 16;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int64_t epart = 0;
        int32_t* drow = a.delta ? a.delta + (size_t)(row_ok[h] ? row[h] : 0) * a.ld_delta : nullptr;
        const bool vec = drow && (a.ld_delta & 3) == 0 && (reinterpret_cast<uintptr_t>(a.delta) & 15) == 0;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          uint32_t rh[32], rl[32];
          tmem_ld32(tm + lane_off + (uint32_t)(h * BN + c0), rh);
          if constexpr (LIMBS == 2) tmem_ld32(tm + lane_off + (uint32_t)(2 * BN + h * BN + c0), rl);
          const int kbase = n0 + c0;
          if (!row_ok[h] || kbase >= a.n) continue;
          const uint32_t dword = dwords[h][c0 >> 5];
#pragma unroll
          for (int j4 = 0; j4 < 32; j4 += 4) {
            int v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = j4 + e;
              const int F = LIMBS == 2 ? 256 * fint(rh[j]) + fint(rl[j]) : fint(rh[j]);
              const int wkk = sdiag[c0 + j];
              const bool dk = (dword >> j) & 1u;
              v[e] = dk ? -F : F + wkk;  // Eq. (3)
              if (dk && kbase + j < a.n) epart += (int64_t)F + wkk;
            }
            const int k0 = kbase + j4;
            if (!drow || k0 >= a.n) continue;
            if (vec && k0 + 3 < a.n) {
              *reinterpret_cast<int4*>(drow + k0) = make_int4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (k0 + e < a.n) drow[k0 + e] = v[e];
            }
          }
        }
        if (row_ok[h] && a.E2)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.E2 + row[h]), (unsigned long long)epart);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TMEM_COLS) : "memory");
}

template <int LIMBS>
__global__ void __launch_bounds__(kThreads, 1)
    k_recompute_umma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapHi,
                     const __grid_constant__ CUtensorMap mapLo, const UmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  recompute_tile<LIMBS>(&mapA, &mapHi, &mapLo, a, blockIdx.x, blockIdx.y, smraw);
}

// every instance's tiles in one launch: CTA q belongs to the instance i with
// prefix[i] <= q < prefix[i+1]
__global__ void __launch_bounds__(kThreads, 1)
    k_recompute_multi(const RecInst* insts, const int32_t* prefix, int ninst) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int cta = blockIdx.x;
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= cta) lo = mid; else hi = mid;
  }
  const RecInst& r = insts[lo];
  const int local = cta - prefix[lo];
  if (r.limbs == 1)
    recompute_tile<1>(&r.mapA, &r.mapHi, &r.mapLo, r.a, local % r.tiles_n, local / r.tiles_n, smraw);
  else
    recompute_tile<2>(&r.mapA, &r.mapHi, &r.mapLo, r.a, local % r.tiles_n, local / r.tiles_n, smraw);
}

void launch_recompute_multi(const RecInst* insts, const int32_t* prefix, int ninst, int ctas,
                            cudaStream_t st) {
  k_recompute_multi<<<ctas, kThreads, umma_smem_bytes(), st>>>(insts, prefix, ninst);
}

bool umma_prepare() {
  const int bytes = (int)umma_smem_bytes();
  return cudaFuncSetAttribute(k_recompute_umma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_recompute_umma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_recompute_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess;
}

void launch_recompute_umma(int limbs, dim3 grid, cudaStream_t st, const CUtensorMap& mapA,
                           const CUtensorMap& mapHi, const CUtensorMap& mapLo, const UmmaArgs& a) {
  if (limbs == 1)
    k_recompute_umma<1><<<grid, kThreads, umma_smem_bytes(), st>>>(mapA, mapHi, mapLo, a);
  else
    k_recompute_umma<2><<<grid, kThreads, umma_smem_bytes(), st>>>(mapA, mapHi, mapLo, a);
}

// E = E2 / 2 (E2 holds sum_k d_k (F_k + W_kk), always even)
__global__ void k_halve(int64_t* E, const int64_t* E2, int count, const DevCtrl* ctrl) {
  if (ctrl && ctrl->done) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
    E[q] = E2[q] / 2;
}

size_t umma_smem_bytes() { return (size_t)STAGES * STAGE_MAX + 1024; }
int umma_tile_m() { return BM; }
int umma_tile_n() { return BN; }
int umma_tile_k() { return BK; }

}  // namespace dabs

namespace dabs {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool make_tmap_bf16(CUtensorMap* map, void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)umma_tile_k(), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace dabs
