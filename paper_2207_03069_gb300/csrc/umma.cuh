// umma.cuh -- tensor-core (tcgen05) batched Delta/energy recompute: kernel
// arguments, launch helpers and the TMA tensor-map builder.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace dabs {

constexpr int DABS_KERNEL_TIMEOUT = 1;  // error code a kernel writes when a bounded wait expires

struct UmmaArgs {
  int count;              // vectors (rows of D)
  int n, n_pad, nw;       // problem size, padded size (multiple of 128), words per vector
  int ld_delta;           // row stride of delta
  const uint32_t* D;      // [count][nw] packed vectors
  const int32_t* diag;    // W_kk
  int32_t* delta;         // [count][ld_delta] or null
  int64_t* E2;            // [count] receives 2 E (zeroed before the launch) or null
  int* err;               // kernel error flag (0 = ok)
  const DevCtrl* ctrl;    // optional: skip when a solve has stopped
};

__global__ void k_bits_to_bf16(const uint32_t* D, int count, int n, int nw, int rows_pad,
                               int n_pad, uint16_t* A, uint32_t one, const DevCtrl* ctrl);
__global__ void k_limbs(const int16_t* W, int n, int ld, int n_pad, int limbs, uint16_t* Whi,
                        uint16_t* Wlo);
// one instance of the batched form's recompute launch
struct RecInst {
  CUtensorMap mapA, mapHi, mapLo;  // 64-byte aligned
  UmmaArgs a;
  int limbs;    // 1 or 2 (as launch_recompute_umma)
  int tiles_n;  // n_pad / umma_tile_n()
};

// the tensor-core recompute: limbs = 1, W as one fp16 operand; 2, two bf16
// limbs (see umma.cu).  umma_prepare sets the kernels' shared-memory limit
// (once); false on a CUDA error.
bool umma_prepare();
void launch_recompute_umma(int limbs, dim3 grid, cudaStream_t st, const CUtensorMap& mapA,
                           const CUtensorMap& mapHi, const CUtensorMap& mapLo, const UmmaArgs& a);
// the recompute of several instances in one launch (insts, prefix in device
// memory; prefix[i] = first CTA of instance i, ctas = prefix[ninst])
void launch_recompute_multi(const RecInst* insts, const int32_t* prefix, int ninst, int ctas,
                            cudaStream_t st);
__global__ void k_halve(int64_t* E, const int64_t* E2, int count, const DevCtrl* ctrl);

size_t umma_smem_bytes();
int umma_tile_m();
int umma_tile_n();
int umma_tile_k();
// 2-D bf16 tensor map (rows x cols, row-major) with a box of 64 columns x
// box_rows rows and 128-byte swizzle
bool make_tmap_bf16(CUtensorMap* map, void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows);

}  // namespace dabs
