// weights.cu -- residency of an instance (the W of Eq. (1), kept in global
// memory as in Section V-A): the caller's rows arrive by one DMA into a
// staging buffer, and these kernels check them (symmetry, no -32768), measure
// them (row sums of |W|, off-diagonal non-zeros per row, their prefix sums)
// and, once the host has read the outcome, commit W, -W and the diagonal and
// build the sparse rows.  Loading an instance thus reads the host buffer once.
#include "kernels.cuh"

namespace dabs {

// One block per 32 x 32 tile pair (ti <= tj): tile A holds rows ti*32.. x
// columns tj*32.., tile B its mirror, rows tj*32.. x columns ti*32...  Every
// entry of W lies in exactly one A or one B, so the per-row sums and counts
// see each entry once.  A mismatch A[r][c] != B[c][r] is an asymmetric pair;
// -32768 is looked for in A only (an entry of B equals its mirror in A unless
// that pair is already asymmetric).  Both are reported by their lowest linear
// index i * n + j.
__global__ void k_weights_tiles(const WeightsArgs a) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  __shared__ int16_t A[32][33], B[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  const int n = a.n;
  for (int r = ty; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + tx;
    A[r][tx] = (i < n && j < n) ? a.Ws[(size_t)i * a.ld + j] : (int16_t)0;
    const int i2 = tj * 32 + r, j2 = ti * 32 + tx;
    B[r][tx] = (i2 < n && j2 < n) ? a.Ws[(size_t)i2 * a.ld + j2] : (int16_t)0;
  }
  __syncthreads();
  unsigned long long bad = ~0ull, low = ~0ull, nmax = ~0ull;
  for (int r = ty; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + tx;
    const int16_t w = A[r][tx];
    nmax = min(nmax, ~(unsigned long long)abs((int)w));
    if (ti != tj) nmax = min(nmax, ~(unsigned long long)abs((int)B[r][tx]));
    if (i < n && j < n) {
      const unsigned long long at = (unsigned long long)i * n + j;
      if (w != B[tx][r]) bad = min(bad, at);
      if (w == INT16_MIN) low = min(low, at);
    }
    // row i over this tile's columns (entries outside W were loaded as 0)
    unsigned s = (unsigned)abs((int)w), c = (w != 0 && j != i) ? 1u : 0u;
    if (ti != tj) {  // the mirror tile: row tj*32 + r, no diagonal entries
      const int16_t v = B[r][tx];
      unsigned s2 = (unsigned)abs((int)v), c2 = v != 0 ? 1u : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      }
      const int i2 = tj * 32 + r;
      if (tx == 0 && i2 < n) {
        atomicAdd(a.rowsum + i2, s2);
        atomicAdd(a.rowcnt + i2, c2);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (tx == 0 && i < n) {
      atomicAdd(a.rowsum + i, s);
      atomicAdd(a.rowcnt + i, c);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad = min(bad, __shfl_xor_sync(0xffffffffu, bad, o));
    low = min(low, __shfl_xor_sync(0xffffffffu, low, o));
    nmax = min(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
  }
  if (tx == 0) {
    if (bad != ~0ull) atomicMin(&a.chk->bad, bad);
    if (low != ~0ull) atomicMin(&a.chk->low, low);
    if (nmax != ~0ull) atomicMin(&a.chk->nmax, nmax);
  }
}

// One block of 1024 threads: R = max_i sum_j |W_ij|, the off-diagonal
// non-zero total, and the exclusive prefix sums of the row counts (rowptr[i],
// rowptr[n] = total, zeros after it).  Each thread scans a contiguous run of
// rows; the runs' totals are scanned across the block.
__global__ void k_weights_rows(const WeightsArgs a) {
  __shared__ unsigned long long part[32];
  __shared__ unsigned rmax[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int n = a.n, per = (n + 1023) / 1024;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  unsigned long long sum = 0;
  unsigned mx = 0;
  for (int i = lo; i < hi; ++i) {
    sum += a.rowcnt[i];
    mx = max(mx, a.rowsum[i]);
  }
  // inclusive scan of the runs' totals: within warps, then across them
  unsigned long long inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 31) part[wid] = inc;
  if (lane == 0) rmax[wid] = mx;
  __syncthreads();
  if (wid == 0) {
    unsigned long long p = part[lane];
    unsigned m = rmax[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, p, o);
      if (lane >= o) p += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    part[lane] = p;  // inclusive over warps
    if (lane == 31) {
      a.chk->nnz = p;
      a.chk->R = m;
    }
  }
  __syncthreads();
  unsigned long long run = inc - sum + (wid > 0 ? part[wid - 1] : 0ull);
  for (int i = lo; i < hi; ++i) {
    a.rowptr[i] = (uint32_t)run;
    run += a.rowcnt[i];
  }
  for (int i = n + t; i < a.rowptr_len; i += 1024) a.rowptr[i] = i == n ? (uint32_t)part[31] : 0u;
}

// W = staged rows, -W and the diagonal, 8 entries (one 16-byte vector) per
// step; rows are ld = 64k entries long, so a vector never spans two rows.
// Columns n..ld-1 are written as zero.  The staging buffer may be Wneg itself.
__global__ void k_weights_commit(const WeightsArgs a) {
  const size_t vecs = (size_t)a.n * a.ld / 8;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < vecs;
       q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q * 8 / a.ld), j0 = (int)(q * 8 % a.ld);
    uint4 v = reinterpret_cast<const uint4*>(a.Ws)[q];
    if (j0 + 8 > a.n) {  // zero the halves at columns >= n
      const auto keep = [&](uint32_t h, int j) {
        return j >= a.n ? 0u : j + 1 >= a.n ? (h & 0xffffu) : h;
      };
      v = make_uint4(keep(v.x, j0), keep(v.y, j0 + 2), keep(v.z, j0 + 4), keep(v.w, j0 + 6));
    }
    if (i >= j0 && i < j0 + 8) {
      const int e = (i - j0) >> 1;
      const uint32_t pair = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
      a.diag[i] = (int32_t)(int16_t)((i - j0) & 1 ? pair >> 16 : pair & 0xffffu);
    }
    reinterpret_cast<uint4*>(a.W)[q] = v;
    reinterpret_cast<uint4*>(a.Wneg)[q] = make_uint4(__vneg2(v.x), __vneg2(v.y), __vneg2(v.z), __vneg2(v.w));
  }
}

// Sparse rows: one warp per row writes the row's off-diagonal non-zeros,
// column ascending, as (k << 16) | (uint16) W_ik from rowptr[i] on.
__global__ void k_sparse_fill(const WeightsArgs a) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= a.n) return;
  const int16_t* row = a.W + (size_t)i * a.ld;
  uint32_t at = a.rowptr[i];
  for (int c0 = 0; c0 < a.n; c0 += 32) {
    const int k = c0 + lane;
    const int16_t w = k < a.n ? row[k] : (int16_t)0;
    const bool keep = w != 0 && k != i;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) a.ent[at + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)k << 16) | (uint16_t)w;
    at += __popc(m);
  }
}

}  // namespace dabs
