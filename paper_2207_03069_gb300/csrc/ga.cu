// ga.cu -- device kernels of the genetic layer (Section IV) and of the solve
// bookkeeping: pool initialisation, offspring (parent selection, 5%/95%
// operation and algorithm choice, the eight genetic operations, Xrossover
// between neighbouring islands), pool merge (packets inserted iff better than
// the worst entry, duplicates rejected), and the per-generation finalisation
// (global best, flip count, stop flag).  Also the CUDA-core batched
// energy/Delta evaluation used by the host-side dabs_energy / dabs_delta.
#include "kernels.cuh"

namespace dabs {

// ---------------------------------------------------------------- init
__global__ void k_pool_init(const PoolArgs a) {
  const int lane = threadIdx.x & 31;
  const int e_glob = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // entry = p*C + e
  if (e_glob >= a.P * a.C) return;
  if (a.cond && *a.cond != 0) return;  // no restart this generation
  const uint32_t p = (uint32_t)(e_glob / a.C), e = (uint32_t)(e_glob % a.C);
  const uint64_t seed = a.ctrl->seed;
  const uint32_t epoch = a.cond ? a.ctrl->restarts + 1 : 0;  // the restart being made
  const int cur = a.ctrl->g & 1;
  uint32_t* x = a.pool_X[cur] + (size_t)e_glob * a.nw;
  for (int w = lane; w < a.nw; w += 32) {
    const uint4 u = draw(seed, (uint32_t)w, e, p, RNG_INIT_BITS | epoch);
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t word = j < 8 ? u.x : j < 16 ? u.y : j < 24 ? u.z : u.w;
      v |= ((word >> (4 * (j & 7))) & 1u) << j;
    }
    x[w] = v & valid_mask(w, a.n);
  }
  if (lane == 0) {
    const uint4 u = draw(seed, 0, e, p, RNG_INIT_TAGS | epoch);
    a.pool_E[cur][e_glob] = INT64_MAX;
    a.pool_algo[cur][e_glob] = (uint8_t)uniform_below(u.x, N_ALGOS);
    a.pool_op[cur][e_glob] = (uint8_t)uniform_below(u.y, N_OPS);
  }
}

// Wneg = -W, element by element (weights lie in [-32767, 32767])
__global__ void k_negate(const int16_t* W, int16_t* Wneg, size_t count) {
  const size_t v = count / 8;  // 8 int16 per 16-byte vector
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < v; q += (size_t)gridDim.x * blockDim.x) {
    const uint4 w = reinterpret_cast<const uint4*>(W)[q];
    reinterpret_cast<uint4*>(Wneg)[q] = make_uint4(__vneg2(w.x), __vneg2(w.y), __vneg2(w.z), __vneg2(w.w));
  }
  for (size_t q = 8 * v + blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x)
    Wneg[q] = (int16_t)-W[q];
}

// X = 0, E = 0, Delta_k = W_kk for every search slot (Section III-B start).
__global__ void k_state_init(const StateArgs a) {
  if (a.cond && *a.cond != 0) return;
  if (a.bump && blockIdx.x == 0 && threadIdx.x == 0) a.bump->restarts += 1;
  const size_t total = (size_t)a.S * a.ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % a.ld);
    a.delta[q] = k < a.n ? a.diag[k] : 0;
  }
  const size_t xw = (size_t)a.S * a.nw;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < xw;
       q += (size_t)gridDim.x * blockDim.x)
    a.X[q] = 0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)a.S;
       q += (size_t)gridDim.x * blockDim.x)
    a.E[q] = 0;
  if (a.gbest_X)
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)a.nw;
         q += (size_t)gridDim.x * blockDim.x)
      a.gbest_X[q] = 0;
}

// Section IV-B, last paragraph: the pools have merged when every entry lies
// within Hamming distance h of the global best.  One warp per entry; any
// entry farther than h sets the flag.  The flag reads 1 (skip) unless
// k_finalize ran in this generation and armed it.
__global__ void k_restart_check(const RestartArgs a) {
  if (*a.flag != 0) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t* PX = a.pool_X[a.ctrl->g & 1];
  for (int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < a.P * a.C; q += warps) {
    const uint32_t* x = PX + (size_t)q * a.nw;
    int d = 0;
    for (int w = lane; w < a.nw; w += 32) d += __popc(x[w] ^ a.gbest_X[w]);
    d = __reduce_add_sync(FULLMASK, d);
    if (d > a.h) {
      if (lane == 0) atomicOr(a.flag, 1u);
      return;
    }
  }
}

// ---------------------------------------------------------------- offspring
__device__ __forceinline__ uint32_t interval_mask(int w, int lo, int hi) {
  // bits of word w inside [lo, hi)
  const int a0 = max(lo, 32 * w), b0 = min(hi, 32 * w + 32);
  if (a0 >= b0) return 0u;
  const int len = b0 - a0;
  const uint32_t m = len == 32 ? FULLMASK : ((1u << len) - 1u);
  return m << (a0 - 32 * w);
}

// the target, algorithm and operation of search s (one warp)
__device__ void offspring_one(const OffArgs& a, int s, int lane) {
  const DevCtrl* ctrl = a.ctrl;
  const uint32_t g = ctrl->g;
  const uint64_t seed = ctrl->seed;
  const int cur = g & 1;
  const uint32_t P = (uint32_t)a.P, C = (uint32_t)a.C;
  const uint32_t p = (uint32_t)s % P, q = (p + 1) % P;
  const uint32_t* PX = a.pool_X[cur];
  // Section IV-A: 5% uniform choice, 95% copy of a random pool row's field
  const uint4 c = draw(seed, 0, g, (uint32_t)s, RNG_CHOICE);
  int op = c.x < kMixThreshold ? (int)uniform_below(c.y, N_OPS)
                               : (int)a.pool_op[cur][p * C + uniform_below(c.y, C)];
  int algo = c.z < kMixThreshold ? (int)uniform_below(c.w, N_ALGOS)
                                 : (int)a.pool_algo[cur][p * C + uniform_below(c.w, C)];
  if (a.abs_mode) {  // the earlier ABS: CyclicMin, mutation after crossover
    op = CROSSOVER;
    algo = CYCLICMIN;
  }
  const uint4 r = draw(seed, 0, g, (uint32_t)s, RNG_PARENT);
  const uint32_t* A = PX + ((size_t)p * C + parent_rank(r.x, C)) * a.nw;
  const uint32_t bp = op == XROSSOVER ? q : p;  // Section IV-B: neighbour island
  const uint32_t* Bv = PX + ((size_t)bp * C + parent_rank(r.y, C)) * a.nw;
  const uint32_t* best = PX + ((size_t)p * C) * a.nw;
  const int hi = a.n / 2, lo = hi < 32 ? hi : 32;
  const int len = lo + (int)uniform_below(r.z, (uint32_t)(hi - lo + 1));
  const int start = (int)uniform_below(r.w, (uint32_t)a.n);
  uint32_t* D = a.D + (size_t)s * a.nw;
  for (int w = lane; w < a.nw; w += 32) {
    const uint4 u = draw(seed, (uint32_t)w, g, (uint32_t)s, RNG_BITS);
    uint32_t hit = 0, coin = 0, coin3 = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t word = j < 8 ? u.x : j < 16 ? u.y : j < 24 ? u.z : u.w;
      const uint32_t nib = (word >> (4 * (j & 7))) & 0xFu;
      hit |= (uint32_t)((nib & 7u) == 0u) << j;
      coin |= (nib & 1u) << j;
      coin3 |= (nib >> 3) << j;
    }
    const uint32_t av = A[w], bv = Bv[w];
    uint32_t v;
    if (a.abs_mode) {  // coin from bit 3 of the nibble, then the mutation mask
      D[w] = (((bv & coin3) | (av & ~coin3)) ^ hit) & valid_mask(w, a.n);
      continue;
    }
    switch (op) {
      case MUTATION: v = av ^ hit; break;
      case CROSSOVER:
      case XROSSOVER: v = (bv & coin) | (av & ~coin); break;
      case ZERO: v = av & ~hit; break;
      case ONE: v = av | hit; break;
      case INTERVALZERO: {
        uint32_t seg = interval_mask(w, start, min(start + len, a.n));
        if (start + len > a.n) seg |= interval_mask(w, 0, start + len - a.n);
        v = av & ~seg;
        break;
      }
      case BEST: v = best[w]; break;
      default: v = coin; break;
    }
    D[w] = v & valid_mask(w, a.n);
  }
  if (lane == 0) {
    a.algo[s] = (uint8_t)algo;
    a.op[s] = (uint8_t)op;
  }
}

__global__ void k_offspring(const OffArgs a) {
  const int lane = threadIdx.x & 31;
  const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (s >= a.S) return;
  if (a.ctrl->done) return;
  offspring_one(a, s, lane);
}

// ---------------------------------------------------------------- merge
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// warp-cooperative hash of a bit vector (only accelerates equality tests)
__device__ __forceinline__ uint64_t warp_hash(const uint32_t* x, int nw, int lane) {
  uint64_t h = 0;
  for (int w = lane; w < nw; w += 32) h ^= mix64(((uint64_t)w << 32) | x[w]);
#pragma unroll
  for (int off = 16; off; off >>= 1) h ^= __shfl_xor_sync(FULLMASK, h, off);
  return h;
}

__device__ __forceinline__ bool same_bits(const uint32_t* x, const uint32_t* y, int nw) {
  for (int w = 0; w < nw; ++w)
    if (x[w] != y[w]) return false;
  return true;
}

constexpr int64_t kEnergyBias = (int64_t)1 << 46;  // |E| < 2^46 for n <= 65536, int16 W

// One CTA per pool.  The sequential insertion of the results in search order
// (enter iff E < E(worst) and no entry holds the same (E, X); placed after
// equal energies; worst dropped) equals: the first C of the union of the old
// entries (first) and the new results (in search order), stably sorted by
// energy, after dropping later copies of an equal (E, X).
__device__ void merge_pool(const MergeArgs& a, int p, unsigned char* smraw) {
  const DevCtrl* ctrl = a.ctrl;
  const uint32_t g = ctrl->g;
  const int cur = g & 1, nxt = cur ^ 1;
  const int C = a.C, P = a.P, nw = a.nw;
  const int R = (a.S - p + P - 1) / P;  // results of this pool: s = p + P*r
  const int M = a.Mmax;                 // power of two >= R
  int64_t* oldE = reinterpret_cast<int64_t*>(smraw);                 // [C]
  uint64_t* oldH = reinterpret_cast<uint64_t*>(oldE + C);            // [C]
  uint64_t* key = oldH + C;                                          // [M]
  uint64_t* cH = key + M;                                            // [M]
  int* uflag = reinterpret_cast<int*>(cH + M);                       // [M]
  int* upos = uflag + M;                                             // [M]
  __shared__ int ncand, nuniq;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t* PE = a.pool_E[cur] + (size_t)p * C;
  const uint32_t* PX = a.pool_X[cur] + (size_t)p * C * nw;
  for (int e = tid; e < C; e += blockDim.x) oldE[e] = PE[e];
  if (tid == 0) ncand = 0;
  __syncthreads();
  const int64_t worst = oldE[C - 1];
  // candidates (E < worst) with a sortable key ((E + bias) << 17 | r)
  for (int r = tid; r < M; r += blockDim.x) {
    uint64_t kv = ~0ull;
    if (r < R) {
      const int s = p + P * r;
      const int64_t e = a.best_E[s];
      if (e < worst) kv = ((uint64_t)(e + kEnergyBias) << 17) | (uint64_t)r;
    }
    key[r] = kv;
  }
  __syncthreads();
  // bitonic sort of M keys (ascending; non-candidates = ~0 sink to the end)
  for (int k = 2; k <= M; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < M; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = key[i], y = key[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { key[i] = y; key[l] = x; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < M; i += blockDim.x)
    if (key[i] != ~0ull) atomicAdd(&ncand, 1);
  // hashes of the old entries and of the candidates
  for (int e = wid; e < C; e += nwarps) {
    const uint64_t h = warp_hash(PX + (size_t)e * nw, nw, lane);
    if (lane == 0) oldH[e] = h;
  }
  __syncthreads();
  const int nc = ncand;
  for (int q = wid; q < nc; q += nwarps) {
    const int r = (int)(key[q] & 0x1FFFFull);
    const uint64_t h = warp_hash(a.best_X + (size_t)(p + P * r) * nw, nw, lane);
    if (lane == 0) cH[q] = h;
  }
  __syncthreads();
  // duplicate test: an equal (E, X) among the old entries or earlier candidates
  for (int q = tid; q < nc; q += blockDim.x) {
    const int64_t e = (int64_t)(key[q] >> 17) - kEnergyBias;
    const int r = (int)(key[q] & 0x1FFFFull);
    const uint32_t* x = a.best_X + (size_t)(p + P * r) * nw;
    bool dup = false;
    // old entries with equal energy (oldE ascending)
    int lo = 0, hi = C;
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (oldE[mid] < e) lo = mid + 1; else hi = mid; }
    for (int k2 = lo; k2 < C && oldE[k2] == e && !dup; ++k2)
      if (oldH[k2] == cH[q] && same_bits(PX + (size_t)k2 * nw, x, nw)) dup = true;
    for (int q2 = q - 1; q2 >= 0 && !dup; --q2) {
      const int64_t e2 = (int64_t)(key[q2] >> 17) - kEnergyBias;
      if (e2 != e) break;
      const int r2 = (int)(key[q2] & 0x1FFFFull);
      if (cH[q2] == cH[q] && same_bits(a.best_X + (size_t)(p + P * r2) * nw, x, nw)) dup = true;
    }
    uflag[q] = dup ? 0 : 1;
  }
  __syncthreads();
  if (tid == 0) {  // compaction order = sorted order
    int u = 0;
    for (int q = 0; q < nc; ++q) { upos[q] = uflag[q] ? u : -1; u += uflag[q]; }
    nuniq = u;
  }
  __syncthreads();
  const int U = nuniq;
  // energies of the unique candidates in sorted order (cH is free now)
  int64_t* uE = reinterpret_cast<int64_t*>(cH);
  for (int q = tid; q < nc; q += blockDim.x)
    if (upos[q] >= 0) uE[upos[q]] = (int64_t)(key[q] >> 17) - kEnergyBias;
  __syncthreads();
  // write the new pool: old entry e goes to e + #{u : uE[u] < oldE[e]};
  // unique candidate u goes to u + #{e : oldE[e] <= uE[u]}; keep ranks < C.
  int64_t* NE = a.pool_E[nxt] + (size_t)p * C;
  uint32_t* NX = a.pool_X[nxt] + (size_t)p * C * nw;
  uint8_t* NA = a.pool_algo[nxt] + (size_t)p * C;
  uint8_t* NO = a.pool_op[nxt] + (size_t)p * C;
  const uint8_t* OA = a.pool_algo[cur] + (size_t)p * C;
  const uint8_t* OO = a.pool_op[cur] + (size_t)p * C;
  for (int e = wid; e < C; e += nwarps) {
    int lo = 0, hi = U;
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (uE[mid] < oldE[e]) lo = mid + 1; else hi = mid; }
    const int rank = e + lo;
    if (rank < C) {
      for (int w = lane; w < nw; w += 32) NX[(size_t)rank * nw + w] = PX[(size_t)e * nw + w];
      if (lane == 0) { NE[rank] = oldE[e]; NA[rank] = OA[e]; NO[rank] = OO[e]; }
    }
  }
  for (int q = wid; q < nc; q += nwarps) {
    const int u = upos[q];
    if (u < 0) continue;
    const int64_t e = uE[u];
    int lo = 0, hi = C;
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (oldE[mid] <= e) lo = mid + 1; else hi = mid; }
    const int rank = u + lo;
    if (rank < C) {
      const int r = (int)(key[q] & 0x1FFFFull);
      const int s = p + P * r;
      const uint32_t* x = a.best_X + (size_t)s * nw;
      for (int w = lane; w < nw; w += 32) NX[(size_t)rank * nw + w] = x[w];
      if (lane == 0) { NE[rank] = e; NA[rank] = a.algo[s]; NO[rank] = a.op[s]; }
    }
  }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge(const MergeArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.ctrl->done) return;
  merge_pool(a, blockIdx.x, smraw);
}

// ---------------------------------------------------------------- finalize
__device__ void finalize_one(const FinArgs& a) {
  DevCtrl* ctrl = a.ctrl;
  __shared__ uint64_t sflips[32];
  __shared__ int64_t sbestE[32];
  __shared__ int sbestS[32];
  __shared__ int winner;
  __shared__ unsigned long long cnt[kStats];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid < kStats) cnt[tid] = 0;
  __syncthreads();
  if (a.stats)  // Table V: main algorithm and genetic operation of every search
    for (int s = tid; s < a.S; s += blockDim.x) {
      atomicAdd(&cnt[min((int)a.algo[s], N_ALGOS - 1)], 1ull);
      atomicAdd(&cnt[N_ALGOS + min((int)a.op[s], N_OPS - 1)], 1ull);
    }
  uint64_t f = 0;
  int64_t be = INT64_MAX;
  int bs = INT_MAX;
  for (int s = tid; s < a.S; s += blockDim.x) {
    f += a.flips[s];
    const int64_t e = a.best_E[s];
    if (e < be) { be = e; bs = s; }  // s ascending per thread: first minimum kept
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    f += __shfl_xor_sync(FULLMASK, f, off);
    const int64_t e2 = __shfl_xor_sync(FULLMASK, be, off);
    const int s2 = __shfl_xor_sync(FULLMASK, bs, off);
    if (e2 < be || (e2 == be && s2 < bs)) { be = e2; bs = s2; }
  }
  if (lane == 0) { sflips[wid] = f; sbestE[wid] = be; sbestS[wid] = bs; }
  __syncthreads();
  if (tid == 0) {
    uint64_t ft = 0;
    int64_t e = INT64_MAX;
    int sb = INT_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ft += sflips[w];
      if (sbestE[w] < e || (sbestE[w] == e && sbestS[w] < sb)) { e = sbestE[w]; sb = sbestS[w]; }
    }
    winner = -1;
    if (e < ctrl->best_E) {  // Step 1 style strict improvement across generations
      ctrl->best_E = e;
      winner = sb;
    }
    ctrl->flips_total += ft;
    ctrl->g += 1;
  }
  __syncthreads();
  if (winner >= 0)
    for (int w = tid; w < a.nw; w += blockDim.x) a.gbest_X[w] = a.best_X[(size_t)winner * a.nw + w];
  if (a.stats && tid == 0 && winner >= 0) {  // Table VI: the finder of the new global best
    cnt[N_ALGOS + N_OPS + min((int)a.algo[winner], N_ALGOS - 1)] += 1;
    cnt[2 * N_ALGOS + N_OPS + min((int)a.op[winner], N_OPS - 1)] += 1;
  }
  __syncthreads();
  if (a.stats && tid < kStats && cnt[tid]) a.stats[tid] += cnt[tid];
  if (a.rflag && tid == 0) *a.rflag = 0;
  if (tid == 0) {
    const bool stop = ctrl->flips_total >= ctrl->budget || ctrl->best_E <= ctrl->target ||
                      (ctrl->max_generations > 0 && ctrl->g >= ctrl->max_generations);
    if (stop) ctrl->done = 1;
  }
}

__global__ void __launch_bounds__(1024) k_finalize(const FinArgs a) {
  if (a.ctrl->done) return;
  finalize_one(a);
}

// ---------------------------------------------------------------- energy / Delta
// Eq. (2) and Eq. (3) for `count` packed vectors: thread k accumulates the
// column sums of W over the set bits j < k and j > k; E adds, per set bit k,
// W_kk plus the lower part, so each pair is counted once.
__global__ void __launch_bounds__(256) k_energy_delta(const EDArgs a) {
  if (a.ctrl && a.ctrl->done) return;
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t* x = a.X + (size_t)v * a.nw;
  int lo = 0, hi = 0;
  const bool in = k < a.n;
  for (int w = 0; w < a.nw; ++w) {
    uint32_t word = x[w];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const int j = 32 * w + b;
      if (in) {
        const int wv = a.W[(size_t)j * a.ld + k];
        if (j < k) lo += wv;
        else if (j > k) hi += wv;
      }
    }
  }
  int64_t econ = 0;
  if (in) {
    const int xk = (x[k >> 5] >> (k & 31)) & 1;
    const int wkk = a.W[(size_t)k * a.ld + k];
    const int F = lo + hi + (xk ? wkk : 0);  // sum_j W_jk x_j
    if (a.delta) a.delta[(size_t)v * a.ld_delta + k] = xk ? -F : F + wkk;  // Eq. (3)
    if (xk) econ = (int64_t)wkk + lo;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) econ += __shfl_xor_sync(FULLMASK, econ, off);
  __shared__ int64_t part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = econ;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
    atomicAdd(reinterpret_cast<unsigned long long*>(a.E + v), (unsigned long long)t);
  }
}

// Launch order of the search slots grouped by main algorithm (any order inside
// a group: it only decides which CTA runs which search, never a result).
__global__ void __launch_bounds__(1024) k_order_by_algo(const uint8_t* algo, int S, int32_t* order,
                                                        const DevCtrl* ctrl, int mod, int lo, int hi) {
  if (ctrl && ctrl->done) return;
  __shared__ int cnt[N_ALGOS], off[N_ALGOS];
  if (threadIdx.x < N_ALGOS) cnt[threadIdx.x] = 0;
  __syncthreads();
  // with mod > 0 only the slots s with lo <= s mod mod < hi are listed (the
  // searches of this context's islands when a solve is split over devices)
  auto listed = [&](int s) { return mod <= 0 || (s % mod >= lo && s % mod < hi); };
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    if (listed(s)) atomicAdd(&cnt[min((int)algo[s], N_ALGOS - 1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < N_ALGOS; ++q) { off[q] = acc; acc += cnt[q]; }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    if (listed(s)) order[atomicAdd(&off[min((int)algo[s], N_ALGOS - 1)], 1)] = s;
}

// X <- D and Delta, E from scratch for every search slot (recompute seeding);
// the energy accumulators must be zero before the launch.
__global__ void k_copy_targets(const uint32_t* D, uint32_t* X, int64_t* E, size_t words, int S,
                               const DevCtrl* ctrl) {
  if (ctrl->done) return;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < words;
       q += (size_t)gridDim.x * blockDim.x)
    X[q] = D[q];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)S;
       q += (size_t)gridDim.x * blockDim.x)
    E[q] = 0;
}


// ---------------------------------------------------------------- batched generation
// The batched form's generation with one launch per stage for every instance
// (Sections III-B and IV per instance): k_gen_pre breeds the targets and
// orders the slots of all instances (one CTA each) and prepares their
// recompute; k_gen_post merges the results into the pools (one CTA per pool)
// and finalises each instance in the last of its merge CTAs.  Each instance
// reads and writes only its own buffers and control block, so its results are
// those of its generations alone.

__global__ void __launch_bounds__(1024) k_gen_pre(const BatchInst* insts) {
  const BatchInst& b = insts[blockIdx.x];
  const OffArgs& o = b.off;
  if (o.ctrl->done) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int s = wid; s < o.S; s += nwarps) offspring_one(o, s, lane);
  __syncthreads();
  // launch order of the slots grouped by main algorithm (which CTA runs which
  // search; never a result)
  __shared__ int cnt[N_ALGOS], off[N_ALGOS];
  if (threadIdx.x < N_ALGOS) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < o.S; s += blockDim.x) atomicAdd(&cnt[min((int)o.algo[s], N_ALGOS - 1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < N_ALGOS; ++q) { off[q] = acc; acc += cnt[q]; }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < o.S; s += blockDim.x)
    b.order[atomicAdd(&off[min((int)o.algo[s], N_ALGOS - 1)], 1)] = s;
  if (b.seed_mode != 1) return;
  // recompute seeding: X = D, the 0/1 operand of the tensor-core recompute
  // (zero rows past S, zero columns past n) and its energy accumulators
  const size_t words = (size_t)o.S * o.nw;
  for (size_t q = threadIdx.x; q < words; q += blockDim.x) b.X[q] = o.D[q];
  for (int r = threadIdx.x; r < b.rows_pad; r += blockDim.x) b.E2[r] = 0;
  const int half = b.n_pad / 2;
  const size_t pairs = (size_t)b.rows_pad * half;
  for (size_t q = threadIdx.x; q < pairs; q += blockDim.x) {
    const int r = (int)(q / half), k = 2 * (int)(q % half);
    uint32_t v = 0;
    if (r < o.S && k < o.n) {
      const uint32_t w = o.D[(size_t)r * o.nw + (k >> 5)];
      const uint32_t b0 = (w >> (k & 31)) & 1u, b1 = (k + 1 < o.n) ? ((w >> ((k + 1) & 31)) & 1u) : 0u;
      v = (b0 ? b.one : 0u) | ((b1 ? b.one : 0u) << 16);
    }
    reinterpret_cast<uint32_t*>(b.A)[q] = v;
  }
}

__global__ void __launch_bounds__(kMergeThreads) k_gen_post(const BatchInst* insts,
                                                            const int32_t* prefix, int ninst) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int cta = blockIdx.x;
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= cta) lo = mid; else hi = mid;
  }
  const BatchInst& b = insts[lo];
  if (b.merge.ctrl->done) return;
  merge_pool(b.merge, cta - prefix[lo], smraw);
  // the last merge CTA of the instance finalises it (after all its pools)
  __shared__ unsigned last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(b.merged, 1u) == (unsigned)b.merge.P - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  finalize_one(b.fin);
  if (threadIdx.x == 0) *b.merged = 0;
}

}  // namespace dabs
