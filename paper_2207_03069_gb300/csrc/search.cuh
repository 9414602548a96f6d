// search.cuh -- the batch-search kernel (Section III-A incremental search,
// Section III-B batch search): one group of NW warps per search slot keeps X,
// the exact int32 Delta vector and the int64 energy in registers, and flips one
// bit per iteration: Step 1 (best one-bit neighbour -> BEST), Step 2 (the
// phase's selector), Step 3 (E += Delta_i, Delta_k += W_ik sigma(x_i) sigma(x_k)
// for k != i by Eq. (4), Delta_i = -Delta_i by Eq. (5)).
//
// The phases (Straight, Greedy, main search) run in one loop per main
// algorithm (run_algo / run_key are templates on it), with one flip site;
// the launch order groups a launch's slots by algorithm, so an SM mostly runs
// one loop body (instruction cache).
//
// Register layout: thread t of a group (NT = 32 NW threads) owns, for chunk
// c = 0..CH-1, the eight consecutive bits k = c*8*NT + 8t + e (e = 0..7).  One
// 128-bit load per chunk brings the thread's eight int16 weights of row i, so
// a whole row is read with fully coalesced 16-byte accesses.  Bit k lives at
// local position p = 8c + e of the thread's Delta array and bit masks.
//
// Keyed form (C::KEY, for instances whose Delta range allows it): d holds
// Delta_k * 2^kb + (k << 1 | x_k) instead of Delta_k.  The update of Eq. (4)
// is the same multiply-add (sigma scaled by 2^kb), and any minimum over d
// then carries the winning bit's index (lowest on ties) and x_k, so no
// second pass finds the arg-min.
//
// Reductions use the warp reduce instructions and, for NW > 1, one
// shared-memory slot round per reduction (double-buffered, one barrier), in
// which lane w reads warp w's slot and a second warp reduction combines
// them.  Ties resolve to the lowest bit index (CyclicMin: the first bit in
// cyclic order from the window start).
//
// sigma(x_k) is one register per bit, or (4-chunk variants of 8 and 16
// warps, held to 128 registers) four signed bytes per register.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace dabs {

template <int NW_, int CH_, int RF_ = ROWS_DENSE, bool KEY_ = false, bool EARLY_ = false>
struct Cfg {
  static constexpr int NW = NW_, CH = CH_;
  static constexpr int RF = RF_;               // row format (RowFormat)
  static constexpr bool KEY = KEY_;            // keyed Delta (see Searcher::run_key)
  // Eq. (5) written by the owner while row i is in flight (Searcher::commit):
  // single-warp searches of one instance per launch.  Launches of several
  // instances (the batched form, whose launches share the SMs with other
  // variants' launches) and groups of warps write it after the update
  // (flip_after), which measured faster there.
  static constexpr bool EARLY = EARLY_ && NW_ == 1;
  // the variants held to 128 registers with 32 bits per thread keep
  // sigma(x_k) as packed signed bytes (four per register) instead of one
  // register per bit
  static constexpr bool SG8 = NW_ >= 8 && CH_ == 4;
  static constexpr int NT = 32 * NW;           // threads per search
  static constexpr int EPT = 8 * CH;           // bits per thread
  static constexpr int SPAN = 8 * NT;          // bits per chunk
  static constexpr int NMW = (EPT + 31) / 32;  // mask words per thread
  static constexpr int SPC = NW == 1 ? 8 : 1;  // searches per CTA (at most)
  static constexpr int CTA = NT * SPC;
  static constexpr int CAP = SPAN * CH;        // largest n this variant holds
};

constexpr unsigned FULL = 0xffffffffu;
enum Phase : int { PH_STRAIGHT = 0, PH_GREEDY = 1, PH_MAIN = 2 };
enum Selector : int { SEL_STRAIGHT = 8, SEL_GREEDY = 9 };

__device__ __forceinline__ int sext_lo(uint32_t w) { return (int)(w << 16) >> 16; }
__device__ __forceinline__ int sext_hi(uint32_t w) { return (int)w >> 16; }
__device__ __forceinline__ int w16(const uint4& v, int e) {
  const uint32_t w = e < 2 ? v.x : e < 4 ? v.y : e < 6 ? v.z : v.w;
  return (e & 1) ? sext_hi(w) : sext_lo(w);
}
__device__ __forceinline__ uint32_t u32of(const uint4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
// f^3 >> 31 for a 21-bit fixed-point ratio f (the cube21 schedule helper)
__device__ __forceinline__ uint64_t cube_of(uint32_t f) {
  const uint64_t f2 = (uint64_t)f * f;
  return (f2 * f) >> 31;
}
// bits [lo, hi) of the 8-bit run starting at b0, as an 8-bit mask
__device__ __forceinline__ uint32_t run_mask(int b0, int lo, int hi) {
  const int a = max(lo, b0), b = min(hi, b0 + 8);
  return a < b ? (((1u << (b - a)) - 1u) << (a - b0)) : 0u;
}

template <class C>
struct SmemSearch {
  int4 red[2][C::NW];        // reduction slots (double buffered)
  int tot[C::CH][C::NW];     // per chunk, per warp candidate counts (k-th pick)
  int pick[4];               // broadcast of a pick made by one thread
  int2 nx[2];                // TwoNeighbor: (x_k, d_k) of the next bit from its owner (by parity)
};

#define DABS_CASES(X)                                                                      \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15)    \
  X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29)      \
  X(30) X(31)

template <class C>
struct Searcher {
  static constexpr int NW = C::NW, CH = C::CH, NT = C::NT, EPT = C::EPT, SPAN = C::SPAN,
                       NMW = C::NMW;
  static_assert(EPT <= 32, "register-resident variants hold at most 32 bits per thread");
  // --- state (registers) ---
  int d[EPT];          // Delta (INT_MAX for bits >= n)
  // sigma(x_k) = 2 x_k - 1 (times 2^kb in the keyed form), one register per
  // bit; or, with Cfg::SG8, +-1 as signed bytes, bit k in byte k % 4 of sg[k / 4]
  int sg[C::SG8 ? EPT / 4 : EPT];
  uint32_t xb[NMW];    // X bits
  uint32_t bb[NMW];    // BEST bits
  uint32_t vb[NMW];    // valid bits (k < n)
  uint32_t db[NMW];    // target D bits
  uint32_t tb[NMW];    // tabu bits
  int64_t E, Ebest;
  uint32_t flips;
  // --- context ---
  SmemSearch<C>* sm;
  int t, lane, warp, buf;
  uint32_t s, g;
  uint64_t seed;
  const int16_t* W;     // W, and Wneg = -W: row i of sigma(x_i) W is read directly
  const int16_t* Wneg;
  const int32_t* diag;  // W_kk
  int n, ld;
  int ring_len, ring_head;  // tabu ring (uniform); entry j lives in lane j's ringv
  int ringv;
  int kb = 0;               // keyed form: bits below the Delta part of a key
  // sparse rows (C::RF != ROWS_DENSE): offsets and entries (shared or global
  // memory), and this search's scratch row in shared memory, all zero between
  // flips
  const uint32_t* srow = nullptr;
  const uint32_t* sent = nullptr;
  int16_t* scr = nullptr;
  const int16_t* sw = nullptr;  // C::RF == ROWS_DENSE_SMEM: W in shared memory

  __device__ __forceinline__ Searcher(const SearchArgs& a, SmemSearch<C>* smem, int tid,
                                      uint32_t sidx, uint32_t gen, uint64_t sd)
      : sm(smem), t(tid), lane(tid & 31), warp(tid >> 5), buf(0), s(sidx), g(gen), seed(sd),
        W(a.W), Wneg(a.Wneg), diag(a.diag), n(a.n), ld(a.ld), ring_len(0), ring_head(0), ringv(0),
        kb(C::KEY ? a.key_bits : 0) {}

  // ------------------------------------------------------------ bit helpers
  __device__ __forceinline__ static bool bit_at(const uint32_t (&m)[NMW], int p) {
    return (m[0] >> (p & 31)) & 1u;  // NMW == 1
  }
  __device__ __forceinline__ int kidx(int p) const { return (p >> 3) * SPAN + 8 * t + (p & 7); }
  __device__ __forceinline__ static int owner_t(int i) { return (i >> 3) & (NT - 1); }
  __device__ __forceinline__ static int local_p(int i) { return ((i >> 3) / NT) * 8 + (i & 7); }
  __device__ __forceinline__ uint32_t key_of(int lp) const {
    return lp < 0 ? UINT_MAX : (((uint32_t)kidx(lp) << 1) | (uint32_t)bit_at(xb, lp));
  }
  // value of d at a run-time position 0 <= p < EPT: a binary select tree on
  // the bits of p (no branch, no local memory)
  __device__ __forceinline__ int get_at(int p) const {
    int v[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) v[q] = d[q];
#pragma unroll
    for (int w = 1; w < EPT; w <<= 1) {
      const bool hi = (p & w) != 0;
#pragma unroll
      for (int q = 0; q < EPT; q += 2 * w) v[q] = hi ? v[q + w] : v[q];
    }
    return v[0];
  }
  // sigma(x_k) of register position Q flips
  template <int Q>
  __device__ __forceinline__ void flip_sigma() {
    if constexpr (C::SG8) sg[Q / 4] ^= (int)(0xFEu << (8 * (Q % 4)));  // 0x01 <-> 0xFF
    else sg[Q] = -sg[Q];
  }
  // sigma(x_k) at register position p (a constant once unrolled): +-1 from
  // its packed byte, or the stored value
  __device__ __forceinline__ int sigma_of(int p) const {
    if constexpr (C::SG8) return (int)(signed char)((uint32_t)sg[p >> 2] >> (8 * (p & 3)));
    else return sg[p];
  }
  // Eq. (5) at a run-time position after the row update (groups of warps,
  // where Delta_i is known to every thread): d = v, sigma flips
  __device__ __forceinline__ void set_flipped(int p, int v) {
    if constexpr (NW > 1 && EPT <= 16) {
      // groups of warps: the other warps wait for this write at the next
      // round, so no indirect branch (a jump table costs over a hundred
      // cycles with one active lane) -- a select per register instead (with
      // 32 registers per thread the selects cost more than the branch)
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const bool hit = q == p;
        d[q] = hit ? v : d[q];
        if constexpr (C::SG8)
          sg[q / 4] ^= hit ? (int)(0xFEu << (8 * (q % 4))) : 0;
        else
          sg[q] = hit ? -sg[q] : sg[q];
      }
      return;
    }
    switch (p) {
#define DABS_SET(q)                         \
  case q:                                   \
    if constexpr (q < EPT) {                \
      d[q < EPT ? q : 0] = v;               \
      flip_sigma<(q < EPT ? q : 0)>();      \
    }                                       \
    break;
      DABS_CASES(DABS_SET)
#undef DABS_SET
      default: break;
    }
  }
  // Eq. (5) at a run-time position p (the owner of bit i = kidx(p)): reads
  // Delta_i, stores the flipped value plus corr, and flips sigma(x_i).  A
  // switch on p keeps d in registers (no local memory).
  __device__ __forceinline__ int flip_at(int p, int i, int xi, int corr) {
    int di = 0;
    switch (p) {
#define DABS_FLIP(q)                                                          \
  case q:                                                                     \
    if constexpr (q < EPT) {                                                  \
      constexpr int qq = q < EPT ? q : 0;                                     \
      const int o = d[qq];                                                    \
      di = C::KEY ? (o >> kb) : o;                                            \
      d[qq] = (C::KEY ? -di * (1 << kb) + ((i << 1) | (xi ^ 1)) : -di) + corr; \
      flip_sigma<qq>();                                                       \
    }                                                                         \
    break;
      DABS_CASES(DABS_FLIP)
#undef DABS_FLIP
      default: break;
    }
    return di;
  }

  // ------------------------------------------------------------ reductions
  template <int K>
  __device__ __forceinline__ void gmin(int (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = __reduce_min_sync(FULL, v[q]);
    if constexpr (NW > 1) {
      if (lane == 0)
        sm->red[buf][warp] = make_int4(v[0], K > 1 ? v[K > 1 ? 1 : 0] : 0, K > 2 ? v[K > 2 ? 2 : 0] : 0, 0);
      __syncthreads();
      // lane w < NW takes warp w's slot; one more warp reduction combines them
      const int4 r = slot(make_int4(INT_MAX, INT_MAX, INT_MAX, 0));
      v[0] = __reduce_min_sync(FULL, r.x);
      if constexpr (K > 1) v[K > 1 ? 1 : 0] = __reduce_min_sync(FULL, r.y);
      if constexpr (K > 2) v[K > 2 ? 2 : 0] = __reduce_min_sync(FULL, r.z);
      buf ^= 1;
    }
  }
  // groups of warps, after the barrier of a round: warp `lane`'s slot in the
  // lanes below NW, `neutral` in the others
  __device__ __forceinline__ int4 slot(int4 neutral) const {
    return lane < NW ? sm->red[buf][lane < NW ? lane : 0] : neutral;
  }
  template <int K>
  __device__ __forceinline__ void gminu(uint32_t (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = __reduce_min_sync(FULL, v[q]);
    if constexpr (NW > 1) {
      if (lane == 0)
        sm->red[buf][warp] = make_int4((int)v[0], K > 1 ? (int)v[K > 1 ? 1 : 0] : 0, 0, 0);
      __syncthreads();
      const int4 r = slot(make_int4(-1, -1, 0, 0));  // UINT_MAX
      v[0] = __reduce_min_sync(FULL, (uint32_t)r.x);
      if constexpr (K > 1) v[K > 1 ? 1 : 0] = __reduce_min_sync(FULL, (uint32_t)r.y);
      buf ^= 1;
    }
  }

  // groups of warps: up to two plain minima v (warp-reduced) and one
  // (value, key) pair -- the group minimum and the lowest key among the
  // warps holding it -- in one shared-memory round
  template <int K>
  __device__ __forceinline__ void gmin_pair(int (&v)[K], int& pv, uint32_t& pk) {
    static_assert(K >= 1 && K <= 2, "at most two plain values");
    if constexpr (NW == 1) return;  // a single warp: the warp values are the group's
    if (lane == 0) sm->red[buf][warp] = make_int4(v[0], K > 1 ? v[K - 1] : 0, pv, (int)pk);
    __syncthreads();
    const int4 r = slot(make_int4(INT_MAX, INT_MAX, INT_MAX, -1));
    v[0] = __reduce_min_sync(FULL, r.x);
    if constexpr (K > 1) v[K - 1] = __reduce_min_sync(FULL, r.y);
    pv = __reduce_min_sync(FULL, r.z);
    pk = __reduce_min_sync(FULL, r.z == pv ? (uint32_t)r.w : UINT_MAX);
    buf ^= 1;
  }
  // Step 1's key for the group minimum m (groups of warps: a round of its own,
  // taken only when the step improves BEST)
  __device__ __forceinline__ uint32_t step1_key(const int (&cma)[CH], int m) {
    uint32_t k[1] = {warp_key(FULL, cma, m)};
    gminu(k);
    return k[0];
  }
  // TwoNeighbor visits bits in a fixed order: in a group of warps the owner of
  // the next bit publishes its x_k and d_k once the current flip is applied,
  // and the group reads them after its next round (slot by iteration parity)
  __device__ __forceinline__ void publish_next(int k, int it_read) {
    if (t == owner_t(k)) {
      const int pk = local_p(k);
      sm->nx[it_read & 1] = make_int2(bit_at(xb, pk) ? 1 : 0, get_at(pk));
    }
  }

  // ------------------------------------------------------------ per-thread scans
  // ------------------------------------------------------------ Step 1 / Step 3
  // BEST <- f_j(X) for j = key >> 1 (Step 1 on strict improvement)
  __device__ __forceinline__ void take_best(uint32_t keyj, int m) {
    const int j = (int)(keyj >> 1);
    bb[0] = xb[0];
    if (t == owner_t(j)) bb[0] ^= 1u << local_p(j);
    Ebest = E + m;
  }

  // Step 3, in two halves so that independent work can run while row i is in
  // flight: row_load issues the loads of row i of sigma(x_i) W (x_i = xi
  // before the flip), row_apply updates E and Delta by Eqs. (4) and (5)
  // (di = Delta_i before the flip) and flips x_i.
  __device__ __forceinline__ static void group_sync() {
    if constexpr (NW == 1) __syncwarp();
    else __syncthreads();
  }
  __device__ __forceinline__ void row_load(int i, int xi, uint4 (&rv)[CH]) const {
    // every selector yields 0 <= i < n; the clamp only keeps a logic error
    // from turning into an out-of-bounds read (parity tests would flag it)
    i = min(max(i, 0), n - 1);
    if constexpr (C::RF == ROWS_DENSE_SMEM) {
      // row i of W from shared memory; sigma(x_i) = -1 negates both halves
      const uint4* row = reinterpret_cast<const uint4*>(sw + (size_t)i * ld);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int off = c * SPAN + 8 * t;
        uint4 v = off < ld ? row[off >> 3] : make_uint4(0, 0, 0, 0);
        if (!xi) v = make_uint4(__vneg2(v.x), __vneg2(v.y), __vneg2(v.z), __vneg2(v.w));
        rv[c] = v;
      }
      return;
    }
    if constexpr (C::RF != ROWS_DENSE) {
      // scatter sigma(x_i) W_ik of the stored entries into the zeroed scratch
      // row, then every thread reads its chunks exactly as from a dense row
      // and clears them again; the first barrier orders the previous flip's
      // clearing before this scatter
      group_sync();
      uint32_t b, e;
      if constexpr (C::RF == ROWS_SPARSE_GLOBAL) {
        b = __ldg(srow + i);
        e = __ldg(srow + i + 1);
      } else {
        b = srow[i];
        e = srow[i + 1];
      }
      for (uint32_t j = b + (uint32_t)t; j < e; j += NT) {
        const uint32_t en = C::RF == ROWS_SPARSE_GLOBAL ? __ldg(sent + j) : sent[j];
        const int w = sext_lo(en);
        scr[en >> 16] = (int16_t)(xi ? w : -w);
      }
      group_sync();
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int off = c * SPAN + 8 * t;
        if (off < ld) {
          uint4* q = reinterpret_cast<uint4*>(scr + off);
          rv[c] = *q;
          *q = make_uint4(0, 0, 0, 0);
        } else {
          rv[c] = make_uint4(0, 0, 0, 0);
        }
      }
      return;
    }
    const int16_t* row = (xi ? W : Wneg) + (size_t)i * ld;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int off = c * SPAN + 8 * t;
      rv[c] = off < ld ? __ldg(reinterpret_cast<const uint4*>(row + off)) : make_uint4(0, 0, 0, 0);
    }
  }
  // Eq. (5) and x_i ^= 1 for a single warp, made while row i is in flight:
  // the owner of bit i reads Delta_i from its register and stores -Delta_i
  // raised by W_ii (in key units), because the row update that follows adds
  // sigma(x_i) W_ii sigma'(x_i) = -W_ii at k = i once sigma(x_i) is flipped
  // (sparse rows hold no diagonal entry: nothing to raise).  Returns Delta_i
  // in every lane.  A group of warps instead knows Delta_i from its
  // selection and writes it after the update (flip_after): a barrier behind
  // the owner's write would keep every warp waiting for it.
  __device__ __forceinline__ int commit(int i, int xi) {
    static_assert(C::EARLY, "single-warp searches of one instance");
    i = min(max(i, 0), n - 1);
    int di = 0;
    if (t == owner_t(i)) {
      constexpr bool sparse = C::RF == ROWS_SPARSE_SMEM || C::RF == ROWS_SPARSE_GLOBAL;
      const int corr = sparse ? 0 : __ldg(diag + i) * (C::KEY ? (1 << kb) : 1);
      const int pi = local_p(i);
      di = flip_at(pi, i, xi, corr);
      xb[0] ^= 1u << pi;
    }
    return __shfl_sync(FULL, di, owner_t(i));
  }
  __device__ __forceinline__ void flip_after(int i, int di, int xi) {
    i = min(max(i, 0), n - 1);
    if (t == owner_t(i)) {
      const int pi = local_p(i);
      // Eq. (5): Delta_i = -Delta_i (and x_i, in the keyed form's low bits)
      set_flipped(pi, C::KEY ? -di * (1 << kb) + ((i << 1) | (xi ^ 1)) : -di);
      xb[0] ^= 1u << pi;
    }
  }
  // Eq. (4) for every k (k = i included: see commit and flip_after), E += Delta_i
  __device__ __forceinline__ void row_apply(const uint4 (&rv)[CH], int di) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int p = 8 * c + e;
        if constexpr (C::SG8 && C::KEY)
          d[p] += (w16(rv[c], e) * sigma_of(p)) << kb;
        else
          d[p] += w16(rv[c], e) * sigma_of(p);
      }
    }
    E += di;
    ++flips;
  }

  // RandomMin draws of one iteration: 16-bit half (k % 8) of the Philox block
  // (flip, g, s, RNG_RANDMIN | k/8) for each owned bit k.  A thread's eight
  // bits of chunk c are k/8 = c NT + t: one whole block per chunk.
  __device__ __forceinline__ void randmin_draw(uint32_t flip_idx, uint4 (&r)[CH]) const {
#pragma unroll
    for (int c = 0; c < CH; ++c)
      r[c] = draw(seed, flip_idx, g, s, RNG_RANDMIN | (uint32_t)(c * NT + t));
  }
  // bit p's 16-bit uniform is below thr
  __device__ __forceinline__ static bool randmin_hit(const uint4 (&r)[CH], int p, uint32_t thr) {
    const int c = p >> 3, e = p & 7;
    return ((u32of(r[c], e >> 1) >> (16 * (e & 1))) & 0xFFFFu) < thr;
  }

  // ------------------------------------------------------------ k-th pick
  // The ((u * count) >> 32)-th set bit of the group-wide candidate mask Cm, in
  // ascending bit order.  Returns key = (i << 1) | x_i.
  __device__ __forceinline__ uint32_t kth(uint32_t Cm, uint32_t u, int* di) {
    int cnt[CH], wt[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      cnt[c] = __popc((Cm >> (8 * c)) & 0xFFu);
      wt[c] = (int)__reduce_add_sync(FULL, (unsigned)cnt[c]);
    }
    int csel = 0, wsel = 0, rel = 0;
    if constexpr (NW == 1) {
      int total = 0;
#pragma unroll
      for (int c = 0; c < CH; ++c) total += wt[c];
      int kk = (int)uniform_below(u, (uint32_t)total);
      bool found = false;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (!found && kk < wt[c]) { csel = c; rel = kk; found = true; }
        if (!found) kk -= wt[c];
      }
    } else {
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < CH; ++c) sm->tot[c][warp] = wt[c];
      }
      __syncthreads();
      // the counts in ascending bit order (chunk, then warp): entry j =
      // c NW + w; lane l holds entries l EPL .. l EPL + EPL - 1, and one
      // prefix over the lanes locates the kk-th candidate's entry
      constexpr int NE = CH * NW, EPL = (NE + 31) / 32;
      const int* tf = &sm->tot[0][0];
      int te[EPL];
      int ls = 0;
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int j = lane * EPL + e;
        te[e] = j < NE ? tf[j < NE ? j : 0] : 0;
        ls += te[e];
      }
      int incl = ls;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(FULL, incl, 31);
      const int kk = (int)uniform_below(u, (uint32_t)total);
      const unsigned bl = __ballot_sync(FULL, incl > kk);  // none when there is no candidate
      int js = lane * EPL, r = kk - (incl - ls);
#pragma unroll
      for (int e = 0; e < EPL - 1; ++e)
        if (r >= te[e] && js == lane * EPL + e) { r -= te[e]; ++js; }
      const int src = bl ? __ffs(bl) - 1 : 0;
      js = __shfl_sync(FULL, js, src);
      r = __shfl_sync(FULL, r, src);
      if (bl) {
        csel = js / NW;
        wsel = js % NW;
        rel = r;
      }
    }
    uint32_t key = 0;
    int dv = 0;  // groups of warps: the pick's stored d value (see flip_after)
    if (warp == wsel) {
      int mycnt = 0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c == csel) mycnt = cnt[c];
      // exclusive prefix of the per-lane counts (0..8) from four bit-sliced
      // ballots: independent votes instead of a serial shuffle scan
      const unsigned below = (1u << lane) - 1u;
      int excl = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) excl += __popc(__ballot_sync(FULL, (mycnt >> b) & 1) & below) << b;
      const int incl = excl + mycnt;
      const bool mine = excl <= rel && rel < incl;
      // position of the (r+1)-th set bit of this lane's byte (r = rank in
      // it): halves, quarters, bits, without a loop
      uint32_t byte = (Cm >> (8 * csel)) & 0xFFu;
      int r = mine ? rel - excl : 0, pos = 0;
      const int c4 = __popc(byte & 0xFu);
      if (r >= c4) { pos += 4; r -= c4; byte >>= 4; }
      const int c2 = __popc(byte & 0x3u);
      if (r >= c2) { pos += 2; r -= c2; byte >>= 2; }
      if (r >= (int)(byte & 1u)) pos += 1;
      const int p = 8 * csel + pos;
      if (mine) {
        key = key_of(p);
        if constexpr (!C::EARLY) dv = get_at(p);
      }
      const unsigned bal = __ballot_sync(FULL, mine);
      const int src = bal ? __ffs(bal) - 1 : 0;
      key = __shfl_sync(FULL, key, src);
      if constexpr (!C::EARLY) dv = __shfl_sync(FULL, dv, src);
      if constexpr (NW > 1) {
        if (lane == 0) { sm->pick[0] = (int)key; sm->pick[1] = dv; }
      }
    }
    if constexpr (NW > 1) {
      __syncthreads();
      key = (uint32_t)sm->pick[0];
      dv = sm->pick[1];
    }
    *di = dv;
    return key;
  }

  // x_i (and, for groups of warps, the stored d value) of a bit chosen
  // without a reduction (TwoNeighbor)
  __device__ __forceinline__ int fetch_x(int i, int* dv) {
    const int pi = local_p(i), ot = owner_t(i);
    int x = bit_at(xb, pi) ? 1 : 0;
    if constexpr (NW == 1) {
      x = __shfl_sync(FULL, x, ot);
      *dv = C::EARLY ? 0 : __shfl_sync(FULL, get_at(pi), ot);
    } else {
      if (t == ot) { sm->pick[2] = get_at(pi); sm->pick[3] = x; }
      __syncthreads();
      *dv = sm->pick[2];
      x = sm->pick[3];
      __syncthreads();
    }
    return x;
  }

  // ------------------------------------------------------------ tabu
  // bit i flipped at this iteration becomes tabu for the next tau iterations;
  // the ring of the last tau flips is spread over the lanes (entry j in lane j)
  __device__ __forceinline__ void tabu_push(int i, int tau) {
    if (tau <= 0) return;
    if (ring_len == tau) {
      const int old = __shfl_sync(FULL, ringv, ring_head);
      if (t == owner_t(old)) tb[0] ^= 1u << local_p(old);
    } else {
      ++ring_len;
    }
    if (lane == ring_head) ringv = i;
    ring_head = ring_head + 1 == tau ? 0 : ring_head + 1;
    if (t == owner_t(i)) tb[0] ^= 1u << local_p(i);
  }

  // ------------------------------------------------------------ bit masks
  // bit p set where pred(p) holds, ORed as a balanced tree (independent terms)
  template <class P>
  __device__ __forceinline__ static uint32_t mask_of(P pred) {
    uint32_t m8[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      uint32_t b[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) b[e] = (uint32_t)pred(8 * c + e) << e;
      m8[c] = ((b[0] | b[1]) | (b[2] | b[3])) | ((b[4] | b[5]) | (b[6] | b[7]));
    }
    if constexpr (CH == 1) return m8[0];
    else if constexpr (CH == 2) return m8[0] | (m8[CH > 1 ? 1 : 0] << 8);
    else return (m8[0] | (m8[CH > 1 ? 1 : 0] << 8)) | ((m8[CH > 2 ? 2 : 0] << 16) | (m8[CH > 3 ? 3 : 0] << 24));
  }

  // ------------------------------------------------------------ chunk minima
  // three-input min/max (DPX) trees: per 8-bit chunk, then across chunks
  __device__ __forceinline__ static int min8(const int (&v)[8]) {
    return __vimin3_s32(__vimin3_s32(v[0], v[1], v[2]), __vimin3_s32(v[3], v[4], v[5]),
                        min(v[6], v[7]));
  }
  __device__ __forceinline__ static int max8(const int (&v)[8]) {
    return __vimax3_s32(__vimax3_s32(v[0], v[1], v[2]), __vimax3_s32(v[3], v[4], v[5]),
                        max(v[6], v[7]));
  }
  __device__ __forceinline__ static int min_of(const int (&cm)[CH]) {
    if constexpr (CH == 1) return cm[0];
    else if constexpr (CH == 2) return min(cm[0], cm[CH > 1 ? 1 : 0]);
    else return min(min(cm[0], cm[CH > 1 ? 1 : 0]), min(cm[CH > 2 ? 2 : 0], cm[CH > 3 ? 3 : 0]));
  }
  // per-chunk minima of d over the bits of M (INT_MAX where none)
  __device__ __forceinline__ void chunk_min(uint32_t M, int (&cm)[CH]) const {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      int v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = ((M >> (8 * c + e)) & 1u) ? d[8 * c + e] : INT_MAX;
      cm[c] = min8(v);
    }
  }
  __device__ __forceinline__ void chunk_min_all(int (&cm)[CH]) const {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      int v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = d[8 * c + e];
      cm[c] = min8(v);
    }
  }
  // key (k << 1 | x_k) of this warp's lowest bit k in M with d == target, found
  // chunk by chunk with a ballot over the chunk minima (UINT_MAX if none)
  __device__ __forceinline__ uint32_t warp_key(uint32_t M, const int (&cm)[CH], int target) const {
    // all chunk ballots at once (independent), then the first chunk that has one
    unsigned bal[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) bal[c] = __ballot_sync(FULL, cm[c] == target);
    int csel = -1;
    unsigned b = 0;
#pragma unroll
    for (int c = CH - 1; c >= 0; --c)
      if (bal[c]) { csel = c; b = bal[c]; }
    if (csel < 0) return UINT_MAX;
    uint32_t mm = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (c == csel)
#pragma unroll
        for (int e = 0; e < 8; ++e)
          mm |= (uint32_t)(((M >> (8 * c + e)) & 1u) && d[8 * c + e] == target) << e;
    const int p = 8 * csel + (mm ? __ffs(mm) - 1 : 0);
    const uint32_t kk = ((uint32_t)kidx(p) << 1) | ((xb[0] >> p) & 1u);
    return __shfl_sync(FULL, kk, __ffs(b) - 1);
  }

  // ------------------------------------------------------------ the batch search
  // Section III-B: seeding (Straight, unless X was set to D already), Greedy,
  // then (main search, Greedy) rounds until at least B flips; TwoNeighbor at
  // most once.  Every iteration first runs Step 1 over all n bits.  The loop
  // is specialised per main algorithm (ALGO) so each body is lean.
  template <int ALGO>
  __device__ __forceinline__ void run_algo(int seed_mode, int T, int tau, uint32_t B) {
    int phase = seed_mode == 0 ? PH_STRAIGHT : PH_GREEDY;
    int runs = 0, it = 0, ws = 0;
    const int Tmain = ALGO == TWONEIGHBOR ? 2 * n - 1 : T;
    // exact floor(a * 2^21 / T) for a = t (rising) and a = T - t (falling),
    // advanced incrementally instead of a 64-bit division per iteration
    const uint32_t Kq = (1u << 21) / (uint32_t)T, Kr = (1u << 21) % (uint32_t)T;
    uint32_t fup = 0, rup = 0, fdn = 1u << 21;
    int rdn = 0;
    uint32_t rnd0 = 0, rnd1 = 0;  // 32 MaxMin/PositiveMin draws, one per lane
    const int cwin = n < 32 ? n : 32;
    // RandomMin's floor c = 32/n in units of 2^-16, rounded up
    const uint32_t c16 = ((1u << 21) + (uint32_t)n - 1) / (uint32_t)n;
    for (;;) {
      int i = 0, xi = 0, di = 0;
      uint32_t kj = UINT_MAX;
      int cma[CH];
      chunk_min_all(cma);  // Step 1: every one-bit neighbour
      int m;
      bool improve;
      if (phase != PH_MAIN && NW > 1) {
        // ---------------- Straight / Greedy, groups of warps: the selection's
        // (value, key) pair rides in Step 1's round
        const bool st = phase == PH_STRAIGHT;
        const uint32_t Ms = (xb[0] ^ db[0]) & vb[0];
        int cms[CH];
        int v[1] = {__reduce_min_sync(FULL, min_of(cma))};
        int pv;
        uint32_t pk;
        if (st) {
          chunk_min(Ms, cms);
          pv = __reduce_min_sync(FULL, min_of(cms));
          pk = pv == INT_MAX ? UINT_MAX : warp_key(Ms, cms, pv);
        } else {
          pv = v[0];
          pk = warp_key(FULL, cma, pv);
        }
        gmin_pair(v, pv, pk);
        m = v[0];
        if (st && pv == INT_MAX) {  // X == D: Straight ends
          phase = PH_GREEDY;
          continue;
        }
        improve = E + m < Ebest;
        if (!st && m >= 0) {  // local minimum: Greedy ends after Step 1
          if (improve) take_best(pk, m);
          if (flips < B && !(ALGO == TWONEIGHBOR && runs >= 1)) {
            phase = PH_MAIN;
            it = 0;
            ws = 0;
            fup = 0;
            rup = 0;
            fdn = 1u << 21;
            rdn = 0;
            tb[0] = 0;
            ring_len = 0;
            ring_head = 0;
            if (ALGO == TWONEIGHBOR) publish_next(0, 0);  // its first bit
            continue;
          }
          break;
        }
        if (st) {
          kj = improve ? step1_key(cma, m) : UINT_MAX;
          di = pv;
        } else {
          kj = pk;
          di = m;
        }
        i = (int)(pk >> 1);
        xi = (int)(pk & 1u);
      } else if (phase != PH_MAIN) {
        // ---------------- Straight / Greedy
        const bool st = phase == PH_STRAIGHT;
        const uint32_t Ms = (xb[0] ^ db[0]) & vb[0];
        int cms[CH];
        if (st) chunk_min(Ms, cms);
        int v[2] = {min_of(cma), st ? min_of(cms) : INT_MAX};
        gmin(v);
        m = v[0];
        if (st && v[1] == INT_MAX) {  // X == D: Straight ends
          phase = PH_GREEDY;
          continue;
        }
        improve = E + m < Ebest;
        if (!st && m >= 0) {  // local minimum: Greedy ends after Step 1
          if (improve) {
            uint32_t k[1] = {warp_key(FULL, cma, m)};
            gminu(k);
            take_best(k[0], m);
          }
          if (flips < B && !(ALGO == TWONEIGHBOR && runs >= 1)) {
            phase = PH_MAIN;
            it = 0;
            ws = 0;
            fup = 0;
            rup = 0;
            fdn = 1u << 21;
            rdn = 0;
            tb[0] = 0;
            ring_len = 0;
            ring_head = 0;
            continue;
          }
          break;
        }
        if (st) {
          uint32_t k[2] = {improve ? warp_key(FULL, cma, m) : UINT_MAX, warp_key(Ms, cms, v[1])};
          gminu(k);
          kj = k[0];
          i = (int)(k[1] >> 1);
          xi = (int)(k[1] & 1u);
          di = v[1];
        } else {
          uint32_t k[1] = {warp_key(FULL, cma, m)};
          gminu(k);
          kj = k[0];
          i = (int)(k[0] >> 1);
          xi = (int)(k[0] & 1u);
          di = m;
        }
      } else {
        // ---------------- main search iteration t = it + 1
        fup += Kq;
        rup += Kr;
        if (rup >= (uint32_t)T) { ++fup; rup -= (uint32_t)T; }
        fdn -= Kq;
        rdn -= (int)Kr;
        if (rdn < 0) { --fdn; rdn += T; }
        const uint32_t F = vb[0] & ~tb[0];  // free (non-tabu) bits
        if (ALGO == TWONEIGHBOR) {
          int v[1] = {min_of(cma)};
          gmin(v);
          m = v[0];
          improve = E + m < Ebest;
          if (improve) {
            uint32_t k[1] = {warp_key(FULL, cma, m)};
            gminu(k);
            kj = k[0];
          }
          i = it == 0 ? 0 : ((it & 1) ? (it + 1) >> 1 : (it >> 1) - 1);
          if constexpr (NW > 1) {
            const int2 nx = sm->nx[it & 1];  // published before the round above
            xi = nx.x;
            di = nx.y;
          } else {
            xi = fetch_x(i, &di);
          }
        } else if (ALGO == MAXMIN || ALGO == POSITIVEMIN) {
          if ((it & 31) == 0) {
            // the flips of iterations it .. it+31 are flips .. flips+31
            const uint4 u = draw(seed, flips + (uint32_t)lane, g, s,
                                 ALGO == MAXMIN ? RNG_MAXMIN : RNG_POSMIN);
            rnd0 = u.x;
            rnd1 = u.y;
          }
          const uint32_t u0 = __shfl_sync(FULL, rnd0, it & 31);
          uint32_t Cm = 0, ukth = 0;
          if (ALGO == MAXMIN) {
            int cmn[CH], cmx[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              int vn[8], vx[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const bool f = (F >> (8 * c + e)) & 1u;
                vn[e] = f ? d[8 * c + e] : INT_MAX;
                vx[e] = f ? d[8 * c + e] : INT_MIN;
              }
              cmn[c] = min8(vn);
              cmx[c] = ~max8(vx);
            }
            int v[3] = {min_of(cma), min_of(cmn), min_of(cmx)};
            gmin(v);
            m = v[0];
            const int mn = v[1], mx = ~v[2];
            const uint64_t q = cube_of(fdn);
            const uint64_t span = (uint64_t)((int64_t)mx - (int64_t)mn);
            const uint64_t R = (q * span) >> 32;
            // threshold in [mn, mx]: fits int32
            const int thr = (int)((int64_t)mn + (int64_t)(((uint64_t)u0 * (R + 1)) >> 32));
            Cm = mask_of([&](int p) { return d[p] <= thr; }) & F;
            ukth = __shfl_sync(FULL, rnd1, it & 31);
          } else {
            int cmp[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              int vp[8];
#pragma unroll
              for (int e = 0; e < 8; ++e)
                vp[e] = (((F >> (8 * c + e)) & 1u) && d[8 * c + e] > 0) ? d[8 * c + e] : INT_MAX;
              cmp[c] = min8(vp);
            }
            int v[2] = {min_of(cma), min_of(cmp)};
            gmin(v);
            m = v[0];
            const int pm = v[1];
            if (pm != INT_MAX) {
              Cm = mask_of([&](int p) { return d[p] <= pm; }) & F;
            } else {
              Cm = F;
            }
            ukth = u0;
          }
          improve = E + m < Ebest;
          if (improve) {
            uint32_t k[1] = {warp_key(FULL, cma, m)};
            gminu(k);
            kj = k[0];
          }
          const uint32_t key = kth(Cm, ukth, &di);
          i = (int)(key >> 1);
          xi = (int)(key & 1u);
        } else if (ALGO == CYCLICMIN) {
          const uint64_t wl = (cube_of(fup) * (uint64_t)n) >> 32;
          const int wsz = (int)(wl < (uint64_t)cwin ? (uint64_t)cwin : (wl > (uint64_t)n ? (uint64_t)n : wl));
          // window [ws, ws + wsz) cyclically: [ws, min(ws+wsz, n)) and [0, ws+wsz-n)
          const int hi1 = min(ws + wsz, n), hi2 = ws + wsz - n;
          uint32_t M1 = 0, M2 = 0;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int b0 = c * SPAN + 8 * t;
            M1 |= run_mask(b0, ws, hi1) << (8 * c);
            M2 |= run_mask(b0, 0, hi2) << (8 * c);
          }
          M1 &= F;
          M2 &= F;
          int cm1[CH], cm2[CH];
          chunk_min(M1, cm1);
          chunk_min(M2, cm2);
          uint32_t wk;  // the window pick's key, relative to ws (cyclic order)
          if constexpr (NW > 1) {
            // this warp's window minimum and its first bit in cyclic order from
            // ws, reduced in Step 1's round
            int v[1] = {__reduce_min_sync(FULL, min_of(cma))};
            int pv = __reduce_min_sync(FULL, min(min_of(cm1), min_of(cm2)));
            uint32_t pk = UINT_MAX;
            if (pv != INT_MAX) {
              const uint32_t k1 = warp_key(M1, cm1, pv), k2 = warp_key(M2, cm2, pv);
              const uint32_t r1 = k1 == UINT_MAX ? UINT_MAX : k1 - ((uint32_t)ws << 1);
              const uint32_t r2 = k2 == UINT_MAX ? UINT_MAX : k2 + ((uint32_t)(n - ws) << 1);
              pk = min(r1, r2);
            }
            gmin_pair(v, pv, pk);
            m = v[0];
            improve = E + m < Ebest;
            kj = improve ? step1_key(cma, m) : UINT_MAX;
            wk = pk;
            di = pv;
          } else {
            int v[2] = {min_of(cma), min(min_of(cm1), min_of(cm2))};
            gmin(v);
            m = v[0];
            improve = E + m < Ebest;
            // first in cyclic order from ws: [ws, n) before [0, ws + wsz - n)
            const uint32_t k1 = warp_key(M1, cm1, v[1]), k2 = warp_key(M2, cm2, v[1]);
            const uint32_t r1 = k1 == UINT_MAX ? UINT_MAX : k1 - ((uint32_t)ws << 1);
            const uint32_t r2 = k2 == UINT_MAX ? UINT_MAX : k2 + ((uint32_t)(n - ws) << 1);
            uint32_t k[2] = {improve ? warp_key(FULL, cma, m) : UINT_MAX, min(r1, r2)};
            gminu(k);
            kj = k[0];
            wk = k[1];
            di = v[1];
          }
          const int sb = ws + (int)(wk >> 1);
          i = sb >= n ? sb - n : sb;
          xi = (int)(wk & 1u);
          ws += wsz;
          if (ws >= n) ws -= n;
        } else {  // RANDOMMIN
          uint32_t thr = (uint32_t)(cube_of(fup) >> 16);
          thr = thr < c16 ? c16 : (thr > 65536u ? 65536u : thr);
          uint4 rr[CH];  // this iteration's draws
          randmin_draw(flips, rr);
          const uint32_t Cm = mask_of([&](int p) { return randmin_hit(rr, p, thr); }) & F;
          int cmc[CH];
          chunk_min(Cm, cmc);
          uint32_t key;
          if constexpr (NW > 1) {
            // the candidates' pair in Step 1's round
            int v[1] = {__reduce_min_sync(FULL, min_of(cma))};
            int pv = __reduce_min_sync(FULL, min_of(cmc));
            uint32_t pk = pv == INT_MAX ? UINT_MAX : warp_key(Cm, cmc, pv);
            gmin_pair(v, pv, pk);
            m = v[0];
            improve = E + m < Ebest;
            kj = improve ? step1_key(cma, m) : UINT_MAX;
            if (pv == INT_MAX) {  // no candidate: argmin over the free bits (rare)
              int cmf[CH];
              chunk_min(F, cmf);
              int vf[1] = {min_of(cmf)};
              gmin(vf);
              pv = vf[0];
              uint32_t kf[1] = {warp_key(F, cmf, pv)};
              gminu(kf);
              pk = kf[0];
            }
            di = pv;
            key = pk;
          } else {
            int v[2] = {min_of(cma), min_of(cmc)};
            gmin(v);
            m = v[0];
            improve = E + m < Ebest;
            uint32_t ks;
            if (v[1] != INT_MAX) {
              di = v[1];
              ks = warp_key(Cm, cmc, di);
            } else {  // no candidate: argmin over the free bits (rare)
              int cmf[CH];
              chunk_min(F, cmf);
              int vf[1] = {min_of(cmf)};
              gmin(vf);
              di = vf[0];
              ks = warp_key(F, cmf, di);
            }
            uint32_t k[2] = {improve ? warp_key(FULL, cma, m) : UINT_MAX, ks};
            gminu(k);
            kj = k[0];
            key = k[1];
          }
          i = (int)(key >> 1);
          xi = (int)(key & 1u);
        }
      }
      if (improve) take_best(kj, m);
      uint4 rv[CH];
      row_load(i, xi, rv);
      // independent of row i: overlaps its load latency
      if constexpr (C::EARLY) di = commit(i, xi);
      if (phase == PH_MAIN && ALGO != TWONEIGHBOR) tabu_push(i, tau);
      row_apply(rv, di);
      if constexpr (!C::EARLY) flip_after(i, di, xi);
      if constexpr (NW > 1 && ALGO == TWONEIGHBOR) {
        if (phase == PH_MAIN && it + 1 < Tmain) {
          const int q = it + 1;  // the next bit differs from bit i
          publish_next((q & 1) ? (q + 1) >> 1 : (q >> 1) - 1, q);
        }
      }
      if (phase == PH_MAIN && ++it == Tmain) {
        phase = PH_GREEDY;
        ++runs;
        tb[0] = 0;
      }
    }
  }

  __device__ __forceinline__ void run(int algo, int seed_mode, int T, int tau, uint32_t B) {
    if constexpr (C::KEY) {
      switch (algo) {
        case MAXMIN: run_key<MAXMIN>(seed_mode, T, tau, B); break;
        case CYCLICMIN: run_key<CYCLICMIN>(seed_mode, T, tau, B); break;
        case RANDOMMIN: run_key<RANDOMMIN>(seed_mode, T, tau, B); break;
        case POSITIVEMIN: run_key<POSITIVEMIN>(seed_mode, T, tau, B); break;
        default: run_key<TWONEIGHBOR>(seed_mode, T, tau, B); break;
      }
    } else {
      switch (algo) {
        case MAXMIN: run_algo<MAXMIN>(seed_mode, T, tau, B); break;
        case CYCLICMIN: run_algo<CYCLICMIN>(seed_mode, T, tau, B); break;
        case RANDOMMIN: run_algo<RANDOMMIN>(seed_mode, T, tau, B); break;
        case POSITIVEMIN: run_algo<POSITIVEMIN>(seed_mode, T, tau, B); break;
        default: run_algo<TWONEIGHBOR>(seed_mode, T, tau, B); break;
      }
    }
  }

  // ------------------------------------------------------------ keyed batch search
  // The same sequence and selectors as run_algo on keys: every arg-min is the
  // minimum key itself, whose low kb bits are (k << 1 | x_k).
  template <int ALGO>
  __device__ __forceinline__ void run_key(int seed_mode, int T, int tau, uint32_t B) {
    int phase = seed_mode == 0 ? PH_STRAIGHT : PH_GREEDY;
    int runs = 0, it = 0, ws = 0;
    const int Tmain = ALGO == TWONEIGHBOR ? 2 * n - 1 : T;
    const uint32_t Kq = (1u << 21) / (uint32_t)T, Kr = (1u << 21) % (uint32_t)T;
    uint32_t fup = 0, rup = 0, fdn = 1u << 21;
    int rdn = 0;
    uint32_t rnd0 = 0, rnd1 = 0;  // 32 MaxMin/PositiveMin draws, one per lane
    const int cwin = n < 32 ? n : 32;
    // RandomMin's floor c = 32/n in units of 2^-16, rounded up
    const uint32_t c16 = ((1u << 21) + (uint32_t)n - 1) / (uint32_t)n;
    const int low = (1 << kb) - 1;  // (k << 1 | x_k) part of a key
    const int unit = 1 << kb;       // Delta = 1 in key units
    for (;;) {
      int sk;  // key of the bit to flip
      int cma[CH];
      chunk_min_all(cma);  // Step 1: every one-bit neighbour
      int mk;              // its minimum key
      if (phase != PH_MAIN) {
        // ---------------- Straight / Greedy
        const bool st = phase == PH_STRAIGHT;
        const uint32_t Ms = (xb[0] ^ db[0]) & vb[0];
        int cms[CH];
        if (st) chunk_min(Ms, cms);
        int v[2] = {min_of(cma), st ? min_of(cms) : INT_MAX};
        gmin(v);
        mk = v[0];
        if (st && v[1] == INT_MAX) {  // X == D: Straight ends
          phase = PH_GREEDY;
          continue;
        }
        const int m = mk >> kb;
        if (E + m < Ebest) take_best((uint32_t)(mk & low), m);
        if (!st && m >= 0) {  // local minimum: Greedy ends after Step 1
          if (flips < B && !(ALGO == TWONEIGHBOR && runs >= 1)) {
            phase = PH_MAIN;
            it = 0;
            ws = 0;
            fup = 0;
            rup = 0;
            fdn = 1u << 21;
            rdn = 0;
            tb[0] = 0;
            ring_len = 0;
            ring_head = 0;
            continue;
          }
          break;
        }
        sk = st ? v[1] : mk;
      } else {
        // ---------------- main search iteration t = it + 1
        fup += Kq;
        rup += Kr;
        if (rup >= (uint32_t)T) { ++fup; rup -= (uint32_t)T; }
        fdn -= Kq;
        rdn -= (int)Kr;
        if (rdn < 0) { --fdn; rdn += T; }
        const uint32_t F = vb[0] & ~tb[0];  // free (non-tabu) bits
        if (ALGO == TWONEIGHBOR) {
          int v[1] = {min_of(cma)};
          gmin(v);
          mk = v[0];
          const int i = it == 0 ? 0 : ((it & 1) ? (it + 1) >> 1 : (it >> 1) - 1);
          int dv;
          const int x = fetch_x(i, &dv);
          sk = C::EARLY ? (i << 1) | x : dv;  // its key (early commit: the low part)
        } else if (ALGO == MAXMIN || ALGO == POSITIVEMIN) {
          if ((it & 31) == 0) {
            const uint4 u = draw(seed, flips + (uint32_t)lane, g, s,
                                 ALGO == MAXMIN ? RNG_MAXMIN : RNG_POSMIN);
            rnd0 = u.x;
            rnd1 = u.y;
          }
          const uint32_t u0 = __shfl_sync(FULL, rnd0, it & 31);
          uint32_t Cm = 0, ukth = 0;
          if (ALGO == MAXMIN) {
            int cmn[CH], cmx[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              int vn[8], vx[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const bool f = (F >> (8 * c + e)) & 1u;
                vn[e] = f ? d[8 * c + e] : INT_MAX;
                vx[e] = f ? d[8 * c + e] : INT_MIN;
              }
              cmn[c] = min8(vn);
              cmx[c] = ~max8(vx);
            }
            int v[3] = {min_of(cma), min_of(cmn), min_of(cmx)};
            gmin(v);
            mk = v[0];
            const int mn = v[1] >> kb, mx = (~v[2]) >> kb;
            const uint64_t q = cube_of(fdn);
            const uint64_t span = (uint64_t)((int64_t)mx - (int64_t)mn);
            const uint64_t R = (q * span) >> 32;
            const int thr = (int)((int64_t)mn + (int64_t)(((uint64_t)u0 * (R + 1)) >> 32));
            const int lim = (thr + 1) * unit;  // Delta <= thr  <=>  key < lim
            Cm = mask_of([&](int p) { return d[p] < lim; }) & F;
            ukth = __shfl_sync(FULL, rnd1, it & 31);
          } else {
            int cmp[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              int vp[8];
#pragma unroll
              for (int e = 0; e < 8; ++e)
                vp[e] = (((F >> (8 * c + e)) & 1u) && d[8 * c + e] >= unit) ? d[8 * c + e] : INT_MAX;
              cmp[c] = min8(vp);
            }
            int v[2] = {min_of(cma), min_of(cmp)};
            gmin(v);
            mk = v[0];
            if (v[1] != INT_MAX) {
              const int lim = ((v[1] >> kb) + 1) * unit;
              Cm = mask_of([&](int p) { return d[p] < lim; }) & F;
            } else {
              Cm = F;
            }
            ukth = u0;
          }
          int dv;
          const uint32_t kk = kth(Cm, ukth, &dv);
          sk = C::EARLY ? (int)kk : dv;  // its key (early commit: the low part)
        } else if (ALGO == CYCLICMIN) {
          const uint64_t wl = (cube_of(fup) * (uint64_t)n) >> 32;
          const int wsz = (int)(wl < (uint64_t)cwin ? (uint64_t)cwin : (wl > (uint64_t)n ? (uint64_t)n : wl));
          const int hi1 = min(ws + wsz, n), hi2 = ws + wsz - n;
          uint32_t M1 = 0, M2 = 0;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int b0 = c * SPAN + 8 * t;
            M1 |= run_mask(b0, ws, hi1) << (8 * c);
            M2 |= run_mask(b0, 0, hi2) << (8 * c);
          }
          M1 &= F;
          M2 &= F;
          int cm1[CH], cm2[CH];
          chunk_min(M1, cm1);
          chunk_min(M2, cm2);
          int v[3] = {min_of(cma), min_of(cm1), min_of(cm2)};
          gmin(v);
          mk = v[0];
          // first in cyclic order from ws: [ws, n) before [0, ws + wsz - n)
          sk = (v[2] == INT_MAX || (v[1] != INT_MAX && (v[1] >> kb) <= (v[2] >> kb))) ? v[1] : v[2];
          ws += wsz;
          if (ws >= n) ws -= n;
        } else {  // RANDOMMIN
          uint32_t thr = (uint32_t)(cube_of(fup) >> 16);
          thr = thr < c16 ? c16 : (thr > 65536u ? 65536u : thr);
          uint4 rr[CH];  // this iteration's draws
          randmin_draw(flips, rr);
          const uint32_t Cm = mask_of([&](int p) { return randmin_hit(rr, p, thr); }) & F;
          int cmc[CH];
          chunk_min(Cm, cmc);
          int v[2] = {min_of(cma), min_of(cmc)};
          gmin(v);
          mk = v[0];
          sk = v[1];
          if (sk == INT_MAX) {  // no candidate: arg-min over the free bits (rare)
            int cmf[CH];
            chunk_min(F, cmf);
            int vf[1] = {min_of(cmf)};
            gmin(vf);
            sk = vf[0];
          }
        }
        const int m = mk >> kb;
        if (E + m < Ebest) take_best((uint32_t)(mk & low), m);
      }
      const int i = (sk & low) >> 1, xi = sk & 1;
      uint4 rv[CH];
      row_load(i, xi, rv);
      // independent of row i: overlaps its load latency
      int di = sk >> kb;  // groups of warps: from the selection
      if constexpr (C::EARLY) di = commit(i, xi);
      if (phase == PH_MAIN && ALGO != TWONEIGHBOR) tabu_push(i, tau);
      row_apply(rv, di);
      if constexpr (!C::EARLY) flip_after(i, di, xi);
      if (phase == PH_MAIN && ++it == Tmain) {
        phase = PH_GREEDY;
        ++runs;
        tb[0] = 0;
      }
    }
  }

  // ------------------------------------------------------------ state I/O
  __device__ __forceinline__ void load(const SearchArgs& a) {
    const uint8_t* xbytes = reinterpret_cast<const uint8_t*>(a.X + (size_t)s * a.nw);
    const uint8_t* dbytes = reinterpret_cast<const uint8_t*>(a.D + (size_t)s * a.nw);
    const int32_t* dl = a.delta + (size_t)s * ld;
    const int nbytes = 4 * a.nw;
    xb[0] = 0; db[0] = 0; vb[0] = 0; bb[0] = 0; tb[0] = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int base = c * SPAN + 8 * t;
      int4 v0 = make_int4(0, 0, 0, 0), v1 = v0;
      if (base < ld) {
        v0 = *reinterpret_cast<const int4*>(dl + base);
        v1 = *reinterpret_cast<const int4*>(dl + base + 4);
      }
      const int vals[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
      const int bi = c * NT + t;
      const uint32_t xbyte = bi < nbytes ? xbytes[bi] : 0u;
      const uint32_t dbyte = bi < nbytes ? dbytes[bi] : 0u;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int p = 8 * c + e;
        const bool valid = base + e < n;
        const int xk = (int)((xbyte >> e) & 1u);
        if constexpr (C::KEY)
          d[p] = valid ? vals[e] * (1 << kb) + (((base + e) << 1) | xk) : INT_MAX;
        else
          d[p] = valid ? vals[e] : INT_MAX;
        if constexpr (C::SG8) {
          if (e % 4 == 0) sg[p / 4] = 0;
          sg[p / 4] |= (int)((xk && valid ? 0x01u : 0xFFu) << (8 * (p % 4)));
        } else {
          sg[p] = (xk && valid ? 1 : -1) * (C::KEY ? (1 << kb) : 1);
        }
        if (valid) {
          vb[0] |= 1u << p;
          xb[0] |= ((xbyte >> e) & 1u) << p;
          db[0] |= ((dbyte >> e) & 1u) << p;
        }
      }
    }
    E = a.E2 ? a.E2[s] / 2 : a.E[s];
    Ebest = INT64_MAX;
    flips = 0;
  }

  __device__ __forceinline__ void store(const SearchArgs& a) {
    uint8_t* xbytes = reinterpret_cast<uint8_t*>(a.X + (size_t)s * a.nw);
    uint8_t* bbytes = reinterpret_cast<uint8_t*>(a.best_X + (size_t)s * a.nw);
    int32_t* dl = a.delta + (size_t)s * ld;
    const int nbytes = 4 * a.nw;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int base = c * SPAN + 8 * t;
      if (base < ld) {
        int vals[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          vals[e] = (base + e < n) ? (C::KEY ? d[8 * c + e] >> kb : d[8 * c + e]) : 0;
        *reinterpret_cast<int4*>(dl + base) = make_int4(vals[0], vals[1], vals[2], vals[3]);
        *reinterpret_cast<int4*>(dl + base + 4) = make_int4(vals[4], vals[5], vals[6], vals[7]);
      }
      const int bi = c * NT + t;
      if (bi < nbytes) {
        xbytes[bi] = (uint8_t)((xb[0] >> (8 * c)) & 0xFFu);
        bbytes[bi] = (uint8_t)((bb[0] >> (8 * c)) & 0xFFu);
      }
    }
    if (t == 0) {
      a.E[s] = E;
      a.best_E[s] = Ebest;
      a.flips[s] = flips;
    }
  }
};

// Eight-warp variants are held to 128 registers so that two searches share an
// SM (8x4 spills a little; measured 21% faster per flip at n = 8192 than one
// search per SM); the others keep one CTA's worth of registers per thread.
template <int NW, int CH, int RF, bool KEY, bool EARLY>
__global__ void __launch_bounds__(Cfg<NW, CH, RF, KEY>::CTA, (NW == 8 ? 2 : 1))
    k_batch_search(const SearchArgs single, const MultiArgs multi) {
  using C = Cfg<NW, CH, RF, KEY, EARLY>;
  __shared__ SmemSearch<C> smem[C::SPC];
  extern __shared__ __align__(16) unsigned char dsm[];
  const int sl = threadIdx.x / C::NT;
  // the launcher may use fewer searches per CTA than the maximum, so that the
  // CTAs spread over all SMs; the other warps of the CTA leave at once
  const int spc = single.spc > 0 ? single.spc : C::SPC;
  // shared-memory W or sparse rows (one instance per launch): the whole CTA
  // copies them into shared memory and clears the scratch rows
  if constexpr (RF == ROWS_DENSE_SMEM) {
    const int w16 = single.n * single.ld / 8;
    uint4* d4 = reinterpret_cast<uint4*>(dsm);
    const uint4* gw = reinterpret_cast<const uint4*>(single.W);
    for (int q = threadIdx.x; q < w16; q += blockDim.x) d4[q] = gw[q];
    __syncthreads();
  }
  int c16 = 0;  // 16-byte units before the scratch rows
  if constexpr (RF == ROWS_SPARSE_SMEM || RF == ROWS_SPARSE_GLOBAL) {
    const int r16 = sparse_row16(single.n), e16 = sparse_ent16(single.sp_nnz);
    uint4* d4 = reinterpret_cast<uint4*>(dsm);
    if constexpr (RF == ROWS_SPARSE_SMEM) {
      const uint4* gr = reinterpret_cast<const uint4*>(single.sp_row);
      const uint4* ge = reinterpret_cast<const uint4*>(single.sp_ent);
      for (int q = threadIdx.x; q < r16; q += blockDim.x) d4[q] = gr[q];
      for (int q = threadIdx.x; q < e16; q += blockDim.x) d4[r16 + q] = ge[q];
      c16 = r16 + e16;
    }
    const int z16 = spc * single.ld / 8;
    for (int q = threadIdx.x; q < z16; q += blockDim.x) d4[c16 + q] = make_uint4(0, 0, 0, 0);
    __syncthreads();
  }
  if (sl >= spc) return;
  const uint32_t slot = blockIdx.x * spc + sl;
  // one instance (single) or several (multi: find the slot's instance)
  const SearchArgs* ap = &single;
  uint32_t local = slot;
  if (multi.insts) {
    if (slot >= (uint32_t)multi.total) return;
    int lo = 0, hi = multi.ninst;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((uint32_t)multi.prefix[mid] <= slot) lo = mid; else hi = mid;
    }
    ap = multi.insts + lo;
    local = slot - (uint32_t)multi.prefix[lo];
  }
  const SearchArgs& a = *ap;
  if (local >= (uint32_t)a.S) return;
  // slots grouped by algorithm keep each SM on one loop body (instruction
  // cache); the search index s, and with it every result, is unchanged
  const uint32_t s = a.order ? (uint32_t)a.order[local] : local;
  const DevCtrl* ctrl = a.ctrl;
  if (ctrl->done) return;
  Searcher<C> sr(a, &smem[sl], threadIdx.x % C::NT, s, ctrl->g, ctrl->seed);
  if constexpr (RF == ROWS_SPARSE_SMEM) {
    sr.srow = reinterpret_cast<const uint32_t*>(dsm);
    sr.sent = sr.srow + 4 * sparse_row16(a.n);
  } else if constexpr (RF == ROWS_SPARSE_GLOBAL) {
    sr.srow = a.sp_row;
    sr.sent = a.sp_ent;
  }
  if constexpr (RF == ROWS_SPARSE_SMEM || RF == ROWS_SPARSE_GLOBAL)
    sr.scr = reinterpret_cast<int16_t*>(dsm + 16 * (size_t)c16) + (size_t)sl * a.ld;
  if constexpr (RF == ROWS_DENSE_SMEM) sr.sw = reinterpret_cast<const int16_t*>(dsm);
  sr.load(a);
  sr.run(a.algo[s], a.seed_mode, a.T, a.tau, a.B);
  sr.store(a);
}

template <int NW, int CH, int RF, bool KEY = false, bool EARLY = true>
void launch_rows(const SearchArgs& a, const MultiArgs& m, unsigned grid, cudaStream_t st) {
  size_t dyn = 0;
  if constexpr (RF != ROWS_DENSE) {
    dyn = sparse_smem_bytes(RF, a.n, a.sp_nnz, a.ld, a.spc);  // also W for ROWS_DENSE_SMEM
    // a size above the device's limit makes the launch fail (the caller reads
    // the error); the host only selects a sparse format that fits
    cudaFuncSetAttribute(k_batch_search<NW, CH, RF, KEY, EARLY>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  }
  k_batch_search<NW, CH, RF, KEY, EARLY><<<grid, Cfg<NW, CH, RF, KEY>::CTA, dyn, st>>>(a, m);
}

// Launches one variant over `slots` searches of one instance (m == nullptr)
// or of the instances listed in *m.  A single instance whose arguments carry
// sparse rows runs the sparse-row kernel of its format.
template <int NW, int CH>
bool launch_variant(const SearchArgs* a, cudaStream_t st, SearchVariant* v, const MultiArgs* m) {
  using C = Cfg<NW, CH>;
  if (v) *v = SearchVariant{NW, CH, C::CAP, C::CTA, C::SPC};
  if (!a) return true;
  const int slots = m ? m->total : a->S;
  if (slots <= 0) return true;
  SearchArgs a2 = *a;
  a2.spc = spc_for(slots, C::SPC);
  const unsigned grid = (unsigned)((slots + a2.spc - 1) / a2.spc);
  const MultiArgs mm = m ? *m : MultiArgs{nullptr, nullptr, 0, 0};
  // the keyed form runs for single-instance launches with dense rows (from
  // global or, one-warp variants, shared memory)
  const int mode = m ? ROWS_DENSE
                     : (a2.sp_mode == ROWS_DENSE_SMEM ? (NW == 1 ? ROWS_DENSE_SMEM : ROWS_DENSE)
                                                      : (a2.sp_row ? a2.sp_mode : ROWS_DENSE));
  if constexpr (NW == 1) {
    if (mode == ROWS_DENSE_SMEM) {
      if (a2.key_bits > 0) launch_rows<NW, CH, ROWS_DENSE_SMEM, true>(a2, mm, grid, st);
      else launch_rows<NW, CH, ROWS_DENSE_SMEM>(a2, mm, grid, st);
      return true;
    }
  }
  if (mode == ROWS_SPARSE_SMEM)
    launch_rows<NW, CH, ROWS_SPARSE_SMEM>(a2, mm, grid, st);
  else if (mode == ROWS_SPARSE_GLOBAL)
    launch_rows<NW, CH, ROWS_SPARSE_GLOBAL>(a2, mm, grid, st);
  else if (!m && a2.key_bits > 0)
    launch_rows<NW, CH, ROWS_DENSE, true>(a2, mm, grid, st);
  else if (!m)
    launch_rows<NW, CH, ROWS_DENSE>(a2, mm, grid, st);
  else  // several instances per launch
    launch_rows<NW, CH, ROWS_DENSE, false, false>(a2, mm, grid, st);
  return true;
}

}  // namespace dabs
