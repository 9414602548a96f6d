// search.cuh -- the batch-search kernel (Section III-A incremental search,
// Section III-B batch search): one group of NW warps per search slot keeps X,
// the exact int32 Delta vector and the int64 energy in registers, and flips one
// bit per iteration: Step 1 (best one-bit neighbour -> BEST), Step 2 (the
// phase's selector), Step 3 (E += Delta_i, Delta_k += W_ik sigma(x_i) sigma(x_k)
// for k != i by Eq. (4), Delta_i = -Delta_i by Eq. (5)).
//
// Register layout: thread t of a group (NT = 32 NW threads) owns, for chunk
// c = 0..CH-1, the eight consecutive bits k = c*8*NT + 8t + e (e = 0..7).  One
// 128-bit load per chunk brings the thread's eight int16 weights of row i, so
// a whole row is read with fully coalesced 16-byte accesses.  Bit k lives at
// local position p = 8c + e of the thread's Delta array and bit masks.
//
// Reductions use the sm_80+ warp reduce instructions and, for NW > 1, one
// shared-memory slot round per reduction (double-buffered, one barrier).
// Ties always resolve to the lowest bit index (for CyclicMin: the first bit in
// cyclic order from the window start).
#pragma once
#include "common.cuh"

namespace dabs {

template <int NW_, int CH_>
struct Cfg {
  static constexpr int NW = NW_, CH = CH_;
  static constexpr int NT = 32 * NW;           // threads per search
  static constexpr int EPT = 8 * CH;           // bits per thread
  static constexpr int SPAN = 8 * NT;          // bits per chunk
  static constexpr int NMW = (EPT + 31) / 32;  // mask words per thread
  static constexpr int SPC = NW == 1 ? 4 : 1;  // searches per CTA
  static constexpr int CTA = NT * SPC;
  static constexpr int CAP = SPAN * CH;        // largest n this variant holds
};

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int sext_lo(uint32_t w) { return (int)(w << 16) >> 16; }
__device__ __forceinline__ int sext_hi(uint32_t w) { return (int)w >> 16; }
__device__ __forceinline__ int w16(const uint4& v, int e) {
  const uint32_t w = e < 2 ? v.x : e < 4 ? v.y : e < 6 ? v.z : v.w;
  return (e & 1) ? sext_hi(w) : sext_lo(w);
}
__device__ __forceinline__ uint32_t u32of(const uint4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

template <class C>
struct SmemSearch {
  int red[2][C::NW][4];      // reduction slots (double buffered)
  int tot[C::CH][C::NW];     // per chunk, per warp candidate counts (k-th pick)
  int pick[4];               // broadcast of a pick made by one thread
  int ring[C::NW][32];       // tabu list (one copy per warp: warp-synchronous updates)
};

template <class C>
struct Searcher {
  static constexpr int NW = C::NW, CH = C::CH, NT = C::NT, EPT = C::EPT, SPAN = C::SPAN,
                       NMW = C::NMW;
  // --- state (registers) ---
  int d[EPT];          // Delta (INT_MAX for bits >= n)
  uint32_t xb[NMW];    // X bits
  uint32_t bb[NMW];    // BEST bits
  uint32_t vb[NMW];    // valid bits (k < n)
  uint32_t db[NMW];    // target D bits
  uint32_t tb[NMW];    // tabu bits
  int64_t E, Ebest;
  uint32_t flips;
  // --- context ---
  const SearchArgs a;
  SmemSearch<C>* sm;
  int t, lane, warp, buf;
  uint32_t s, g;
  uint64_t seed;
  const int16_t* W;
  int n, ld;
  // tabu ring (uniform): flipped bits of the last tau main iterations
  int ring_len, ring_head;

  __device__ __forceinline__ Searcher(const SearchArgs& args, SmemSearch<C>* smem, int tid, uint32_t sidx,
                      uint32_t gen, uint64_t sd)
      : a(args), sm(smem), t(tid), lane(tid & 31), warp(tid >> 5), buf(0), s(sidx), g(gen),
        seed(sd), W(args.W), n(args.n), ld(args.ld) {}

  // ------------------------------------------------------------ bit helpers
  __device__ __forceinline__ static bool bit(const uint32_t (&m)[NMW], int p) {
    return (m[p >> 5] >> (p & 31)) & 1u;
  }
  // same for a run-time position (no dynamic register-array indexing)
  __device__ __forceinline__ static bool bit_at(const uint32_t (&m)[NMW], int p) {
    uint32_t w = 0;
#pragma unroll
    for (int q = 0; q < NMW; ++q)
      if (q == (p >> 5)) w = m[q];
    return (w >> (p & 31)) & 1u;
  }
  __device__ __forceinline__ int kidx(int p) const { return (p >> 3) * SPAN + 8 * t + (p & 7); }
  __device__ __forceinline__ static int owner_t(int i) { return (i >> 3) & (NT - 1); }
  __device__ __forceinline__ static int local_p(int i) { return ((i >> 3) / NT) * 8 + (i & 7); }
  __device__ __forceinline__ void toggle(uint32_t (&m)[NMW], int p) {
#pragma unroll
    for (int q = 0; q < NMW; ++q)
      if (q == (p >> 5)) m[q] ^= 1u << (p & 31);
  }
  // value of d at a run-time position p (same p in all threads of the group)
  __device__ __forceinline__ int get_at(int p) const {
    int v = 0;
#pragma unroll
    for (int q = 0; q < EPT; ++q)
      if (q == p) v = d[q];
    return v;
  }
  __device__ __forceinline__ void set_at(int p, int v) {
#pragma unroll
    for (int q = 0; q < EPT; ++q)
      if (q == p) d[q] = v;
  }

  // ------------------------------------------------------------ reductions
  __device__ __forceinline__ void gsync() {
    if constexpr (NW == 1) __syncwarp();
    else __syncthreads();
  }
  // group min of up to three int values (warp reduce, then a slot round)
  template <int K>
  __device__ __forceinline__ void gmin(int (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = __reduce_min_sync(FULL, v[q]);
    if constexpr (NW > 1) {
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) sm->red[buf][warp][q] = v[q];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < K; ++q) {
        int r = sm->red[buf][0][q];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = min(r, sm->red[buf][w][q]);
        v[q] = r;
      }
      buf ^= 1;
    }
  }
  template <int K>
  __device__ __forceinline__ void gminu(uint32_t (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = __reduce_min_sync(FULL, v[q]);
    if constexpr (NW > 1) {
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) sm->red[buf][warp][q] = (int)v[q];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < K; ++q) {
        uint32_t r = (uint32_t)sm->red[buf][0][q];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = min(r, (uint32_t)sm->red[buf][w][q]);
        v[q] = r;
      }
      buf ^= 1;
    }
  }

  // ------------------------------------------------------------ per-thread scans
  __device__ __forceinline__ int tmin_all() const {
    int m = INT_MAX;
#pragma unroll
    for (int p = 0; p < EPT; ++p) m = min(m, d[p]);
    return m;
  }
  __device__ __forceinline__ int tmin_mask(const uint32_t (&M)[NMW]) const {
    int m = INT_MAX;
#pragma unroll
    for (int p = 0; p < EPT; ++p)
      if (bit(M, p)) m = min(m, d[p]);
    return m;
  }
  // key = (k << 1) | x_k of the lowest k with d == v (UINT_MAX if none)
  __device__ __forceinline__ uint32_t tkey_eq(int v) const {
    uint32_t key = UINT_MAX;
#pragma unroll
    for (int p = EPT - 1; p >= 0; --p)
      if (d[p] == v) key = ((uint32_t)kidx(p) << 1) | (uint32_t)bit(xb, p);
    return key;
  }
  __device__ __forceinline__ uint32_t tkey_eq_mask(int v, const uint32_t (&M)[NMW]) const {
    uint32_t key = UINT_MAX;
#pragma unroll
    for (int p = EPT - 1; p >= 0; --p)
      if (bit(M, p) && d[p] == v) key = ((uint32_t)kidx(p) << 1) | (uint32_t)bit(xb, p);
    return key;
  }

  // ------------------------------------------------------------ Step 1 / Step 3
  // BEST <- f_j(X) for j = key >> 1 (Step 1 on strict improvement)
  __device__ __forceinline__ void take_best(uint32_t keyj, int m) {
    const int j = (int)(keyj >> 1);
#pragma unroll
    for (int q = 0; q < NMW; ++q) bb[q] = xb[q];
    if (t == owner_t(j)) toggle(bb, local_p(j));
    Ebest = E + m;
  }

  // Step 3: flip bit i (x_i = xi before the flip, di = Delta_i before the flip)
  __device__ __forceinline__ void flip(int i, int xi, int di) {
    // every selector yields 0 <= i < n; the clamp only keeps a logic error
    // from turning into an out-of-bounds read (parity tests would flag it)
    i = min(max(i, 0), n - 1);
    const int16_t* row = W + (size_t)i * ld;
    uint4 rv[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int off = c * SPAN + 8 * t;
      rv[c] = off < ld ? __ldg(reinterpret_cast<const uint4*>(row + off)) : make_uint4(0, 0, 0, 0);
    }
    const uint32_t xim = xi ? FULL : 0u;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int p = 8 * c + e;
        // -1 where x_k != x_i: sigma(x_i) sigma(x_k) = (m | 1)
        const int m = -(int)(((xb[p >> 5] ^ xim) >> (p & 31)) & 1u);
        d[p] += w16(rv[c], e) * (m | 1);
      }
    }
    const int pi = local_p(i);
    const bool own = (t == owner_t(i));
    if (own) {
      set_at(pi, -di);  // Eq. (5)
      toggle(xb, pi);
    }
    E += di;
    ++flips;
  }

  // ------------------------------------------------------------ k-th pick
  // The ((u * count) >> 32)-th set bit of the group-wide candidate mask Cm, in
  // ascending bit order.  Returns key = (i << 1) | x_i and Delta_i via *di.
  __device__ __forceinline__ uint32_t kth(const uint32_t (&Cm)[NMW], uint32_t u, int* di) {
    int cnt[CH], wt[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      cnt[c] = __popc((Cm[(8 * c) >> 5] >> ((8 * c) & 31)) & 0xFFu);
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
      int total = 0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int w = 0; w < NW; ++w) total += sm->tot[c][w];
      int kk = (int)uniform_below(u, (uint32_t)total);
      bool found = false;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int tw = sm->tot[c][w];
          if (!found && kk < tw) { csel = c; wsel = w; rel = kk; found = true; }
          if (!found) kk -= tw;
        }
    }
    uint32_t key = 0;
    int dv = 0;
    if (warp == wsel) {
      int mycnt = 0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c == csel) mycnt = cnt[c];
      int incl = mycnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
      }
      const int excl = incl - mycnt;
      const bool mine = excl <= rel && rel < incl;
      if (mine) {
        uint32_t byte = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c == csel) byte = (Cm[(8 * c) >> 5] >> ((8 * c) & 31)) & 0xFFu;
        int r = rel - excl;
        int e = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if ((byte >> q) & 1u) {
            if (r == 0) e = q;
            --r;
          }
        const int p = 8 * csel + e;
        key = ((uint32_t)kidx(p) << 1) | (uint32_t)bit_at(xb, p);
        dv = get_at(p);
      }
      const unsigned bal = __ballot_sync(FULL, mine);
      const int src = __ffs(bal) - 1;
      key = __shfl_sync(FULL, key, src);
      dv = __shfl_sync(FULL, dv, src);
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

  // Delta_i and x_i of a bit chosen without a reduction (TwoNeighbor)
  __device__ __forceinline__ uint32_t fetch(int i, int* di) {
    const int pi = local_p(i), ot = owner_t(i);
    int v = get_at(pi);
    uint32_t x = bit_at(xb, pi) ? 1u : 0u;
    if constexpr (NW == 1) {
      v = __shfl_sync(FULL, v, ot);
      x = __shfl_sync(FULL, x, ot);
    } else {
      if (t == ot) { sm->pick[2] = v; sm->pick[3] = (int)x; }
      __syncthreads();
      v = sm->pick[2];
      x = (uint32_t)sm->pick[3];
      __syncthreads();
    }
    *di = v;
    return ((uint32_t)i << 1) | x;
  }

  // ------------------------------------------------------------ phases
  // Greedy (Section III-A): Step 1, stop at a local minimum, else flip argmin.
  __device__ __forceinline__ void greedy() {
    for (;;) {
      int v[1] = {tmin_all()};
      gmin(v);
      const int m = v[0];
      const bool improve = E + m < Ebest;
      if (m >= 0 && !improve) break;
      uint32_t k[1] = {tkey_eq(m)};
      gminu(k);
      if (improve) take_best(k[0], m);
      if (m >= 0) break;
      flip((int)(k[0] >> 1), (int)(k[0] & 1u), m);
    }
  }

  // Straight (Section III-A): walk to D flipping the argmin over x_k != d_k.
  __device__ __forceinline__ void straight() {
    for (;;) {
      uint32_t M[NMW];
#pragma unroll
      for (int q = 0; q < NMW; ++q) M[q] = (xb[q] ^ db[q]) & vb[q];
      int v[2] = {tmin_all(), tmin_mask(M)};
      gmin(v);
      if (v[1] == INT_MAX) break;  // X == D
      const int m = v[0], ms = v[1];
      const bool improve = E + m < Ebest;
      uint32_t k[2] = {improve ? tkey_eq(m) : UINT_MAX, tkey_eq_mask(ms, M)};
      gminu(k);
      if (improve) take_best(k[0], m);
      flip((int)(k[1] >> 1), (int)(k[1] & 1u), ms);
    }
  }

  __device__ __forceinline__ void step1_only(int m) {
    if (E + m < Ebest) {
      uint32_t k[1] = {tkey_eq(m)};
      gminu(k);
      take_best(k[0], m);
    }
  }

  __device__ __forceinline__ void tabu_free(uint32_t (&F)[NMW]) const {
#pragma unroll
    for (int q = 0; q < NMW; ++q) F[q] = vb[q] & ~tb[q];
  }
  // bit i flipped at this iteration becomes tabu for the next tau iterations
  __device__ __forceinline__ void tabu_push(int i, int tau) {
    if (tau <= 0) return;
    int* ring = sm->ring[warp];
    if (ring_len == tau) {
      const int old = ring[ring_head];
      if (t == owner_t(old)) toggle(tb, local_p(old));
    } else {
      ++ring_len;
    }
    __syncwarp();
    if (lane == 0) ring[ring_head] = i;
    __syncwarp();
    ring_head = ring_head + 1 == tau ? 0 : ring_head + 1;
    if (t == owner_t(i)) toggle(tb, local_p(i));
  }

  __device__ __forceinline__ void main_search(int algo, int T, int tau) {
    if (algo == TWONEIGHBOR) {
      for (int q = 0; q < 2 * n - 1; ++q) {
        const int i = q == 0 ? 0 : ((q & 1) ? (q + 1) >> 1 : (q >> 1) - 1);
        int v[1] = {tmin_all()};
        gmin(v);
        step1_only(v[0]);
        int di;
        const uint32_t key = fetch(i, &di);
        flip(i, (int)(key & 1u), di);
      }
      return;
    }
#pragma unroll
    for (int q = 0; q < NMW; ++q) tb[q] = 0;
    ring_len = 0;
    ring_head = 0;
    const int cwin = n < 32 ? n : 32;
    const uint32_t c16 = ((1u << 21) + (uint32_t)n - 1) / (uint32_t)n;
    int ws = 0;  // CyclicMin window start
    for (int it = 1; it <= T; ++it) {
      uint32_t F[NMW];
      tabu_free(F);
      int i = 0, xi = 0, di = 0;
      if (algo == MAXMIN) {
        int mx = INT_MIN;
#pragma unroll
        for (int p = 0; p < EPT; ++p)
          if (bit(F, p)) mx = max(mx, d[p]);
        int v[3] = {tmin_all(), tmin_mask(F), ~mx};
        gmin(v);
        step1_only(v[0]);
        const int mn = v[1];
        const int mxg = ~v[2];
        const uint64_t q = cube21((uint64_t)(T - it), (uint64_t)T);
        const uint64_t span = (uint64_t)((int64_t)mxg - (int64_t)mn);
        const uint64_t R = (q * span) >> 32;
        const uint4 u = draw(seed, flips, g, s, RNG_MAXMIN);
        const int64_t thr = (int64_t)mn + (int64_t)(((uint64_t)u.x * (R + 1)) >> 32);
        uint32_t Cm[NMW];
#pragma unroll
        for (int w = 0; w < NMW; ++w) Cm[w] = 0;
#pragma unroll
        for (int p = 0; p < EPT; ++p)
          if (bit(F, p) && (int64_t)d[p] <= thr) Cm[p >> 5] |= 1u << (p & 31);
        const uint32_t key = kth(Cm, u.y, &di);
        i = (int)(key >> 1);
        xi = (int)(key & 1u);
      } else if (algo == POSITIVEMIN) {
        int pm = INT_MAX;
#pragma unroll
        for (int p = 0; p < EPT; ++p)
          if (bit(F, p) && d[p] > 0) pm = min(pm, d[p]);
        int v[2] = {tmin_all(), pm};
        gmin(v);
        step1_only(v[0]);
        const int pmg = v[1];
        uint32_t Cm[NMW];
#pragma unroll
        for (int w = 0; w < NMW; ++w) Cm[w] = 0;
#pragma unroll
        for (int p = 0; p < EPT; ++p)
          if (bit(F, p) && (pmg == INT_MAX || d[p] <= pmg)) Cm[p >> 5] |= 1u << (p & 31);
        const uint4 u = draw(seed, flips, g, s, RNG_POSMIN);
        const uint32_t key = kth(Cm, u.x, &di);
        i = (int)(key >> 1);
        xi = (int)(key & 1u);
      } else if (algo == CYCLICMIN) {
        uint64_t wl = (cube21((uint64_t)it, (uint64_t)T) * (uint64_t)n) >> 32;
        if (wl < (uint64_t)cwin) wl = (uint64_t)cwin;
        if (wl > (uint64_t)n) wl = (uint64_t)n;
        const int wsz = (int)wl;
        int bm = INT_MAX;
        uint32_t Wm[NMW];
#pragma unroll
        for (int w = 0; w < NMW; ++w) Wm[w] = 0;
#pragma unroll
        for (int p = 0; p < EPT; ++p) {
          int r = kidx(p) - ws;
          if (r < 0) r += n;
          if (bit(F, p) && r < wsz) {
            Wm[p >> 5] |= 1u << (p & 31);
            bm = min(bm, d[p]);
          }
        }
        int v[2] = {tmin_all(), bm};
        gmin(v);
        const int m = v[0], mw = v[1];
        const bool improve = E + m < Ebest;
        // selection key: (cyclic offset from the window start << 1) | x
        uint32_t kc = UINT_MAX;
#pragma unroll
        for (int p = EPT - 1; p >= 0; --p) {
          int r = kidx(p) - ws;
          if (r < 0) r += n;
          if (bit(Wm, p) && d[p] == mw) kc = min(kc, ((uint32_t)r << 1) | (uint32_t)bit(xb, p));
        }
        uint32_t k[2] = {improve ? tkey_eq(m) : UINT_MAX, kc};
        gminu(k);
        if (improve) take_best(k[0], m);
        int sel = ws + (int)(k[1] >> 1);
        if (sel >= n) sel -= n;
        i = sel;
        xi = (int)(k[1] & 1u);
        di = mw;
        ws += wsz;
        if (ws >= n) ws -= n;
      } else {  // RANDOMMIN
        uint64_t thr = cube21((uint64_t)it, (uint64_t)T) >> 16;
        if (thr < c16) thr = c16;
        if (thr > 65536u) thr = 65536u;
        uint32_t Cm[NMW];
#pragma unroll
        for (int w = 0; w < NMW; ++w) Cm[w] = 0;
        int bc = INT_MAX;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const uint4 u = draw(seed, flips, g, s, RNG_RANDMIN | (uint32_t)(c * NT + t));
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int p = 8 * c + e;
            const uint32_t u16 = (u32of(u, e >> 1) >> (16 * (e & 1))) & 0xFFFFu;
            if (bit(F, p) && u16 < (uint32_t)thr) {
              Cm[p >> 5] |= 1u << (p & 31);
              bc = min(bc, d[p]);
            }
          }
        }
        int v[3] = {tmin_all(), bc, tmin_mask(F)};
        gmin(v);
        const int m = v[0];
        const bool improve = E + m < Ebest;
        const bool have = v[1] != INT_MAX;
        const int ms = have ? v[1] : v[2];
        uint32_t k[2] = {improve ? tkey_eq(m) : UINT_MAX, have ? tkey_eq_mask(ms, Cm) : tkey_eq_mask(ms, F)};
        gminu(k);
        if (improve) take_best(k[0], m);
        i = (int)(k[1] >> 1);
        xi = (int)(k[1] & 1u);
        di = ms;
      }
      flip(i, xi, di);
      tabu_push(i, tau);
    }
#pragma unroll
    for (int q = 0; q < NMW; ++q) tb[q] = 0;
  }

  // ------------------------------------------------------------ state I/O
  __device__ __forceinline__ void load() {
    const uint8_t* xbytes = reinterpret_cast<const uint8_t*>(a.X + (size_t)s * a.nw);
    const uint8_t* dbytes = reinterpret_cast<const uint8_t*>(a.D + (size_t)s * a.nw);
    const int32_t* dl = a.delta + (size_t)s * ld;
    const int nbytes = 4 * a.nw;
#pragma unroll
    for (int q = 0; q < NMW; ++q) { xb[q] = 0; db[q] = 0; vb[q] = 0; bb[q] = 0; tb[q] = 0; }
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
        d[p] = valid ? vals[e] : INT_MAX;
        if (valid) {
          vb[p >> 5] |= 1u << (p & 31);
          xb[p >> 5] |= ((xbyte >> e) & 1u) << (p & 31);
          db[p >> 5] |= ((dbyte >> e) & 1u) << (p & 31);
        }
      }
    }
    E = a.E[s];
    Ebest = INT64_MAX;
    flips = 0;
  }

  __device__ __forceinline__ void store() {
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
        for (int e = 0; e < 8; ++e) vals[e] = (base + e < n) ? d[8 * c + e] : 0;
        *reinterpret_cast<int4*>(dl + base) = make_int4(vals[0], vals[1], vals[2], vals[3]);
        *reinterpret_cast<int4*>(dl + base + 4) = make_int4(vals[4], vals[5], vals[6], vals[7]);
      }
      const int bi = c * NT + t;
      if (bi < nbytes) {
        xbytes[bi] = (uint8_t)((xb[(8 * c) >> 5] >> ((8 * c) & 31)) & 0xFFu);
        bbytes[bi] = (uint8_t)((bb[(8 * c) >> 5] >> ((8 * c) & 31)) & 0xFFu);
      }
    }
    if (t == 0) {
      a.E[s] = E;
      a.best_E[s] = Ebest;
      a.flips[s] = flips;
    }
  }
};

template <int NW, int CH>
__global__ void __launch_bounds__(Cfg<NW, CH>::CTA) k_batch_search(const SearchArgs a) {
  using C = Cfg<NW, CH>;
  __shared__ SmemSearch<C> smem[C::SPC];
  const int sl = threadIdx.x / C::NT;
  const uint32_t s = blockIdx.x * C::SPC + sl;
  if (s >= (uint32_t)a.S) return;
  const DevCtrl* ctrl = a.ctrl;
  if (ctrl->done) return;
  Searcher<C> sr(a, &smem[sl], threadIdx.x % C::NT, s, ctrl->g, ctrl->seed);
  sr.load();
  if (a.seed_mode == 0) sr.straight();
  sr.greedy();
  const int algo = a.algo[s];
  int runs = 0;
  // Section III-B: (main search, Greedy) rounds until at least b*n flips;
  // TwoNeighbor at most once.
  while (sr.flips < a.B && !(algo == TWONEIGHBOR && runs >= 1)) {
    sr.main_search(algo, a.T, a.tau);
    ++runs;
    sr.greedy();
  }
  sr.store();
}

}  // namespace dabs
