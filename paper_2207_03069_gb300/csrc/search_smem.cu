// search_smem.cu -- the batch search (Section III-A incremental search,
// Section III-B batch search) with Delta in shared memory: one warp per
// search and one search per CTA, so that large instances keep many searches
// per SM (as many as their shared memory allows) instead of spreading one
// search over many warps that meet at a barrier for every reduction.
//
// Lane l owns the L = 32 LW consecutive bits k = l L .. l L + L - 1 (LW the
// power of two >= ceil(n / 1024), so that owner and position are shifts and
// masks), so ascending bit order is lane order, then position: a
// minimum with the lowest index is a (value, index) pair reduced over lanes,
// and the k-th candidate of MaxMin / PositiveMin is one prefix over lanes.
// Each search's shared memory holds
//   dS[32][LP]   the stored Delta_k: Delta_k for a free bit, Delta_k + 2^30
//                for a tabu bit, INT_MAX for k >= n, so that every minimum
//                over the free (non-tabu) bits is a plain minimum; Step 1,
//                which also ranges over the tabu bits, adds the tabu ring's
//                entries (LP = L + 4 spreads the lanes over the banks);
//   sS[32][LP]   sigma(x_k) (0 for k >= n);
//   rS[32 L]     row i of sigma(x_i) W, fetched by one cp.async.bulk copy
//                completing on an mbarrier (bounded wait); lane l walks its
//                block starting at group l, which keeps the row, Delta and
//                sigma reads of a quarter-warp on distinct banks;
//   xS, tS, bS   X, target D and BEST bits, LW words per lane.
// Eq. (4) is one multiply-add per owned bit; Eq. (5) and the tabu penalties
// are single shared-memory stores.  Requires |Delta_k| < 2^29 in every state
// (R = max_k sum_j |W_kj| < 2^29, checked on the host).
#include <climits>

#include "dabs.h"
#include "kernels.cuh"
#include "umma.cuh"

namespace dabs {
namespace {

constexpr unsigned FULL_S = 0xffffffffu;
constexpr int kPen = 1 << 30;   // added to the stored Delta of a tabu bit
constexpr int kFree = 1 << 29;  // stored values below this belong to free bits
constexpr int kSent = INT_MAX;  // stored value of the bits k >= n
constexpr uint64_t kWaitNs = 2000000000ull;
enum : int { P_STRAIGHT = 0, P_GREEDY = 1, P_MAIN = 2 };

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int sx_lo(uint32_t w) { return (int)(w << 16) >> 16; }
__device__ __forceinline__ int sx_hi(uint32_t w) { return (int)w >> 16; }
__device__ __forceinline__ uint64_t cube21f(uint32_t f) {
  const uint64_t f2 = (uint64_t)f * f;
  return (f2 * f) >> 31;
}
__device__ __forceinline__ int min4(const int4& v) {
  return min(__vimin3_s32(v.x, v.y, v.z), v.w);
}
__device__ __forceinline__ int at4(const int4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

struct SmemSearch {
  // layout
  int n, ld, LW, L, LP, LWP, lane, base;
  int lsh;  // log2 L
  int* dS;
  int* sS;
  int16_t* rS;
  uint32_t* xS;
  uint32_t* tS;
  uint32_t* bS;
  uint64_t* bar;
  uint32_t parity;
  // problem and stream
  const int16_t* W;
  const int16_t* Wneg;
  uint64_t seed;
  uint32_t s, g;
  int* err;
  bool failed;
  bool stall;  // test hook: issue no copy for the next row, so its wait runs out
  // state
  int64_t E, Ebest;
  uint32_t flips;
  int ring_len, ring_head, ringv;

  __device__ int* dptr(int k) const { return dS + (k >> lsh) * LP + (k & (L - 1)); }
  __device__ int* sptr(int k) const { return sS + (k >> lsh) * LP + (k & (L - 1)); }
  __device__ uint32_t* xword(uint32_t* bits, int k) const {
    return bits + (k >> lsh) * LWP + ((k & (L - 1)) >> 5);
  }
  __device__ uint32_t xbit(int k) const { return (*xword(xS, k) >> (k & 31)) & 1u; }
  __device__ int4 ld4(int q) const {
    const int* __restrict__ p = dS + lane * LP + 4 * q;
    return *reinterpret_cast<const int4*>(p);
  }

  // (value, index) of the warp's minimum, lowest index on ties
  __device__ static void wmin(int& v, int& k) {
    const int m = __reduce_min_sync(FULL_S, v);
    k = __reduce_min_sync(FULL_S, v == m ? k : INT_MAX);
    v = m;
  }
  // running (value, index) minimum of this lane: a group's minimum replaces
  // it only when smaller, so the lowest index is kept
  __device__ void track(int gm, int q, int& mv, int& mq) const {
    if (gm < mv) { mv = gm; mq = q; }
  }
  __device__ int locate(int mv, int mq) const {  // index of value mv in group mq
    if (mv == INT_MAX) return INT_MAX;
    const int4 v = ld4(mq);
    const int e = v.x == mv ? 0 : v.y == mv ? 1 : v.z == mv ? 2 : 3;
    return base + 4 * mq + e;
  }

  // ---------------------------------------------------------------- scans
  // minimum over all stored values (= over the free bits)
  __device__ void scan_plain(int& fv, int& fk) const {
    int mv = INT_MAX, mq = 0;
#pragma unroll 8
    for (int q = 0; q < L / 4; ++q) track(min4(ld4(q)), q, mv, mq);
    fv = mv;
    fk = locate(mv, mq);
  }
  // Straight: also the minimum over the bits where X and D differ
  __device__ void scan_straight(int& fv, int& fk, int& sv, int& sk) const {
    int mv = INT_MAX, mq = 0, ms = INT_MAX, ks = INT_MAX;
    for (int w = 0; w < LW; ++w) {
      const uint32_t mw = xS[lane * LWP + w] ^ tS[lane * LWP + w];
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        const int q = 8 * w + qq;
        const int4 v = ld4(q);
        track(min4(v), q, mv, mq);
        const uint32_t nib = (mw >> (4 * qq)) & 0xFu;
        if (nib) {
          const int a = (nib & 1u) ? v.x : INT_MAX, b = (nib & 2u) ? v.y : INT_MAX;
          const int c = (nib & 4u) ? v.z : INT_MAX, d = (nib & 8u) ? v.w : INT_MAX;
          const int gm = min(__vimin3_s32(a, b, c), d);
          if (gm < ms) {
            ms = gm;
            ks = base + 4 * q + (a == gm ? 0 : b == gm ? 1 : c == gm ? 2 : 3);
          }
        }
      }
    }
    fv = mv;
    fk = locate(mv, mq);
    sv = ms;
    sk = ks;
  }
  // minimum over the bits of this lane in [lo, hi) (stored value, lowest index)
  __device__ void scan_range(int lo, int hi, int& rv, int& rk) const {
    rv = INT_MAX;
    rk = INT_MAX;
    const int a = max(lo, base), b = min(hi, base + L);
    if (a >= b) return;
    const int q0 = (a - base) >> 2, q1 = (b - 1 - base) >> 2;
    for (int q = q0; q <= q1; ++q) {
      const int4 v = ld4(q);
      const int k0 = base + 4 * q;
      int e4[4] = {v.x, v.y, v.z, v.w};
      if (q == q0 || q == q1) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (k0 + e < a || k0 + e >= b) e4[e] = INT_MAX;
      }
      const int gm = min(__vimin3_s32(e4[0], e4[1], e4[2]), e4[3]);
      if (gm < rv) {
        rv = gm;
        rk = k0 + (e4[0] == gm ? 0 : e4[1] == gm ? 1 : e4[2] == gm ? 2 : 3);
      }
    }
  }
  // RandomMin: also the minimum over the candidates (bit k's 16-bit uniform,
  // half k % 8 of block k / 8, below the threshold)
  __device__ void scan_random(uint32_t thr, int& fv, int& fk, int& cv, int& ck) const {
    int mv = INT_MAX, mq = 0, mc = INT_MAX, kc = INT_MAX;
    for (int b = 0; b < L / 8; ++b) {
      const uint4 u = draw(seed, flips, g, s, RNG_RANDMIN | (uint32_t)((base >> 3) + b));
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * b + qq;
        const int4 v = ld4(q);
        track(min4(v), q, mv, mq);
        const uint32_t w0 = qq == 0 ? u.x : u.z, w1 = qq == 0 ? u.y : u.w;
        const int a0 = (w0 & 0xFFFFu) < thr ? v.x : INT_MAX;
        const int a1 = (w0 >> 16) < thr ? v.y : INT_MAX;
        const int a2 = (w1 & 0xFFFFu) < thr ? v.z : INT_MAX;
        const int a3 = (w1 >> 16) < thr ? v.w : INT_MAX;
        const int gm = min(__vimin3_s32(a0, a1, a2), a3);
        if (gm < mc) {
          mc = gm;
          kc = base + 4 * q + (a0 == gm ? 0 : a1 == gm ? 1 : a2 == gm ? 2 : 3);
        }
      }
    }
    fv = mv;
    fk = locate(mv, mq);
    cv = mc;
    ck = kc;
  }
  // MaxMin: also the maximum over the free bits
  __device__ void scan_maxmin(int& fv, int& fk, int& mx) const {
    int mv = INT_MAX, mq = 0, xm = INT_MIN;
#pragma unroll 8
    for (int q = 0; q < L / 4; ++q) {
      const int4 v = ld4(q);
      track(min4(v), q, mv, mq);
      const int a = v.x < kFree ? v.x : INT_MIN, b = v.y < kFree ? v.y : INT_MIN;
      const int c = v.z < kFree ? v.z : INT_MIN, d = v.w < kFree ? v.w : INT_MIN;
      xm = max(xm, max(__vimax3_s32(a, b, c), d));
    }
    fv = mv;
    fk = locate(mv, mq);
    mx = xm;
  }
  // PositiveMin: also min over (unsigned)(Delta - 1): the smallest positive
  // Delta of a free bit, or >= kFree - 1 when there is none
  __device__ void scan_posmin(int& fv, int& fk, uint32_t& um) const {
    int mv = INT_MAX, mq = 0;
    uint32_t u = UINT_MAX;
#pragma unroll 8
    for (int q = 0; q < L / 4; ++q) {
      const int4 v = ld4(q);
      track(min4(v), q, mv, mq);
      u = min(u, min(min((uint32_t)(v.x - 1), (uint32_t)(v.y - 1)),
                     min((uint32_t)(v.z - 1), (uint32_t)(v.w - 1))));
    }
    fv = mv;
    fk = locate(mv, mq);
    um = u;
  }
  // the ((u * count) >> 32)-th free bit with stored value <= thr (thr < kFree),
  // ascending index: per-lane counts, a prefix over lanes, then the owning
  // lane walks its groups
  __device__ void kth(int thr, uint32_t u, int& kv, int& kk) const {
    int cnt = 0;
#pragma unroll 8
    for (int q = 0; q < L / 4; ++q) {
      const int4 v = ld4(q);
      cnt += (v.x <= thr) + (v.y <= thr) + (v.z <= thr) + (v.w <= thr);
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL_S, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULL_S, incl, 31);
    const int pick = (int)uniform_below(u, (uint32_t)total);
    const bool mine = pick >= incl - cnt && pick < incl;
    int rk = INT_MAX, rv = 0;
    if (mine) {
      int r = pick - (incl - cnt);
      for (int q = 0; q < L / 4; ++q) {
        const int4 v = ld4(q);
        const int c = (v.x <= thr) + (v.y <= thr) + (v.z <= thr) + (v.w <= thr);
        if (r < c) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int x = at4(v, e);
            if (x <= thr && rk == INT_MAX) {
              if (r == 0) { rk = base + 4 * q + e; rv = x; }
              --r;
            }
          }
          break;
        }
        r -= c;
      }
    }
    const unsigned bal = __ballot_sync(FULL_S, mine);
    const int src = bal ? __ffs(bal) - 1 : 0;
    kk = __shfl_sync(FULL_S, rk, src);
    kv = __shfl_sync(FULL_S, rv, src);
  }

  // ---------------------------------------------------------------- BEST
  __device__ void take_best(int j, int m) {
    for (int w = 0; w < LW; ++w) bS[lane * LWP + w] = xS[lane * LWP + w];
    __syncwarp();
    if (lane == 0) *xword(bS, j) ^= 1u << (j & 31);
    __syncwarp();
    Ebest = E + m;
  }

  // ---------------------------------------------------------------- row i
  // One bulk copy of row i of sigma(x_i) W (ld int16, 16-byte multiple) into rS.
  __device__ void row_fetch(int i, int xi) {
    const int16_t* row = (xi ? W : Wneg) + (size_t)i * ld;
    __syncwarp();
    if (stall) return;  // nothing arrives on the mbarrier: row_wait runs out
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads of rS before the copy
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                   "r"((uint32_t)ld * 2u)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              su32(rS)),
          "l"(row), "r"((uint32_t)ld * 2u), "r"(su32(bar))
          : "memory");
    }
  }
  // bounded wait for the current row; false (and the error flag) on timeout
  __device__ bool row_wait() {
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0;; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(su32(bar)), "r"(parity)
          : "memory");
      if (ok) break;
      if ((it & 63) == 63 && now_ns() - t0 > kWaitNs) {
        if (err && lane == 0) atomicExch(err, DABS_KERNEL_TIMEOUT);
        return false;
      }
    }
    parity ^= 1u;
    return true;
  }
  // Eq. (4) on this lane's block: Delta_k += W_ik sigma(x_i) sigma(x_k),
  // eight bits at a time, starting at group `lane` (bank spread)
  __device__ void row_apply() {
    const int16_t* __restrict__ rr = rS + base;
    int* __restrict__ dd = dS + lane * LP;
    const int* __restrict__ ss = sS + lane * LP;
    const int G = L / 8;
#pragma unroll 4
    for (int t = 0; t < G; ++t) {
      const int q2 = (t + lane) & (G - 1);  // G is a power of two
      if (base + 8 * q2 >= ld) continue;  // past the row: sigma is 0 there
      const uint4 w = *reinterpret_cast<const uint4*>(rr + 8 * q2);
      int4 d0 = *reinterpret_cast<const int4*>(dd + 8 * q2);
      int4 d1 = *reinterpret_cast<const int4*>(dd + 8 * q2 + 4);
      const int4 s0 = *reinterpret_cast<const int4*>(ss + 8 * q2);
      const int4 s1 = *reinterpret_cast<const int4*>(ss + 8 * q2 + 4);
      d0.x += sx_lo(w.x) * s0.x;
      d0.y += sx_hi(w.x) * s0.y;
      d0.z += sx_lo(w.y) * s0.z;
      d0.w += sx_hi(w.y) * s0.w;
      d1.x += sx_lo(w.z) * s1.x;
      d1.y += sx_hi(w.z) * s1.y;
      d1.z += sx_lo(w.w) * s1.z;
      d1.w += sx_hi(w.w) * s1.w;
      *reinterpret_cast<int4*>(dd + 8 * q2) = d0;
      *reinterpret_cast<int4*>(dd + 8 * q2 + 4) = d1;
    }
  }

  // ---------------------------------------------------------------- the batch search
  template <int ALGO>
  __device__ void run(int seed_mode, int T, int tau, uint32_t B) {
    int phase = seed_mode == 0 ? P_STRAIGHT : P_GREEDY;
    int runs = 0, it = 0, ws = 0;
    const int Tmain = ALGO == TWONEIGHBOR ? 2 * n - 1 : T;
    const bool use_tabu = ALGO != TWONEIGHBOR && tau > 0;
    const uint32_t Kq = (1u << 21) / (uint32_t)T, Kr = (1u << 21) % (uint32_t)T;
    uint32_t fup = 0, rup = 0, fdn = 1u << 21;
    int rdn = 0;
    uint32_t rnd0 = 0, rnd1 = 0;
    const int cwin = n < 32 ? n : 32;
    // RandomMin's floor c = 32/n in units of 2^-16, rounded up
    const uint32_t c16 = ((1u << 21) + (uint32_t)n - 1) / (uint32_t)n;
    for (;;) {
      int i, di, m, j;
      if (phase != P_MAIN) {
        // ---------------- Straight / Greedy (no tabu bits)
        const bool st = phase == P_STRAIGHT;
        int fv, fk, sv = INT_MAX, sk = INT_MAX;
        if (st) scan_straight(fv, fk, sv, sk);
        else scan_plain(fv, fk);
        wmin(fv, fk);
        if (st) {
          wmin(sv, sk);
          if (sv == INT_MAX) {  // X == D: Straight ends
            phase = P_GREEDY;
            continue;
          }
        }
        m = fv;
        j = fk;
        if (E + m < Ebest) take_best(j, m);
        if (!st && m >= 0) {  // local minimum: Greedy ends after Step 1
          if (flips < B && !(ALGO == TWONEIGHBOR && runs >= 1)) {
            phase = P_MAIN;
            it = 0;
            ws = 0;
            fup = 0;
            rup = 0;
            fdn = 1u << 21;
            rdn = 0;
            ring_len = 0;
            ring_head = 0;
            continue;
          }
          break;
        }
        i = st ? sk : fk;
        di = st ? sv : fv;
      } else {
        // ---------------- main search iteration t = it + 1
        fup += Kq;
        rup += Kr;
        if (rup >= (uint32_t)T) { ++fup; rup -= (uint32_t)T; }
        fdn -= Kq;
        rdn -= (int)Kr;
        if (rdn < 0) { --fdn; rdn += T; }
        int fv, fk;  // minimum over the free bits
        if (ALGO == TWONEIGHBOR) {
          scan_plain(fv, fk);
          i = it == 0 ? 0 : ((it & 1) ? (it + 1) >> 1 : (it >> 1) - 1);
          di = *dptr(i);  // no tabu bits in TwoNeighbor
        } else if (ALGO == MAXMIN || ALGO == POSITIVEMIN) {
          if ((it & 31) == 0) {
            const uint4 u = draw(seed, flips + (uint32_t)lane, g, s,
                                 ALGO == MAXMIN ? RNG_MAXMIN : RNG_POSMIN);
            rnd0 = u.x;
            rnd1 = u.y;
          }
          const uint32_t u0 = __shfl_sync(FULL_S, rnd0, it & 31);
          int thr;
          uint32_t uk;
          if (ALGO == MAXMIN) {
            int mx;
            scan_maxmin(fv, fk, mx);
            mx = __reduce_max_sync(FULL_S, mx);
            const int mn = __reduce_min_sync(FULL_S, fv);
            const uint64_t q = cube21f(fdn);
            const uint64_t span = (uint64_t)((int64_t)mx - (int64_t)mn);
            const uint64_t R = (q * span) >> 32;
            thr = (int)((int64_t)mn + (int64_t)(((uint64_t)u0 * (R + 1)) >> 32));
            uk = __shfl_sync(FULL_S, rnd1, it & 31);
          } else {
            uint32_t um;
            scan_posmin(fv, fk, um);
            um = __reduce_min_sync(FULL_S, um);
            thr = um < (uint32_t)(kFree - 1) ? (int)um + 1 : kFree - 1;
            uk = u0;
          }
          kth(thr, uk, di, i);
        } else if (ALGO == CYCLICMIN) {
          scan_plain(fv, fk);
          const uint64_t wl = (cube21f(fup) * (uint64_t)n) >> 32;
          const int wsz = (int)(wl < (uint64_t)cwin ? (uint64_t)cwin : (wl > (uint64_t)n ? (uint64_t)n : wl));
          int v1, k1, v2, k2;
          scan_range(ws, min(ws + wsz, n), v1, k1);
          scan_range(0, ws + wsz - n, v2, k2);
          wmin(v1, k1);
          wmin(v2, k2);
          // first in cyclic order from ws: [ws, n) before [0, ws + wsz - n)
          const bool one = v2 == INT_MAX || (v1 != INT_MAX && v1 <= v2);
          i = one ? k1 : k2;
          di = one ? v1 : v2;
          ws += wsz;
          if (ws >= n) ws -= n;
        } else {  // RANDOMMIN
          uint32_t thr = (uint32_t)(cube21f(fup) >> 16);
          thr = thr < c16 ? c16 : (thr > 65536u ? 65536u : thr);
          int cv, ck;
          scan_random(thr, fv, fk, cv, ck);
          wmin(cv, ck);
          if (cv >= kFree) {  // no free candidate: arg-min over the free bits (rare)
            int gv = fv, gk = fk;
            wmin(gv, gk);
            cv = gv;
            ck = gk;
          }
          i = ck;
          di = cv;
        }
        // Step 1 over all n bits: the free minimum and the tabu ring
        if (lane < ring_len) {
          const int rv = *dptr(ringv) - kPen;
          if (rv < fv || (rv == fv && ringv < fk)) { fv = rv; fk = ringv; }
        }
        wmin(fv, fk);
        m = fv;
        j = fk;
        if (E + m < Ebest) take_best(j, m);
      }
      i = min(max(i, 0), n - 1);
      const int xi = (int)xbit(i);
      row_fetch(i, xi);
      // tabu: i enters; when the ring is full its oldest entry leaves
      int leave = -1;
      if (phase == P_MAIN && use_tabu) {
        if (ring_len == tau) leave = __shfl_sync(FULL_S, ringv, ring_head);
        else ++ring_len;
        if (lane == ring_head) ringv = i;
        ring_head = ring_head + 1 == tau ? 0 : ring_head + 1;
      }
      if (!row_wait()) {
        failed = true;
        return;
      }
      row_apply();
      __syncwarp();
      if (lane == 0) {
        *dptr(i) = -di + (phase == P_MAIN && use_tabu ? kPen : 0);  // Eq. (5)
        *sptr(i) = -*sptr(i);
        *xword(xS, i) ^= 1u << (i & 31);
        if (leave >= 0) *dptr(leave) -= kPen;
      }
      __syncwarp();
      E += di;
      ++flips;
      if (phase == P_MAIN && ++it == Tmain) {  // main run ends: its tabu bits are released
        if (use_tabu && lane < ring_len) *dptr(ringv) -= kPen;
        __syncwarp();
        ring_len = 0;
        ring_head = 0;
        phase = P_GREEDY;
        ++runs;
      }
    }
  }
};

}  // namespace

// Shared memory of one search (16-byte aligned sections, see the file comment).
__host__ __device__ inline void smem_search_layout(int n, int* LW, uint32_t* off_d, uint32_t* off_s,
                                                   uint32_t* off_r, uint32_t* off_x, uint32_t* bytes) {
  int lw = 1;
  while (1024 * lw < n) lw <<= 1;
  const int L = 32 * lw, LP = L + 4;
  const int LWP = lw | 1;
  const uint32_t bits = (uint32_t)(((32 * LWP * 4) + 15) / 16 * 16);
  uint32_t o = 16;  // mbarrier
  *off_d = o;
  o += 32u * LP * 4u;
  *off_s = o;
  o += 32u * LP * 4u;
  *off_r = o;
  o += 32u * L * 2u;
  *off_x = o;
  o += 3u * bits;
  *LW = lw;
  *bytes = o;
}

size_t smem_search_bytes(int n) {
  int lw;
  uint32_t a, b, c, d, bytes;
  smem_search_layout(n, &lw, &a, &b, &c, &d, &bytes);
  return bytes;
}

__global__ void __launch_bounds__(32) k_batch_search_smem(const SearchArgs single, const MultiArgs multi) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x;
  const uint32_t slot = blockIdx.x;
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
  const uint32_t s = a.order ? (uint32_t)a.order[local] : local;
  const DevCtrl* ctrl = a.ctrl;
  if (ctrl->done) return;

  SmemSearch sr;
  uint32_t off_d, off_s, off_r, off_x, bytes;
  smem_search_layout(a.n, &sr.LW, &off_d, &off_s, &off_r, &off_x, &bytes);
  sr.n = a.n;
  sr.ld = a.ld;
  sr.L = 32 * sr.LW;
  sr.lsh = 31 - __clz(sr.L);
  sr.LP = sr.L + 4;
  sr.LWP = sr.LW | 1;
  sr.lane = lane;
  sr.base = lane * sr.L;
  sr.bar = reinterpret_cast<uint64_t*>(sm);
  sr.dS = reinterpret_cast<int*>(sm + off_d);
  sr.sS = reinterpret_cast<int*>(sm + off_s);
  sr.rS = reinterpret_cast<int16_t*>(sm + off_r);
  const uint32_t bits = (uint32_t)(((32 * sr.LWP * 4) + 15) / 16 * 16);
  sr.xS = reinterpret_cast<uint32_t*>(sm + off_x);
  sr.tS = reinterpret_cast<uint32_t*>(sm + off_x + bits);
  sr.bS = reinterpret_cast<uint32_t*>(sm + off_x + 2 * bits);
  sr.parity = 0;
  sr.W = a.W;
  sr.Wneg = a.Wneg;
  sr.seed = ctrl->seed;
  sr.s = s;
  sr.g = ctrl->g;
  sr.err = a.serr;
  sr.failed = false;
  sr.stall = a.stall_test != 0;
  sr.ring_len = 0;
  sr.ring_head = 0;
  sr.ringv = 0;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(sr.bar)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // load: bits of this lane's words, Delta and sigma of its block
  const int nw = a.nw;
  for (int w = 0; w < sr.LW; ++w) {
    const int gw = lane * sr.LW + w;
    sr.xS[lane * sr.LWP + w] = gw < nw ? a.X[(size_t)s * nw + gw] : 0u;
    sr.tS[lane * sr.LWP + w] = gw < nw ? a.D[(size_t)s * nw + gw] : 0u;
    sr.bS[lane * sr.LWP + w] = 0u;
  }
  const int32_t* dl = a.delta + (size_t)s * a.ld;
  for (int e = 0; e < sr.L; ++e) {
    const int k = sr.base + e;
    const bool valid = k < a.n;
    const uint32_t xb = (sr.xS[lane * sr.LWP + e / 32] >> (e % 32)) & 1u;
    sr.dS[lane * sr.LP + e] = valid ? dl[k] : kSent;
    sr.sS[lane * sr.LP + e] = valid ? (xb ? 1 : -1) : 0;
  }
  sr.E = a.E2 ? a.E2[s] / 2 : a.E[s];
  sr.Ebest = INT64_MAX;
  sr.flips = 0;
  __syncwarp();
  switch (a.algo[s]) {
    case MAXMIN: sr.run<MAXMIN>(a.seed_mode, a.T, a.tau, a.B); break;
    case CYCLICMIN: sr.run<CYCLICMIN>(a.seed_mode, a.T, a.tau, a.B); break;
    case RANDOMMIN: sr.run<RANDOMMIN>(a.seed_mode, a.T, a.tau, a.B); break;
    case POSITIVEMIN: sr.run<POSITIVEMIN>(a.seed_mode, a.T, a.tau, a.B); break;
    default: sr.run<TWONEIGHBOR>(a.seed_mode, a.T, a.tau, a.B); break;
  }
  if (sr.failed) {
    sr.row_wait();  // give a copy still in flight (bounded) time to land
    return;
  }
  __syncwarp();
  // store
  int32_t* dw = a.delta + (size_t)s * a.ld;
  for (int e = 0; e < sr.L; ++e) {
    const int k = sr.base + e;
    if (k < a.ld) dw[k] = k < a.n ? sr.dS[lane * sr.LP + e] : 0;
  }
  for (int w = 0; w < sr.LW; ++w) {
    const int gw = lane * sr.LW + w;
    if (gw < nw) {
      a.X[(size_t)s * nw + gw] = sr.xS[lane * sr.LWP + w];
      a.best_X[(size_t)s * nw + gw] = sr.bS[lane * sr.LWP + w];
    }
  }
  if (lane == 0) {
    a.E[s] = sr.E;
    a.best_E[s] = sr.Ebest;
    a.flips[s] = sr.flips;
  }
}

bool launch_search_smem(const SearchArgs* a, cudaStream_t st, SearchVariant* v, const MultiArgs* m) {
  if (v) *v = SearchVariant{1, 0, DABS_N_MAX, 32, 1};
  if (!a) return true;
  const int slots = m ? m->total : a->S;
  if (slots <= 0) return true;
  const size_t bytes = smem_search_bytes(m ? m->max_n : a->n);
  cudaFuncSetAttribute(k_batch_search_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_batch_search_smem<<<(unsigned)slots, 32, bytes, st>>>(*a, m ? *m : MultiArgs{nullptr, nullptr, 0, 0, 0});
  return true;
}

}  // namespace dabs
