/*
 * dabs_oracle.c -- plain CPU oracle of the DABS hot path (test infrastructure
 * only; see dabs_oracle.h).  Written from the paper's text: Section III-A
 * (incremental search, Eqs. (3)-(5), Steps 1-4, the search algorithms and
 * tabu), Section III-B (batch search and flip factors), Section III-C
 * (packets), Section IV (genetic operations, solution pools, island model).
 *
 * Readings fixed here where the paper is silent, garbled or real-valued
 * (the CUDA library implements the same readings independently):
 *  R1  Energy (Eq. (2), index set garbled): E = sum_i W_ii x_i +
 *      sum_{i<j} W_ij x_i x_j with W symmetric -- each pair once, the form
 *      Eqs. (3)-(5) are derived from.
 *  R2  Step 1: minE over all n one-bit neighbours, lowest index on ties;
 *      BEST is replaced only on strict improvement.  E(BEST) starts at
 *      INT64_MAX at the start of every batch search, so BEST only ever holds
 *      one-bit neighbours examined in Step 1.
 *  R3  Greedy: Step 1, then stop (without flipping) if min Delta >= 0,
 *      otherwise flip the argmin (lowest index on ties).
 *  R4  Straight: stop when X == D; otherwise Step 1, then flip the argmin of
 *      Delta over {k : x_k != d_k} (lowest index on ties).
 *  R5  Iteration-dependent ratios use one integer helper,
 *      cube21(a, T) = (floor(a * 2^21 / T))^3 >> 31, i.e. (a/T)^3 in units
 *      of 2^-32 with a 21-bit ratio.
 *  R6  MaxMin: min/max of Delta over non-tabu bits; R = (cube21(T-t, T) *
 *      (max-min)) >> 32; threshold d = min + ((u0 * (R+1)) >> 32); the
 *      candidates are the non-tabu bits with Delta <= d; the pick is the
 *      ((u1 * count) >> 32)-th candidate in ascending index order.
 *  R7  CyclicMin: c = min(32, n); window width w_t = clamp((cube21(t,T) * n)
 *      >> 32, c, n) for t = 1..T; the first window starts at bit 0 of each
 *      CyclicMin run and each next one starts where the last one ended
 *      (cyclically); argmin over non-tabu bits of the window, ties to the
 *      first bit in cyclic order from the window start.
 *  R8  RandomMin: p(t) = max((t/T)^3, c) with c = 32/n is held in units of
 *      2^-16: thr = clamp(cube21(t,T) >> 16, ceil(2^21 / n), 65536), so the
 *      floor ceil(32 * 2^16 / n) / 2^16 is c rounded up to the next 2^-16 for
 *      every n (exactly c when n divides 2^21) and p = 1 when n <= 32; bit k
 *      is a candidate iff its 16-bit uniform < thr; argmin of Delta over
 *      non-tabu candidates (lowest index on ties); if there is no candidate,
 *      argmin over all non-tabu bits.
 *  R9  PositiveMin: posmin = min Delta > 0 over non-tabu bits; candidates are
 *      non-tabu bits with Delta <= posmin (all non-tabu bits if no positive
 *      Delta exists); the pick is the ((u0 * count) >> 32)-th candidate.
 *  R10 TwoNeighbor: flips 0, then k, k-1 for k = 1..n-1 (2n-1 flips); no tabu;
 *      at most once per batch search, which ends after the following Greedy.
 *  R11 Tabu: period tau = min(tabu, n-1); a bit flipped at main-search
 *      iteration t is excluded at iterations t+1..t+tau of the same run; the
 *      list starts empty at each main run; Straight, Greedy and TwoNeighbor
 *      neither use nor fill it.  With tabu <= 31 every candidate set above is
 *      non-empty.
 *  R12 T = max(1, floor(n * s)) flips per main search (except TwoNeighbor);
 *      the batch search ends at the first check with total >= B, with
 *      B = ceil(n * b); the check runs after every Greedy.
 *  R13 Seeding: mode 0 walks X to D with Straight (the paper); mode 1 sets
 *      X = D and recomputes Delta and E from scratch (no flips, no Step 1).
 *  R14 Parent selection: rank = (t * m) >> 64 with t = (u^3) >> 32 for a
 *      32-bit uniform u (the floor(r^3 m) of Section IV-A); the pool is kept
 *      sorted ascending by energy, older entries first on ties.
 *  R15 Operation and algorithm choice: with u0 < floor(0.05 * 2^32) pick
 *      uniformly ((u1 * 8) >> 32, resp. (u3 * 5) >> 32), otherwise copy the
 *      field of pool row (u1 * C) >> 32 (resp. (u3 * C) >> 32).
 *  R16 Per-bit draws: each 32-bit word of X gets one Philox block, i.e. a
 *      4-bit nibble per bit.  Mutation/Zero/One touch a bit iff the low three
 *      bits of its nibble are zero (probability 1/8, also for One);
 *      Crossover/Xrossover take parent B iff bit 0 of the nibble is set;
 *      Random uses that bit as the value.
 *  R17 IntervalZero: len = lo + ((u2 * (hi-lo+1)) >> 32), hi = floor(n/2),
 *      lo = min(32, hi); start = (u3 * n) >> 32; the segment wraps around.
 *  R18 Islands: search s belongs to pool s mod P; Xrossover takes parent B
 *      from pool (p+1) mod P.
 *  R19 Generations are synchronous: all targets of generation g are bred from
 *      the pools as they stood after generation g-1; results are merged in
 *      search order.  A result enters its pool iff E < E(worst) and no entry
 *      holds the same (E, X); it is placed after entries of equal energy and
 *      the worst entry is dropped.  Pools start with random vectors,
 *      E = INT64_MAX and random algorithm/operation fields.
 *  R20 Global best: first result (generation, then search order) with the
 *      lowest energy.  A solve stops at the first generation boundary with
 *      total flips >= budget, best E <= target or generations == limit.
 *  R22 Statistics (Tables V and VI): per generation, every search counts its
 *      main algorithm and genetic operation; a generation whose best result
 *      improves the global best credits that result's algorithm and operation
 *      (the first finder).
 *  R21 Random numbers: Philox4x32-10 keyed by (seed lo, seed hi) with counter
 *      (x, y, z, w):
 *        MaxMin      (flip, g, s, 1<<24)         u0 threshold, u1 pick
 *        PositiveMin (flip, g, s, 2<<24)         u0 pick
 *        RandomMin   (flip, g, s, 3<<24 | k/8)   16-bit half (k%8) of the block
 *        choice      (0, g, s, 4<<24)            u0..u3 of R15
 *        parents     (0, g, s, 5<<24)            u0 rank A, u1 rank B, u2/u3 R17
 *        bits        (word, g, s, 6<<24)         R16
 *        pool init   (word, entry, pool, 7<<24 | r)  bit 0 of each nibble
 *        pool tags   (0, entry, pool, 8<<24 | r)     algo (u0*5)>>32, op (u1*8)>>32
 *      where flip is the number of flips already made in the batch search and
 *      r the number of restarts so far (R23).
 *  R23 Restart (Section IV-B, last paragraph): "all pools merged" is read as
 *      every entry of every pool lying within Hamming distance h (a parameter)
 *      of the global best.  Tested after each generation's merge and global
 *      best update (when restarts are enabled); if it holds, r += 1, every pool
 *      is drawn afresh as at the start with epoch r, and every search restarts
 *      from X = 0, E = 0, Delta = diag.  The global best, the flip count, the
 *      generation index and the statistics carry on.
 *  R24 ABS mode (Section I, the earlier Adaptive Bulk Search): every search
 *      runs CyclicMin and every target is a mutation after a crossover of
 *      two parents of its own pool (ranks as R14).  Per bit, with the bits
 *      draw of R16: coin = bit 3 of the nibble picks parent B, then the bit
 *      is inverted iff its low three bits are 0.  The result is recorded as
 *      a Crossover for R22.
 */
#include "dabs_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define MIX_THRESHOLD 214748364u /* floor(0.05 * 2^32) */

/* ------------------------------------------------------------------------ */
/* Eq. (2): energy as a plain double loop, each pair (i<j) once (R1).       */
int64_t orc_energy(const int16_t* W, int32_t n, const uint8_t* X) {
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (!X[i]) continue;
        e += W[(int64_t)i * n + i];
        for (int32_t j = i + 1; j < n; ++j)
            if (X[j]) e += W[(int64_t)i * n + j];
    }
    return e;
}

/* Eq. (3): Delta_k = -sigma(x_k) * sum_j W_jk x_j + W_kk * (1 - x_k). */
void orc_delta(const int16_t* W, int32_t n, const uint8_t* X, int32_t* delta) {
    for (int32_t k = 0; k < n; ++k) {
        int64_t sum = 0;
        for (int32_t j = 0; j < n; ++j)
            if (X[j]) sum += W[(int64_t)j * n + k];
        int64_t sigma = 2 * (int64_t)X[k] - 1;
        delta[k] = (int32_t)(-sigma * sum + (int64_t)W[(int64_t)k * n + k] * (1 - X[k]));
    }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications, the key bumped by the Weyl constants between
 * rounds.                                                                   */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t out[4]) {
    uint32_t ctr[4] = {x, y, z, w};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* uniform integer in [0, m) by multiply-shift */
static uint32_t uidx(uint32_t u, uint32_t m) { return (uint32_t)(((uint64_t)u * m) >> 32); }

/* Section IV-A: the (floor(r^3 m)+1)-th packet, r in [0,1) (R14). */
uint32_t orc_parent_rank(uint32_t u, uint32_t m) {
    unsigned __int128 cube = (unsigned __int128)((uint64_t)u * u) * u;
    uint64_t t = (uint64_t)(cube >> 32);
    return (uint32_t)(((unsigned __int128)t * m) >> 64);
}

/* (a/T)^3 in units of 2^-32 (R5); a <= T. */
uint64_t orc_cube21(uint64_t a, uint64_t T) {
    uint64_t f = (a << 21) / T;
    return (f * f * f) >> 31;
}

/* R8: RandomMin's candidate probability p(t) = max((t/T)^3, 32/n) in units of
 * 2^-16 (Section III-A, RandomMin).                                         */
uint32_t orc_randmin_threshold(uint64_t t, uint64_t T, int32_t n) {
    uint64_t thr = orc_cube21(t, T) >> 16;
    uint64_t floor_c = ((1ull << 21) + (uint64_t)n - 1) / (uint64_t)n; /* ceil(32 * 2^16 / n) */
    if (thr < floor_c) thr = floor_c;
    if (thr > 65536) thr = 65536;
    return (uint32_t)thr;
}

/* R8/R21: the 16-bit uniform of every bit k < n for the RandomMin iteration
 * made as flip `flip` of search s in generation g.                          */
void orc_randmin_draws(uint64_t seed, uint32_t flip, uint32_t g, uint32_t s, int32_t n,
                       uint16_t* u16) {
    uint32_t u[4];
    for (int32_t k = 0; k < n; ++k) {
        if ((k & 7) == 0) draw(seed, flip, g, s, (3u << 24) | (uint32_t)(k >> 3), u);
        u16[k] = (uint16_t)(u[(k & 7) >> 1] >> (16 * (k & 1)));
    }
}

/* R6: MaxMin's threshold d, drawn uniformly from [mn, D(t)] with
 * D(t) = mn + ((T-t)/T)^3 (mx - mn) (Section III-A, MaxMin); *R_out gets
 * the width floor(((T-t)/T)^3 (mx - mn)) of the interval.                   */
int64_t orc_maxmin_threshold(int32_t mn, int32_t mx, uint64_t t, uint64_t T, uint32_t u0,
                             uint64_t* R_out) {
    uint64_t q = orc_cube21(T - t, T);
    uint64_t span = (uint64_t)((int64_t)mx - (int64_t)mn);
    uint64_t R = (q * span) >> 32;
    if (R_out) *R_out = R;
    return (int64_t)mn + (int64_t)(((uint64_t)u0 * (R + 1)) >> 32);
}

/* Section III-B: another (main search, Greedy) round is run while fewer than
 * B = b*n flips were made; TwoNeighbor runs at most once (R10, R12).        */
int orc_batch_continue(uint64_t total, uint64_t B, int32_t main_runs, int32_t algo) {
    if (total >= B) return 0;
    if (algo == ORC_TWONEIGHBOR && main_runs >= 1) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* One incremental search (Section III-A) acting on persistent state.        */
typedef struct {
    const int16_t* W;
    int32_t n;
    uint64_t seed;
    uint32_t g, s;
    uint8_t* X;
    int32_t* delta;
    int64_t* E;
    uint8_t* best_X;
    int64_t best_E;
    uint64_t flips;
    int32_t phase;
    int32_t* trace_idx;
    int32_t* trace_phase;
    int64_t trace_cap;
    int32_t check;
    int32_t bad;
    int32_t* last; /* tabu: iteration of the last flip in the current main run */
    int32_t* scratch;
    orc_sel_trace* sel; /* optional per-flip record of the selectors' quantities */
} search_run;

/* Step 1: examine every one-bit neighbour, keep the best in BEST (R2).
 * Returns min Delta and its lowest index in *j.                             */
static int32_t step1(search_run* b, int32_t* j_out) {
    int32_t j = 0, m = b->delta[0];
    for (int32_t i = 1; i < b->n; ++i)
        if (b->delta[i] < m) { m = b->delta[i]; j = i; }
    int64_t cand = *b->E + m;
    if (cand < b->best_E) {
        memcpy(b->best_X, b->X, (size_t)b->n);
        b->best_X[j] ^= 1;
        b->best_E = cand;
    }
    *j_out = j;
    return m;
}

/* Step 3: X <- f_i(X), E <- E + Delta_i, Delta by Eqs. (4) and (5). */
static void flip(search_run* b, int32_t i) {
    const int32_t n = b->n;
    const int16_t* Wi = b->W + (int64_t)i * n;
    int32_t di = b->delta[i];
    *b->E += di;
    int32_t si = 2 * b->X[i] - 1;
    for (int32_t k = 0; k < n; ++k) {
        if (k == i) continue;
        int32_t sk = 2 * b->X[k] - 1;
        b->delta[k] += Wi[k] * si * sk; /* Eq. (4), pre-flip x_i and x_k */
    }
    b->delta[i] = -di; /* Eq. (5) */
    b->X[i] ^= 1;
    if (b->trace_idx && (int64_t)b->flips < b->trace_cap) {
        b->trace_idx[b->flips] = i;
        if (b->trace_phase) b->trace_phase[b->flips] = b->phase;
    }
    b->flips += 1;
    if (b->check && !b->bad) {
        orc_delta(b->W, n, b->X, b->scratch);
        if (orc_energy(b->W, n, b->X) != *b->E) b->bad = 1;
        for (int32_t k = 0; k < n; ++k)
            if (b->scratch[k] != b->delta[k]) b->bad = 1;
    }
}

static void greedy(search_run* b) {
    b->phase = ORC_PH_GREEDY;
    for (;;) {
        int32_t j;
        int32_t m = step1(b, &j);
        if (m >= 0) break; /* local minimum: Delta_k >= 0 for all k */
        flip(b, j);
    }
}

static void straight(search_run* b, const uint8_t* D) {
    b->phase = ORC_PH_STRAIGHT;
    for (;;) {
        int32_t i = -1;
        for (int32_t k = 0; k < b->n; ++k)
            if (b->X[k] != D[k] && (i < 0 || b->delta[k] < b->delta[i])) i = k;
        if (i < 0) break; /* X == D */
        int32_t j;
        step1(b, &j);
        flip(b, i);
    }
}

/* selector record of the iteration about to flip (test instrumentation) */
static void sel_record(search_run* b, int64_t a, int64_t r, uint32_t count) {
    if (!b->sel || (int64_t)b->flips >= b->sel->cap) return;
    b->sel->a[b->flips] = a;
    b->sel->r[b->flips] = r;
    b->sel->count[b->flips] = (int32_t)count;
}

static int is_tabu(const search_run* b, int32_t k, int32_t t, int32_t tau) {
    return b->last[k] > 0 && t - b->last[k] <= tau;
}

/* k-th (0-based) bit of the candidate mask in ascending index order */
static int32_t kth_candidate(const uint8_t* cand, int32_t n, uint32_t k) {
    for (int32_t i = 0; i < n; ++i)
        if (cand[i]) {
            if (k == 0) return i;
            --k;
        }
    return -1;
}

static void main_search(search_run* b, int32_t algo, int32_t T, int32_t tau) {
    const int32_t n = b->n;
    b->phase = ORC_PH_MAIN;
    int32_t j;
    if (algo == ORC_TWONEIGHBOR) {
        for (int32_t q = 0; q < 2 * n - 1; ++q) {
            int32_t i = (q == 0) ? 0 : ((q & 1) ? (q + 1) / 2 : q / 2 - 1);
            step1(b, &j);
            flip(b, i);
        }
        return;
    }
    for (int32_t k = 0; k < n; ++k) b->last[k] = 0;
    uint8_t* cand = (uint8_t*)malloc((size_t)n);
    uint16_t* u16 = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)n);
    int32_t win_start = 0;
    const int32_t c_win = n < 32 ? n : 32;
    for (int32_t t = 1; t <= T; ++t) {
        if (b->sel && (int64_t)b->flips < b->sel->cap) {
            int32_t nf = 0;
            for (int32_t k = 0; k < n; ++k) nf += !is_tabu(b, k, t, tau);
            b->sel->free[b->flips] = nf;
        }
        step1(b, &j);
        int32_t i = -1;
        uint32_t u[4];
        if (algo == ORC_MAXMIN) {
            int32_t mn = 0, mx = 0, any = 0;
            for (int32_t k = 0; k < n; ++k) {
                if (is_tabu(b, k, t, tau)) continue;
                if (!any || b->delta[k] < mn) mn = b->delta[k];
                if (!any || b->delta[k] > mx) mx = b->delta[k];
                any = 1;
            }
            draw(b->seed, (uint32_t)b->flips, b->g, b->s, 1u << 24, u);
            uint64_t R;
            int64_t d = orc_maxmin_threshold(mn, mx, (uint64_t)t, (uint64_t)T, u[0], &R);
            uint32_t count = 0;
            for (int32_t k = 0; k < n; ++k) {
                cand[k] = !is_tabu(b, k, t, tau) && (int64_t)b->delta[k] <= d;
                count += cand[k];
            }
            i = kth_candidate(cand, n, uidx(u[1], count));
            sel_record(b, d, (int64_t)R, count);
        } else if (algo == ORC_CYCLICMIN) {
            uint64_t w = (orc_cube21((uint64_t)t, (uint64_t)T) * (uint64_t)n) >> 32;
            if (w < (uint64_t)c_win) w = (uint64_t)c_win;
            if (w > (uint64_t)n) w = (uint64_t)n;
            for (int32_t r = 0; r < (int32_t)w; ++r) {
                int32_t k = (win_start + r) % n;
                if (is_tabu(b, k, t, tau)) continue;
                if (i < 0 || b->delta[k] < b->delta[i]) i = k;
            }
            win_start = (int32_t)((win_start + (int64_t)w) % n);
            sel_record(b, (int64_t)w, 0, 0);
        } else if (algo == ORC_RANDOMMIN) {
            uint32_t thr = orc_randmin_threshold((uint64_t)t, (uint64_t)T, n);
            orc_randmin_draws(b->seed, (uint32_t)b->flips, b->g, b->s, n, u16);
            uint32_t count = 0;
            for (int32_t k = 0; k < n; ++k) {
                if (is_tabu(b, k, t, tau) || u16[k] >= thr) continue;
                ++count;
                if (i < 0 || b->delta[k] < b->delta[i]) i = k;
            }
            if (i < 0)
                for (int32_t k = 0; k < n; ++k)
                    if (!is_tabu(b, k, t, tau) && (i < 0 || b->delta[k] < b->delta[i])) i = k;
            sel_record(b, thr, 0, count);
        } else { /* ORC_POSITIVEMIN */
            int32_t pm = 0, anypos = 0;
            for (int32_t k = 0; k < n; ++k)
                if (!is_tabu(b, k, t, tau) && b->delta[k] > 0 && (!anypos || b->delta[k] < pm)) {
                    pm = b->delta[k];
                    anypos = 1;
                }
            uint32_t count = 0;
            for (int32_t k = 0; k < n; ++k) {
                cand[k] = !is_tabu(b, k, t, tau) && (!anypos || b->delta[k] <= pm);
                count += cand[k];
            }
            draw(b->seed, (uint32_t)b->flips, b->g, b->s, 2u << 24, u);
            i = kth_candidate(cand, n, uidx(u[0], count));
            sel_record(b, anypos ? pm : INT64_MAX, 0, count);
        }
        flip(b, i);
        b->last[i] = t;
    }
    free(cand);
    free(u16);
}

static uint64_t main_flips(const orc_params* p, int32_t n) {
    uint64_t T = ((uint64_t)n * (uint64_t)p->s_num) / (uint64_t)p->s_den;
    return T < 1 ? 1 : T;
}
static uint64_t batch_flips(const orc_params* p, int32_t n) {
    return ((uint64_t)n * (uint64_t)p->b_num + (uint64_t)p->b_den - 1) / (uint64_t)p->b_den;
}

int orc_batch_search(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed, uint32_t g,
                     uint32_t s, uint8_t* X, int32_t* delta, int64_t* E, const uint8_t* D,
                     int32_t algo, uint8_t* best_X, int64_t* best_E, uint64_t* flips,
                     int32_t* trace_idx, int32_t* trace_phase, int64_t trace_cap, int32_t check) {
    return orc_batch_search_sel(W, n, p, seed, g, s, X, delta, E, D, algo, best_X, best_E, flips,
                                trace_idx, trace_phase, trace_cap, check, NULL);
}

int orc_batch_search_sel(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed,
                         uint32_t g, uint32_t s, uint8_t* X, int32_t* delta, int64_t* E,
                         const uint8_t* D, int32_t algo, uint8_t* best_X, int64_t* best_E,
                         uint64_t* flips, int32_t* trace_idx, int32_t* trace_phase,
                         int64_t trace_cap, int32_t check, orc_sel_trace* sel) {
    search_run b;
    memset(&b, 0, sizeof b);
    b.sel = sel;
    b.W = W; b.n = n; b.seed = seed; b.g = g; b.s = s;
    b.X = X; b.delta = delta; b.E = E; b.best_X = best_X; b.best_E = INT64_MAX;
    b.trace_idx = trace_idx; b.trace_phase = trace_phase; b.trace_cap = trace_cap;
    b.check = check;
    b.last = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    b.scratch = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    memset(best_X, 0, (size_t)n);
    const int32_t T = (int32_t)main_flips(p, n);
    const int32_t tau = p->tabu < n - 1 ? p->tabu : n - 1;
    const uint64_t B = batch_flips(p, n);

    if (p->seed_mode == 0) {
        straight(&b, D);
    } else {
        memcpy(X, D, (size_t)n);
        orc_delta(W, n, X, delta);
        *E = orc_energy(W, n, X);
    }
    greedy(&b);
    int32_t runs = 0;
    while (orc_batch_continue(b.flips, B, runs, algo)) {
        main_search(&b, algo, T, tau);
        ++runs;
        greedy(&b);
    }
    *best_E = b.best_E;
    *flips = b.flips;
    free(b.last);
    free(b.scratch);
    return b.bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Solver: solution pools (Section IV) and per-search persistent state.     */
struct orc_solver {
    const int16_t* W;
    int16_t* W_own;
    int32_t n;
    orc_params p;
    uint64_t seed;
    int32_t S, P, C;
    uint8_t* pool_X; /* [P][C][n] */
    int64_t* pool_E; /* [P][C]    */
    int32_t* pool_algo;
    int32_t* pool_op;
    uint8_t* X;      /* [S][n] */
    int32_t* delta;  /* [S][n] */
    int64_t* E;      /* [S]    */
    uint8_t* D;      /* [S][n] */
    int32_t* algo;
    int32_t* op;
    uint8_t* res_X;
    int64_t* res_E;
    uint64_t* res_flips;
    uint8_t* gbest_X;
    int64_t gbest_E;
    uint64_t flips_total;
    uint32_t g;
    uint64_t algo_count[ORC_N_ALGOS], op_count[ORC_N_OPS];
    uint64_t best_algo[ORC_N_ALGOS], best_op[ORC_N_OPS];
    uint32_t restarts;
};

static int nibble(const uint32_t u[4], int32_t j) { return (int)((u[j >> 3] >> (4 * (j & 7))) & 0xFu); }

/* Section III-B: every search starts at X = 0, E = 0, Delta_k = W_kk. */
static void reset_searches(orc_solver* so) {
    const size_t S = (size_t)so->S, N = (size_t)so->n;
    memset(so->X, 0, S * N);
    memset(so->E, 0, S * sizeof(int64_t));
    for (size_t s = 0; s < S; ++s)
        for (int32_t k = 0; k < so->n; ++k) so->delta[s * N + k] = so->W[(int64_t)k * so->n + k];
}

/* Section IV-A: random vectors with +infinity energy, random fields; the
 * epoch r separates the draws of each restart (R23). */
static void init_pools(orc_solver* so, uint32_t r) {
    const int32_t n = so->n;
    const size_t C = (size_t)so->C, N = (size_t)n;
    for (uint32_t pp = 0; pp < (uint32_t)so->P; ++pp)
        for (uint32_t e = 0; e < (uint32_t)C; ++e) {
            uint8_t* x = so->pool_X + ((size_t)pp * C + e) * N;
            uint32_t u[4];
            for (int32_t k = 0; k < n; ++k) {
                draw(so->seed, (uint32_t)(k >> 5), e, pp, (7u << 24) | r, u);
                x[k] = (uint8_t)(nibble(u, k & 31) & 1);
            }
            so->pool_E[pp * C + e] = INT64_MAX;
            draw(so->seed, 0, e, pp, (8u << 24) | r, u);
            so->pool_algo[pp * C + e] = (int32_t)uidx(u[0], ORC_N_ALGOS);
            so->pool_op[pp * C + e] = (int32_t)uidx(u[1], ORC_N_OPS);
        }
}

/* R23: all pools merged around the global best? */
static int pools_merged(const orc_solver* so) {
    const size_t PC = (size_t)so->P * so->C, N = (size_t)so->n;
    for (size_t q = 0; q < PC; ++q) {
        int64_t d = 0;
        for (size_t k = 0; k < N; ++k) d += so->pool_X[q * N + k] != so->gbest_X[k];
        if (d > so->p.restart_dist) return 0;
    }
    return 1;
}

orc_solver* orc_solver_create(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed) {
    orc_solver* so = (orc_solver*)calloc(1, sizeof *so);
    so->W_own = (int16_t*)malloc((size_t)n * n * sizeof(int16_t));
    memcpy(so->W_own, W, (size_t)n * n * sizeof(int16_t));
    so->W = so->W_own;
    so->n = n; so->p = *p; so->seed = seed;
    so->S = p->searches; so->P = p->pools; so->C = p->pool_cap;
    const size_t S = (size_t)so->S, P = (size_t)so->P, C = (size_t)so->C, N = (size_t)n;
    so->pool_X = (uint8_t*)calloc(P * C * N, 1);
    so->pool_E = (int64_t*)calloc(P * C, sizeof(int64_t));
    so->pool_algo = (int32_t*)calloc(P * C, sizeof(int32_t));
    so->pool_op = (int32_t*)calloc(P * C, sizeof(int32_t));
    so->X = (uint8_t*)calloc(S * N, 1);
    so->delta = (int32_t*)calloc(S * N, sizeof(int32_t));
    so->E = (int64_t*)calloc(S, sizeof(int64_t));
    so->D = (uint8_t*)calloc(S * N, 1);
    so->algo = (int32_t*)calloc(S, sizeof(int32_t));
    so->op = (int32_t*)calloc(S, sizeof(int32_t));
    so->res_X = (uint8_t*)calloc(S * N, 1);
    so->res_E = (int64_t*)calloc(S, sizeof(int64_t));
    so->res_flips = (uint64_t*)calloc(S, sizeof(uint64_t));
    so->gbest_X = (uint8_t*)calloc(N, 1);
    so->gbest_E = INT64_MAX;
    reset_searches(so);
    init_pools(so, 0);
    return so;
}

void orc_solver_destroy(orc_solver* so) {
    if (!so) return;
    free(so->W_own); free(so->pool_X); free(so->pool_E); free(so->pool_algo); free(so->pool_op);
    free(so->X); free(so->delta); free(so->E); free(so->D); free(so->algo); free(so->op);
    free(so->res_X); free(so->res_E); free(so->res_flips); free(so->gbest_X);
    free(so);
}

/* Section IV-A genetic operations and Section IV-B Xrossover for search s. */
static void breed(const orc_solver* so, uint32_t g, uint32_t s, uint8_t* D, int32_t* algo_out,
                  int32_t* op_out) {
    const int32_t n = so->n;
    const uint32_t P = (uint32_t)so->P, C = (uint32_t)so->C;
    const uint32_t pp = s % P, qq = (pp + 1) % P;
    uint32_t c[4], r[4], u[4];
    draw(so->seed, 0, g, s, 4u << 24, c);
    int32_t op = (c[0] < MIX_THRESHOLD) ? (int32_t)uidx(c[1], ORC_N_OPS)
                                         : so->pool_op[pp * C + uidx(c[1], C)];
    int32_t algo = (c[2] < MIX_THRESHOLD) ? (int32_t)uidx(c[3], ORC_N_ALGOS)
                                           : so->pool_algo[pp * C + uidx(c[3], C)];
    if (so->p.abs_mode) { /* R24 */
        op = ORC_CROSSOVER;
        algo = ORC_CYCLICMIN;
    }
    draw(so->seed, 0, g, s, 5u << 24, r);
    const uint8_t* A = so->pool_X + ((size_t)pp * C + orc_parent_rank(r[0], C)) * (size_t)n;
    const uint32_t bpool = (op == ORC_XROSSOVER) ? qq : pp;
    const uint8_t* Bv = so->pool_X + ((size_t)bpool * C + orc_parent_rank(r[1], C)) * (size_t)n;
    const uint8_t* best = so->pool_X + ((size_t)pp * C) * (size_t)n;
    for (int32_t k = 0; k < n; ++k) {
        draw(so->seed, (uint32_t)(k >> 5), g, s, 6u << 24, u);
        int nib = nibble(u, k & 31);
        int hit = (nib & 7) == 0, coin = nib & 1;
        if (so->p.abs_mode) { /* R24: crossover, then mutation */
            D[k] = (uint8_t)(((nib >> 3) ? Bv[k] : A[k]) ^ hit);
            continue;
        }
        switch (op) {
            case ORC_MUTATION: D[k] = (uint8_t)(A[k] ^ hit); break;
            case ORC_CROSSOVER:
            case ORC_XROSSOVER: D[k] = coin ? Bv[k] : A[k]; break;
            case ORC_ZERO: D[k] = hit ? 0 : A[k]; break;
            case ORC_ONE: D[k] = hit ? 1 : A[k]; break;
            case ORC_INTERVALZERO: D[k] = A[k]; break;
            case ORC_BEST: D[k] = best[k]; break;
            default: D[k] = (uint8_t)coin; break; /* ORC_RANDOM */
        }
    }
    if (op == ORC_INTERVALZERO) {
        uint32_t hi = (uint32_t)n / 2, lo = hi < 32 ? hi : 32;
        uint32_t len = lo + uidx(r[2], hi - lo + 1);
        uint32_t start = uidx(r[3], (uint32_t)n);
        for (uint32_t t = 0; t < len; ++t) D[(start + t) % (uint32_t)n] = 0;
    }
    *algo_out = algo;
    *op_out = op;
}

void orc_solver_offspring(orc_solver* so, uint32_t g, uint8_t* D, int32_t* algo, int32_t* op) {
    for (uint32_t s = 0; s < (uint32_t)so->S; ++s)
        breed(so, g, s, D + (size_t)s * so->n, &algo[s], &op[s]);
}

static void pool_insert(orc_solver* so, uint32_t pp, const uint8_t* x, int64_t e, int32_t algo,
                        int32_t op) {
    const int32_t n = so->n;
    const uint32_t C = (uint32_t)so->C;
    int64_t* PE = so->pool_E + (size_t)pp * C;
    uint8_t* PX = so->pool_X + (size_t)pp * C * n;
    if (!(e < PE[C - 1])) return;
    for (uint32_t k = 0; k < C; ++k)
        if (PE[k] == e && memcmp(PX + (size_t)k * n, x, (size_t)n) == 0) return;
    uint32_t pos = 0;
    while (pos < C && PE[pos] <= e) ++pos;
    for (uint32_t k = C - 1; k > pos; --k) {
        PE[k] = PE[k - 1];
        memcpy(PX + (size_t)k * n, PX + (size_t)(k - 1) * n, (size_t)n);
        so->pool_algo[pp * C + k] = so->pool_algo[pp * C + k - 1];
        so->pool_op[pp * C + k] = so->pool_op[pp * C + k - 1];
    }
    PE[pos] = e;
    memcpy(PX + (size_t)pos * n, x, (size_t)n);
    so->pool_algo[pp * C + pos] = algo;
    so->pool_op[pp * C + pos] = op;
}

void orc_pool_merge(orc_solver* so, const uint8_t* best_X, const int64_t* best_E,
                    const int32_t* algo, const int32_t* op) {
    for (uint32_t s = 0; s < (uint32_t)so->S; ++s)
        pool_insert(so, s % (uint32_t)so->P, best_X + (size_t)s * so->n, best_E[s], algo[s], op[s]);
    int32_t winner = -1;
    for (uint32_t s = 0; s < (uint32_t)so->S; ++s) {
        so->algo_count[algo[s]] += 1;
        so->op_count[op[s]] += 1;
        if (best_E[s] < so->gbest_E) {
            so->gbest_E = best_E[s];
            memcpy(so->gbest_X, best_X + (size_t)s * so->n, (size_t)so->n);
            winner = (int32_t)s;
        }
    }
    if (winner >= 0) { /* Table VI: the finder of the new global best */
        so->best_algo[algo[winner]] += 1;
        so->best_op[op[winner]] += 1;
    }
}

typedef struct {
    orc_solver* so;
    uint32_t s0, s1;
} worker_arg;

static void* worker(void* a) {
    worker_arg* w = (worker_arg*)a;
    orc_solver* so = w->so;
    const size_t N = (size_t)so->n;
    for (uint32_t s = w->s0; s < w->s1; ++s)
        orc_batch_search(so->W, so->n, &so->p, so->seed, so->g, s, so->X + s * N, so->delta + s * N,
                         &so->E[s], so->D + s * N, so->algo[s], so->res_X + s * N, &so->res_E[s],
                         &so->res_flips[s], NULL, NULL, 0, 0);
    return NULL;
}

uint64_t orc_solver_generation(orc_solver* so, int32_t threads) {
    orc_solver_offspring(so, so->g, so->D, so->algo, so->op);
    if (threads < 1) threads = 1;
    if (threads > so->S) threads = so->S;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    worker_arg* args = (worker_arg*)malloc(sizeof(worker_arg) * (size_t)threads);
    for (int32_t t = 0; t < threads; ++t) {
        args[t].so = so;
        args[t].s0 = (uint32_t)((int64_t)so->S * t / threads);
        args[t].s1 = (uint32_t)((int64_t)so->S * (t + 1) / threads);
        if (threads == 1) worker(&args[t]);
        else pthread_create(&th[t], NULL, worker, &args[t]);
    }
    if (threads > 1)
        for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
    orc_pool_merge(so, so->res_X, so->res_E, so->algo, so->op);
    uint64_t f = 0;
    for (int32_t s = 0; s < so->S; ++s) f += so->res_flips[s];
    so->flips_total += f;
    so->g += 1;
    if (so->p.restart && pools_merged(so)) { /* R23 */
        so->restarts += 1;
        init_pools(so, so->restarts);
        reset_searches(so);
    }
    return f;
}

void orc_solver_get_pools(const orc_solver* so, uint8_t* X, int64_t* E, int32_t* algo, int32_t* op) {
    const size_t PC = (size_t)so->P * so->C;
    if (X) memcpy(X, so->pool_X, PC * so->n);
    if (E) memcpy(E, so->pool_E, PC * sizeof(int64_t));
    if (algo) memcpy(algo, so->pool_algo, PC * sizeof(int32_t));
    if (op) memcpy(op, so->pool_op, PC * sizeof(int32_t));
}

void orc_solver_set_pools(orc_solver* so, const uint8_t* X, const int64_t* E, const int32_t* algo,
                          const int32_t* op) {
    const size_t PC = (size_t)so->P * so->C;
    memcpy(so->pool_X, X, PC * so->n);
    memcpy(so->pool_E, E, PC * sizeof(int64_t));
    memcpy(so->pool_algo, algo, PC * sizeof(int32_t));
    memcpy(so->pool_op, op, PC * sizeof(int32_t));
}

void orc_solver_get_state(const orc_solver* so, uint8_t* X, int32_t* delta, int64_t* E) {
    const size_t S = (size_t)so->S, N = (size_t)so->n;
    if (X) memcpy(X, so->X, S * N);
    if (delta) memcpy(delta, so->delta, S * N * sizeof(int32_t));
    if (E) memcpy(E, so->E, S * sizeof(int64_t));
}

void orc_solver_get_results(const orc_solver* so, uint8_t* best_X, int64_t* best_E, uint64_t* flips,
                            int32_t* algo, int32_t* op) {
    const size_t S = (size_t)so->S, N = (size_t)so->n;
    if (best_X) memcpy(best_X, so->res_X, S * N);
    if (best_E) memcpy(best_E, so->res_E, S * sizeof(int64_t));
    if (flips) memcpy(flips, so->res_flips, S * sizeof(uint64_t));
    if (algo) memcpy(algo, so->algo, S * sizeof(int32_t));
    if (op) memcpy(op, so->op, S * sizeof(int32_t));
}

void orc_solver_get_stats(const orc_solver* so, uint64_t* algo_count, uint64_t* op_count,
                          uint64_t* best_algo, uint64_t* best_op) {
    memcpy(algo_count, so->algo_count, sizeof so->algo_count);
    memcpy(op_count, so->op_count, sizeof so->op_count);
    memcpy(best_algo, so->best_algo, sizeof so->best_algo);
    memcpy(best_op, so->best_op, sizeof so->best_op);
}

uint32_t orc_solver_get_restarts(const orc_solver* so) { return so->restarts; }

void orc_solver_get_best(const orc_solver* so, uint8_t* X, int64_t* E, uint64_t* flips_total,
                         uint32_t* generations) {
    if (X) memcpy(X, so->gbest_X, (size_t)so->n);
    if (E) *E = so->gbest_E;
    if (flips_total) *flips_total = so->flips_total;
    if (generations) *generations = so->g;
}

int orc_solve(const int16_t* W, int32_t n, const orc_params* p, uint64_t budget, uint64_t seed,
              int64_t target, int32_t threads, uint8_t* best_X, int64_t* best_E, uint64_t* flips,
              uint32_t* generations) {
    orc_solver* so = orc_solver_create(W, n, p, seed);
    for (;;) {
        orc_solver_generation(so, threads);
        if (so->flips_total >= budget) break;
        if (so->gbest_E <= target) break;
        if (p->max_generations > 0 && so->g >= (uint32_t)p->max_generations) break;
    }
    orc_solver_get_best(so, best_X, best_E, flips, generations);
    orc_solver_destroy(so);
    return 0;
}
