/*
 * dabs_oracle.h -- plain, slow CPU oracle of the Diverse Adaptive Bulk Search
 * (DABS) hot path.  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA
 * library bit for bit.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm may load it; the product path never does.
 *
 * It shares no code, header, table or constant generator with the CUDA
 * library under paper_2207_03069_gb300/csrc.  Every function states the
 * passage of the paper (Nakano et al., "Diverse Adaptive Bulk Search: a
 * Framework for Solving QUBO Problems on Multiple GPUs") it follows.
 *
 * Conventions (the "readings" where the paper is silent or garbled are listed
 * in the comment block at the top of dabs_oracle.c):
 *   - W is a symmetric n x n int16 matrix, row-major, leading dimension n.
 *   - X, D, BEST are byte vectors of n entries, each 0 or 1.
 *   - energies are int64, Delta values int32.
 */
#ifndef DABS_ORACLE_H
#define DABS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MAXMIN = 0, ORC_CYCLICMIN = 1, ORC_RANDOMMIN = 2, ORC_POSITIVEMIN = 3,
       ORC_TWONEIGHBOR = 4, ORC_N_ALGOS = 5 };
enum { ORC_MUTATION = 0, ORC_CROSSOVER = 1, ORC_XROSSOVER = 2, ORC_ZERO = 3, ORC_ONE = 4,
       ORC_INTERVALZERO = 5, ORC_BEST = 6, ORC_RANDOM = 7, ORC_N_OPS = 8 };
/* phase tags written to a batch-search trace */
enum { ORC_PH_STRAIGHT = 0, ORC_PH_GREEDY = 1, ORC_PH_MAIN = 2 };

typedef struct {
    int32_t searches;        /* S: concurrent batch searches                  */
    int32_t pools;           /* P: islands (solution pools)                   */
    int32_t pool_cap;        /* C: packets per pool                           */
    int32_t tabu;            /* tabu period (0..31)                           */
    int32_t s_num, s_den;    /* search flip factor s = s_num / s_den          */
    int32_t b_num, b_den;    /* batch flip factor  b = b_num / b_den          */
    int32_t seed_mode;       /* 0 = Straight walk to D, 1 = from-scratch X=D  */
    int32_t max_generations; /* 0 = unlimited                                 */
    int32_t restart;         /* 1 = restart when the pools have merged (R23)  */
    int32_t restart_dist;    /* h: merged = every entry within distance h     */
    int32_t abs_mode;        /* 1 = ABS: CyclicMin, crossover then mutation   */
} orc_params;

/* ---- definitions (Section I-A Eq. (2); Section III Eq. (3)) ---- */
int64_t orc_energy(const int16_t* W, int32_t n, const uint8_t* X);
void    orc_delta(const int16_t* W, int32_t n, const uint8_t* X, int32_t* delta);

/* ---- counter-based random numbers (Philox4x32-10, Salmon et al. SC'11) ---- */
void     orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_parent_rank(uint32_t u, uint32_t m);          /* Section IV-A */
uint64_t orc_cube21(uint64_t a, uint64_t T);               /* (a/T)^3 in 2^-32 units */
int      orc_batch_continue(uint64_t total, uint64_t B, int32_t main_runs, int32_t algo);
/* Section III-A RandomMin: p(t) in units of 2^-16 (reading R8) and the per-bit
 * 16-bit uniforms of the iteration made as flip `flip` of search s, gen g */
uint32_t orc_randmin_threshold(uint64_t t, uint64_t T, int32_t n);
void     orc_randmin_draws(uint64_t seed, uint32_t flip, uint32_t g, uint32_t s, int32_t n,
                           uint16_t* u16);
/* Section III-A MaxMin: threshold d in [mn, D(t)] (reading R6); *R_out (may be
 * NULL) receives the interval width floor(((T-t)/T)^3 (mx - mn)) */
int64_t  orc_maxmin_threshold(int32_t mn, int32_t mx, uint64_t t, uint64_t T, uint32_t u0,
                              uint64_t* R_out);

/* ---- one batch search (Section III-B) on persistent state X, delta, E ----
 * trace_idx/trace_phase (optional, may be NULL) receive one entry per flip,
 * up to trace_cap entries.  check != 0 recomputes Delta and E from scratch
 * after every flip and returns -1 on the first mismatch.                    */
int orc_batch_search(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed,
                     uint32_t g, uint32_t s, uint8_t* X, int32_t* delta, int64_t* E,
                     const uint8_t* D, int32_t algo, uint8_t* best_X, int64_t* best_E,
                     uint64_t* flips, int32_t* trace_idx, int32_t* trace_phase,
                     int64_t trace_cap, int32_t check);

/* Per-flip record of the main searches' selectors, indexed by flip number
 * (entries of other phases are left untouched), up to cap entries:
 *   a     MaxMin threshold d; RandomMin threshold (units of 2^-16);
 *         PositiveMin posmin (INT64_MAX if no positive Delta); CyclicMin width
 *   r     MaxMin interval width R (0 otherwise)
 *   count candidates: MaxMin and PositiveMin (non-tabu, Delta <= bound),
 *         RandomMin (non-tabu bits whose uniform is below the threshold)
 *   free  non-tabu bits at that iteration                                   */
typedef struct {
    int64_t* a;
    int64_t* r;
    int32_t* count;
    int32_t* free;
    int64_t cap;
} orc_sel_trace;
int orc_batch_search_sel(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed,
                         uint32_t g, uint32_t s, uint8_t* X, int32_t* delta, int64_t* E,
                         const uint8_t* D, int32_t algo, uint8_t* best_X, int64_t* best_E,
                         uint64_t* flips, int32_t* trace_idx, int32_t* trace_phase,
                         int64_t trace_cap, int32_t check, orc_sel_trace* sel);

/* ---- solver object: pools + per-search state, one generation at a time ---- */
typedef struct orc_solver orc_solver;
orc_solver* orc_solver_create(const int16_t* W, int32_t n, const orc_params* p, uint64_t seed);
void        orc_solver_destroy(orc_solver* so);
/* runs one generation (offspring, batch searches on `threads` host threads,
 * pool merge, global best).  Returns the flips of this generation.          */
uint64_t    orc_solver_generation(orc_solver* so, int32_t threads);
/* breeds the targets of generation g from the current pools without running */
void        orc_solver_offspring(orc_solver* so, uint32_t g, uint8_t* D, int32_t* algo, int32_t* op);
void        orc_solver_get_pools(const orc_solver* so, uint8_t* X, int64_t* E, int32_t* algo, int32_t* op);
void        orc_solver_set_pools(orc_solver* so, const uint8_t* X, const int64_t* E,
                                 const int32_t* algo, const int32_t* op);
void        orc_solver_get_state(const orc_solver* so, uint8_t* X, int32_t* delta, int64_t* E);
void        orc_solver_get_results(const orc_solver* so, uint8_t* best_X, int64_t* best_E,
                                   uint64_t* flips, int32_t* algo, int32_t* op);
void        orc_solver_get_best(const orc_solver* so, uint8_t* X, int64_t* E,
                                uint64_t* flips_total, uint32_t* generations);
/* Tables V/VI counters: per-search algorithm/operation counts and the
 * algorithm/operation of each result that improved the global best */
void        orc_solver_get_stats(const orc_solver* so, uint64_t* algo_count, uint64_t* op_count,
                                 uint64_t* best_algo, uint64_t* best_op);
/* restarts made so far (Section IV-B, all pools merged) */
uint32_t    orc_solver_get_restarts(const orc_solver* so);
/* merges externally given results into the pools (Section IV, packets) */
void        orc_pool_merge(orc_solver* so, const uint8_t* best_X, const int64_t* best_E,
                           const int32_t* algo, const int32_t* op);

/* whole solve (stops at the first generation boundary where flips >= budget,
 * best <= target, or max_generations is reached)                            */
int orc_solve(const int16_t* W, int32_t n, const orc_params* p, uint64_t budget, uint64_t seed,
              int64_t target, int32_t threads, uint8_t* best_X, int64_t* best_E,
              uint64_t* flips, uint32_t* generations);

#ifdef __cplusplus
}
#endif
#endif
