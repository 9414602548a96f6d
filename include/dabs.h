/*
 * dabs.h -- C ABI of libdabs.so, a GB300 (sm_103a) implementation of the
 * bulk local search of Diverse Adaptive Bulk Search (DABS) for QUBO
 * (Nakano, Takafuji, Ito et al., "Diverse Adaptive Bulk Search: a Framework
 * for Solving QUBO Problems on Multiple GPUs").
 *
 * Problem (Section I-A, Eq. (2)): minimise E(X) = sum_i W_ii x_i +
 * sum_{i<j} W_ij x_i x_j over X in {0,1}^n, for a symmetric int16 matrix W
 * with entries in [-32767, 32767] (each unordered pair counted once).  A matrix written with every ordered
 * pair counted converts to this form by W'_ij = W_ij + W_ji (i != j).
 *
 * Conventions of every call:
 *  - Return 0 (DABS_OK) on success, a negative DABS_E_* code on error; no
 *    call aborts the process.  dabs_strerror() names the code and
 *    dabs_last_error() gives the context's last message.
 *  - "host" buffers are ordinary CPU memory owned by the caller; "device"
 *    buffers are CUDA global memory on the context's device, owned by the
 *    caller.  The library keeps no pointer to a caller buffer after a call
 *    returns.  Calls on host buffers are synchronous.  Calls on device
 *    buffers are enqueued on the context's stream (see dabs_set_stream) and
 *    return before the GPU work completes.
 *  - Bit vectors on the device are packed: bit k of a vector is bit (k % 32)
 *    of 32-bit word k / 32; a vector occupies ceil(n / 32) words and its bits
 *    >= n must be zero.  On the host, X vectors are n bytes of 0 or 1.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Energies are int64; Delta values are int32 (exact for n <= 65535).
 */
#ifndef DABS_H
#define DABS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DABS_OK 0
#define DABS_E_INVALID_ARG (-1)  /* bad size, pointer, parameter or bit value   */
#define DABS_E_NOT_SYMMETRIC (-2)/* W is not symmetric                          */
#define DABS_E_TOO_LARGE (-3)    /* n or a parameter above what the build holds */
#define DABS_E_OOM (-4)          /* device allocation failed                    */
#define DABS_E_TIMEOUT (-5)      /* a bounded device wait ran out               */
#define DABS_E_CUDA (-6)         /* any other CUDA runtime error                */
#define DABS_E_BUSY (-7)         /* the context is in a state that forbids it   */
#define DABS_E_NO_DEVICE (-8)    /* no CUDA device of compute capability 10.3   */

#define DABS_N_MAX 16384         /* largest n of the register-resident search   */

enum { DABS_MAXMIN = 0, DABS_CYCLICMIN = 1, DABS_RANDOMMIN = 2, DABS_POSITIVEMIN = 3,
       DABS_TWONEIGHBOR = 4 };
enum { DABS_MUTATION = 0, DABS_CROSSOVER = 1, DABS_XROSSOVER = 2, DABS_ZERO = 3, DABS_ONE = 4,
       DABS_INTERVALZERO = 5, DABS_BEST = 6, DABS_RANDOM = 7 };

/* Solver parameters (Sections III-B and IV).  Defaults (dabs_params_default):
 * 32 searches, 4 pools, pool_cap 100 and tabu 8 (the paper's experiments),
 * s = 1/10, b = 1, Straight seeding, no generation limit, no restarts, DABS
 * (not ABS) breeding.                                                       */
typedef struct dabs_params {
    int32_t searches;        /* concurrent batch searches S (1..65535)          */
    int32_t pools;           /* solution pools P (islands), 1..S                */
    int32_t pool_cap;        /* packets per pool C, 1..1024                     */
    int32_t tabu;            /* tabu period, 0..31                              */
    int32_t s_num, s_den;    /* search flip factor s: T = max(1, floor(n s))    */
    int32_t b_num, b_den;    /* batch flip factor b: B = ceil(n b)              */
    int32_t seed_mode;       /* 0: Straight walk to each target (Section III-B);
                                1: X = target, Delta and E recomputed           */
    int32_t max_generations; /* 0 = unlimited                                  */
    int32_t restart;         /* 1: when every pool entry lies within Hamming
                                distance restart_dist of the global best (the
                                pools have merged, Section IV-B), draw all
                                pools afresh and restart every search from
                                X = 0; the global best carries on.  0: never */
    int32_t restart_dist;    /* h of the merge test (negative: never merged)  */
    int32_t abs_mode;        /* 1: the earlier Adaptive Bulk Search (Section I):
                                CyclicMin only, and every target is a mutation
                                after a crossover of two parents of its own
                                pool.  0: DABS                                */
} dabs_params;

typedef struct dabs_ctx dabs_ctx;

/* Fills *p with the defaults above. */
int dabs_params_default(dabs_params* p);

/* Creates a context on the current CUDA device: copies W (host, n*n int16,
 * row-major, symmetric) to device memory once (rows padded to a multiple of
 * 64 entries) and allocates the solver state for *p.  Errors: INVALID_ARG
 * (null pointer, n < 1, bad params), NOT_SYMMETRIC, TOO_LARGE (n > DABS_N_MAX
 * or S / P > 4096), NO_DEVICE, OOM; INVALID_ARG also when an entry is
 * -32768 (the library keeps -W on the device).  On error *out is NULL.     */
int dabs_create(const int16_t* W, int32_t n, const dabs_params* p, dabs_ctx** out);

/* Frees every device and host resource of ctx (NULL is accepted). */
void dabs_destroy(dabs_ctx* ctx);

/* Message of a DABS_E_* code, and the context's last error message. */
const char* dabs_strerror(int code);
const char* dabs_last_error(const dabs_ctx* ctx);

/* Uses `stream` (a cudaStream_t, NULL = the context's own stream) for all
 * further device work of ctx. */
int dabs_set_stream(dabs_ctx* ctx, void* stream);

/* Replaces the weights with another symmetric n x n matrix of the same n
 * (host buffer, read once by one copy), keeping the solver state
 * allocations.  The checks run on the device before anything is replaced:
 * NOT_SYMMETRIC (the message names the lowest i * n + j with W_ij != W_ji)
 * or INVALID_ARG (an entry -32768), and on error the context is unchanged. */
int dabs_load_weights(dabs_ctx* ctx, const int16_t* W);

/* Eq. (2): energy of one host vector X (n bytes, each 0 or 1). */
int dabs_energy(dabs_ctx* ctx, const uint8_t* X, int64_t* E);

/* Eq. (3): Delta_k(X) = E(f_k(X)) - E(X) for all k of one host vector. */
int dabs_delta(dabs_ctx* ctx, const uint8_t* X, int32_t* delta);

/* Batched Eq. (2)/(3) on device buffers: X (count packed vectors), E
 * (count int64), delta (count x ld_delta int32, or NULL).  Asynchronous. */
int dabs_energy_delta_dev(dabs_ctx* ctx, const uint32_t* X, int32_t count, int64_t* E,
                          int32_t* delta, int32_t ld_delta);

/* Eq. (2)/(3) for `count` packed device vectors on the tensor cores
 * (tcgen05 MMA on bf16 limbs: W = 256 hi + lo, 8-bit limbs, fp32 accumulation
 * exact for n <= 65,793), same outputs as dabs_energy_delta_dev.  count must
 * not exceed the context's searches rounded up to 128.  Asynchronous; a
 * bounded device wait that ran out is reported by dabs_kernel_status. */
int dabs_recompute_dev(dabs_ctx* ctx, const uint32_t* X, int32_t count, int64_t* E,
                       int32_t* delta, int32_t ld_delta);
/* Recompute seeding (seed_mode = 1) on 0 = CUDA cores, 1 = tensor cores (the
 * default for contexts created with seed_mode = 1). */
int dabs_set_recompute(dabs_ctx* ctx, int32_t mode);
/* Waits for the context's stream; DABS_E_TIMEOUT if a kernel's bounded wait
 * ran out since the last call (the flag is then cleared). */
int dabs_kernel_status(dabs_ctx* ctx);
/* Test hook (no counterpart in the paper): the next dabs_bulk_search_dev of a
 * context on variant (1, 0) issues no copy for its first row, so that row's
 * bounded wait runs out (about 4 s: the wait, then the wait for a copy in
 * flight), the search stops without storing, and dabs_kernel_status reports
 * DABS_E_TIMEOUT; the context stays usable.  INVALID_ARG on other variants. */
int dabs_test_stall_next_search(dabs_ctx* ctx);

/* Whole solve (Sections III and IV): pools initialised with random vectors,
 * every search starting at X = 0; generations of (offspring, batch search,
 * pool merge) until, at a generation boundary, the total number of flips
 * reaches `budget`, the best energy is <= `target` (INT64_MIN: no target),
 * or max_generations is reached.  Writes the best vector (host, n bytes),
 * its energy and the flips made.  Deterministic in (W, params, budget, seed,
 * target).  DABS_E_TIMEOUT (as dabs_kernel_status) if a kernel's bounded
 * device wait ran out during the solve; dabs_batch_solve checks every
 * instance the same way.                                                     */
int dabs_solve(dabs_ctx* ctx, uint64_t budget, uint64_t seed, int64_t target, uint8_t* best_X,
               int64_t* best_E, uint64_t* flips);

/* ---- batched form: many instances per launch ---------------------------
 * Solves the k contexts together (Sections III and IV per instance): every
 * generation runs each instance's offspring, recompute, merge and finalise
 * kernels and one batch-search launch per kernel variant covering all the
 * instances of that variant; the variants' launches run concurrently, the
 * one with the most work first.  An instance uses the variant chosen for it
 * by dabs_set_variant or dabs_autotune; otherwise the default for many
 * instances in flight (8 warps x 2 chunks for 2048 < n <= 4096, where a
 * context alone uses 4 x 4).  Each instance stops on its own
 * budget/target/generation limit; instance i's results (best_X[i], n_i host
 * bytes; best_E[i]; flips[i]) equal dabs_solve(ctxs[i], budgets[i], seeds[i],
 * targets[i]) alone.  targets, best_X, best_E, flips may be NULL.
 * Synchronous. */
int dabs_batch_solve(dabs_ctx* const* ctxs, int32_t k, const uint64_t* budgets,
                     const uint64_t* seeds, const int64_t* targets, uint8_t* const* best_X,
                     int64_t* best_E, uint64_t* flips);

/* The same batched form one step at a time (dabs_batch_solve is built on
 * it).  dabs_batch_create takes k distinct contexts (k >= 1) and a
 * cudaStream_t (NULL: the batch makes its own); while the batch lives every
 * context's work is enqueued on that stream (their own streams are restored
 * by dabs_batch_destroy), and each context's inspection calls
 * (dabs_solve_status, dabs_solve_best, dabs_read_pools, ...) stay valid.
 * dabs_batch_begin starts every instance's solve as dabs_solve_begin(ctxs[i],
 * seeds[i], budgets[i], targets[i]) would (targets may be NULL: none).
 * dabs_batch_generations runs `count` generations of every instance still
 * running, then waits for the stream and retires the instances whose solve
 * has stopped; *running (may be NULL) receives how many remain.  After g
 * generations instance i is in the state g calls of
 * dabs_solve_generations(ctxs[i], 1) leave it in alone.  INVALID_ARG for a
 * NULL or repeated context, or generations before begin. */
typedef struct dabs_batch dabs_batch;
int  dabs_batch_create(dabs_ctx* const* ctxs, int32_t k, void* stream, dabs_batch** out);
int  dabs_batch_begin(dabs_batch* b, const uint64_t* budgets, const uint64_t* seeds,
                      const int64_t* targets);
int  dabs_batch_generations(dabs_batch* b, int32_t count, int32_t* running);
/* Measurement of a batch since its creation (waits for its stream): the
 * instances still running, the batch-search launch groups in use, the kernels
 * launched on the device, and the summed device time (ms) of the
 * generations' batch-search phases.  Any output may be NULL. */
int  dabs_batch_info(dabs_batch* b, int32_t* running, int32_t* search_groups,
                     uint64_t* launches, double* search_ms);
void dabs_batch_destroy(dabs_batch* b);

/* ---- served form: request queue with continuous batching ----------------
 * A server owns a queue of solve requests.  dabs_server_step admits queued
 * requests (first come, first served) while the device bytes of their
 * contexts fit the HBM budget and advances the admitted ones in rounds of
 * the given number of generations in batched form.  Requests run in two
 * size classes (n <= 2048, n > 2048), each with its own stream and rounds,
 * so small requests are not held at the pace of the largest one's
 * generations; requests that arrive while a class's round runs join at its
 * next round.  A finished request's context is kept and reused (a new W
 * loaded into it) by a later request of the same n and parameters, and
 * freed when the budget needs its bytes.  Each request's result equals
 * dabs_solve alone.  Latency = completion (detected at the end of a round)
 * minus submission. */
typedef struct dabs_server dabs_server;
int dabs_server_create(size_t hbm_budget_bytes, dabs_server** out);
void dabs_server_destroy(dabs_server* s);
/* Copies W (host, n*n int16, symmetric) into the request; TOO_LARGE if the
 * request alone exceeds the budget or n > DABS_N_MAX.  Does not block. */
int dabs_server_submit(dabs_server* s, const int16_t* W, int32_t n, const dabs_params* p,
                       uint64_t budget, uint64_t seed, int64_t target, uint64_t* ticket);
/* One scheduling step: retires the requests of every class whose round has
 * ended, admits queued requests and starts a round in every class with work
 * and none in flight; when no round had ended, it first waits for one (so
 * every call advances the solve).  *pending = queued + running requests. */
int dabs_server_step(dabs_server* s, int32_t generations, int32_t* pending);
/* status: 0 queued, 1 running, 2 done (outputs written, best_X n bytes),
 * negative = the request failed with that DABS_E_* code. */
int dabs_server_poll(dabs_server* s, uint64_t ticket, uint8_t* best_X, int64_t* best_E,
                     uint64_t* flips, double* latency_s, int32_t* status);
int dabs_server_info(const dabs_server* s, size_t* used_bytes, int32_t* queued, int32_t* running);
/* Admission also stops while the running requests' batch searches hold more
 * than max_warps resident warps (searches x warps per search; default two
 * waves, 64 x SM count; 0 = no cap).  A request is always admitted when
 * nothing runs. */
int dabs_server_set_limits(dabs_server* s, int64_t max_warps);

/* ---- stepwise form of dabs_solve (device-resident state) ---------------- */
/* Resets pools, search state and counters for a new solve.  Asynchronous. */
int dabs_solve_begin(dabs_ctx* ctx, uint64_t seed, uint64_t budget, int64_t target);
/* Enqueues `count` generations; generations after the stop condition are
 * no-ops on the device.  By default the four kernels of a generation are
 * captured once as a CUDA graph (on the context's stream) and the graph is
 * launched `count` times; a change of variant, row format, keyed form,
 * recompute mode, stream or weights captures it again.  Asynchronous. */
int dabs_solve_generations(dabs_ctx* ctx, int32_t count);
/* 1 (default): generations run as CUDA graph launches; 0: kernel by kernel.
 * Results are the same. */
int dabs_set_graphs(dabs_ctx* ctx, int32_t enable);
/* Waits for the stream, then reports the counters. */
int dabs_solve_status(dabs_ctx* ctx, uint64_t* flips, uint32_t* generations, int64_t* best_E,
                      int32_t* done);
/* Waits for the stream, then reports the pool restarts made so far
 * (dabs_params.restart). */
int dabs_solve_restarts(dabs_ctx* ctx, uint32_t* restarts);
/* Waits for the stream, then copies the best vector (host, n bytes) and E. */
int dabs_solve_best(dabs_ctx* ctx, uint8_t* best_X, int64_t* best_E);

/* ---- one batch search per slot on caller buffers (Section III-B) --------
 * For slots s < count: state X (packed), delta (ld int32 per slot, see
 * dabs_info), E; target D (packed); algo (one byte per slot, DABS_MAXMIN..
 * DABS_TWONEIGHBOR).  Runs seeding (Straight, or nothing when seed_mode = 1:
 * the state must then already equal the target), Greedy and (main search,
 * Greedy) rounds until b*n flips, drawing random numbers for generation g
 * and slot s of `seed`.  Outputs per slot: BEST (packed), E(BEST), flips.
 * All pointers are device buffers.  Asynchronous.                         */
int dabs_bulk_search_dev(dabs_ctx* ctx, uint64_t seed, uint32_t g, int32_t count, uint32_t* X,
                         int32_t* delta, int64_t* E, const uint32_t* D, const uint8_t* algo,
                         uint32_t* best_X, int64_t* best_E, uint32_t* flips);

/* ---- the batch search without device allocation -------------------------
 * No counterpart in the paper: an engineering entry point.  It runs the same
 * batch search as dabs_bulk_search_dev (identical results) for callers that
 * cannot allocate device memory -- e.g. code whose device memory is owned by
 * another allocator (a framework's caching allocator or a fixed arena) that
 * must not see cudaMalloc/cudaFree, which may synchronise the device and
 * fragment the arena.  No context is needed and nothing is allocated: the
 * negated weight copy, the diagonal, the slot launch order and the control
 * block live in one file-scope device array of 2 MiB + 128 KiB + 256 B that
 * every GPU which loads the library keeps until the process exits.
 *   W      device, n x ld int16 row-major, 16-byte aligned, ld a multiple of
 *          8, columns >= n zero, entries in [-32767, 32767]; an entry of
 *          -32768 is found on the device and refuses the call there: no
 *          search runs and every slot gets best_E = INT64_MAX, flips = 0
 *   p      tabu, s_num/s_den, b_num/b_den and seed_mode are used
 *   X, delta (count x ld int32, 16-byte aligned), E, D, algo, best_X, best_E,
 *   flips  as in dabs_bulk_search_dev (device buffers of the caller)
 *   stream the cudaStream_t to enqueue on (NULL = default stream)
 * Limits: n * ld <= 1048576 and count <= 16384, else DABS_E_TOO_LARGE.
 * The first call on a device looks up the array's device address (once per
 * device and CUDA context, with that device current; after a cudaDeviceReset
 * the next call looks it up again); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (each call rewrites the parts it reads), so calls whose GPU work overlaps
 * race: order them on one stream.  Asynchronous.                            */
int dabs_bulk_search_noalloc(const int16_t* W, int32_t n, int32_t ld, const dabs_params* p,
                             uint64_t seed, uint32_t g, int32_t count, uint32_t* X,
                             int32_t* delta, int64_t* E, const uint32_t* D, const uint8_t* algo,
                             uint32_t* best_X, int64_t* best_E, uint32_t* flips, void* stream);

/* ---- measurement (no counterpart in the paper) --------------------------
 * Read bandwidth (GB/s) of `bytes` of device memory at `buf` (16-byte
 * aligned), read `reps` times back to back after three warm-up passes on
 * `stream` (NULL: the default stream).  A buffer well under the L2's size
 * stays resident, which measures the L2 read bandwidth the batch search's
 * row reads are compared with when W fits the L2.  Synchronous; allocates a
 * 4-byte result slot. */
int dabs_measure_read_gbs(const void* buf, size_t bytes, int32_t reps, void* stream, double* gbs);

/* ---- inspection (host copies; synchronous) ------------------------------ */
/* n, padded row length ld, packed words per vector, S, P, C, and the
 * kernel variant (warps per search, 8-bit chunks per thread). */
int dabs_info(const dabs_ctx* ctx, int32_t* n, int32_t* ld, int32_t* words, int32_t* searches,
              int32_t* pools, int32_t* pool_cap, int32_t* warps, int32_t* chunks);
/* Chooses the batch-search variant: `warps` warps per search with `chunks`
 * 8-bit chunks per thread and Delta in registers (n up to 256 warps chunks),
 * or (1, 0): one warp per search with Delta in shared memory, one search per
 * CTA (n up to DABS_N_MAX; every Delta must stay below 2^29 in magnitude,
 * i.e. max_k sum_j |W_kj| < 2^29; it reads dense rows, fetched per lane block
 * by bulk copies into shared memory, and its waits are bounded: a wait that
 * runs out sets the flag dabs_kernel_status reports).  Returns TOO_LARGE if
 * the variant cannot run the instance.  Sparse rows stay selected only if
 * they fit the new variant. */
int dabs_set_variant(dabs_ctx* ctx, int32_t warps, int32_t chunks);
/* Row format of the batch search (Step 3, Eq. (4) reads row i of W):
 *   DABS_ROWS_DENSE          the dense int16 rows of W in global memory;
 *   DABS_ROWS_SPARSE_SMEM    every CTA keeps the off-diagonal non-zeros of all
 *                            rows (column << 16 | 16-bit weight, 4 bytes each,
 *                            plus n+1 row offsets) in shared memory;
 *   DABS_ROWS_SPARSE_GLOBAL  the same entries read from global memory (L2);
 *   DABS_ROWS_DENSE_SMEM     every CTA keeps all of W (n x ld int16) in shared
 *                            memory (one-warp variants, n up to about 330 on
 *                            this GPU) and reads row i with 128-bit shared
 *                            loads, negating it when x_i = 0.
 * With sparse rows a flip scatters row i into a zeroed per-search scratch row
 * in shared memory, so it reads 4 bytes per non-zero instead of 2n bytes.
 * Sparse rows are stored while the non-zeros are at most max(n^2/4, 64); TOO_LARGE
 * when they are not, or when the format's shared memory (the copy, about
 * 56,000 entries at most on this GPU, and ld int16 per search of a CTA)
 * exceeds the device's opt-in size per block.  The default is dense rows
 * (the fastest measured on Max-Cut n = 800 and a 5,627-node sparse Ising
 * model: the flip loop is bound by its dependency chain, not by the row
 * read); dabs_autotune times all three.  Results do not depend on the format.
 * Batched launches (dabs_batch_solve, the server) read dense rows. */
enum { DABS_ROWS_DENSE = 0, DABS_ROWS_SPARSE_SMEM = 1, DABS_ROWS_SPARSE_GLOBAL = 2,
       DABS_ROWS_DENSE_SMEM = 3 };
int dabs_set_rows(dabs_ctx* ctx, int32_t mode);
/* Keyed form of the batch search: each thread keeps Delta_k * 2^kb +
 * (k << 1 | x_k) instead of Delta_k, so that every minimum of Step 1 and of
 * the selectors also yields the lowest winning index and x_k, with no second
 * pass.  Available when (2R + 2) 2^kb < 2^31, kb = bitlen(n-1) + 1, R =
 * max_k sum_j |W_kj| (every Delta lies in [-R, R]); on by default (enable = 1)
 * and used for single-instance launches with dense rows.  Results do not
 * depend on it.  dabs_get_keyed reports the switch and kb (0: the instance
 * does not allow it). */
int dabs_set_keyed(dabs_ctx* ctx, int32_t enable);
int dabs_get_keyed(const dabs_ctx* ctx, int32_t* enabled, int32_t* key_bits);
/* Current row format and the number of stored off-diagonal non-zeros (-1
 * when sparse rows are not stored). */
int dabs_get_rows(const dabs_ctx* ctx, int32_t* mode, int32_t* nnz);
/* Runs a throwaway solve on the context's workload for `generations` warm-up
 * generations, breeds the next generation's targets, then times the batch
 * search of that same generation with every built variant that holds n (each
 * from the same snapshot of the search state) and keeps the fastest per flip
 * (results never depend on the variant).
 * table (may be NULL) receives DABS_N_VARIANTS nanoseconds-per-flip entries
 * in the order (warps x chunks) 1x1 1x2 1x4 2x1 2x2 2x4 4x1 4x2 4x4 8x1 8x2
 * 8x4 16x1 16x2 16x4 1x0 with dense rows, then the same 16 for each other row
 * format in the order of their codes (dabs_set_rows), 0 where a variant
 * cannot hold n or the row format is unavailable.  Sets the fastest variant
 * and row format.  Resets the solve state; call before dabs_solve_begin.
 * Synchronous. */
#define DABS_N_VARIANTS 64
int dabs_autotune(dabs_ctx* ctx, int32_t generations, int32_t* warps, int32_t* chunks,
                  float* ns_per_flip, float* table);
/* Counters of the running solve (the paper's Tables V and VI): runs of each
 * main algorithm (DABS_MAXMIN..) and uses of each genetic operation
 * (DABS_MUTATION..) over all searches and generations, and the algorithm and
 * operation of every result that improved the global best.  Any pointer may
 * be NULL; arrays of 5 and 8 entries.  Synchronous. */
int dabs_read_stats(dabs_ctx* ctx, uint64_t* algo_count, uint64_t* op_count, uint64_t* best_algo,
                    uint64_t* best_op);
/* Checkpoint of a solve at a generation boundary: pools, per-search state,
 * global best, counters and the control block, into a host buffer (call with
 * buf = NULL to learn *size).  dabs_restore loads it into a context created
 * with the same W, n and parameters; the solve then continues exactly as the
 * original would have.  Synchronous. */
int dabs_checkpoint(dabs_ctx* ctx, void* buf, size_t cap, size_t* size);
int dabs_restore(dabs_ctx* ctx, const void* buf, size_t size);
/* Current pools (the ones the next generation breeds from): X [P][C][words],
 * E [P][C], algo [P][C], op [P][C].  Any pointer may be NULL. */
int dabs_read_pools(dabs_ctx* ctx, uint32_t* X, int64_t* E, uint8_t* algo, uint8_t* op);
int dabs_write_pools(dabs_ctx* ctx, const uint32_t* X, const int64_t* E, const uint8_t* algo,
                     const uint8_t* op);
/* Per-search state X [S][words], delta [S][ld], E [S]. */
int dabs_read_state(dabs_ctx* ctx, uint32_t* X, int32_t* delta, int64_t* E);
/* Last generation's targets D [S][words], algo, op and results BEST [S][words],
 * E(BEST) [S], flips [S]. */
int dabs_read_generation(dabs_ctx* ctx, uint32_t* D, uint8_t* algo, uint8_t* op,
                         uint32_t* best_X, int64_t* best_E, uint32_t* flips);
/* Overwrites the results buffers (for a merge-only step). */
int dabs_write_results(dabs_ctx* ctx, const uint32_t* best_X, const int64_t* best_E,
                       const uint32_t* flips, const uint8_t* algo, const uint8_t* op);
/* Runs one stage of the current generation: 0 offspring (+ recompute when
 * seed_mode = 1), 1 batch search, 2 pool merge, 3 finalise (advances the
 * generation).  Asynchronous. */
int dabs_run_stage(dabs_ctx* ctx, int32_t stage);
/* A solve split over devices by island (Section IV-B: the solution pools
 * are islands; search s breeds from island s mod P): stage 1 then runs only
 * the searches s with lo <= s mod modulus < hi (modulus = P for whole
 * islands); the other slots' results are written by dabs_write_results
 * before the merge (paper_2207_03069_gb300/islands.py exchanges them).
 * modulus = 0 runs every search (the default).  Applies to dabs_run_stage
 * only; INVALID_ARG unless 0 <= lo < hi <= modulus. */
int dabs_set_search_slots(dabs_ctx* ctx, int32_t modulus, int32_t lo, int32_t hi);

#ifdef __cplusplus
}
#endif
#endif
