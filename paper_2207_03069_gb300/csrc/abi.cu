// abi.cu -- the C ABI of libdabs.so (declared in include/dabs.h): context
// lifetime, weight residency, the per-generation launch sequence
// (offspring -> [recompute] -> batch search -> pool merge -> finalise), the
// stepwise and whole solve, and inspection calls.  No exception crosses the
// ABI; every CUDA error becomes a DABS_E_* code with a message in the context.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace dabs;

namespace dabs_internal {

int fail(dabs_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

template <class T>
int dalloc(dabs_ctx* ctx, T** ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  CK(cudaMalloc(&p, bytes));
  ctx->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return DABS_OK;
}

bool params_ok(const dabs_params* p) {
  return p->searches >= 1 && p->searches <= 65535 && p->pools >= 1 && p->pools <= p->searches &&
         p->pool_cap >= 1 && p->pool_cap <= 1024 && p->tabu >= 0 && p->tabu <= 31 &&
         p->s_num >= 0 && p->s_den >= 1 && p->b_num >= 0 && p->b_den >= 1 &&
         (p->seed_mode == 0 || p->seed_mode == 1) && p->max_generations >= 0 &&
         (p->restart == 0 || p->restart == 1) && (p->abs_mode == 0 || p->abs_mode == 1);
}

// the smallest variant that holds n, in the order measured fastest per size
// band on this GPU (n <= 256, 512, 1024, 2048, 4096, 8192, 16384).  Alone
// (one instance's searches, about one wave), 4 warps x 4 chunks is fastest
// for 2048 < n <= 4096; with many instances in flight (batched, served) 8
// warps x 2 chunks is, and 8 warps x 1 chunk for 1024 < n <= 2048: more
// warps per SM hide more of the per-flip latency (measured on 64 instances
// of n in [256, 4096]: 12% and 3% less time per generation).  Server
// admission (batch.cu) counts warps with the second order.
bool default_variant(int n, SearchVariant* v, bool many) {
  static const int alone[][2] = {{1, 1}, {1, 2}, {1, 4}, {4, 2}, {4, 4}, {8, 4}, {16, 4}};
  static const int batched[][2] = {{1, 1}, {1, 2}, {1, 4}, {8, 1}, {8, 2}, {8, 4}, {16, 4}};
  for (auto& o : many ? batched : alone) {
    SearchVariant q;
    if (launch_search(o[0], o[1], nullptr, nullptr, &q) && q.cap >= n) {
      *v = q;
      return true;
    }
  }
  return false;
}

int tc_limbs(dabs_ctx* ctx);
bool rows_ok(const dabs_ctx* ctx, const SearchVariant& v, int mode);

// Loads W (host, n x n, row-major): one DMA into the -W buffer as staging,
// then the checks and row measurements on the device (weights.cu).  Only
// their outcome comes back to the host; when it rejects W, -W is rebuilt
// from the unchanged W and the context is as before the call.
int upload_weights(dabs_ctx* ctx, const int16_t* W) {
  const int n = ctx->n, ld = ctx->ld;
  cudaStream_t st = ctx->stream;
  // launch arguments that depend on W's values (a captured generation stays
  // valid while they do not change: W itself is read through fixed pointers)
  const int old_kb = ctx->key_bits, old_nnz = ctx->sp_nnz, old_rows = ctx->rows_mode;
  const uint32_t* old_ent = ctx->sp_ent;
  WeightsArgs a{};
  a.Ws = ctx->Wneg;
  a.W = ctx->W;
  a.Wneg = ctx->Wneg;
  a.diag = ctx->diag;
  a.n = n;
  a.ld = ld;
  a.rowsum = ctx->wrow;
  a.rowcnt = ctx->wrow + n;
  a.rowptr = ctx->wptr;
  a.rowptr_len = 4 * sparse_row16(n);
  a.chk = ctx->wchk;
  // stream order keeps the DMA behind any generation still reading -W
  CK(cudaMemcpy2DAsync(ctx->Wneg, (size_t)ld * sizeof(int16_t), W, (size_t)n * sizeof(int16_t),
                       (size_t)n * sizeof(int16_t), (size_t)n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(ctx->wrow, 0, 2 * (size_t)n * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(ctx->wchk, 0xff, sizeof(WCheck), st));
  const unsigned tiles = (unsigned)((n + 31) / 32);
  k_weights_tiles<<<dim3(tiles, tiles), dim3(32, 8), 0, st>>>(a);
  CKLAUNCH();
  k_weights_rows<<<1, 1024, 0, st>>>(a);
  CKLAUNCH();
  CK(cudaMemcpyAsync(ctx->h_wchk, ctx->wchk, sizeof(WCheck), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const WCheck c = *ctx->h_wchk;
  const unsigned vec_blocks = (unsigned)std::min<size_t>(((size_t)n * ld / 8 + 255) / 256, 4096);
  if (c.bad != ~0ull || c.low != ~0ull) {
    k_negate<<<vec_blocks, 256, 0, st>>>(ctx->W, ctx->Wneg, (size_t)n * ld);
    CKLAUNCH();
    CK(cudaStreamSynchronize(st));
    if (c.bad != ~0ull) {
      const int i = (int)(c.bad / n), j = (int)(c.bad % n);
      return fail(ctx, DABS_E_NOT_SYMMETRIC, "W[%d][%d] != W[%d][%d]", i, j, j, i);
    }
    return fail(ctx, DABS_E_INVALID_ARG, "W[%d][%d] = -32768 (weights must lie in [-32767, 32767])",
                (int)(c.low / n), (int)(c.low % n));
  }
  k_weights_commit<<<vec_blocks, 256, 0, st>>>(a);
  CKLAUNCH();
  ctx->w_hash_ok = false;
  ctx->max_abs = (int)~c.nmax;
  const int64_t R = (int64_t)c.R;
  const size_t nnz_all = (size_t)c.nnz;
  // keyed Delta: |Delta_k| <= R_k = sum_j |W_kj| in every state, and a key
  // (Delta << kb | k << 1 | x_k) plus the diagonal term added to it before
  // Eq. (5) overwrites it must stay inside int32
  {
    int kb = 1;
    while ((1 << (kb - 1)) < n) ++kb;  // bitlen(n - 1) + 1
    ctx->key_bits = ((2 * R + 2) << kb) < (int64_t)INT32_MAX ? kb : 0;
    // the shared-memory Delta variant marks tabu bits with +2^30: |Delta| < 2^29
    ctx->smem_ok = R < (1 << 29) - 1 &&
                   smem_search_bytes(n) + 1024 <= (size_t)std::max(ctx->smem_optin, 0);
  }
  // sparse rows: the off-diagonal non-zeros of each row, column ascending,
  // kept while they take at most half the bytes of the dense rows (or 64
  // entries, for tiny instances)
  const size_t limit = std::max<size_t>((size_t)n * n / 4, 64);
  ctx->sp_nnz = -1;
  if (nnz_all <= limit) {
    const int nnz = (int)nnz_all;
    const size_t cap = 4 * (size_t)sparse_ent16(nnz);
    if (cap > ctx->sp_cap) {
      CK(cudaStreamSynchronize(st));
      if (ctx->sp_ent) cudaFree(ctx->sp_ent);
      ctx->sp_ent = nullptr;
      ctx->sp_cap = 0;
      CK(cudaMalloc(&ctx->sp_ent, cap * 4));
      ctx->sp_cap = cap;
    }
    a.ent = ctx->sp_ent;
    CK(cudaMemcpyAsync(ctx->sp_row, ctx->wptr, 4 * (size_t)sparse_row16(n) * 4, cudaMemcpyDeviceToDevice, st));
    if (cap > (size_t)nnz) CK(cudaMemsetAsync(ctx->sp_ent + nnz, 0, (cap - nnz) * 4, st));
    k_sparse_fill<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(a);
    CKLAUNCH();
    ctx->sp_nnz = nnz;
  }
  if (!rows_ok(ctx, ctx->var, ctx->rows_mode)) ctx->rows_mode = ROWS_DENSE;
  if (ctx->key_bits != old_kb || ctx->sp_nnz != old_nnz || ctx->rows_mode != old_rows ||
      ctx->sp_ent != old_ent)
    graph_stale(ctx);
  if (ctx->tc_ready) return tc_limbs(ctx);
  return DABS_OK;
}

// hash of W (ties checkpoints to their instance), from the device copy on
// first use after a load: four independent xor-multiply chains over the
// row-major n x n bytes in 64-bit words, then the tail bytes
static int weights_hash(dabs_ctx* ctx, uint64_t* out) {
  if (!ctx->w_hash_ok) {
    const int n = ctx->n;
    std::vector<int16_t> h((size_t)n * n);
    CK(cudaMemcpy2DAsync(h.data(), (size_t)n * sizeof(int16_t), ctx->W, (size_t)ctx->ld * sizeof(int16_t),
                         (size_t)n * sizeof(int16_t), (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const unsigned char* by = reinterpret_cast<const unsigned char*>(h.data());
    const size_t nb = h.size() * sizeof(int16_t);
    const uint64_t P = 1099511628211ull;
    uint64_t ln[4] = {1469598103934665603ull, 0x9E3779B97F4A7C15ull, 0xC2B2AE3D27D4EB4Full,
                      0x165667B19E3779F9ull};
    size_t q = 0;
    for (; q + 32 <= nb; q += 32)
      for (int l = 0; l < 4; ++l) {
        uint64_t w;
        memcpy(&w, by + q + 8 * l, 8);
        ln[l] = (ln[l] ^ w) * P;
      }
    for (; q < nb; ++q) ln[0] = (ln[0] ^ by[q]) * P;
    uint64_t hv = ln[0];
    for (int l = 1; l < 4; ++l) hv = (hv ^ ((ln[l] << (16 * l)) | (ln[l] >> (64 - 16 * l)))) * P;
    ctx->w_hash = hv ^ (uint64_t)nb;
    ctx->w_hash_ok = true;
  }
  *out = ctx->w_hash;
  return DABS_OK;
}

// a row format is usable with variant v: sparse rows are stored, and the
// shared memory they need (the copy for ROWS_SPARSE_SMEM, one scratch row per
// search of a CTA) fits the opt-in size of a block with 2 KiB to spare for
// the kernel's static arrays
bool rows_ok(const dabs_ctx* ctx, const SearchVariant& v, int mode) {
  if (v.ch == 0) return mode == ROWS_DENSE;  // the shared-memory Delta variant reads dense rows
  if (mode == ROWS_DENSE) return true;
  if (mode == ROWS_DENSE_SMEM)  // one-warp variants; W and 2 KiB fit a block
    return v.nw == 1 && sparse_smem_bytes(mode, ctx->n, 0, ctx->ld, v.spc) + 2048 <= (size_t)ctx->smem_optin;
  if (ctx->sp_nnz < 0 || (mode != ROWS_SPARSE_SMEM && mode != ROWS_SPARSE_GLOBAL)) return false;
  const size_t need = sparse_smem_bytes(mode, ctx->n, ctx->sp_nnz, ctx->ld, v.spc) + 2048;
  return need <= (size_t)ctx->smem_optin;
}

// dense rows: measured on this GPU, the sparse formats save bytes but add a
// scatter and two group barriers per flip, which the latency-bound flip loop
// feels more than the (L2-resident) dense row read; dabs_set_rows or the
// autotuner select them where they win
int default_rows(const dabs_ctx*) { return ROWS_DENSE; }

// the tensor-core operands of the loaded W: one fp16 operand when it is
// exact (|W_ij| <= 2048) and every partial sum stays below 2^24 in fp32
// (n max|W_ij| < 2^24), else two bf16 limbs (allocated on first need)
int tc_limbs(dabs_ctx* ctx) {
  const size_t total = (size_t)ctx->n_pad * ctx->n_pad;
  const int limbs = (ctx->max_abs <= 2048 && (int64_t)ctx->n * ctx->max_abs < (1 << 24)) ? 1 : 2;
  if (limbs == 2 && !ctx->Wlo) {
    int rc;
    CK(cudaStreamSynchronize(ctx->stream));
    if ((rc = dalloc(ctx, &ctx->Wlo, total)) != DABS_OK) return rc;
    if (!make_tmap_bf16(&ctx->mapLo, ctx->Wlo, ctx->n_pad, ctx->n_pad, umma_tile_n()))
      return fail(ctx, DABS_E_CUDA, "cuTensorMapEncodeTiled failed");
  }
  k_limbs<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      ctx->W, ctx->n, ctx->ld, ctx->n_pad, limbs, ctx->Whi, ctx->Wlo);
  CKLAUNCH();
  if (limbs != ctx->tc_limbs_n) graph_stale(ctx);
  ctx->tc_limbs_n = limbs;
  return DABS_OK;
}

// allocates the tensor-core recompute buffers and builds the TMA maps (once)
int tc_setup(dabs_ctx* ctx) {
  if (ctx->tc_ready) return DABS_OK;
  const int bm = umma_tile_m(), bn = umma_tile_n();
  const int bnk = std::max(bn, umma_tile_k());  // both tile widths divide the padding (powers of two)
  ctx->n_pad = (ctx->n + bnk - 1) / bnk * bnk;
  ctx->rows_pad = (std::max(ctx->S, 1) + bm - 1) / bm * bm;
  int rc;
  if ((rc = dalloc(ctx, &ctx->Whi, (size_t)ctx->n_pad * ctx->n_pad)) != DABS_OK) return rc;
  if ((rc = dalloc(ctx, &ctx->Abf, (size_t)ctx->rows_pad * ctx->n_pad)) != DABS_OK) return rc;
  if ((rc = dalloc(ctx, &ctx->E2, (size_t)ctx->rows_pad)) != DABS_OK) return rc;
  if ((rc = dalloc(ctx, &ctx->kerr, 1)) != DABS_OK) return rc;
  CK(cudaMemsetAsync(ctx->kerr, 0, sizeof(int), ctx->stream));
  if (!make_tmap_bf16(&ctx->mapA, ctx->Abf, ctx->rows_pad, ctx->n_pad, bm) ||
      !make_tmap_bf16(&ctx->mapHi, ctx->Whi, ctx->n_pad, ctx->n_pad, bn))
    return fail(ctx, DABS_E_CUDA, "cuTensorMapEncodeTiled failed");
  // the one-limb form's maps stand in for the unused second limb
  ctx->mapLo = ctx->mapHi;
  if (!umma_prepare()) return fail(ctx, DABS_E_CUDA, "tensor-core kernel set-up failed");
  if ((rc = tc_limbs(ctx)) != DABS_OK) return rc;
  ctx->tc_ready = true;
  return DABS_OK;
}

// Eq. (2)/(3) for `count` packed vectors on the tensor cores
int tc_recompute(dabs_ctx* ctx, const uint32_t* X, int count, int64_t* E, int32_t* delta,
                 int ld_delta, const DevCtrl* ctrl) {
  cudaStream_t st = ctx->stream;
  const size_t pairs = (size_t)ctx->rows_pad * (ctx->n_pad / 2);
  const uint32_t one = ctx->tc_limbs_n == 1 ? 0x3C00u : 0x3F80u;  // 1.0 in fp16 / bf16
  k_bits_to_bf16<<<(unsigned)std::min<size_t>((pairs + 255) / 256, 4096), 256, 0, st>>>(
      X, count, ctx->n, ctx->nw, ctx->rows_pad, ctx->n_pad, ctx->Abf, one, ctrl);
  CKSTAGE();
  CK(cudaMemsetAsync(ctx->E2, 0, sizeof(int64_t) * ctx->rows_pad, st));
  UmmaArgs u{count, ctx->n, ctx->n_pad, ctx->nw, ld_delta, X, ctx->diag, delta, ctx->E2, ctx->kerr, ctrl};
  const dim3 grid(ctx->n_pad / umma_tile_n(), (count + umma_tile_m() - 1) / umma_tile_m());
  launch_recompute_umma(ctx->tc_limbs_n, grid, st, ctx->mapA, ctx->mapHi, ctx->mapLo, u);
  CKSTAGE();
  k_halve<<<(count + 255) / 256, 256, 0, st>>>(E, ctx->E2, count, ctrl);
  CKSTAGE();
  return DABS_OK;
}

SearchArgs solve_search_args(dabs_ctx* ctx) {
  SearchArgs a{};
  a.W = ctx->W;
  a.Wneg = ctx->Wneg;
  a.diag = ctx->diag;
  a.n = ctx->n; a.ld = ctx->ld; a.nw = ctx->nw; a.S = ctx->S;
  a.T = ctx->T; a.tau = ctx->tau; a.B = ctx->B; a.seed_mode = ctx->p.seed_mode;
  a.ctrl = ctx->ctrl;
  a.X = ctx->X; a.delta = ctx->delta; a.E = ctx->E; a.D = ctx->D; a.algo = ctx->algo;
  a.best_X = ctx->bestX; a.best_E = ctx->bestE; a.flips = ctx->flips;
  a.order = ctx->order;
  a.key_bits = ctx->keyed ? ctx->key_bits : 0;
  a.serr = ctx->serr;
  a.sp_mode = ctx->rows_mode;
  if (ctx->rows_mode == ROWS_SPARSE_SMEM || ctx->rows_mode == ROWS_SPARSE_GLOBAL) {
    a.sp_row = ctx->sp_row;
    a.sp_ent = ctx->sp_ent;
    a.sp_nnz = ctx->sp_nnz;
  }
  return a;
}

int stage(dabs_ctx* ctx, int which) {
  cudaStream_t st = ctx->stream;
  if (which == 0) {
    OffArgs o{};
    o.n = ctx->n; o.nw = ctx->nw; o.S = ctx->S; o.P = ctx->P; o.C = ctx->C; o.ctrl = ctx->ctrl;
    for (int b = 0; b < 2; ++b) { o.pool_X[b] = ctx->poolX[b]; o.pool_algo[b] = ctx->poolA[b]; o.pool_op[b] = ctx->poolO[b]; }
    o.D = ctx->D; o.algo = ctx->algo; o.op = ctx->op; o.abs_mode = ctx->p.abs_mode;
    k_offspring<<<(ctx->S * 32 + 255) / 256, 256, 0, st>>>(o);
    CKSTAGE();
    if (ctx->p.seed_mode == 1) {
      const size_t words = (size_t)ctx->S * ctx->nw;
      k_copy_targets<<<148, 256, 0, st>>>(ctx->D, ctx->X, ctx->E, words, ctx->S, ctx->ctrl);
      CKSTAGE();
      if (ctx->recompute_mode == 1) {
        const int rc = tc_recompute(ctx, ctx->D, ctx->S, ctx->E, ctx->delta, ctx->ld, ctx->ctrl);
        if (rc) return rc;
      } else {
        EDArgs e{ctx->W, ctx->n, ctx->ld, ctx->nw, ctx->X, ctx->delta, ctx->ld, ctx->E, ctx->ctrl};
        k_energy_delta<<<dim3((ctx->n + 255) / 256, ctx->S), 256, 0, st>>>(e);
        CKSTAGE();
      }
    }
  } else if (which == 1 || which == 4) {
    const bool split = which == 1 && ctx->slot_mod > 0;
    k_order_by_algo<<<1, 1024, 0, st>>>(ctx->algo, ctx->S, ctx->order, ctx->ctrl,
                                        split ? ctx->slot_mod : 0, ctx->slot_lo, ctx->slot_hi);
    CKSTAGE();
    if (which == 4) return DABS_OK;  // launch order only (batched search follows)
    SearchArgs a = solve_search_args(ctx);
    if (split) {
      if (ctx->slot_count == 0) return DABS_OK;
      a.S = ctx->slot_count;  // the listed slots only
    }
    if (!launch_search(ctx->var.nw, ctx->var.ch, &a, st, nullptr))
      return fail(ctx, DABS_E_INVALID_ARG, "no batch-search variant %d/%d", ctx->var.nw, ctx->var.ch);
    CKSTAGE();
  } else if (which == 2) {
    MergeArgs m{};
    m.nw = ctx->nw; m.S = ctx->S; m.P = ctx->P; m.C = ctx->C; m.Mmax = ctx->Mmax; m.ctrl = ctx->ctrl;
    for (int b = 0; b < 2; ++b) { m.pool_X[b] = ctx->poolX[b]; m.pool_E[b] = ctx->poolE[b]; m.pool_algo[b] = ctx->poolA[b]; m.pool_op[b] = ctx->poolO[b]; }
    m.best_X = ctx->bestX; m.best_E = ctx->bestE; m.algo = ctx->algo; m.op = ctx->op;
    k_merge<<<ctx->P, kMergeThreads, ctx->merge_smem, st>>>(m);
    CKSTAGE();
  } else if (which == 3) {
    const bool restart = ctx->p.restart != 0;
    if (restart) CK(cudaMemsetAsync(ctx->rflag, 1, sizeof(uint32_t), st));  // skip unless armed
    FinArgs f{ctx->nw, ctx->S, ctx->ctrl, ctx->bestX, ctx->bestE, ctx->flips, ctx->gbestX,
              ctx->algo, ctx->op, ctx->stats, restart ? ctx->rflag : nullptr};
    k_finalize<<<1, 1024, 0, st>>>(f);
    CKSTAGE();
    if (restart) {  // Section IV-B: restart once every pool has merged around the best
      const int entries = ctx->P * ctx->C;
      RestartArgs r{ctx->nw, ctx->P, ctx->C, ctx->p.restart_dist, ctx->ctrl,
                    {ctx->poolX[0], ctx->poolX[1]}, ctx->gbestX, ctx->rflag};
      k_restart_check<<<std::min((entries * 32 + 255) / 256, 1216), 256, 0, st>>>(r);
      CKSTAGE();
      PoolArgs pa{};
      pa.n = ctx->n; pa.nw = ctx->nw; pa.P = ctx->P; pa.C = ctx->C; pa.ctrl = ctx->ctrl;
      pa.cond = ctx->rflag;
      for (int b = 0; b < 2; ++b) { pa.pool_X[b] = ctx->poolX[b]; pa.pool_E[b] = ctx->poolE[b]; pa.pool_algo[b] = ctx->poolA[b]; pa.pool_op[b] = ctx->poolO[b]; }
      k_pool_init<<<(entries * 32 + 255) / 256, 256, 0, st>>>(pa);
      CKSTAGE();
      StateArgs sa{ctx->n, ctx->ld, ctx->nw, ctx->S, ctx->diag, ctx->X, ctx->delta, ctx->E,
                   nullptr, ctx->rflag, ctx->ctrl};
      k_state_init<<<304, 256, 0, st>>>(sa);
      CKSTAGE();
    }
  } else {
    return fail(ctx, DABS_E_INVALID_ARG, "stage %d", which);
  }
  return DABS_OK;
}

int read_ctrl(dabs_ctx* ctx, DevCtrl* out) {
  CK(cudaMemcpyAsync(ctx->h_ctrl, ctx->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *out = *ctx->h_ctrl;
  return DABS_OK;
}

int check_bits(dabs_ctx* ctx, const uint8_t* X) {
  for (int k = 0; k < ctx->n; ++k)
    if (X[k] > 1) return fail(ctx, DABS_E_INVALID_ARG, "X[%d] = %d is not 0 or 1", k, X[k]);
  return DABS_OK;
}

}  // namespace dabs_internal

using namespace dabs_internal;

namespace dabs {
int spc_for(int slots, int maxspc) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 152;
  }
  const int want = (slots + sms - 1) / sms;
  return std::min(maxspc, std::max(1, want));
}

bool launch_search(int nw, int ch, const SearchArgs* a, cudaStream_t st, SearchVariant* v,
                   const MultiArgs* m) {
  if (nw == 1 && ch == 0) return launch_search_smem(a, st, v, m);  // Delta in shared memory
  switch (nw) {
    case 1: return launch_search_w1(ch, a, st, v, m);
    case 2: return launch_search_w2(ch, a, st, v, m);
    case 4: return launch_search_w4(ch, a, st, v, m);
    case 8: return launch_search_w8(ch, a, st, v, m);
    case 16: return launch_search_w16(ch, a, st, v, m);
    default: return false;
  }
}
}  // namespace dabs

extern "C" {

int dabs_params_default(dabs_params* p) {
  if (!p) return DABS_E_INVALID_ARG;
  *p = dabs_params{32, 4, 100, 8, 1, 10, 1, 1, 0, 0, 0, 0, 0};
  return DABS_OK;
}

const char* dabs_strerror(int code) {
  switch (code) {
    case DABS_OK: return "ok";
    case DABS_E_INVALID_ARG: return "invalid argument";
    case DABS_E_NOT_SYMMETRIC: return "weight matrix is not symmetric";
    case DABS_E_TOO_LARGE: return "size above the supported maximum";
    case DABS_E_OOM: return "device memory allocation failed";
    case DABS_E_TIMEOUT: return "bounded device wait ran out";
    case DABS_E_CUDA: return "CUDA runtime error";
    case DABS_E_BUSY: return "context busy";
    case DABS_E_NO_DEVICE: return "no compute capability 10.3 CUDA device";
    default: return "unknown error";
  }
}

const char* dabs_last_error(const dabs_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

void dabs_destroy(dabs_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->sp_ent) cudaFree(ctx->sp_ent);
  if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
  if (ctx->h_wchk) cudaFreeHost(ctx->h_wchk);
  if (ctx->own) cudaStreamDestroy(ctx->own);
  delete ctx;
}

int dabs_create(const int16_t* W, int32_t n, const dabs_params* p, dabs_ctx** out) {
  if (!out) return DABS_E_INVALID_ARG;
  *out = nullptr;
  if (!W || !p || n < 1 || !params_ok(p)) return DABS_E_INVALID_ARG;
  if (n > DABS_N_MAX) return DABS_E_TOO_LARGE;
  const int R = (p->searches + p->pools - 1) / p->pools;
  if (R > 4096) return DABS_E_TOO_LARGE;
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DABS_E_NO_DEVICE;
  if (cudaGetDevice(&dev) != cudaSuccess) return DABS_E_NO_DEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DABS_E_NO_DEVICE;
  if (prop.major != 10 || prop.minor != 3) return DABS_E_NO_DEVICE;
  dabs_ctx* ctx = new (std::nothrow) dabs_ctx;
  if (!ctx) return DABS_E_OOM;
  ctx->dev = dev;
  ctx->n = n;
  ctx->ld = (n + 63) / 64 * 64;
  ctx->nw = (n + 31) / 32;
  ctx->p = *p;
  uint64_t T = (uint64_t)n * (uint64_t)p->s_num / (uint64_t)p->s_den;
  ctx->T = (int)(T < 1 ? 1 : (T > (1u << 30) ? (1u << 30) : T));
  ctx->tau = p->tabu < n - 1 ? p->tabu : n - 1;
  ctx->B = (uint32_t)(((uint64_t)n * p->b_num + p->b_den - 1) / p->b_den);
  ctx->S = p->searches; ctx->P = p->pools; ctx->C = p->pool_cap;
  int M = 1;
  while (M < R) M <<= 1;
  ctx->Mmax = M;
  ctx->merge_smem = (size_t)ctx->C * 16 + (size_t)M * 24;
  if (!default_variant(n, &ctx->var, false)) { dabs_destroy(ctx); return DABS_E_TOO_LARGE; }
  int rc;
#define TRY(x) do { if ((rc = (x)) != DABS_OK) { *out = nullptr; int r_ = rc; dabs_destroy(ctx); return r_; } } while (0)
  if (cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking) != cudaSuccess) {
    dabs_destroy(ctx);
    return DABS_E_CUDA;
  }
  ctx->stream = ctx->own;
  const size_t S = ctx->S, PC = (size_t)ctx->P * ctx->C, nw = ctx->nw, ld = ctx->ld;
  {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    ctx->smem_optin = optin;
  }
  TRY(dalloc(ctx, &ctx->sp_row, 4 * (size_t)sparse_row16(n)));
  TRY(dalloc(ctx, &ctx->W, (size_t)n * ld));
  TRY(cudaMemsetAsync(ctx->W, 0, (size_t)n * ld * sizeof(int16_t), ctx->stream) == cudaSuccess ? DABS_OK : DABS_E_CUDA);
  TRY(dalloc(ctx, &ctx->Wneg, (size_t)n * ld));
  TRY(dalloc(ctx, &ctx->diag, (size_t)n));
  TRY(dalloc(ctx, &ctx->wrow, 2 * (size_t)n));
  TRY(dalloc(ctx, &ctx->wptr, 4 * (size_t)sparse_row16(n)));
  TRY(dalloc(ctx, &ctx->wchk, 1));
  TRY(dalloc(ctx, &ctx->ctrl, 1));
  TRY(dalloc(ctx, &ctx->bulk_ctrl, 1));
  for (int b = 0; b < 2; ++b) {
    TRY(dalloc(ctx, &ctx->poolX[b], PC * nw));
    TRY(dalloc(ctx, &ctx->poolE[b], PC));
    TRY(dalloc(ctx, &ctx->poolA[b], PC));
    TRY(dalloc(ctx, &ctx->poolO[b], PC));
  }
  TRY(dalloc(ctx, &ctx->X, S * nw));
  TRY(dalloc(ctx, &ctx->delta, S * ld));
  TRY(dalloc(ctx, &ctx->E, S));
  TRY(dalloc(ctx, &ctx->D, S * nw));
  TRY(dalloc(ctx, &ctx->algo, S));
  TRY(dalloc(ctx, &ctx->op, S));
  TRY(dalloc(ctx, &ctx->bestX, S * nw));
  TRY(dalloc(ctx, &ctx->bestE, S));
  TRY(dalloc(ctx, &ctx->flips, S));
  TRY(dalloc(ctx, &ctx->order, S));
  TRY(dalloc(ctx, &ctx->gbestX, nw));
  TRY(dalloc(ctx, &ctx->stats, kStats));
  TRY(dalloc(ctx, &ctx->rflag, 1));
  TRY(dalloc(ctx, &ctx->serr, 1));
  TRY(cudaMemsetAsync(ctx->serr, 0, sizeof(int), ctx->stream) == cudaSuccess ? DABS_OK : DABS_E_CUDA);
  TRY(dalloc(ctx, &ctx->one_X, nw));
  TRY(dalloc(ctx, &ctx->one_d, ld));
  TRY(dalloc(ctx, &ctx->one_E, 1));
  if (cudaMallocHost(&ctx->h_ctrl, sizeof(DevCtrl)) != cudaSuccess) { dabs_destroy(ctx); return DABS_E_OOM; }
  if (cudaMallocHost(&ctx->h_wchk, sizeof(WCheck)) != cudaSuccess) { dabs_destroy(ctx); return DABS_E_OOM; }
  if (ctx->merge_smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ctx->merge_smem) != cudaSuccess) {
      dabs_destroy(ctx);
      return DABS_E_TOO_LARGE;
    }
  }
  TRY(upload_weights(ctx, W));
  ctx->rows_mode = default_rows(ctx);
  if (p->seed_mode == 1) {  // recompute seeding runs on the tensor cores by default
    TRY(tc_setup(ctx));
    ctx->recompute_mode = 1;
  }
  // a fresh context is a solve with seed 0 that has not run yet
  TRY(dabs_solve_begin(ctx, 0, UINT64_MAX, INT64_MIN));
  TRY(cudaStreamSynchronize(ctx->stream) == cudaSuccess ? DABS_OK : DABS_E_CUDA);
#undef TRY
  *out = ctx;
  return DABS_OK;
}

int dabs_set_stream(dabs_ctx* ctx, void* stream) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_load_weights(dabs_ctx* ctx, const int16_t* W) {
  if (!ctx || !W) return DABS_E_INVALID_ARG;
  return upload_weights(ctx, W);
}

int dabs_energy_delta_dev(dabs_ctx* ctx, const uint32_t* X, int32_t count, int64_t* E,
                          int32_t* delta, int32_t ld_delta) {
  if (!ctx || !X || !E || count < 0 || (delta && ld_delta < ctx->n)) return DABS_E_INVALID_ARG;
  if (count == 0) return DABS_OK;
  if (count > 65535) return fail(ctx, DABS_E_TOO_LARGE, "count %d > 65535", count);
  CK(cudaMemsetAsync(E, 0, sizeof(int64_t) * count, ctx->stream));
  EDArgs e{ctx->W, ctx->n, ctx->ld, ctx->nw, X, delta, ld_delta, E, nullptr};
  k_energy_delta<<<dim3((ctx->n + 255) / 256, count), 256, 0, ctx->stream>>>(e);
  CKLAUNCH();
  return DABS_OK;
}

static int one_vector(dabs_ctx* ctx, const uint8_t* X, int64_t* E, int32_t* delta) {
  int rc = check_bits(ctx, X);
  if (rc) return rc;
  std::vector<uint32_t> packed(ctx->nw, 0u);
  for (int k = 0; k < ctx->n; ++k) packed[k >> 5] |= (uint32_t)X[k] << (k & 31);
  CK(cudaMemcpyAsync(ctx->one_X, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
  rc = dabs_energy_delta_dev(ctx, ctx->one_X, 1, ctx->one_E, delta ? ctx->one_d : nullptr, ctx->ld);
  if (rc) return rc;
  int64_t e = 0;
  CK(cudaMemcpyAsync(&e, ctx->one_E, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
  if (delta)
    CK(cudaMemcpyAsync(delta, ctx->one_d, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (E) *E = e;
  return DABS_OK;
}

int dabs_energy(dabs_ctx* ctx, const uint8_t* X, int64_t* E) {
  if (!ctx || !X || !E) return DABS_E_INVALID_ARG;
  return one_vector(ctx, X, E, nullptr);
}

int dabs_delta(dabs_ctx* ctx, const uint8_t* X, int32_t* delta) {
  if (!ctx || !X || !delta) return DABS_E_INVALID_ARG;
  return one_vector(ctx, X, nullptr, delta);
}

int dabs_solve_begin(dabs_ctx* ctx, uint64_t seed, uint64_t budget, int64_t target) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  DevCtrl c{};
  c.seed = seed;
  c.g = 0;
  c.done = 0;
  c.flips_total = 0;
  c.budget = budget;
  c.target = target;
  c.max_generations = (uint32_t)ctx->p.max_generations;
  c.best_E = INT64_MAX;
  *ctx->h_ctrl = c;
  CK(cudaMemcpyAsync(ctx->ctrl, ctx->h_ctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->stats, 0, sizeof(unsigned long long) * kStats, ctx->stream));
  StateArgs s{ctx->n, ctx->ld, ctx->nw, ctx->S, ctx->diag, ctx->X, ctx->delta, ctx->E, ctx->gbestX,
              nullptr, nullptr};
  k_state_init<<<304, 256, 0, ctx->stream>>>(s);
  CKLAUNCH();
  PoolArgs pa{};
  pa.n = ctx->n; pa.nw = ctx->nw; pa.P = ctx->P; pa.C = ctx->C; pa.ctrl = ctx->ctrl;
  for (int b = 0; b < 2; ++b) { pa.pool_X[b] = ctx->poolX[b]; pa.pool_E[b] = ctx->poolE[b]; pa.pool_algo[b] = ctx->poolA[b]; pa.pool_op[b] = ctx->poolO[b]; }
  const int entries = ctx->P * ctx->C;
  k_pool_init<<<(entries * 32 + 255) / 256, 256, 0, ctx->stream>>>(pa);
  CKLAUNCH();
  return DABS_OK;
}

int dabs_run_stage(dabs_ctx* ctx, int32_t which) {
  if (!ctx) return DABS_E_INVALID_ARG;
  return stage(ctx, which);
}

// Captures one generation (the four stages) on the context's stream as a
// CUDA graph.  Every kernel reads the generation index, seed and stop flag
// from the device control block, so the same graph serves every generation.
static int capture_generation(dabs_ctx* ctx) {
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  ctx->graph_ok = false;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  int rc = DABS_OK;
  for (int st = 0; st < 4 && rc == DABS_OK; ++st) rc = stage(ctx, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (rc != DABS_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != DABS_OK ? rc : fail(ctx, DABS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    ctx->gexec = nullptr;
    return fail(ctx, DABS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
  }
  ctx->graph_ok = true;
  return DABS_OK;
}

int dabs_solve_generations(dabs_ctx* ctx, int32_t count) {
  if (!ctx || count < 0) return DABS_E_INVALID_ARG;
  if (ctx->graphs && count > 0) {
    if (!ctx->graph_ok) {
      const int rc = capture_generation(ctx);
      if (rc) return rc;
    }
    for (int32_t q = 0; q < count; ++q) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    return DABS_OK;
  }
  for (int32_t q = 0; q < count; ++q)
    for (int st = 0; st < 4; ++st) {
      const int rc = stage(ctx, st);
      if (rc) return rc;
    }
  return DABS_OK;
}

int dabs_set_graphs(dabs_ctx* ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return DABS_E_INVALID_ARG;
  ctx->graphs = enable;
  return DABS_OK;
}

int dabs_solve_status(dabs_ctx* ctx, uint64_t* flips, uint32_t* generations, int64_t* best_E,
                      int32_t* done) {
  if (!ctx) return DABS_E_INVALID_ARG;
  DevCtrl c;
  const int rc = read_ctrl(ctx, &c);
  if (rc) return rc;
  if (flips) *flips = c.flips_total;
  if (generations) *generations = c.g;
  if (best_E) *best_E = c.best_E;
  if (done) *done = (int32_t)c.done;
  return DABS_OK;
}

int dabs_solve_restarts(dabs_ctx* ctx, uint32_t* restarts) {
  if (!ctx || !restarts) return DABS_E_INVALID_ARG;
  DevCtrl c;
  const int rc = read_ctrl(ctx, &c);
  if (rc) return rc;
  *restarts = c.restarts;
  return DABS_OK;
}

int dabs_solve_best(dabs_ctx* ctx, uint8_t* best_X, int64_t* best_E) {
  if (!ctx) return DABS_E_INVALID_ARG;
  DevCtrl c;
  int rc = read_ctrl(ctx, &c);
  if (rc) return rc;
  if (best_X) {
    std::vector<uint32_t> packed(ctx->nw);
    CK(cudaMemcpy(packed.data(), ctx->gbestX, packed.size() * 4, cudaMemcpyDeviceToHost));
    for (int k = 0; k < ctx->n; ++k) best_X[k] = (uint8_t)((packed[k >> 5] >> (k & 31)) & 1u);
  }
  if (best_E) *best_E = c.best_E;
  return DABS_OK;
}

int dabs_solve(dabs_ctx* ctx, uint64_t budget, uint64_t seed, int64_t target, uint8_t* best_X,
               int64_t* best_E, uint64_t* flips) {
  if (!ctx) return DABS_E_INVALID_ARG;
  int rc = dabs_solve_begin(ctx, seed, budget, target);
  if (rc) return rc;
  int chunk = 1;
  for (;;) {
    rc = dabs_solve_generations(ctx, chunk);
    if (rc) return rc;
    int32_t done = 0;
    rc = dabs_solve_status(ctx, flips, nullptr, nullptr, &done);
    if (rc) return rc;
    if (done) break;
    if (chunk < 64) chunk <<= 1;
  }
  if ((rc = dabs_kernel_status(ctx))) return rc;  // a bounded device wait that ran out
  return dabs_solve_best(ctx, best_X, best_E);
}

int dabs_bulk_search_dev(dabs_ctx* ctx, uint64_t seed, uint32_t g, int32_t count, uint32_t* X,
                         int32_t* delta, int64_t* E, const uint32_t* D, const uint8_t* algo,
                         uint32_t* best_X, int64_t* best_E, uint32_t* flips) {
  if (!ctx || count < 0 || (count > 0 && (!X || !delta || !E || !D || !algo || !best_X || !best_E || !flips)))
    return DABS_E_INVALID_ARG;
  if (count == 0) return DABS_OK;
  DevCtrl c{};
  c.seed = seed;
  c.g = g;
  CK(cudaMemcpyAsync(ctx->bulk_ctrl, &c, sizeof c, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  SearchArgs a = solve_search_args(ctx);
  a.S = count;
  a.ctrl = ctx->bulk_ctrl;
  a.order = nullptr;
  if (count <= ctx->S) {
    k_order_by_algo<<<1, 1024, 0, ctx->stream>>>(algo, count, ctx->order, ctx->bulk_ctrl, 0, 0, 0);
    CKLAUNCH();
    a.order = ctx->order;
  }
  a.X = X; a.delta = delta; a.E = E; a.D = D; a.algo = algo;
  a.best_X = best_X; a.best_E = best_E; a.flips = flips;
  a.stall_test = ctx->stall_test;
  if (!launch_search(ctx->var.nw, ctx->var.ch, &a, ctx->stream, nullptr))
    return fail(ctx, DABS_E_INVALID_ARG, "no batch-search variant");
  ctx->stall_test = 0;  // the hook covers one launch
  CKLAUNCH();
  return DABS_OK;
}

int dabs_test_stall_next_search(dabs_ctx* ctx) {
  if (!ctx) return DABS_E_INVALID_ARG;
  if (ctx->var.ch != 0) return fail(ctx, DABS_E_INVALID_ARG, "the hook needs variant (1, 0)");
  ctx->stall_test = 1;
  return DABS_OK;
}

int dabs_info(const dabs_ctx* ctx, int32_t* n, int32_t* ld, int32_t* words, int32_t* searches,
              int32_t* pools, int32_t* pool_cap, int32_t* warps, int32_t* chunks) {
  if (!ctx) return DABS_E_INVALID_ARG;
  if (n) *n = ctx->n;
  if (ld) *ld = ctx->ld;
  if (words) *words = ctx->nw;
  if (searches) *searches = ctx->S;
  if (pools) *pools = ctx->P;
  if (pool_cap) *pool_cap = ctx->C;
  if (warps) *warps = ctx->var.nw;
  if (chunks) *chunks = ctx->var.ch;
  return DABS_OK;
}

int dabs_set_variant(dabs_ctx* ctx, int32_t warps, int32_t chunks) {
  if (!ctx) return DABS_E_INVALID_ARG;
  SearchVariant v;
  if (!launch_search(warps, chunks, nullptr, nullptr, &v))
    return fail(ctx, DABS_E_INVALID_ARG, "variant %d/%d not built", warps, chunks);
  if (v.cap < ctx->n) return fail(ctx, DABS_E_TOO_LARGE, "variant holds %d < n", v.cap);
  if (v.ch == 0 && !ctx->smem_ok)
    return fail(ctx, DABS_E_TOO_LARGE, "Delta range or size does not fit the shared-memory variant");
  ctx->var = v;
  ctx->var_set = true;
  if (!rows_ok(ctx, v, ctx->rows_mode)) ctx->rows_mode = ROWS_DENSE;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_set_rows(dabs_ctx* ctx, int32_t mode) {
  if (!ctx || mode < DABS_ROWS_DENSE || mode > DABS_ROWS_DENSE_SMEM) return DABS_E_INVALID_ARG;
  if (!rows_ok(ctx, ctx->var, mode))
    return fail(ctx, DABS_E_TOO_LARGE, "row format %d unavailable (%d stored entries)", mode, ctx->sp_nnz);
  ctx->rows_mode = mode;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_set_search_slots(dabs_ctx* ctx, int32_t modulus, int32_t lo, int32_t hi) {
  if (!ctx || modulus < 0 || (modulus > 0 && (lo < 0 || hi <= lo || hi > modulus)))
    return DABS_E_INVALID_ARG;
  ctx->slot_mod = modulus;
  ctx->slot_lo = modulus > 0 ? lo : 0;
  ctx->slot_hi = modulus > 0 ? hi : 0;
  int cnt = 0;
  for (int s = 0; s < ctx->S; ++s) cnt += modulus <= 0 || (s % modulus >= lo && s % modulus < hi);
  ctx->slot_count = cnt;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_set_keyed(dabs_ctx* ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return DABS_E_INVALID_ARG;
  ctx->keyed = enable;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_get_keyed(const dabs_ctx* ctx, int32_t* enabled, int32_t* key_bits) {
  if (!ctx) return DABS_E_INVALID_ARG;
  if (enabled) *enabled = ctx->keyed;
  if (key_bits) *key_bits = ctx->key_bits;
  return DABS_OK;
}

int dabs_get_rows(const dabs_ctx* ctx, int32_t* mode, int32_t* nnz) {
  if (!ctx) return DABS_E_INVALID_ARG;
  if (mode) *mode = ctx->rows_mode;
  if (nnz) *nnz = ctx->sp_nnz;
  return DABS_OK;
}

int dabs_autotune(dabs_ctx* ctx, int32_t generations, int32_t* warps, int32_t* chunks,
                  float* ns_per_flip, float* table) {
  if (!ctx || generations < 1) return DABS_E_INVALID_ARG;
  constexpr int NV = DABS_N_VARIANTS / 4;  // per RowFormat: dense, sparse shared, sparse global, dense shared
  static const int cand[NV][2] = {{1, 1}, {1, 2}, {1, 4}, {2, 1}, {2, 2}, {2, 4}, {4, 1}, {4, 2},
                                  {4, 4}, {8, 1}, {8, 2}, {8, 4}, {16, 1}, {16, 2}, {16, 4}, {1, 0}};
  if (table)
    for (int q = 0; q < DABS_N_VARIANTS; ++q) table[q] = 0.f;
  // warm a throwaway solve for `generations` generations, breed the next
  // targets, snapshot the search state, then time every variant's batch
  // search of that same generation from the same snapshot
  int rc = dabs_solve_begin(ctx, 0x5eed, UINT64_MAX, INT64_MIN);
  if (rc) return rc;
  if ((rc = dabs_solve_generations(ctx, generations))) return rc;
  if ((rc = stage(ctx, 0)) || (rc = stage(ctx, 4))) return rc;
  const size_t xb = (size_t)ctx->S * ctx->nw * 4, db = (size_t)ctx->S * ctx->ld * 4,
               eb = (size_t)ctx->S * 8;
  void* snap = nullptr;
  CK(cudaMalloc(&snap, xb + db + eb));
  unsigned char* sp = static_cast<unsigned char*>(snap);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const SearchVariant keep = ctx->var;
  const int keep_rows = ctx->rows_mode;
  SearchVariant best = keep;
  int best_rows = keep_rows;
  float best_ns = 0.f;
  do {
    if ((rc = cudaMemcpyAsync(sp, ctx->X, xb, cudaMemcpyDeviceToDevice, ctx->stream)) ||
        (rc = cudaMemcpyAsync(sp + xb, ctx->delta, db, cudaMemcpyDeviceToDevice, ctx->stream)) ||
        (rc = cudaMemcpyAsync(sp + xb + db, ctx->E, eb, cudaMemcpyDeviceToDevice, ctx->stream)) ||
        (rc = cudaEventCreate(&e0)) || (rc = cudaEventCreate(&e1))) {
      rc = fail(ctx, DABS_E_CUDA, "autotune set-up failed");
      break;
    }
    for (int ci = 0; ci < DABS_N_VARIANTS && !rc; ++ci) {
      SearchVariant v;
      const int rows = ci / NV;  // RowFormat
      if (!launch_search(cand[ci % NV][0], cand[ci % NV][1], nullptr, nullptr, &v) || v.cap < ctx->n)
        continue;
      if (v.ch == 0 && !ctx->smem_ok) continue;
      if (!rows_ok(ctx, v, rows)) continue;
      cudaMemcpyAsync(ctx->X, sp, xb, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->delta, sp + xb, db, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ctx->E, sp + xb + db, eb, cudaMemcpyDeviceToDevice, ctx->stream);
      ctx->rows_mode = rows;
      const SearchArgs a = solve_search_args(ctx);
      cudaEventRecord(e0, ctx->stream);
      launch_search(v.nw, v.ch, &a, ctx->stream, nullptr);
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        rc = fail(ctx, DABS_E_CUDA, "autotune launch failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      std::vector<uint32_t> fl(ctx->S);
      cudaMemcpy(fl.data(), ctx->flips, fl.size() * 4, cudaMemcpyDeviceToHost);
      double total = 0;
      for (uint32_t f : fl) total += f;
      const float ns = total > 0 ? (float)(ms * 1e6 / total) : 1e30f;
      if (table) table[ci] = ns;
      if (best_ns == 0.f || ns < best_ns) { best_ns = ns; best = v; best_rows = rows; }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(snap);
  if (rc != DABS_OK) { ctx->var = keep; ctx->rows_mode = keep_rows; return rc; }
  ctx->var = best;
  ctx->var_set = true;
  ctx->rows_mode = best_rows;
  graph_stale(ctx);
  if (warps) *warps = best.nw;
  if (chunks) *chunks = best.ch;
  if (ns_per_flip) *ns_per_flip = best_ns;
  return dabs_solve_begin(ctx, 0, UINT64_MAX, INT64_MIN);
}

int dabs_set_recompute(dabs_ctx* ctx, int32_t mode) {
  if (!ctx || (mode != 0 && mode != 1)) return DABS_E_INVALID_ARG;
  if (mode == 1) {
    const int rc = tc_setup(ctx);
    if (rc) return rc;
  }
  ctx->recompute_mode = mode;
  graph_stale(ctx);
  return DABS_OK;
}

int dabs_recompute_dev(dabs_ctx* ctx, const uint32_t* X, int32_t count, int64_t* E,
                       int32_t* delta, int32_t ld_delta) {
  if (!ctx || !X || !E || count < 0 || (delta && ld_delta < ctx->n)) return DABS_E_INVALID_ARG;
  int rc = tc_setup(ctx);
  if (rc) return rc;
  if (count > ctx->rows_pad)
    return fail(ctx, DABS_E_TOO_LARGE, "count %d > %d rows of the recompute buffer", count, ctx->rows_pad);
  if (count == 0) return DABS_OK;
  return tc_recompute(ctx, X, count, E, delta, ld_delta, nullptr);
}

int dabs_kernel_status(dabs_ctx* ctx) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int* flag : {ctx->kerr, ctx->serr}) {
    if (!flag) continue;
    int e = 0;
    CK(cudaMemcpy(&e, flag, sizeof e, cudaMemcpyDeviceToHost));
    if (e) {
      CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      return fail(ctx, DABS_E_TIMEOUT, "a device wait ran out (kernel error %d)", e);
    }
  }
  return DABS_OK;
}

int dabs_read_stats(dabs_ctx* ctx, uint64_t* algo_count, uint64_t* op_count, uint64_t* best_algo,
                    uint64_t* best_op) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long h[kStats];
  CK(cudaMemcpy(h, ctx->stats, sizeof h, cudaMemcpyDeviceToHost));
  for (int q = 0; q < N_ALGOS; ++q) {
    if (algo_count) algo_count[q] = h[q];
    if (best_algo) best_algo[q] = h[N_ALGOS + N_OPS + q];
  }
  for (int q = 0; q < N_OPS; ++q) {
    if (op_count) op_count[q] = h[N_ALGOS + q];
    if (best_op) best_op[q] = h[2 * N_ALGOS + N_OPS + q];
  }
  return DABS_OK;
}

// ---- checkpoint / restore: the whole device state of a solve at a
// generation boundary (pools, per-search state, global best, counters)
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, n, S, P, C, pad;
  dabs_params p;
  uint64_t w_hash, bytes;
};
struct Piece {
  void* ptr;
  size_t bytes;
};
std::vector<Piece> ckpt_pieces(dabs_ctx* c) {
  const size_t S = c->S, PC = (size_t)c->P * c->C, nw = c->nw, ld = c->ld;
  std::vector<Piece> v = {{c->ctrl, sizeof(DevCtrl)}, {c->X, S * nw * 4}, {c->delta, S * ld * 4},
                          {c->E, S * 8}, {c->D, S * nw * 4}, {c->bestX, S * nw * 4}, {c->bestE, S * 8},
                          {c->flips, S * 4}, {c->algo, S}, {c->op, S}, {c->gbestX, nw * 4},
                          {c->stats, sizeof(unsigned long long) * kStats}};
  for (int b = 0; b < 2; ++b) {
    v.push_back({c->poolX[b], PC * nw * 4});
    v.push_back({c->poolE[b], PC * 8});
    v.push_back({c->poolA[b], PC});
    v.push_back({c->poolO[b], PC});
  }
  return v;
}
}  // namespace

int dabs_checkpoint(dabs_ctx* ctx, void* buf, size_t cap, size_t* size) {
  if (!ctx || !size) return DABS_E_INVALID_ARG;
  const auto pieces = ckpt_pieces(ctx);
  size_t total = sizeof(CkptHeader);
  for (auto& q : pieces) total += q.bytes;
  *size = total;
  if (!buf) return DABS_OK;
  if (cap < total) return fail(ctx, DABS_E_INVALID_ARG, "checkpoint buffer of %zu < %zu bytes", cap, total);
  CK(cudaStreamSynchronize(ctx->stream));
  uint64_t wh = 0;
  if (const int rc = weights_hash(ctx, &wh)) return rc;
  CkptHeader h{};
  memcpy(h.magic, "DABSCKP1", 8);
  h.version = 2;
  h.n = ctx->n; h.S = ctx->S; h.P = ctx->P; h.C = ctx->C;
  h.p = ctx->p;
  h.w_hash = wh;
  h.bytes = total;
  unsigned char* o = static_cast<unsigned char*>(buf);
  memcpy(o, &h, sizeof h);
  o += sizeof h;
  for (auto& q : pieces) {
    CK(cudaMemcpy(o, q.ptr, q.bytes, cudaMemcpyDeviceToHost));
    o += q.bytes;
  }
  return DABS_OK;
}

int dabs_restore(dabs_ctx* ctx, const void* buf, size_t size) {
  if (!ctx || !buf || size < sizeof(CkptHeader)) return DABS_E_INVALID_ARG;
  CkptHeader h;
  memcpy(&h, buf, sizeof h);
  uint64_t wh = 0;
  if (const int rc = weights_hash(ctx, &wh)) return rc;
  if (memcmp(h.magic, "DABSCKP1", 8) != 0 || h.version != 2 || h.bytes != size || h.n != ctx->n ||
      h.S != ctx->S || h.P != ctx->P || h.C != ctx->C || h.w_hash != wh ||
      memcmp(&h.p, &ctx->p, sizeof h.p) != 0)
    return fail(ctx, DABS_E_INVALID_ARG, "checkpoint does not match this context");
  const auto pieces = ckpt_pieces(ctx);
  size_t total = sizeof h;
  for (auto& q : pieces) total += q.bytes;
  if (total != size) return fail(ctx, DABS_E_INVALID_ARG, "checkpoint size mismatch");
  CK(cudaStreamSynchronize(ctx->stream));
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof h;
  for (auto& q : pieces) {
    CK(cudaMemcpy(q.ptr, in, q.bytes, cudaMemcpyHostToDevice));
    in += q.bytes;
  }
  return DABS_OK;
}

static int cur_buf(dabs_ctx* ctx, int* b) {
  DevCtrl c;
  const int rc = read_ctrl(ctx, &c);
  if (rc) return rc;
  *b = (int)(c.g & 1u);
  return DABS_OK;
}

int dabs_read_pools(dabs_ctx* ctx, uint32_t* X, int64_t* E, uint8_t* algo, uint8_t* op) {
  if (!ctx) return DABS_E_INVALID_ARG;
  int b = 0, rc = cur_buf(ctx, &b);
  if (rc) return rc;
  const size_t PC = (size_t)ctx->P * ctx->C;
  if (X) CK(cudaMemcpy(X, ctx->poolX[b], PC * ctx->nw * 4, cudaMemcpyDeviceToHost));
  if (E) CK(cudaMemcpy(E, ctx->poolE[b], PC * 8, cudaMemcpyDeviceToHost));
  if (algo) CK(cudaMemcpy(algo, ctx->poolA[b], PC, cudaMemcpyDeviceToHost));
  if (op) CK(cudaMemcpy(op, ctx->poolO[b], PC, cudaMemcpyDeviceToHost));
  return DABS_OK;
}

int dabs_write_pools(dabs_ctx* ctx, const uint32_t* X, const int64_t* E, const uint8_t* algo,
                     const uint8_t* op) {
  if (!ctx || !X || !E || !algo || !op) return DABS_E_INVALID_ARG;
  int b = 0, rc = cur_buf(ctx, &b);
  if (rc) return rc;
  const size_t PC = (size_t)ctx->P * ctx->C;
  CK(cudaMemcpy(ctx->poolX[b], X, PC * ctx->nw * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->poolE[b], E, PC * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->poolA[b], algo, PC, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->poolO[b], op, PC, cudaMemcpyHostToDevice));
  return DABS_OK;
}

int dabs_read_state(dabs_ctx* ctx, uint32_t* X, int32_t* delta, int64_t* E) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t S = ctx->S;
  if (X) CK(cudaMemcpy(X, ctx->X, S * ctx->nw * 4, cudaMemcpyDeviceToHost));
  if (delta) CK(cudaMemcpy(delta, ctx->delta, S * ctx->ld * 4, cudaMemcpyDeviceToHost));
  if (E) CK(cudaMemcpy(E, ctx->E, S * 8, cudaMemcpyDeviceToHost));
  return DABS_OK;
}

int dabs_read_generation(dabs_ctx* ctx, uint32_t* D, uint8_t* algo, uint8_t* op, uint32_t* best_X,
                         int64_t* best_E, uint32_t* flips) {
  if (!ctx) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t S = ctx->S;
  if (D) CK(cudaMemcpy(D, ctx->D, S * ctx->nw * 4, cudaMemcpyDeviceToHost));
  if (algo) CK(cudaMemcpy(algo, ctx->algo, S, cudaMemcpyDeviceToHost));
  if (op) CK(cudaMemcpy(op, ctx->op, S, cudaMemcpyDeviceToHost));
  if (best_X) CK(cudaMemcpy(best_X, ctx->bestX, S * ctx->nw * 4, cudaMemcpyDeviceToHost));
  if (best_E) CK(cudaMemcpy(best_E, ctx->bestE, S * 8, cudaMemcpyDeviceToHost));
  if (flips) CK(cudaMemcpy(flips, ctx->flips, S * 4, cudaMemcpyDeviceToHost));
  return DABS_OK;
}

int dabs_write_results(dabs_ctx* ctx, const uint32_t* best_X, const int64_t* best_E,
                       const uint32_t* flips, const uint8_t* algo, const uint8_t* op) {
  if (!ctx || !best_X || !best_E || !flips || !algo || !op) return DABS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t S = ctx->S;
  CK(cudaMemcpy(ctx->bestX, best_X, S * ctx->nw * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->bestE, best_E, S * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->flips, flips, S * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->algo, algo, S, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->op, op, S, cudaMemcpyHostToDevice));
  return DABS_OK;
}

}  // extern "C"
