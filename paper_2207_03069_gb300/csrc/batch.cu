// batch.cu -- the batched and served forms of the solve.
//
// Batched: many contexts (instances of different n, each with its own pools,
// searches, seed, budget and target) advance generation by generation on one
// stream; their per-instance kernels (offspring, recompute, merge, finalise)
// are small, and all their batch searches run in one multi-instance launch
// per kernel variant, so the GPU is filled by the union of the instances.
// Every instance's result is the one dabs_solve gives it alone: its kernels
// read only its own buffers and its own control block.
//
// Served: a request queue admitted into contexts while an HBM budget allows
// (first come, first served), batched as above, with requests that arrive
// while others run admitted between rounds (continuous batching), and their
// contexts freed as they finish.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <deque>
#include <new>
#include <map>
#include <memory>
#include <vector>

#include "ctx.cuh"

using namespace dabs_internal;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int check(cudaError_t e) { return e == cudaSuccess ? DABS_OK : (e == cudaErrorMemoryAllocation ? DABS_E_OOM : DABS_E_CUDA); }

// Groups the active contexts by batch-search variant and keeps, per group, a
// device table of their SearchArgs and slot offsets.
struct Batcher {
  cudaStream_t stream = nullptr;
  bool own = false;
  struct Group {
    SearchVariant var{};
    std::vector<dabs_ctx*> ctxs;
    SearchArgs* d_insts = nullptr;
    int32_t* d_prefix = nullptr;
    int cap = 0;
    int total = 0;
  };
  std::vector<Group> groups;
  std::vector<dabs_ctx*> active;
  SearchArgs* h_insts = nullptr;  // pinned staging
  int32_t* h_prefix = nullptr;
  int h_cap = 0;
  // the groups' batch searches run concurrently, one side stream per group
  // after the first, forked from and joined back into `stream`
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;  // ev[0] fork, ev[1 + g] join of side stream g
  // the fused generation (every instance's offspring in one launch, the
  // recompute of all instances in one launch, the variant groups' searches,
  // every instance's merge and finalise in one launch), replayed from a CUDA
  // graph; used when no instance restarts its pools and every recompute runs
  // on the tensor cores
  bool fused = false;
  BatchInst* d_binst = nullptr;
  int32_t* d_post_prefix = nullptr;
  RecInst* d_rec = nullptr;
  int32_t* d_rec_prefix = nullptr;
  uint32_t* d_merged = nullptr;
  int fcap = 0;
  int nrec = 0, rec_ctas = 0, post_ctas = 0;
  size_t post_smem = 0;
  // the fused generation as three captured graphs (before the searches, the
  // searches, after them), so that the search phase can be timed by events
  // recorded on the stream between them
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
  bool use_graph = true;
  // measurement: kernels launched by generation() (all instances), and the
  // device time of the batch-search phase (fork to join) of each generation
  uint64_t search_launches = 0;
  std::vector<cudaEvent_t> t_ev;  // a (start, end) pair per generation since the last collect
  size_t t_used = 0;
  double search_ms = 0;

  ~Batcher() {
    if (stream) cudaStreamSynchronize(stream);
    for (cudaStream_t s : side) cudaStreamSynchronize(s);
    for (auto& g : groups) {
      cudaFree(g.d_insts);
      cudaFree(g.d_prefix);
    }
    for (cudaGraphExec_t& g : gexec)
      if (g) cudaGraphExecDestroy(g);
    cudaFree(d_binst);
    cudaFree(d_post_prefix);
    cudaFree(d_rec);
    cudaFree(d_rec_prefix);
    cudaFree(d_merged);
    if (h_insts) cudaFreeHost(h_insts);
    if (h_prefix) cudaFreeHost(h_prefix);
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : t_ev) cudaEventDestroy(e);
    if (own && stream) cudaStreamDestroy(stream);
  }

  // waits for the main stream and every side stream (also after a failed
  // generation, whose forked launches were never joined)
  int sync_all() {
    int rc = check(cudaStreamSynchronize(stream));
    for (cudaStream_t s : side) {
      const int r = check(cudaStreamSynchronize(s));
      if (!rc) rc = r;
    }
    return rc;
  }

  int ensure_side(size_t k) {
    if (ev.empty()) {
      cudaEvent_t e;
      int rc = check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      if (rc) return rc;
      ev.push_back(e);
    }
    while (side.size() < k) {
      cudaStream_t s;
      cudaEvent_t e;
      int rc = check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      if (rc) return rc;
      side.push_back(s);
      if ((rc = check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)))) return rc;
      ev.push_back(e);
    }
    return DABS_OK;
  }

  int init() {
    if (stream) return DABS_OK;
    own = true;
    return check(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
  }

  // rebuild the groups for `active` (contexts must use `stream`)
  int rebuild() {
    int rc = sync_all();
    if (rc) return rc;
    collect_search_time();
    std::vector<Group> ng;
    for (dabs_ctx* c : active) {
      const SearchVariant cv = batch_variant(c);
      Group* g = nullptr;
      for (auto& x : ng)
        if (x.var.nw == cv.nw && x.var.ch == cv.ch) g = &x;
      if (!g) {
        ng.push_back(Group{});
        g = &ng.back();
        g->var = cv;
      }
      g->ctxs.push_back(c);
    }
    // the most work first inside each launch too (longest-processing-time
    // order): its searches' CTAs are dispatched first, so the tail of the
    // launch is made of the shortest searches
    for (auto& g : ng)
      std::stable_sort(g.ctxs.begin(), g.ctxs.end(), [](const dabs_ctx* x, const dabs_ctx* y) {
        return (double)x->S * x->n * x->n > (double)y->S * y->n * y->n;
      });
    // reuse device tables
    for (size_t i = 0; i < ng.size(); ++i) {
      if (i < groups.size()) {
        ng[i].d_insts = groups[i].d_insts;
        ng[i].d_prefix = groups[i].d_prefix;
        ng[i].cap = groups[i].cap;
        groups[i].d_insts = nullptr;
        groups[i].d_prefix = nullptr;
      }
    }
    for (auto& g : groups) {
      cudaFree(g.d_insts);
      cudaFree(g.d_prefix);
    }
    // largest group first: its CTAs are dispatched first, and the smaller
    // groups' CTAs fill the SMs its tail leaves idle
    std::stable_sort(ng.begin(), ng.end(), [](const Group& x, const Group& y) {
      double wx = 0, wy = 0;
      for (const dabs_ctx* c : x.ctxs) wx += (double)c->S * c->n * c->n;
      for (const dabs_ctx* c : y.ctxs) wy += (double)c->S * c->n * c->n;
      return wx > wy;
    });
    groups.swap(ng);
    if (groups.size() > 1 && (rc = ensure_side(groups.size() - 1))) return rc;
    for (cudaGraphExec_t& g : gexec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    fused = !active.empty();
    for (const dabs_ctx* c : active)
      fused = fused && c->p.restart == 0 &&
              (c->p.seed_mode == 0 || (c->recompute_mode == 1 && c->tc_ready));
    if (fused && (rc = fused_tables())) return rc;
    int need = 1;
    for (auto& g : groups) need = std::max<int>(need, (int)g.ctxs.size());
    if (need > h_cap) {
      if (h_insts) cudaFreeHost(h_insts);
      if (h_prefix) cudaFreeHost(h_prefix);
      h_insts = nullptr;
      h_prefix = nullptr;
      if ((rc = check(cudaMallocHost(&h_insts, sizeof(SearchArgs) * need)))) return rc;
      if ((rc = check(cudaMallocHost(&h_prefix, sizeof(int32_t) * (need + 1))))) return rc;
      h_cap = need;
    }
    for (auto& g : groups) {
      const int k = (int)g.ctxs.size();
      if (k > g.cap) {
        cudaFree(g.d_insts);
        cudaFree(g.d_prefix);
        g.d_insts = nullptr;
        g.d_prefix = nullptr;
        if ((rc = check(cudaMalloc(&g.d_insts, sizeof(SearchArgs) * k)))) return rc;
        if ((rc = check(cudaMalloc(&g.d_prefix, sizeof(int32_t) * (k + 1))))) return rc;
        g.cap = k;
      }
      int acc = 0;
      for (int i = 0; i < k; ++i) {
        h_insts[i] = solve_search_args(g.ctxs[i]);
        if (fused && g.ctxs[i]->p.seed_mode == 1) h_insts[i].E2 = g.ctxs[i]->E2;
        h_prefix[i] = acc;
        acc += g.ctxs[i]->S;
      }
      h_prefix[k] = acc;
      g.total = acc;
      if ((rc = check(cudaMemcpyAsync(g.d_insts, h_insts, sizeof(SearchArgs) * k, cudaMemcpyHostToDevice, stream))))
        return rc;
      if ((rc = check(cudaMemcpyAsync(g.d_prefix, h_prefix, sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, stream))))
        return rc;
      // staging is reused by the next group: wait for these copies
      if ((rc = check(cudaStreamSynchronize(stream)))) return rc;
    }
    return DABS_OK;
  }

  // device tables of the fused generation for `active`
  int fused_tables() {
    int rc;
    const int k = (int)active.size();
    if (k > fcap) {
      cudaFree(d_binst);
      cudaFree(d_post_prefix);
      cudaFree(d_rec);
      cudaFree(d_rec_prefix);
      cudaFree(d_merged);
      d_binst = nullptr;
      d_post_prefix = d_rec_prefix = nullptr;
      d_rec = nullptr;
      d_merged = nullptr;
      fcap = 0;
      if ((rc = check(cudaMalloc(&d_binst, sizeof(BatchInst) * k)))) return rc;
      if ((rc = check(cudaMalloc(&d_post_prefix, sizeof(int32_t) * (k + 1))))) return rc;
      if ((rc = check(cudaMalloc(&d_rec, sizeof(RecInst) * k)))) return rc;
      if ((rc = check(cudaMalloc(&d_rec_prefix, sizeof(int32_t) * (k + 1))))) return rc;
      if ((rc = check(cudaMalloc(&d_merged, sizeof(uint32_t) * k)))) return rc;
      fcap = k;
    }
    std::vector<BatchInst> hb(k);
    std::vector<int32_t> hpp(k + 1), hrp(k + 1);
    std::vector<RecInst> hr;
    int acc = 0, racc = 0;
    post_smem = 0;
    for (int i = 0; i < k; ++i) {
      dabs_ctx* c = active[i];
      BatchInst& b = hb[i];
      b = BatchInst{};
      OffArgs& o = b.off;
      o.n = c->n; o.nw = c->nw; o.S = c->S; o.P = c->P; o.C = c->C; o.ctrl = c->ctrl;
      for (int q = 0; q < 2; ++q) { o.pool_X[q] = c->poolX[q]; o.pool_algo[q] = c->poolA[q]; o.pool_op[q] = c->poolO[q]; }
      o.D = c->D; o.algo = c->algo; o.op = c->op; o.abs_mode = c->p.abs_mode;
      MergeArgs& m = b.merge;
      m.nw = c->nw; m.S = c->S; m.P = c->P; m.C = c->C; m.Mmax = c->Mmax; m.ctrl = c->ctrl;
      for (int q = 0; q < 2; ++q) { m.pool_X[q] = c->poolX[q]; m.pool_E[q] = c->poolE[q]; m.pool_algo[q] = c->poolA[q]; m.pool_op[q] = c->poolO[q]; }
      m.best_X = c->bestX; m.best_E = c->bestE; m.algo = c->algo; m.op = c->op;
      b.fin = FinArgs{c->nw, c->S, c->ctrl, c->bestX, c->bestE, c->flips, c->gbestX,
                      c->algo, c->op, c->stats, nullptr};
      b.order = c->order;
      b.seed_mode = c->p.seed_mode;
      b.X = c->X;
      b.merged = d_merged + i;
      hpp[i] = acc;
      acc += c->P;
      post_smem = std::max(post_smem, c->merge_smem);
      if (c->p.seed_mode == 1) {
        b.A = c->Abf;
        b.rows_pad = c->rows_pad;
        b.n_pad = c->n_pad;
        b.one = c->tc_limbs_n == 1 ? 0x3C00u : 0x3F80u;
        b.E2 = c->E2;
        RecInst r{};
        r.mapA = c->mapA;
        r.mapHi = c->mapHi;
        r.mapLo = c->mapLo;
        r.a = UmmaArgs{c->S, c->n, c->n_pad, c->nw, c->ld, c->D, c->diag, c->delta, c->E2,
                       c->kerr, c->ctrl};
        r.limbs = c->tc_limbs_n;
        r.tiles_n = c->n_pad / umma_tile_n();
        hrp[hr.size()] = racc;
        racc += r.tiles_n * ((c->rows_pad + umma_tile_m() - 1) / umma_tile_m());
        hr.push_back(r);
      }
    }
    hpp[k] = acc;
    post_ctas = acc;
    nrec = (int)hr.size();
    hrp[nrec] = racc;
    rec_ctas = racc;
    if ((rc = check(cudaMemcpyAsync(d_binst, hb.data(), sizeof(BatchInst) * k, cudaMemcpyHostToDevice, stream))))
      return rc;
    if ((rc = check(cudaMemcpyAsync(d_post_prefix, hpp.data(), sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, stream))))
      return rc;
    if (nrec > 0) {
      if ((rc = check(cudaMemcpyAsync(d_rec, hr.data(), sizeof(RecInst) * nrec, cudaMemcpyHostToDevice, stream))))
        return rc;
      if ((rc = check(cudaMemcpyAsync(d_rec_prefix, hrp.data(), sizeof(int32_t) * (nrec + 1), cudaMemcpyHostToDevice, stream))))
        return rc;
    }
    if ((rc = check(cudaMemsetAsync(d_merged, 0, sizeof(uint32_t) * k, stream)))) return rc;
    if (post_smem > 48 * 1024 &&
        (rc = check(cudaFuncSetAttribute(k_gen_post, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)post_smem))))
      return rc;
    // the host vectors are freed on return: wait for the copies
    return check(cudaStreamSynchronize(stream));
  }

  // the variant groups' batch-search launches, concurrently on side streams
  int searches() {
    int rc;
    const size_t G = groups.size();
    if (G > 1 && (rc = check(cudaEventRecord(ev[0], stream)))) return rc;
    for (size_t gi = 0; gi < G; ++gi) {
      const Group& g = groups[gi];
      cudaStream_t st = gi == 0 ? stream : side[gi - 1];
      if (gi > 0 && (rc = check(cudaStreamWaitEvent(st, ev[0], 0)))) return rc;
      int32_t max_n = 0;
      for (const dabs_ctx* c : g.ctxs) max_n = std::max(max_n, (int32_t)c->n);
      const MultiArgs m{g.d_insts, g.d_prefix, (int32_t)g.ctxs.size(), g.total, max_n};
      const SearchArgs first = solve_search_args(g.ctxs[0]);
      if (!launch_search(g.var.nw, g.var.ch, &first, st, nullptr, &m)) return DABS_E_INVALID_ARG;
      if ((rc = check(cudaGetLastError()))) return rc;
      if (gi > 0 && (rc = check(cudaEventRecord(ev[gi], st)))) return rc;
    }
    for (size_t gi = 1; gi < G; ++gi)
      if ((rc = check(cudaStreamWaitEvent(stream, ev[gi], 0)))) return rc;
    return DABS_OK;
  }

  // the kernels of one part of the fused generation on `stream` (also used
  // for capture): 0 offspring and recompute, 1 the searches, 2 merge and
  // finalise
  int fused_part(int part) {
    int rc;
    if (part == 0) {
      k_gen_pre<<<(unsigned)active.size(), 1024, 0, stream>>>(d_binst);
      if ((rc = check(cudaGetLastError()))) return rc;
      if (nrec > 0) {
        launch_recompute_multi(d_rec, d_rec_prefix, nrec, rec_ctas, stream);
        if ((rc = check(cudaGetLastError()))) return rc;
      }
      return DABS_OK;
    }
    if (part == 1) return searches();
    k_gen_post<<<(unsigned)post_ctas, kMergeThreads, post_smem, stream>>>(d_binst, d_post_prefix,
                                                                         (int)active.size());
    return check(cudaGetLastError());
  }

  int capture(int part) {
    int rc = check(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    if (rc) return rc;
    rc = fused_part(part);
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(stream, &gr);
    if (!rc && e == cudaSuccess) rc = check(cudaGraphInstantiate(&gexec[part], gr, 0));
    else if (!rc) rc = check(e);
    if (gr) cudaGraphDestroy(gr);
    if (rc) {
      cudaGetLastError();
      gexec[part] = nullptr;
    }
    return rc;
  }

  int generation_fused() {
    int rc;
    for (int part = 0; part < 3 && use_graph; ++part)
      if (!gexec[part] && (rc = capture(part))) return rc;
    while (t_ev.size() < t_used + 2) {
      cudaEvent_t e;
      if ((rc = check(cudaEventCreate(&e)))) return rc;
      t_ev.push_back(e);
    }
    cudaEvent_t t0 = t_ev[t_used], t1 = t_ev[t_used + 1];
    t_used += 2;
    for (int part = 0; part < 3; ++part) {
      if (part == 1 && (rc = check(cudaEventRecord(t0, stream)))) return rc;
      rc = use_graph ? check(cudaGraphLaunch(gexec[part], stream)) : fused_part(part);
      if (rc) return rc;
      if (part == 1 && (rc = check(cudaEventRecord(t1, stream)))) return rc;
    }
    search_launches += groups.size();
    launches_fused += 2 + (nrec > 0 ? 1 : 0);
    return DABS_OK;
  }

  // adds the search phases timed since the last call (the stream must have
  // been synchronised)
  void collect_search_time() {
    for (size_t i = 0; i + 1 < t_used; i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, t_ev[i], t_ev[i + 1]) == cudaSuccess) search_ms += ms;
      else cudaGetLastError();  // a pair never recorded (a failed generation): no error left behind
    }
    t_used = 0;
  }

  uint64_t launches_fused = 0;  // the fused generation's non-search kernels

  // one generation of every active context
  int generation() {
    if (fused) return generation_fused();
    int rc;
    for (dabs_ctx* c : active)
      if ((rc = stage(c, 0)) || (rc = stage(c, 4))) return rc;
    const size_t G = groups.size();
    while (t_ev.size() < t_used + 2) {
      cudaEvent_t e;
      if ((rc = check(cudaEventCreate(&e)))) return rc;
      t_ev.push_back(e);
    }
    cudaEvent_t t0 = t_ev[t_used], t1 = t_ev[t_used + 1];
    t_used += 2;
    if ((rc = check(cudaEventRecord(t0, stream)))) return rc;
    if (G > 1 && (rc = check(cudaEventRecord(ev[0], stream)))) return rc;
    for (size_t gi = 0; gi < G; ++gi) {
      const Group& g = groups[gi];
      cudaStream_t st = gi == 0 ? stream : side[gi - 1];
      if (gi > 0 && (rc = check(cudaStreamWaitEvent(st, ev[0], 0)))) return rc;
      int32_t max_n = 0;
      for (const dabs_ctx* c : g.ctxs) max_n = std::max(max_n, (int32_t)c->n);
      const MultiArgs m{g.d_insts, g.d_prefix, (int32_t)g.ctxs.size(), g.total, max_n};
      const SearchArgs first = solve_search_args(g.ctxs[0]);
      if (!launch_search(g.var.nw, g.var.ch, &first, st, nullptr, &m)) return DABS_E_INVALID_ARG;
      if ((rc = check(cudaGetLastError()))) return rc;
      ++search_launches;
      if (gi > 0 && (rc = check(cudaEventRecord(ev[gi], st)))) return rc;
    }
    for (size_t gi = 1; gi < G; ++gi)
      if ((rc = check(cudaStreamWaitEvent(stream, ev[gi], 0)))) return rc;
    if ((rc = check(cudaEventRecord(t1, stream)))) return rc;
    for (dabs_ctx* c : active)
      if ((rc = stage(c, 2)) || (rc = stage(c, 3))) return rc;
    return DABS_OK;
  }
};

// all control blocks of `ctxs` in one round trip
int read_done(std::vector<dabs_ctx*>& ctxs, std::vector<DevCtrl>& out, cudaStream_t st) {
  out.resize(ctxs.size());
  for (size_t i = 0; i < ctxs.size(); ++i) {
    const int rc = check(cudaMemcpyAsync(ctxs[i]->h_ctrl, ctxs[i]->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, st));
    if (rc) return rc;
  }
  const int rc = check(cudaStreamSynchronize(st));
  if (rc) return rc;
  for (size_t i = 0; i < ctxs.size(); ++i) out[i] = *ctxs[i]->h_ctrl;
  return DABS_OK;
}

}  // namespace

// A batch: contexts advanced together generation by generation on one
// stream (the contexts' own streams are switched to it while the batch lives).
struct dabs_batch {
  Batcher b;
  std::vector<dabs_ctx*> all;
  std::vector<cudaStream_t> saved;
  std::vector<uint64_t> launches0;  // the contexts' launch counters at creation
  bool begun = false;
};

extern "C" int dabs_batch_create(dabs_ctx* const* ctxs, int32_t k, void* stream, dabs_batch** out) {
  if (!out || k < 1 || !ctxs) return DABS_E_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < k; ++i) {
    if (!ctxs[i]) return DABS_E_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return DABS_E_INVALID_ARG;  // one context at most once
  }
  dabs_batch* bt = new (std::nothrow) dabs_batch;
  if (!bt) return DABS_E_OOM;
  int rc = DABS_OK;
  if (stream) bt->b.stream = static_cast<cudaStream_t>(stream);
  else rc = bt->b.init();
  if (rc) {
    delete bt;
    return rc;
  }
  bt->all.assign(ctxs, ctxs + k);
  bt->saved.resize(k);
  for (int i = 0; i < k; ++i) bt->launches0.push_back(ctxs[i]->launches);
  for (int i = 0; i < k; ++i) {
    bt->saved[i] = ctxs[i]->stream;
    cudaStreamSynchronize(bt->saved[i]);
    ctxs[i]->stream = bt->b.stream;
    graph_stale(ctxs[i]);
  }
  *out = bt;
  return DABS_OK;
}

extern "C" void dabs_batch_destroy(dabs_batch* bt) {
  if (!bt) return;
  bt->b.sync_all();
  for (size_t i = 0; i < bt->all.size(); ++i) {
    bt->all[i]->stream = bt->saved[i];
    graph_stale(bt->all[i]);
  }
  delete bt;
}

extern "C" int dabs_batch_begin(dabs_batch* bt, const uint64_t* budgets, const uint64_t* seeds,
                                const int64_t* targets) {
  if (!bt || !budgets || !seeds) return DABS_E_INVALID_ARG;
  int rc = bt->b.sync_all();
  for (size_t i = 0; i < bt->all.size() && !rc; ++i)
    rc = dabs_solve_begin(bt->all[i], seeds[i], budgets[i], targets ? targets[i] : INT64_MIN);
  if (rc) return rc;
  bt->b.active = bt->all;
  rc = bt->b.rebuild();
  bt->begun = rc == DABS_OK;
  return rc;
}

extern "C" int dabs_batch_generations(dabs_batch* bt, int32_t count, int32_t* running) {
  if (!bt || count < 0) return DABS_E_INVALID_ARG;
  if (!bt->begun) return DABS_E_INVALID_ARG;
  int rc = DABS_OK;
  if (!bt->b.active.empty() && count > 0) {
    for (int q = 0; q < count && !rc; ++q) rc = bt->b.generation();
    std::vector<DevCtrl> cs;
    if (!rc) rc = read_done(bt->b.active, cs, bt->b.stream);
    if (!rc) bt->b.collect_search_time();
    if (!rc) {
      std::vector<dabs_ctx*> still;
      for (size_t i = 0; i < bt->b.active.size(); ++i)
        if (!cs[i].done) still.push_back(bt->b.active[i]);
      if (still.size() != bt->b.active.size()) {
        bt->b.active.swap(still);
        if (!bt->b.active.empty()) rc = bt->b.rebuild();
      }
    }
  }
  if (running) *running = (int32_t)bt->b.active.size();
  return rc;
}

extern "C" int dabs_batch_info(dabs_batch* bt, int32_t* running, int32_t* search_groups,
                               uint64_t* launches, double* search_ms) {
  if (!bt) return DABS_E_INVALID_ARG;
  const int rc = bt->b.sync_all();
  if (rc) return rc;
  bt->b.collect_search_time();
  uint64_t l = bt->b.search_launches + bt->b.launches_fused;
  for (size_t i = 0; i < bt->all.size(); ++i) l += bt->all[i]->launches - bt->launches0[i];
  if (running) *running = (int32_t)bt->b.active.size();
  if (search_groups) *search_groups = (int32_t)bt->b.groups.size();
  if (launches) *launches = l;
  if (search_ms) *search_ms = bt->b.search_ms;
  return DABS_OK;
}

extern "C" int dabs_batch_solve(dabs_ctx* const* ctxs, int32_t k, const uint64_t* budgets,
                                const uint64_t* seeds, const int64_t* targets,
                                uint8_t* const* best_X, int64_t* best_E, uint64_t* flips) {
  if (k < 0 || (k > 0 && (!ctxs || !budgets || !seeds))) return DABS_E_INVALID_ARG;
  for (int i = 0; i < k; ++i)
    if (!ctxs[i]) return DABS_E_INVALID_ARG;
  if (k == 0) return DABS_OK;
  dabs_batch* bt = nullptr;
  int rc = dabs_batch_create(ctxs, k, nullptr, &bt);
  if (rc) return rc;
  rc = dabs_batch_begin(bt, budgets, seeds, targets);
  int chunk = 1, running = k;
  while (!rc && running > 0) {
    rc = dabs_batch_generations(bt, chunk, &running);
    if (chunk < 16) chunk <<= 1;
  }
  for (int i = 0; i < k && !rc; ++i) {
    rc = dabs_kernel_status(ctxs[i]);  // a bounded device wait that ran out
    if (!rc && (best_X || best_E))
      rc = dabs_solve_best(ctxs[i], best_X ? best_X[i] : nullptr, best_E ? &best_E[i] : nullptr);
    if (!rc && flips) rc = dabs_solve_status(ctxs[i], &flips[i], nullptr, nullptr, nullptr);
  }
  dabs_batch_destroy(bt);
  return rc;
}

// ------------------------------------------------------------------ server
namespace {

struct Request {
  uint64_t ticket = 0;
  std::vector<int16_t> W;
  int32_t n = 0;
  dabs_params p{};
  uint64_t budget = 0, seed = 0;
  int64_t target = INT64_MIN;
  size_t bytes = 0;
  int64_t warps = 0;  // resident warps of its batch searches (searches x warps per search)
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, < 0 failed (error code)
  dabs_ctx* ctx = nullptr;
  std::vector<uint8_t> best_X;
  int64_t best_E = INT64_MAX;
  uint64_t flips = 0;
};

// device bytes a context for (n, p) allocates (dabs_create's buffers)
size_t ctx_bytes(int32_t n, const dabs_params& p) {
  const size_t ld = (size_t)(n + 63) / 64 * 64, nw = (size_t)(n + 31) / 32;
  const size_t S = (size_t)p.searches, PC = (size_t)p.pools * p.pool_cap;
  size_t b = 2 * (size_t)n * ld * 2 + (size_t)n * 4;                 // W, -W, diag
  b += 2 * PC * (nw * 4 + 8 + 2);                                    // pools
  b += S * (3 * nw * 4 + ld * 4 + 8 + 2 + 8 + 4 + 4);                // search state, results
  if (p.seed_mode == 1) {                                             // tensor recompute
    const size_t np = (size_t)(n + 127) / 128 * 128, rows = (S + 127) / 128 * 128;
    b += 2 * np * np * 2 + rows * np * 2 + rows * 8;
  }
  return b + 64 * 1024;
}

}  // namespace

// A size class of requests advanced together: its own batcher (and stream),
// the requests it runs, those admitted while its generation was in flight,
// and that generation's end event (after the copies of the control blocks).
// Small and large requests sit in different classes, so the small ones are
// not held at the pace of the largest one's generations: the classes' rounds
// overlap on the GPU.
struct ServeClass {
  Batcher batch;
  std::vector<Request*> running;  // in batch.active order
  std::vector<Request*> joining;
  bool dirty = false, inflight = false;
  cudaEvent_t ev = nullptr;
};

constexpr int kServeClasses = 3;
int serve_class(int32_t n) { return n <= 2048 ? 0 : (n <= 4096 ? 1 : 2); }

struct dabs_server {
  size_t budget = 0, used = 0;  // device bytes of running and idle contexts
  int64_t max_warps = 0, running_warps = 0;
  uint64_t next = 1;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  ServeClass cls[kServeClasses];
  // contexts of finished requests, kept for the next request of the same n
  // and parameters (a new W is loaded into them); freed when the budget needs
  // their bytes, so that a retirement does not wait on the device
  struct Idle {
    dabs_ctx* ctx;
    size_t bytes;
  };
  std::deque<Idle> idle;
};

extern "C" int dabs_server_create(size_t hbm_budget_bytes, dabs_server** out) {
  if (!out || hbm_budget_bytes == 0) return DABS_E_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DABS_E_NO_DEVICE;
  dabs_server* s = new (std::nothrow) dabs_server;
  if (!s) return DABS_E_OOM;
  s->budget = hbm_budget_bytes;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  s->max_warps = 2LL * 32 * (sms > 0 ? sms : 152);  // about two full waves of warps
  for (ServeClass& c : s->cls) {
    int rc = c.batch.init();
    if (!rc) rc = check(cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming));
    if (rc) {
      dabs_server_destroy(s);
      return rc;
    }
  }
  *out = s;
  return DABS_OK;
}

extern "C" void dabs_server_destroy(dabs_server* s) {
  if (!s) return;
  for (ServeClass& c : s->cls) c.batch.sync_all();
  for (auto& kv : s->all)
    if (kv.second->ctx) dabs_destroy(kv.second->ctx);
  for (auto& i : s->idle) dabs_destroy(i.ctx);
  for (ServeClass& c : s->cls)
    if (c.ev) cudaEventDestroy(c.ev);
  delete s;
}

extern "C" int dabs_server_submit(dabs_server* s, const int16_t* W, int32_t n, const dabs_params* p,
                                  uint64_t budget, uint64_t seed, int64_t target, uint64_t* ticket) {
  if (!s || !W || !p || !ticket || n < 1) return DABS_E_INVALID_ARG;
  if (n > DABS_N_MAX) return DABS_E_TOO_LARGE;
  auto r = std::make_unique<Request>();
  r->ticket = s->next++;
  r->W.assign(W, W + (size_t)n * n);
  r->n = n;
  r->p = *p;
  r->budget = budget;
  r->seed = seed;
  r->target = target;
  r->bytes = ctx_bytes(n, *p);
  if (r->bytes > s->budget) return DABS_E_TOO_LARGE;
  {
    SearchVariant v{};  // the variant its batch searches will run with
    r->warps = (int64_t)p->searches * (default_variant(n, &v, true) ? v.nw : 1);
  }
  r->t_submit = now_s();
  *ticket = r->ticket;
  s->queue.push_back(r.get());
  s->all[r->ticket] = std::move(r);
  return DABS_OK;
}

namespace {

bool same_params(const dabs_params& a, const dabs_params& b) {
  return std::memcmp(&a, &b, sizeof(dabs_params)) == 0;
}

// retires the finished requests of every class whose generation has ended
// (wait: block until one has); returns how many classes ended
int serve_collect(dabs_server* s, bool wait, int* ended) {
  *ended = 0;
  for (;;) {
    for (ServeClass& c : s->cls) {
      if (!c.inflight) continue;
      const cudaError_t q = cudaEventQuery(c.ev);
      if (q == cudaErrorNotReady) continue;
      int rc = check(q);
      if (rc) return rc;
      c.inflight = false;
      ++*ended;
      c.batch.collect_search_time();
      std::vector<Request*> still;
      for (Request* r : c.running) {
        dabs_ctx* x = r->ctx;
        if (!x->h_ctrl->done) {  // copied after the generation
          still.push_back(r);
          continue;
        }
        const uint64_t flips = x->h_ctrl->flips_total;
        r->best_X.resize(r->n);
        x->stream = x->own;
        rc = dabs_solve_best(x, r->best_X.data(), &r->best_E);
        r->flips = flips;
        r->t_done = now_s();
        r->state = rc ? rc : 2;
        r->ctx = nullptr;
        s->idle.push_back({x, r->bytes});
        s->running_warps -= r->warps;
        r->W.clear();
        r->W.shrink_to_fit();
        c.dirty = true;
      }
      c.running.swap(still);
    }
    if (*ended || !wait) return DABS_OK;
    bool any = false;
    for (ServeClass& c : s->cls) any = any || c.inflight;
    if (!any) return DABS_OK;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// admits queued requests, first come first served, while their bytes fit the
// budget (idle contexts freed oldest first to make room) and the warp cap
// holds; a context of the same n and parameters is reused
int serve_admit(dabs_server* s) {
  for (;;) {
    if (s->queue.empty()) return DABS_OK;
    Request* r = s->queue.front();
    int nrun = 0;
    for (ServeClass& c : s->cls) nrun += (int)(c.running.size() + c.joining.size());
    if (nrun > 0 && s->max_warps > 0 && s->running_warps + r->warps > s->max_warps) return DABS_OK;
    // a reusable context: its bytes are already counted
    dabs_ctx* x = nullptr;
    for (size_t i = 0; i < s->idle.size(); ++i)
      if (s->idle[i].ctx->n == r->n && same_params(s->idle[i].ctx->p, r->p)) {
        x = s->idle[i].ctx;
        s->idle.erase(s->idle.begin() + (long)i);
        break;
      }
    if (!x) {
      while (s->used + r->bytes > s->budget && !s->idle.empty()) {
        dabs_destroy(s->idle.front().ctx);
        s->used -= s->idle.front().bytes;
        s->idle.pop_front();
      }
      if (s->used + r->bytes > s->budget) return DABS_OK;
    }
    s->queue.pop_front();
    int rc;
    if (x) {
      rc = dabs_load_weights(x, r->W.data());
      if (rc) {
        dabs_destroy(x);
        s->used -= r->bytes;
        x = nullptr;
      }
    }
    if (!x) {
      rc = dabs_create(r->W.data(), r->n, &r->p, &x);
      if (rc) {
        r->state = rc;
        r->t_done = now_s();
        continue;
      }
      s->used += r->bytes;
    }
    // the solve starts on the context's own stream; then it joins its class
    rc = dabs_solve_begin(x, r->seed, r->budget, r->target);
    if (!rc) rc = check(cudaStreamSynchronize(x->own));
    if (rc) {
      r->state = rc;
      r->t_done = now_s();
      s->idle.push_back({x, r->bytes});
      continue;
    }
    ServeClass& c = s->cls[serve_class(r->n)];
    x->stream = c.batch.stream;
    r->ctx = x;
    r->state = 1;
    r->t_start = now_s();
    s->running_warps += r->warps;
    c.joining.push_back(r);
  }
}

// starts `generations` generations in every class with work and none in flight
int serve_launch(dabs_server* s, int generations) {
  int rc;
  for (ServeClass& c : s->cls) {
    if (c.inflight) continue;
    if (!c.joining.empty()) {
      c.running.insert(c.running.end(), c.joining.begin(), c.joining.end());
      c.joining.clear();
      c.dirty = true;
    }
    if (c.running.empty()) continue;
    if (c.dirty) {
      c.batch.active.clear();
      for (Request* r : c.running) c.batch.active.push_back(r->ctx);
      if ((rc = c.batch.rebuild())) return rc;
      c.dirty = false;
    }
    for (int q = 0; q < generations; ++q)
      if ((rc = c.batch.generation())) return rc;
    for (Request* r : c.running)
      if ((rc = check(cudaMemcpyAsync(r->ctx->h_ctrl, r->ctx->ctrl, sizeof(DevCtrl),
                                      cudaMemcpyDeviceToHost, c.batch.stream))))
        return rc;
    if ((rc = check(cudaEventRecord(c.ev, c.batch.stream)))) return rc;
    c.inflight = true;
  }
  return DABS_OK;
}

}  // namespace

// One scheduling step: retire the requests of every class whose round has
// ended, admit queued requests, and start a round of `generations`
// generations in every class with work and no round in flight.  When no
// round had ended, the step first waits for one, so every call advances the
// solve; rounds of different classes overlap on the device.  *pending
// receives the number of queued plus running requests.
extern "C" int dabs_server_step(dabs_server* s, int32_t generations, int32_t* pending) {
  if (!s || generations < 1) return DABS_E_INVALID_ARG;
  int ended = 0, rc;
  if ((rc = serve_collect(s, false, &ended))) return rc;
  if ((rc = serve_admit(s))) return rc;
  if ((rc = serve_launch(s, generations))) return rc;
  if (!ended) {
    if ((rc = serve_collect(s, true, &ended))) return rc;
    if ((rc = serve_admit(s))) return rc;
    if ((rc = serve_launch(s, generations))) return rc;
  }
  if (pending) {
    size_t p = s->queue.size();
    for (ServeClass& c : s->cls) p += c.running.size() + c.joining.size();
    *pending = (int32_t)p;
  }
  return DABS_OK;
}

// status: 0 queued, 1 running, 2 done (outputs written), < 0 failed
extern "C" int dabs_server_poll(dabs_server* s, uint64_t ticket, uint8_t* best_X, int64_t* best_E,
                                uint64_t* flips, double* latency_s, int32_t* status) {
  if (!s) return DABS_E_INVALID_ARG;
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return DABS_E_INVALID_ARG;
  Request* r = it->second.get();
  if (status) *status = r->state;
  if (r->state == 2) {
    if (best_X) std::copy(r->best_X.begin(), r->best_X.end(), best_X);
    if (best_E) *best_E = r->best_E;
    if (flips) *flips = r->flips;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
  }
  return DABS_OK;
}

extern "C" int dabs_server_set_limits(dabs_server* s, int64_t max_warps) {
  if (!s || max_warps < 0) return DABS_E_INVALID_ARG;
  s->max_warps = max_warps;
  return DABS_OK;
}

extern "C" int dabs_server_info(const dabs_server* s, size_t* used_bytes, int32_t* queued,
                                int32_t* running) {
  if (!s) return DABS_E_INVALID_ARG;
  if (used_bytes) *used_bytes = s->used;
  if (queued) *queued = (int32_t)s->queue.size();
  if (running) {
    size_t r = 0;
    for (const ServeClass& c : s->cls) r += c.running.size() + c.joining.size();
    *running = (int32_t)r;
  }
  return DABS_OK;
}
