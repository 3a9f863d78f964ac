// batch.cu — batched uneven scenes in one persistent launch, CUDA-graph
// capture of that launch sequence, and the launch-shape autotuner.
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ctx_internal.h"

using namespace firert;

namespace {

fire_status_t cst(cudaError_t e) {
  if (e == cudaSuccess) return FIRE_OK;
  return e == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA;
}

#define BCK(call)                            \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cst(e_);   \
  } while (0)

// validate the scenes and fill the host descriptor table and prefix sums
fire_status_t build_items(const fire_ctx *c, const fire_batch_item_t *items, int n_items,
                          SceneItem *h_items, long long *h_prefix, long long *total) {
  long long tot = 0;
  for (int i = 0; i < n_items; i++) {
    const fire_batch_item_t &it = items[i];
    if (it.n_pix < 0) return FIRE_ERR_ARG;
    if (it.n_pix > 0 && (!it.radiance || !it.wv_bin)) return FIRE_ERR_ARG;
    SceneItem &s = h_items[i];
    s.rad = it.radiance;
    s.wv = it.wv_bin;
    s.n = it.n_pix;
    s.out.state = it.out.state;
    s.out.ET = it.out.ET;
    s.out.sdT = it.out.sdT;
    s.out.alpha = it.out.alpha;
    s.out.cov = it.out.cov;
    s.out.var_ET = it.out.var_ET;
    s.out.cost = it.out.cost;
    s.out.rms = it.out.rms;
    s.out.hfdi = it.out.hfdi;
    s.out.status = it.out.status;
    s.out.iters = it.out.iters;
    s.out.resid = it.out.resid_spec;
    h_prefix[i] = tot;
    tot += it.n_pix;
  }
  h_prefix[n_items] = tot;
  *total = tot;
  (void)c;
  return FIRE_OK;
}

int any_resid(const fire_batch_item_t *items, int n_items) {
  for (int i = 0; i < n_items; i++)
    if (items[i].out.resid_spec) return 1;
  return 0;
}

fire_status_t ensure_items(fire_ctx *c, int n_items) {
  if (n_items <= c->items_cap) return FIRE_OK;
  dev_free(c->d_items);
  dev_free(c->d_prefix);
  c->d_items = nullptr;
  c->d_prefix = nullptr;
  c->items_cap = 0;
  BCK(dev_malloc((void **)&c->d_items, sizeof(SceneItem) * n_items));
  BCK(dev_malloc((void **)&c->d_prefix, sizeof(long long) * (n_items + 1)));
  c->items_cap = n_items;
  return FIRE_OK;
}

}  // namespace

struct fire_graph {
  fire_ctx *ctx;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  SceneItem *h_items;       // pinned: the copy node's source
  long long *h_prefix;
  SceneItem *d_items;       // this graph's own descriptor table
  long long *d_prefix;
  // own hand-over scratch, claim counters, statistics and error word, so
  // that later calls on the context (which may regrow its scratch) leave the
  // captured pointers valid
  float *d_s1x, *d_s2x, *d_s2g;
  int *d_s1meta, *d_err;
  unsigned long long *d_work;
};

extern "C" {

fire_status_t fire_retrieve_batch(fire_ctx_t *c, const fire_batch_item_t *items, int32_t n_items,
                                  const fire_priors_t *pri, int32_t gate_mode,
                                  fire_stream_t stream) {
  if (!c || (n_items > 0 && !items) || n_items < 0) return FIRE_ERR_ARG;
  if (gate_mode != FIRE_FIT_ALL && gate_mode != FIRE_FIT_HFDI) return FIRE_ERR_ARG;
  if (n_items == 0) return FIRE_OK;
  fire_priors_t pd;
  if (!pri) {
    fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
    pri = &pd;
  }
  if (pri->init_mode != FIRE_INIT_DEFAULT) return FIRE_ERR_ARG;   // batched: default start only
  cudaStream_t st = (cudaStream_t)stream;
  SceneItem *h_items = new (std::nothrow) SceneItem[n_items];
  long long *h_prefix = new (std::nothrow) long long[n_items + 1];
  if (!h_items || !h_prefix) {
    delete[] h_items;
    delete[] h_prefix;
    return FIRE_ERR_NOMEM;
  }
  long long total = 0;
  fire_status_t e = build_items(c, items, n_items, h_items, h_prefix, &total);
  if (e == FIRE_OK) e = ensure_items(c, n_items);
  LMLaunch p;
  if (e == FIRE_OK) e = prepare_launch(c, pri, total, gate_mode == FIRE_FIT_HFDI, p);
  if (e == FIRE_OK) p.s.want_resid = any_resid(items, n_items);
  if (e == FIRE_OK) {
    // synchronous copies: the host tables are released before returning
    if (cudaMemcpyAsync(c->d_items, h_items, sizeof(SceneItem) * n_items, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->d_prefix, h_prefix, sizeof(long long) * (n_items + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      e = FIRE_ERR_CUDA;
  }
  delete[] h_items;
  delete[] h_prefix;
  if (e != FIRE_OK) return e;
  if (total == 0) return FIRE_OK;
  p.s.items = c->d_items;
  p.s.prefix = c->d_prefix;
  p.s.n_items = n_items;
  if (cudaMemsetAsync(c->d_work, 0, (size_t)(2 + ST_COUNT) * 8, st) != cudaSuccess) return FIRE_ERR_CUDA;
  return run_fit(c, p, false, st);
}

fire_status_t fire_graph_capture(fire_ctx_t *c, const fire_batch_item_t *items, int32_t n_items,
                                 const fire_priors_t *pri, int32_t gate_mode, fire_graph_t **out) {
  if (!out) return FIRE_ERR_ARG;
  *out = nullptr;
  if (!c || !items || n_items <= 0) return FIRE_ERR_ARG;
  if (gate_mode != FIRE_FIT_ALL && gate_mode != FIRE_FIT_HFDI) return FIRE_ERR_ARG;
  fire_priors_t pd;
  if (!pri) {
    fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
    pri = &pd;
  }
  if (pri->init_mode != FIRE_INIT_DEFAULT) return FIRE_ERR_ARG;
  fire_graph *g = new (std::nothrow) fire_graph();
  if (!g) return FIRE_ERR_NOMEM;
  memset(g, 0, sizeof(*g));
  g->ctx = c;
  fire_status_t e = FIRE_OK;
  long long total = 0;
  if (cudaMallocHost((void **)&g->h_items, sizeof(SceneItem) * n_items) != cudaSuccess ||
      cudaMallocHost((void **)&g->h_prefix, sizeof(long long) * (n_items + 1)) != cudaSuccess ||
      dev_malloc((void **)&g->d_items, sizeof(SceneItem) * n_items) != cudaSuccess ||
      dev_malloc((void **)&g->d_prefix, sizeof(long long) * (n_items + 1)) != cudaSuccess)
    e = FIRE_ERR_NOMEM;
  if (e == FIRE_OK) e = build_items(c, items, n_items, g->h_items, g->h_prefix, &total);
  const size_t nn = (size_t)(total > 0 ? total : 1);
  if (e == FIRE_OK &&
      (dev_malloc((void **)&g->d_s1x, nn * (c->t.K + 2) * 4) != cudaSuccess ||
       dev_malloc((void **)&g->d_s1meta, nn * 4) != cudaSuccess ||
       dev_malloc((void **)&g->d_s2x, nn * 32 * 4) != cudaSuccess ||
       dev_malloc((void **)&g->d_s2g, nn * 6 * 4) != cudaSuccess ||
       dev_malloc((void **)&g->d_work, (size_t)(2 + ST_COUNT) * 8) != cudaSuccess ||
       dev_malloc((void **)&g->d_err, sizeof(int)) != cudaSuccess))
    e = FIRE_ERR_NOMEM;
  LMLaunch p;
  if (e == FIRE_OK) e = prepare_launch(c, pri, total, gate_mode == FIRE_FIT_HFDI, p, false);
  if (e == FIRE_OK) {
    p.s.want_resid = any_resid(items, n_items);
    p.w.s1x = g->d_s1x;
    p.w.s1meta = g->d_s1meta;
    p.w.s2x = g->d_s2x;
    p.w.s2g = g->d_s2g;
    p.w.counter = g->d_work;
    p.w.stats = g->d_work + 2;
    p.w.err = g->d_err;
  }
  cudaStream_t cs = nullptr;
  if (e == FIRE_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) e = FIRE_ERR_CUDA;
  if (e == FIRE_OK) {
    p.s.items = g->d_items;
    p.s.prefix = g->d_prefix;
    p.s.n_items = n_items;
    int blocks = 0;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(g->d_items, g->h_items, sizeof(SceneItem) * n_items,
                                                cudaMemcpyHostToDevice, cs);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(g->d_prefix, g->h_prefix, sizeof(long long) * (n_items + 1),
                                                cudaMemcpyHostToDevice, cs);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_work, 0, (size_t)(2 + ST_COUNT) * 8, cs);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_err, 0, sizeof(int), cs);
    if (ce == cudaSuccess) ce = launch_lm(p, c->num_sms, cs, &blocks, c->tune_variant);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&g->exec, graph, 0);
    g->graph = graph;
    if (ce != cudaSuccess) e = cst(ce);
  }
  if (cs) cudaStreamDestroy(cs);
  if (e != FIRE_OK) {
    fire_graph_destroy(g);
    return e;
  }
  *out = g;
  return FIRE_OK;
}

fire_status_t fire_graph_launch(fire_graph_t *g, fire_stream_t stream) {
  if (!g || !g->exec) return FIRE_ERR_ARG;
  BCK(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return FIRE_OK;
}

void fire_graph_destroy(fire_graph_t *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFreeHost(g->h_items);
  cudaFreeHost(g->h_prefix);
  dev_free(g->d_items);
  dev_free(g->d_prefix);
  dev_free(g->d_s1x);
  dev_free(g->d_s1meta);
  dev_free(g->d_s2x);
  dev_free(g->d_s2g);
  dev_free(g->d_work);
  dev_free(g->d_err);
  delete g;
}

fire_status_t fire_autotune(fire_ctx_t *c, const float *radiance, const uint16_t *wv_bin, int64_t n,
                            fire_tune_t *best, fire_stream_t stream) {
  if (!c || !radiance || !wv_bin || n < 1) return FIRE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fire_priors_t pd;
  fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
  const int variants[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8}, claims[4] = {1, 2, 4, 8};
  cudaEvent_t a, b;
  BCK(cudaEventCreate(&a));
  BCK(cudaEventCreate(&b));
  float best_ms = 1e30f;
  int bv = c->tune_variant, bc = c->tune_claim;
  fire_status_t e = FIRE_OK;
  for (int vi = 0; vi < 9 && e == FIRE_OK; vi++)
    for (int ci = 0; ci < 4 && e == FIRE_OK; ci++) {
      c->tune_variant = variants[vi];
      c->tune_claim = claims[ci];
      LMLaunch p;
      e = prepare_launch(c, &pd, n, 0, p);
      if (e != FIRE_OK) break;
      p.s.rad = radiance;
      p.s.wv = wv_bin;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && e == FIRE_OK; rep++) {   // first run warms up
        if (cudaMemsetAsync(c->d_work, 0, (size_t)(2 + ST_COUNT) * 8, st) != cudaSuccess ||
            cudaEventRecord(a, st) != cudaSuccess) { e = FIRE_ERR_CUDA; break; }
        e = run_fit(c, p, false, st);
        if (e == FIRE_OK && (cudaEventRecord(b, st) != cudaSuccess ||
                             cudaEventSynchronize(b) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
          e = FIRE_ERR_CUDA;
      }
      if (e == FIRE_OK && ms < best_ms) {
        best_ms = ms;
        bv = variants[vi];
        bc = claims[ci];
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->tune_variant = bv;
  c->tune_claim = bc;
  if (best) {
    best->variant = bv;
    best->claim = bc;
    best->ms = best_ms;
  }
  return e;
}

fire_status_t fire_set_tuning(fire_ctx_t *c, int32_t variant, int32_t claim) {
  if (!c || variant < 0 || variant > 8 || claim < 1 || claim > 64) return FIRE_ERR_ARG;
  c->tune_variant = variant;
  c->tune_claim = claim;
  return FIRE_OK;
}

}  // extern "C"
