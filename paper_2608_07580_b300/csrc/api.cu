// api.cu — the C ABI (include/firert.h): argument validation, context and
// device-memory management, host staging and kernel launches. No retrieval
// arithmetic runs on the host: tables, forward model and fits are kernels.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/firert.h"
#include "internal.cuh"
#include "mlp_internal.h"

using namespace firert;

#include "ctx_internal.h"


namespace {

fire_status_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FIRE_OK;
  if (e == cudaErrorMemoryAllocation) return FIRE_ERR_NOMEM;
  return FIRE_ERR_CUDA;
}

#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// contiguous band range [lo, lo + n) whose centres fall in [wlo, whi]
// (or in the union of two intervals); n = 0 if none
void band_range(const float *wl, int nb, float a_lo, float a_hi, float b_lo, float b_hi,
                int *lo, int *n) {
  int first = -1, last = -1;
  for (int b = 0; b < nb; b++) {
    bool in = (wl[b] >= a_lo && wl[b] <= a_hi) || (wl[b] >= b_lo && wl[b] <= b_hi);
    if (in) {
      if (first < 0) first = b;
      last = b;
    }
  }
  *lo = first < 0 ? 0 : first;
  *n = first < 0 ? 0 : last - first + 1;
}

int nearest_band(const float *wl, int nb, float lam) {
  int best = 0;
  for (int b = 1; b < nb; b++)
    if (fabsf(wl[b] - lam) < fabsf(wl[best] - lam)) best = b;
  return best;
}

static_assert(kSolverLM == FIRE_SOLVER_LM && kSolverAdam == FIRE_SOLVER_ADAM,
              "kernel solver codes follow the public ones");

void fill_kconfig(KConfig &k, const fire_config_t &c, const fire_priors_t &p, int K, int nb) {
  memset(&k, 0, sizeof(k));
  for (int i = 0; i < K + 2; i++) {
    k.lo1[i] = p.lo1[i];
    k.hi1[i] = p.hi1[i];
    k.pm1[i] = p.pm1[i];
    k.pp1[i] = p.pp1[i];
  }
  for (int i = 0; i < 6; i++) {
    k.lo2[i] = p.lo2[i];
    k.hi2[i] = p.hi2[i];
    k.pm2[i] = p.pm2[i];
    k.pp2[i] = p.pp2[i];
  }
  for (int i = 0; i < K + 2; i++) k.zk1[i] = k.hi1[i] > k.lo1[i] ? 2.f / (k.hi1[i] - k.lo1[i]) : 0.f;
  for (int i = 0; i < 6; i++) k.zk2[i] = k.hi2[i] > k.lo2[i] ? 2.f / (k.hi2[i] - k.lo2[i]) : 0.f;
  k.init_alpha1 = p.init_alpha1;
  k.init_T1 = p.init_T1;
  k.init_sigma = p.init_sigma;
  k.init_mu_h_floor = p.init_mu_h_floor;
  k.init_mu_s_ceil = p.init_mu_s_ceil;
  k.init_eta_lo = p.init_eta_lo;
  k.init_eta_hi = p.init_eta_hi;
  k.max_it1 = c.max_it1;
  k.max_it2 = c.max_it2;
  k.tau0 = c.tau0;
  k.tol_g = c.tol_g;
  k.tol_x = c.tol_x;
  k.tol_f = c.tol_f;
  k.kappa_max = c.kappa_max;
  k.dfloor = c.dfloor;
  k.noise_rel = c.noise_rel;
  k.noise_abs = c.noise_abs;
  k.weighted = c.weighted || p.noise_sd ? 1 : 0;
  k.hfdi_thresh = c.hfdi_thresh;
  k.ident_sd_et = c.ident_sd_et;
  k.ident_alpha_snr = c.ident_alpha_snr;
  k.wait_spins = c.wait_spins > 0 ? (long long)c.wait_spins : (1ll << 26);
  k.has_nsd = p.noise_sd ? 1 : 0;
  if (p.noise_sd)
    for (int b = 0; b < nb && b < kMaxBands; b++) k.nsd[b] = p.noise_sd[b];
  k.solver = c.solver;
  k.adam_steps1 = c.adam_steps1;
  k.adam_steps2 = c.adam_steps2;
  k.adam_lr1 = (float)c.adam_lr1;
  k.adam_lr2 = (float)c.adam_lr2;
  k.adam_clip = (float)c.adam_clip;
  k.adam_eps = (float)c.adam_eps;
  k.adam_b1 = (float)c.adam_beta1;
  k.adam_b2 = (float)c.adam_beta2;
  k.adam_omb1 = (float)(1.0 - c.adam_beta1);   // 1 - 0.999f would be off by 1.3e-5
  k.adam_omb2 = (float)(1.0 - c.adam_beta2);
  k.adam_b1d = c.adam_beta1;
  k.adam_b2d = c.adam_beta2;
  if (c.solver == FIRE_SOLVER_ADAM) {
    // the paper's Adam minimises Eq. (loss) as printed: no prior term
    for (int i = 0; i < kMaxK + 2; i++) k.pp1[i] = 0.f;
    for (int i = 0; i < 6; i++) k.pp2[i] = 0.f;
  }
}


template <class T>
fire_status_t dev_alloc(T **p, size_t bytes) {
  cudaError_t e = dev_malloc((void **)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA;
  }
  return FIRE_OK;
}

fire_status_t ensure_s1(fire_ctx *c, int64_t n) {
  if (n <= c->s1_cap) return FIRE_OK;
  dev_free(c->d_s1x);
  dev_free(c->d_s1meta);
  dev_free(c->d_s2x);
  dev_free(c->d_s2g);
  c->d_s1x = nullptr;
  c->d_s1meta = nullptr;
  c->d_s2x = c->d_s2g = nullptr;
  c->s1_cap = 0;
  fire_status_t e = dev_alloc(&c->d_s1x, (size_t)n * (c->t.K + 2) * 4);
  if (e == FIRE_OK) e = dev_alloc(&c->d_s1meta, (size_t)n * 4);
  if (e == FIRE_OK) e = dev_alloc(&c->d_s2x, (size_t)n * 32 * 4);
  if (e == FIRE_OK) e = dev_alloc(&c->d_s2g, (size_t)n * 6 * 4);
  if (e == FIRE_OK) c->s1_cap = n;
  return e;
}

// carve per-pixel output arrays for n pixels out of one buffer (the
// residual spectrum [n][nb] only when nb > 0)
size_t outputs_bytes(int64_t n, int K, int nb = 0) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t szf = (size_t)n * 4;
  return al(szf * (K + 8)) + 7 * al(szf) + al(szf * 21) + al((size_t)n) + al((size_t)n * 4) +
         al(szf * nb);
}
KOut carve_outputs(void *buf, int64_t n, int K, int nb = 0) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t szf = (size_t)n * 4;
  char *q = (char *)buf;
  auto carve = [&](size_t b) { char *r = q; q += al(b); return r; };
  KOut o;
  o.state = (float *)carve(szf * (K + 8));
  o.ET = (float *)carve(szf);
  o.sdT = (float *)carve(szf);
  o.alpha = (float *)carve(szf);
  o.var_ET = (float *)carve(szf);
  o.cost = (float *)carve(szf);
  o.rms = (float *)carve(szf);
  o.hfdi = (float *)carve(szf);
  o.cov = (float *)carve(szf * 21);
  o.status = (uint8_t *)carve((size_t)n);
  o.iters = (uint16_t *)carve((size_t)n * 4);
  o.resid = nb > 0 ? (float *)carve(szf * nb) : nullptr;
  return o;
}

}  // namespace

namespace firert {

bool priors_valid(const fire_priors_t &p, int K) {
  for (int i = 0; i < K; i++)
    if (p.lo1[i] != 0.f || p.hi1[i] != 1.f) return false;  // fractions live on [0, 1]
  for (int i = 0; i < K + 2; i++)
    if (!(p.hi1[i] >= p.lo1[i]) || !(p.pp1[i] >= 0.f)) return false;
  for (int i = 0; i < 6; i++)
    if (!(p.hi2[i] >= p.lo2[i]) || !(p.pp2[i] >= 0.f)) return false;
  if (!(p.lo1[K + 1] > 0.f) || !(p.lo2[1] > 0.f) || !(p.lo2[3] > 0.f)) return false;  // T, sigma > 0
  if (p.init_mode != FIRE_INIT_DEFAULT && p.init_mode != FIRE_INIT_GIVEN &&
      p.init_mode != FIRE_INIT_MLP)
    return false;
  return true;
}

bool noise_sd_valid(const fire_priors_t &p, int nb) {
  if (!p.noise_sd) return true;
  for (int b = 0; b < nb; b++)
    if (!(p.noise_sd[b] > 0.f) || !isfinite(p.noise_sd[b])) return false;
  return true;
}

}  // namespace firert

namespace firert {

// The fit of p (device pointers set), with the learned start when asked:
// network inference -> LM from those starts -> default-start re-fit of the
// pixels the fallback rule flags -> keep the lower cost.
cudaEvent_t *timing_events(fire_ctx *c) {
  if (!c->timing) return nullptr;
  while (c->tev.size() < c->tev_used + 4) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->tev.push_back(e);
  }
  cudaEvent_t *ev = c->tev.data() + c->tev_used;
  c->tev_used += 4;
  return ev;
}

fire_status_t run_fit(fire_ctx *c, LMLaunch &p, bool learned, cudaStream_t st) {
  int blocks = 0;
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  if (!learned) {
    CK(launch_lm(p, c->num_sms, st, &blocks, c->tune_variant, timing_events(c)));
    c->last_launches = 3;
    return FIRE_OK;
  }
  const int64_t n = p.s.n_pix;
  const int K = c->t.K;
  if (n > c->mlp_cap) {
    dev_free(c->d_mlp_init);
    dev_free(c->d_fb_idx);
    dev_free(c->d_fb_cost);
    c->d_mlp_init = nullptr;
    c->d_fb_idx = nullptr;
    c->d_fb_cost = nullptr;
    c->mlp_cap = 0;
    fire_status_t e = dev_alloc(&c->d_mlp_init, (size_t)n * (K + 8) * 4);
    if (e == FIRE_OK) e = dev_alloc(&c->d_fb_idx, (size_t)n * 8);
    if (e == FIRE_OK) e = dev_alloc(&c->d_fb_cost, (size_t)n * 4);
    if (e == FIRE_OK && !c->d_fb_count) e = dev_alloc(&c->d_fb_count, 8);
    if (e != FIRE_OK) return e;
    c->mlp_cap = n;
  }
  fire_status_t e = fire_mlp_infer(c->mlp, p.s.rad, n, nullptr, c->d_mlp_init, (fire_stream_t)st);
  if (e != FIRE_OK) return e;
  CK(cudaMemsetAsync(c->d_fb_count, 0, 8, st));
  p.s.init = c->d_mlp_init;
  p.s.init_best = 1;
  p.w.fb_idx = c->d_fb_idx;
  p.w.fb_cost = c->d_fb_cost;
  p.w.fb_count = c->d_fb_count;
  CK(launch_lm(p, c->num_sms, st, &blocks, c->tune_variant, timing_events(c)));
  unsigned long long nfb = 0;
  CK(cudaMemcpyAsync(&nfb, c->d_fb_count, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  c->last_launches = 3 + 6;   // network (inference kernels) + fit
  if (nfb == 0) return FIRE_OK;
  if ((int64_t)nfb > c->cmp_cap) {
    dev_free(c->d_cmp);
    c->d_cmp = nullptr;
    c->cmp_cap = 0;
    e = dev_alloc((char **)&c->d_cmp, outputs_bytes((int64_t)nfb, K, c->t.nb));
    if (e != FIRE_OK) return e;
    c->cmp_cap = (int64_t)nfb;
  }
  KOut cmp = carve_outputs(c->d_cmp, (int64_t)nfb, K, p.o.resid ? c->t.nb : 0);
  LMLaunch q = p;
  q.s.n_pix = (int64_t)nfb;
  q.s.idx = c->d_fb_idx;
  q.s.init = nullptr;
  q.s.init_best = 0;
  q.w.fb_idx = nullptr;
  q.w.fb_cost = nullptr;
  q.w.fb_count = nullptr;
  q.o = cmp;
  q.o.hfdi = nullptr;
  CK(cudaMemsetAsync(c->d_work, 0, 2 * 8, st));   // claim counters only; stats accumulate
  CK(launch_lm(q, c->num_sms, st, &blocks, c->tune_variant));
  CK(launch_merge_fallback(c->d_fb_idx, c->d_fb_cost, (long long)nfb, cmp, p.o, K, c->t.nb, st));
  c->last_launches += 4;
  return FIRE_OK;
}

// common launch set-up of a fit over n pixels (tables, constants, scratch)
fire_status_t prepare_launch(fire_ctx *c, const fire_priors_t *pri, int64_t n, int gate, LMLaunch &p,
                             bool ctx_scratch) {
  memset(&p, 0, sizeof(p));
  if (!priors_valid(*pri, c->t.K) || !noise_sd_valid(*pri, c->t.nb)) return FIRE_ERR_ARG;
  p.t = c->t;
  fill_kconfig(p.c, c->cfg, *pri, c->t.K, c->t.nb);
  p.s.n_pix = n;
  p.s.gate = gate;
  p.s.claim = c->tune_claim;
  p.w.counter = c->d_work;
  p.w.stats = c->d_work + 2;
  p.w.err = c->d_err;
  if (!ctx_scratch) return FIRE_OK;
  fire_status_t e = ensure_s1(c, n);
  if (e != FIRE_OK) return e;
  p.w.s1x = c->d_s1x;
  p.w.s1meta = c->d_s1meta;
  p.w.s2x = c->d_s2x;
  p.w.s2g = c->d_s2g;
  return FIRE_OK;
}

}  // namespace firert


extern "C" {

fire_status_t fire_ctx_set_mlp(fire_ctx_t *c, fire_mlp_t *m) {
  if (!c) return FIRE_ERR_ARG;
  c->mlp = m;
  return FIRE_OK;
}

void fire_default_config(fire_config_t *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->win1_lo = 350.f;   // Omega_1 (Sec. 2.6)
  c->win1_hi = 2500.f;
  c->win2h_lo = 900.f;  // Omega_2^hot, Omega_2^smol (Sec. 2.3)
  c->win2h_hi = 1800.f;
  c->win2s_lo = 1500.f;
  c->win2s_hi = 2500.f;
  c->max_it1 = 100;
  // 1.5 x the FP64 oracle's 400: the FP32 normal matrix resolves the flat
  // directions of the near-degenerate mixture to ~1e-5 of its diagonal, so in
  // those valleys this path takes more steps to meet the same convergence
  // tests (at 400 it ended ~0.05 % of the fire pixels the oracle converges at
  // the cap)
  c->max_it2 = 600;
  c->tau0 = 1.f;
  c->tol_g = 1e-8f;
  c->tol_x = 1e-7f;
  c->tol_f = 1e-10f;
  c->kappa_max = 1e6f;
  c->dfloor = 1e-12f;
  c->noise_rel = 0.005f;
  c->noise_abs = 1e-4f;
  c->weighted = 0;
  c->hfdi_thresh = -0.1f;  // Sec. 2.1
  c->hfdi_lambda_hi = 2430.f;
  c->hfdi_lambda_lo = 2061.f;
  c->ident_sd_et = 100.f;
  c->ident_alpha_snr = 3.f;
  c->solver = FIRE_SOLVER_LM;
  c->adam_steps1 = 30;      // Sec. 2.6: 30 steps at 0.03, then 100 at 0.015
  c->adam_steps2 = 100;
  c->adam_lr1 = 0.03;
  c->adam_lr2 = 0.015;
  c->adam_clip = 1.0;
  c->adam_beta1 = 0.9;      // Eq. (adam) defaults
  c->adam_beta2 = 0.999;
  c->adam_eps = 1e-8;
}

void fire_default_priors(fire_priors_t *p, int32_t K, int32_t nt, float tlo, float thi) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  if (K < 1 || K > FIRE_MAX_ENDM || nt < 2) return;
  float dT = (thi - tlo) / (float)(nt - 1);
  for (int k = 0; k < K; k++) {
    p->lo1[k] = 0.f;
    p->hi1[k] = 1.f;
  }
  p->lo1[K] = 0.f;      // alpha1
  p->hi1[K] = 1.f;
  p->lo1[K + 1] = tlo;  // T1 on the temperature grid
  p->hi1[K + 1] = thi;
  // weak prior in z: alpha towards 0 at 1e-6 (it only regularises J^T J
  // where alpha vanishes); T1 and the mixture shape towards the box centre
  // at 1 (the regulariser of the near-degenerate mixture)
  p->pm1[K] = -1.f;
  p->pp1[K] = 1e-6f;
  p->pm1[K + 1] = 0.f;
  p->pp1[K + 1] = 1.f;
  const float lo2[6] = {900.f, dT, tlo, dT, 0.f, 0.f};
  const float hi2[6] = {thi, 500.f, 1000.f, 500.f, 1.f, 1.f};
  for (int i = 0; i < 6; i++) {
    p->lo2[i] = lo2[i];
    p->hi2[i] = hi2[i];
    p->pm2[i] = i == 5 ? -1.f : 0.f;
    p->pp2[i] = i == 5 ? 1e-6f : 1.f;
  }
  p->init_alpha1 = 0.f;   // no fire until the data say so (the prior's mean for alpha)
  p->init_T1 = 800.f;
  p->init_sigma = 100.f;
  p->init_mu_h_floor = 1000.f;
  p->init_mu_s_ceil = 700.f;
  p->init_eta_lo = 0.05f;
  p->init_eta_hi = 0.95f;
  p->init_mode = FIRE_INIT_DEFAULT;
  p->init_state = nullptr;
}

// the status a fit reports for its device error word: 1 from a bounded wait
// that gave up, 0x100 | site from a failed index check (FIRERT_DEBUG)
static fire_status_t err_status(int err) {
  if (!err) return FIRE_OK;
  return (err & kErrBounds) ? FIRE_ERR_BOUNDS : FIRE_ERR_TIMEOUT;
}

int32_t fire_build_flags(void) {
#ifdef FIRERT_DEBUG
  return 1;
#else
  return 0;
#endif
}

fire_status_t fire_debug_word(fire_ctx_t *c, int32_t *word) {
  if (!c || !word) return FIRE_ERR_ARG;
  CK(cudaDeviceSynchronize());
  int err = 0;
  CK(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  *word = err;
  return FIRE_OK;
}

const char *fire_status_str(fire_status_t s) {
  switch (s) {
    case FIRE_OK: return "ok";
    case FIRE_ERR_ARG: return "invalid argument";
    case FIRE_ERR_CUDA: return "CUDA error";
    case FIRE_ERR_NOMEM: return "out of memory";
    case FIRE_ERR_SHAPE: return "unsupported shape";
    case FIRE_ERR_TIMEOUT: return "device wait timed out";
    case FIRE_ERR_CHECKPOINT: return "bad checkpoint";
    case FIRE_ERR_STATE: return "invalid state";
    case FIRE_ERR_BOUNDS: return "index check failed (bounds-checked build)";
  }
  return "unknown status";
}

void fire_ctx_destroy(fire_ctx_t *ctx) {
  if (!ctx) return;
  for (cudaEvent_t e : ctx->chunk_ev) cudaEventDestroy(e);
  if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
  if (ctx->fit_st2) cudaStreamDestroy(ctx->fit_st2);
  dev_free(ctx->d_ctr);
  dev_free(ctx->d_image);
  dev_free(ctx->d_planck_full);
  dev_free(ctx->d_planck64);
  dev_free(ctx->d_plop);
  dev_free(ctx->d_wvtab);
  dev_free(ctx->d_wl);
  dev_free(ctx->d_sat);
  dev_free(ctx->d_work);
  dev_free(ctx->d_err);
  dev_free(ctx->d_stage);
  dev_free(ctx->d_s1x);
  dev_free(ctx->d_s1meta);
  dev_free(ctx->d_s2x);
  dev_free(ctx->d_s2g);
  dev_free(ctx->d_mlp_init);
  dev_free(ctx->d_fb_idx);
  dev_free(ctx->d_fb_cost);
  dev_free(ctx->d_fb_count);
  dev_free(ctx->d_cmp);
  dev_free(ctx->d_items);
  dev_free(ctx->d_prefix);
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  delete ctx;
}

fire_status_t fire_ctx_create(fire_ctx_t **out, const fire_tables_t *tb, const fire_config_t *cfg) {
  if (!out) return FIRE_ERR_ARG;
  *out = nullptr;
  if (!tb || !tb->wavelength_nm || !tb->solar_irr || !tb->tau_down || !tb->tau_up ||
      !tb->endmembers)
    return FIRE_ERR_ARG;
  const int nb = tb->n_bands, K = tb->n_endm, nt = tb->n_tgrid, nwv = tb->n_wv;
  if (nb < 8 || nb > FIRE_MAX_BANDS || K < 1 || K > FIRE_MAX_ENDM || nt < 2 ||
      nt > FIRE_MAX_TGRID || nwv < 1 || nwv > FIRE_MAX_WV)
    return FIRE_ERR_SHAPE;
  if (K != 3 && K != 5) return FIRE_ERR_SHAPE;  // compiled kernel variants
  if (!(tb->tgrid_hi > tb->tgrid_lo) || !(tb->tgrid_lo > 0.f) || !(tb->cos_sza > 0.f))
    return FIRE_ERR_ARG;
  for (int b = 1; b < nb; b++)
    if (!(tb->wavelength_nm[b] > tb->wavelength_nm[b - 1])) return FIRE_ERR_ARG;
  if (cfg && (cfg->solver < FIRE_SOLVER_LM || cfg->solver > FIRE_SOLVER_ADAM ||
              (cfg->solver == FIRE_SOLVER_ADAM &&
               (cfg->adam_steps1 < 0 || cfg->adam_steps2 < 0 || cfg->adam_steps1 > 65535 ||
                cfg->adam_steps2 > 65535 || !(cfg->adam_lr1 >= 0.0) || !(cfg->adam_lr2 >= 0.0) ||
                !(cfg->adam_clip > 0.0) || !(cfg->adam_beta1 >= 0.0 && cfg->adam_beta1 < 1.0) ||
                !(cfg->adam_beta2 >= 0.0 && cfg->adam_beta2 < 1.0) || !(cfg->adam_eps > 0.0)))))
    return FIRE_ERR_ARG;
  fire_ctx *c = new (std::nothrow) fire_ctx();
  if (!c) return FIRE_ERR_NOMEM;
  if (cfg) c->cfg = *cfg;
  else fire_default_config(&c->cfg);
  // host copies for the water-vapour presolve's depth table
  c->h_wl.assign(tb->wavelength_nm, tb->wavelength_nm + nb);
  c->h_e0.assign(tb->solar_irr, tb->solar_irr + nb);
  c->h_td.assign(tb->tau_down, tb->tau_down + (size_t)nwv * nb);
  c->h_tu.assign(tb->tau_up, tb->tau_up + (size_t)nwv * nb);
  c->h_cos = tb->cos_sza;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

  KTables &t = c->t;
  memset(&t, 0, sizeof(t));
  t.nb = nb;
  t.nwv = nwv;
  t.K = K;
  t.nt = nt;
  t.tglo = tb->tgrid_lo;
  t.tgstep = (tb->tgrid_hi - tb->tgrid_lo) / (float)(nt - 1);
  const fire_config_t &cf = c->cfg;
  band_range(tb->wavelength_nm, nb, cf.win1_lo, cf.win1_hi, cf.win1_lo, cf.win1_hi, &t.b1lo, &t.n1);
  band_range(tb->wavelength_nm, nb, cf.win2h_lo, cf.win2h_hi, cf.win2s_lo, cf.win2s_hi, &t.b2lo,
             &t.n2);
  if (t.n1 < K + 3 || t.n2 < 7 || t.n1 > 512 || t.n2 > 512) {
    delete c;
    return FIRE_ERR_SHAPE;
  }
  t.bh = nearest_band(tb->wavelength_nm, nb, cf.hfdi_lambda_hi);
  t.bl = nearest_band(tb->wavelength_nm, nb, cf.hfdi_lambda_lo);
  ImageLayout &L = t.lay;
  int o = 0;
  auto take = [&](int n) { int r = o; o += (n + 3) & ~3; return r; };
  L.off_c2l = take(nb);
  L.off_c1l5 = take(nb);
  L.off_endm = take(K * nb);
  L.off_win1 = take(nb);
  L.off_win2 = take(nb);
  L.n2s = (t.n2 + 31) & ~31;
  L.off_planck = take(nt * L.n2s);
  L.total = o;
  t.plrows = (t.n2 + 7) & ~7;
  if (lm_smem_bytes(t) > 200 * 1024) {
    delete c;
    return FIRE_ERR_SHAPE;
  }

  // upload raw tables, build the device tables with a kernel
  fire_status_t st = FIRE_OK;
  float *raw = nullptr;
  size_t nraw = (size_t)nb * 2 + (size_t)nwv * nb * 4 + (size_t)K * nb;
  do {
    if ((st = dev_alloc(&c->d_image, (size_t)L.total * 4)) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_planck_full, (size_t)nt * nb * 4)) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_planck64, (size_t)nt * t.n2 * 8)) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_plop, planck_operand_bytes(t))) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_wvtab, (size_t)nwv * nb * sizeof(float4))) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_work, (size_t)(2 + ST_COUNT) * 8)) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_err, sizeof(int))) != FIRE_OK) break;
    if ((st = cuda_status(cudaMemset(c->d_err, 0, sizeof(int)))) != FIRE_OK) break;
    if ((st = dev_alloc(&raw, nraw * 4)) != FIRE_OK) break;
    if ((st = dev_alloc(&c->d_wl, (size_t)nb * 4)) != FIRE_OK) break;
    if ((st = cuda_status(cudaMemcpy(c->d_wl, tb->wavelength_nm, nb * 4, cudaMemcpyHostToDevice))) != FIRE_OK)
      break;
    if (tb->sat_level) {
      if ((st = dev_alloc(&c->d_sat, (size_t)nb * 4)) != FIRE_OK) break;
      if ((st = cuda_status(cudaMemcpy(c->d_sat, tb->sat_level, nb * 4, cudaMemcpyHostToDevice))) != FIRE_OK) break;
    }
    float *d_wl = raw, *d_e0 = raw + nb, *d_td = d_e0 + nb, *d_tu = d_td + (size_t)nwv * nb;
    float *d_ra = d_tu + (size_t)nwv * nb, *d_sa = d_ra + (size_t)nwv * nb;
    float *d_en = d_sa + (size_t)nwv * nb;
    size_t wb = (size_t)nwv * nb * 4;
    cudaMemcpy(d_wl, tb->wavelength_nm, nb * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d_e0, tb->solar_irr, nb * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d_td, tb->tau_down, wb, cudaMemcpyHostToDevice);
    cudaMemcpy(d_tu, tb->tau_up, wb, cudaMemcpyHostToDevice);
    if (tb->rho_atm) cudaMemcpy(d_ra, tb->rho_atm, wb, cudaMemcpyHostToDevice);
    else cudaMemset(d_ra, 0, wb);
    if (tb->sph_alb) cudaMemcpy(d_sa, tb->sph_alb, wb, cudaMemcpyHostToDevice);
    else cudaMemset(d_sa, 0, wb);
    cudaMemcpy(d_en, tb->endmembers, (size_t)K * nb * 4, cudaMemcpyHostToDevice);
    t.image = c->d_image;
    t.wvtab = c->d_wvtab;
    t.sat = c->d_sat;
    const float win[6] = {cf.win1_lo, cf.win1_hi, cf.win2h_lo, cf.win2h_hi, cf.win2s_lo, cf.win2s_hi};
    if ((st = cuda_status(launch_build_tables(t, d_wl, d_e0, tb->cos_sza, d_td, d_tu, d_ra, d_sa,
                                              d_en, c->d_image, c->d_wvtab, win, 0))) != FIRE_OK)
      break;
    if ((st = cuda_status(launch_planck_operand(t, c->d_plop, 0))) != FIRE_OK) break;
    t.plop = c->d_plop;
    if ((st = cuda_status(launch_planck_full(t, d_wl, c->d_planck_full, 0))) != FIRE_OK) break;
    t.planck_full = c->d_planck_full;
    if ((st = cuda_status(launch_planck64(t, d_wl, c->d_planck64, 0))) != FIRE_OK) break;
    t.planck64 = c->d_planck64;
    // the tensor-core stage 2 where the tables fit it
    c->tune_variant = lm_tc_ok(t) ? 6 : 3;
    st = cuda_status(cudaDeviceSynchronize());
  } while (0);
  if (raw) dev_free(raw);
  if (st != FIRE_OK) {
    fire_ctx_destroy(c);
    return st;
  }
  *out = c;
  return FIRE_OK;
}

}  // extern "C"

void fire_ctx_tables(const fire_ctx_t *c, KTables *t, KConfig *k) {
  *t = c->t;
  fire_priors_t p;
  fire_default_priors(&p, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
  fill_kconfig(*k, c->cfg, p, c->t.K, c->t.nb);
}

extern "C" {

fire_status_t fire_window_bands(fire_ctx_t *c, int32_t *b1lo, int32_t *n1, int32_t *b2lo,
                                int32_t *n2) {
  if (!c) return FIRE_ERR_ARG;
  if (b1lo) *b1lo = c->t.b1lo;
  if (n1) *n1 = c->t.n1;
  if (b2lo) *b2lo = c->t.b2lo;
  if (n2) *n2 = c->t.n2;
  return FIRE_OK;
}

// host scenes of at least two minimum chunks are fitted in chunks whose
// copies overlap the fits of the others: a small first chunk (its copy is
// the only one nothing overlaps), larger middle ones, and a small last one
// (its outputs are the only ones copied back after the last fit); sixteenths
// of the scene, no chunk under kChunkMin pixels
static constexpr int64_t kChunkMin = 65536;
static constexpr int kChunks = 5;
static constexpr int kChunkSixteenths[kChunks] = {1, 3, 5, 5, 2};

fire_status_t fire_retrieve(fire_ctx_t *c, const fire_scene_t *sc, const fire_priors_t *pri,
                            const fire_outputs_t *out, fire_stream_t stream) {
  if (!c || !sc || !out) return FIRE_ERR_ARG;
  if (sc->n_pix < 0) return FIRE_ERR_ARG;
  if (sc->mem != FIRE_MEM_DEVICE && sc->mem != FIRE_MEM_HOST) return FIRE_ERR_ARG;
  if (sc->gate_mode != FIRE_FIT_ALL && sc->gate_mode != FIRE_FIT_HFDI) return FIRE_ERR_ARG;
  fire_priors_t pd;
  if (!pri) {
    fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
    pri = &pd;
  }
  if (!priors_valid(*pri, c->t.K)) return FIRE_ERR_ARG;
  if (pri->init_mode == FIRE_INIT_GIVEN && !pri->init_state) return FIRE_ERR_ARG;
  if (pri->init_mode == FIRE_INIT_MLP && !c->mlp) return FIRE_ERR_STATE;
  const bool learned = pri->init_mode == FIRE_INIT_MLP;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(c->d_work, 0, (size_t)(2 + ST_COUNT) * 8, st));
  c->last_launches = 0;
  if (sc->n_pix == 0) return FIRE_OK;
  if (!sc->radiance || !sc->wv_bin) return FIRE_ERR_ARG;
  const int64_t n = sc->n_pix;
  const int K = c->t.K, NS = K + 8;

  LMLaunch p;
  {
    fire_status_t e = prepare_launch(c, pri, n, sc->gate_mode == FIRE_FIT_HFDI, p);
    if (e != FIRE_OK) return e;
  }

  // per-pixel output sizes (bytes), in the order staged for host scenes
  const size_t szf = (size_t)n * 4;
  const size_t s_state = szf * NS, s_cov = szf * 21, s_u8 = (size_t)n, s_it = (size_t)n * 4;
  if (sc->mem == FIRE_MEM_DEVICE) {
    p.s.rad = sc->radiance;
    p.s.wv = sc->wv_bin;
    p.s.init = pri->init_mode == FIRE_INIT_GIVEN ? pri->init_state : nullptr;
    p.o.state = out->state;
    p.o.ET = out->ET;
    p.o.sdT = out->sdT;
    p.o.alpha = out->alpha;
    p.o.cov = out->cov;
    p.o.var_ET = out->var_ET;
    p.o.cost = out->cost;
    p.o.rms = out->rms;
    p.o.hfdi = out->hfdi;
    p.o.status = out->status;
    p.o.iters = out->iters;
    p.o.resid = out->resid_spec;
    p.s.want_resid = out->resid_spec != nullptr;
    return run_fit(c, p, learned, st);
  }

  // host scene: stage inputs and outputs through one device buffer
  const size_t s_rad = (size_t)n * c->t.nb * 4, s_wv = (size_t)n * 2;
  const size_t s_init = pri->init_mode == FIRE_INIT_GIVEN ? szf * NS : 0;
  const size_t s_res = out->resid_spec ? s_rad : 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t need = al(s_rad) + al(s_wv) + al(s_init) + al(s_state) + 7 * al(szf) + al(s_cov) +
                al(s_u8) + al(s_it) + al(s_res);
  if (need > c->stage_bytes) {
    dev_free(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    fire_status_t e = dev_alloc((char **)&c->d_stage, need);
    if (e != FIRE_OK) return e;
    c->stage_bytes = need;
  }
  char *q = (char *)c->d_stage;
  auto carve = [&](size_t b) { char *r = q; q += al(b); return r; };
  float *d_rad = (float *)carve(s_rad);
  uint16_t *d_wv = (uint16_t *)carve(s_wv);
  float *d_init = s_init ? (float *)carve(s_init) : nullptr;
  float *o_state = (float *)carve(s_state), *o_ET = (float *)carve(szf), *o_sdT = (float *)carve(szf);
  float *o_alpha = (float *)carve(szf), *o_var = (float *)carve(szf), *o_cost = (float *)carve(szf);
  float *o_rms = (float *)carve(szf), *o_hfdi = (float *)carve(szf), *o_cov = (float *)carve(s_cov);
  uint8_t *o_status = (uint8_t *)carve(s_u8);
  uint16_t *o_it = (uint16_t *)carve(s_it);
  float *o_res = s_res ? (float *)carve(s_res) : nullptr;
  p.s.rad = d_rad;
  p.s.wv = d_wv;
  p.s.init = d_init;
  p.o.state = out->state ? o_state : nullptr;
  p.o.ET = out->ET ? o_ET : nullptr;
  p.o.sdT = out->sdT ? o_sdT : nullptr;
  p.o.alpha = out->alpha ? o_alpha : nullptr;
  p.o.var_ET = out->var_ET ? o_var : nullptr;
  p.o.cost = out->cost ? o_cost : nullptr;
  p.o.rms = out->rms ? o_rms : nullptr;
  p.o.hfdi = out->hfdi ? o_hfdi : nullptr;
  p.o.cov = out->cov ? o_cov : nullptr;
  p.o.status = out->status ? o_status : nullptr;
  p.o.iters = out->iters ? o_it : nullptr;
  p.o.resid = o_res;
  p.s.want_resid = o_res != nullptr;
  if (learned) {
    // the fallback merge compares costs: keep them even if not requested
    p.o.cost = o_cost;
    p.o.status = o_status;
  }
  if (!learned && n >= 2 * kChunkMin) {
    // plain or given start: the scene in chunks whose copies overlap the
    // fits of the others; consecutive chunks fit on two streams, each with
    // its own claim counters and its slice of the stage scratch, so a
    // chunk's fit starts on the SMs that the previous chunk's last pixels
    // leave idle. Each pixel's fit is independent of the chunking, so the
    // results are those of one launch bit for bit
    int64_t c0[kChunks + 1];
    int nch = 0;
    c0[0] = 0;
    for (int k = 0; k < kChunks && c0[nch] < n; k++) {
      int64_t m = std::max<int64_t>(kChunkMin, n * kChunkSixteenths[k] / 16);
      if (n - c0[nch] - m < kChunkMin || k == kChunks - 1) m = n - c0[nch];   // the rest
      c0[nch + 1] = c0[nch] + m;
      nch++;
    }
    if (!c->copy_st) CK(cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
    if (!c->fit_st2) CK(cudaStreamCreateWithFlags(&c->fit_st2, cudaStreamNonBlocking));
    if (!c->d_ctr) {
      fire_status_t e = dev_alloc(&c->d_ctr, (size_t)2 * kChunks * 8);
      if (e != FIRE_OK) return e;
    }
    while ((int)c->chunk_ev.size() < 2 * nch + 2) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->chunk_ev.push_back(e);
    }
    cudaEvent_t *ev_in = c->chunk_ev.data(), *ev_fit = ev_in + nch;
    cudaEvent_t ev_start = ev_in[2 * nch], ev_done = ev_in[2 * nch + 1];
    cudaStream_t cp = c->copy_st, fs[2] = {st, c->fit_st2};
    // copies and fits start after the caller's earlier work on the staging
    // buffer and the cleared statistics
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    CK(cudaEventRecord(ev_start, st));
    CK(cudaStreamWaitEvent(cp, ev_start, 0));
    CK(cudaStreamWaitEvent(fs[1], ev_start, 0));
    for (int i = 0; i < nch; i++) {
      const int64_t a = c0[i], m = c0[i + 1] - c0[i];
      CK(cudaMemcpyAsync(d_rad + a * c->t.nb, sc->radiance + a * c->t.nb, (size_t)m * c->t.nb * 4,
                         cudaMemcpyHostToDevice, cp));
      CK(cudaMemcpyAsync(d_wv + a, sc->wv_bin + a, (size_t)m * 2, cudaMemcpyHostToDevice, cp));
      if (d_init)
        CK(cudaMemcpyAsync(d_init + a * NS, pri->init_state + a * NS, (size_t)m * NS * 4,
                           cudaMemcpyHostToDevice, cp));
      CK(cudaEventRecord(ev_in[i], cp));
    }
    int blocks = 0;
    c->last_launches = 0;
    for (int i = 0; i < nch; i++) {
      const int64_t a = c0[i], m = c0[i + 1] - c0[i];
      LMLaunch q = p;
      q.s.n_pix = m;
      q.s.rad = d_rad + a * c->t.nb;
      q.s.wv = d_wv + a;
      q.s.init = d_init ? d_init + a * NS : nullptr;
      auto off = [&](auto *ptr, int64_t w) { return ptr ? ptr + a * w : ptr; };
      q.o.state = off(p.o.state, NS);
      q.o.ET = off(p.o.ET, 1);
      q.o.sdT = off(p.o.sdT, 1);
      q.o.alpha = off(p.o.alpha, 1);
      q.o.var_ET = off(p.o.var_ET, 1);
      q.o.cost = off(p.o.cost, 1);
      q.o.rms = off(p.o.rms, 1);
      q.o.hfdi = off(p.o.hfdi, 1);
      q.o.cov = off(p.o.cov, 21);
      q.o.status = off(p.o.status, 1);
      q.o.iters = off(p.o.iters, 2);
      q.o.resid = off(p.o.resid, c->t.nb);
      q.w.counter = c->d_ctr + 2 * i;
      q.w.s1x = p.w.s1x + a * (c->t.K + 2);
      q.w.s1meta = p.w.s1meta + a;
      q.w.s2x = p.w.s2x + a * 32;
      q.w.s2g = p.w.s2g + a * 6;
      cudaStream_t si = fs[i & 1];
      CK(cudaStreamWaitEvent(si, ev_in[i], 0));
      CK(cudaMemsetAsync(q.w.counter, 0, 2 * 8, si));   // claim counters; statistics accumulate
      CK(launch_lm(q, c->num_sms, si, &blocks, c->tune_variant));
      c->last_launches += 3;
      CK(cudaEventRecord(ev_fit[i], si));
      CK(cudaStreamWaitEvent(cp, ev_fit[i], 0));
      struct { void *h; void *d; size_t b; } back[] = {
          {out->state, q.o.state, (size_t)m * NS * 4}, {out->ET, q.o.ET, (size_t)m * 4},
          {out->sdT, q.o.sdT, (size_t)m * 4}, {out->alpha, q.o.alpha, (size_t)m * 4},
          {out->var_ET, q.o.var_ET, (size_t)m * 4}, {out->cost, q.o.cost, (size_t)m * 4},
          {out->rms, q.o.rms, (size_t)m * 4}, {out->hfdi, q.o.hfdi, (size_t)m * 4},
          {out->cov, q.o.cov, (size_t)m * 21 * 4}, {out->status, q.o.status, (size_t)m},
          {out->iters, q.o.iters, (size_t)m * 4},
          {out->resid_spec, q.o.resid, (size_t)m * c->t.nb * 4}};
      const size_t eo[] = {(size_t)a * NS * 4, (size_t)a * 4, (size_t)a * 4, (size_t)a * 4,
                           (size_t)a * 4, (size_t)a * 4, (size_t)a * 4, (size_t)a * 4,
                           (size_t)a * 21 * 4, (size_t)a, (size_t)a * 4,
                           (size_t)a * c->t.nb * 4};
      for (int k = 0; k < 12; k++)
        if (back[k].h)
          CK(cudaMemcpyAsync((char *)back[k].h + eo[k], back[k].d, back[k].b,
                             cudaMemcpyDeviceToHost, cp));
    }
    CK(cudaEventRecord(ev_done, cp));
    CK(cudaStreamWaitEvent(st, ev_done, 0));
    CK(cudaStreamSynchronize(st));
    int err = 0;
    CK(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return err_status(err);
  }
  CK(cudaMemcpyAsync(d_rad, sc->radiance, s_rad, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_wv, sc->wv_bin, s_wv, cudaMemcpyHostToDevice, st));
  if (d_init) CK(cudaMemcpyAsync(d_init, pri->init_state, s_init, cudaMemcpyHostToDevice, st));
  {
    fire_status_t e = run_fit(c, p, learned, st);
    if (e != FIRE_OK) return e;
  }
  struct { void *h; void *d; size_t b; } back[] = {
      {out->state, o_state, s_state}, {out->ET, o_ET, szf}, {out->sdT, o_sdT, szf},
      {out->alpha, o_alpha, szf}, {out->var_ET, o_var, szf}, {out->cost, o_cost, szf},
      {out->rms, o_rms, szf}, {out->hfdi, o_hfdi, szf}, {out->cov, o_cov, s_cov},
      {out->status, o_status, s_u8}, {out->iters, o_it, s_it}, {out->resid_spec, o_res, s_res}};
  for (auto &b : back)
    if (b.h) CK(cudaMemcpyAsync(b.h, b.d, b.b, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int err = 0;
  CK(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  return err_status(err);
}

fire_status_t fire_set_kernel_timing(fire_ctx_t *c, int32_t on) {
  if (!c) return FIRE_ERR_ARG;
  c->timing = on != 0;
  c->tev_used = 0;
  return FIRE_OK;
}

fire_status_t fire_get_kernel_times(fire_ctx_t *c, float *ms, int32_t *n_fits) {
  if (!c || !ms) return FIRE_ERR_ARG;
  ms[0] = ms[1] = ms[2] = 0.f;
  const size_t n = c->tev_used / 4;
  if (n_fits) *n_fits = (int32_t)n;
  if (n == 0) return FIRE_OK;
  CK(cudaEventSynchronize(c->tev[c->tev_used - 1]));
  for (size_t i = 0; i < n; i++) {
    for (int k = 0; k < 3; k++) {
      float v = 0.f;
      CK(cudaEventElapsedTime(&v, c->tev[4 * i + k], c->tev[4 * i + k + 1]));
      ms[k] += v;
    }
  }
  c->tev_used = 0;
  return FIRE_OK;
}

fire_status_t fire_get_stats(fire_ctx_t *c, fire_stats_t *s) {
  if (!c || !s) return FIRE_ERR_ARG;
  unsigned long long h[2 + ST_COUNT];
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(h, c->d_work, sizeof(h), cudaMemcpyDeviceToHost));
  int err = 0;
  CK(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  memset(s, 0, sizeof(*s));
  const unsigned long long *v = h + 2;
  s->n_pixels = v[ST_NPIX];
  s->sum_it1 = v[ST_IT1];
  s->sum_it2 = v[ST_IT2];
  s->n_fp64_pixels = v[ST_FP64];
  s->band_evals1 = v[ST_BAND1];
  s->band_evals2 = v[ST_BAND2];
  s->node_band_evals2 = v[ST_NODEBAND2];
  s->solves64_1 = v[ST_S64_1];
  s->solves64_2 = v[ST_S64_2];
  s->mma_rounds2 = v[ST_MMA2];
  s->n_post64 = v[ST_POST64];
  for (int k = 0; k < 8; k++) s->status_counts[k] = v[ST_STATUS0 + k];
  // algorithmic flops of the method (FMA = 2), per band and evaluation of
  // each stage's model, Jacobian, normal equations and cost (the build's own
  // increment-form decrease and FP32 rounding-floor estimate not counted):
  //  stage 1 (P = K + 1 reduced variables): surface mixture 2K, solar term
  //    5, Planck factor and its T derivative 9, model and residual 4,
  //    Jacobian 2K + 6, weighted Jacobian P, J^T W J P (P + 1), J^T W r 2P,
  //    cost 3: 4K + 27 + P (P + 1) + 3P (71 for K = 3);
  //  stage 2: mixture model and residual 6, Jacobian 13, weighted Jacobian
  //    6, J^T W J 42, J^T W r 12, cost 3 = 82, plus the six moment sums
  //    (two components x three) over the grid: 12 per band and node
  const int K = c->t.K, P1 = K + 1;
  const double f1 = 4.0 * K + 27.0 + P1 * (P1 + 1.0) + 3.0 * P1;
  const double f2 = 6.0 + 13.0 + 6.0 + 42.0 + 12.0 + 3.0;
  s->flops1 = f1 * (double)s->band_evals1;
  s->flops2 = f2 * (double)s->band_evals2 + 12.0 * (double)s->node_band_evals2;
  s->flops = s->flops1 + s->flops2;
  s->kernel_launches = c->last_launches;
  return err_status(err);
}

fire_status_t fire_forward(fire_ctx_t *c, int32_t mode, const float *state, const uint16_t *wv,
                           int64_t n, float nrel, float nabs, uint64_t seed, uint64_t sid,
                           int64_t pix0, float *L_out, fire_stream_t stream) {
  if (!c) return FIRE_ERR_ARG;
  if (mode != 1 && mode != 2) return FIRE_ERR_ARG;
  if (n < 0 || !(nrel >= 0.f) || !(nabs >= 0.f)) return FIRE_ERR_ARG;
  if (n == 0) return FIRE_OK;
  if (!state || !wv || !L_out) return FIRE_ERR_ARG;
  return cuda_status(launch_forward(c->t, mode, state, wv, n, nrel, nabs, seed, sid, pix0, L_out,
                                    (cudaStream_t)stream));
}

fire_status_t fire_normal_equations(fire_ctx_t *c, int32_t stage, const float *radiance,
                                    const uint16_t *wv_bin, const float *states, int64_t n,
                                    const fire_priors_t *pri, float *H, float *g, float *cost,
                                    fire_stream_t stream) {
  if (!c || (stage != 1 && stage != 2) || n < 0) return FIRE_ERR_ARG;
  if (n == 0) return FIRE_OK;
  if (!radiance || !wv_bin || !states || !H || !g || !cost) return FIRE_ERR_ARG;
  fire_priors_t pd;
  if (!pri) {
    fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
    pri = &pd;
  }
  LMLaunch p;
  memset(&p, 0, sizeof(p));
  if (!priors_valid(*pri, c->t.K) || !noise_sd_valid(*pri, c->t.nb)) return FIRE_ERR_ARG;
  p.t = c->t;
  fill_kconfig(p.c, c->cfg, *pri, c->t.K, c->t.nb);
  p.s.n_pix = n;
  p.s.rad = radiance;
  p.s.wv = wv_bin;
  p.w.err = c->d_err;
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), (cudaStream_t)stream));
  return cuda_status(launch_normal_eq(p, stage, states, H, g, cost, (cudaStream_t)stream,
                                      c->tune_variant));
}

fire_status_t fire_gemm_bf16(const fire_gemm_t *q, fire_stream_t stream) {
  if (!q || !q->A || !q->B || q->M < 0 || q->N < 0 || q->K < 0) return FIRE_ERR_ARG;
  if (q->epi < 0 || q->epi > 3 || (q->epi == 3 && !q->mask)) return FIRE_ERR_ARG;
  if ((q->K & 7) || (q->lda & 7) || (q->ldb & 7) || q->lda < q->K || q->ldb < q->K)
    return FIRE_ERR_SHAPE;
  GemmArgs g;
  g.A = (const __nv_bfloat16 *)q->A;
  g.B = (const __nv_bfloat16 *)q->B;
  g.lda = q->lda;
  g.ldb = q->ldb;
  g.M = q->M;
  g.N = q->N;
  g.K = q->K;
  g.epi = q->epi;
  g.bias = q->bias;
  g.mask = (const __nv_bfloat16 *)q->mask;
  g.ldm = q->ldm;
  g.Cf = q->Cf;
  g.ldc = q->ldc;
  g.Cb = (__nv_bfloat16 *)q->Cb;
  g.ldcb = q->ldcb;
  g.CbT = (__nv_bfloat16 *)q->CbT;
  g.ldcbT = q->ldcbT;
  g.accumulate = q->accumulate;
  g.err = q->err;
  return cuda_status(launch_gemm(g, (cudaStream_t)stream));
}

// the band whose centre is nearest to lam (the first of equals)
static int nearest_band(const std::vector<float> &wl, double lam) {
  int best = 0;
  for (int b = 1; b < (int)wl.size(); b++)
    if (fabs((double)wl[b] - lam) < fabs((double)wl[best] - lam)) best = b;
  return best;
}

fire_status_t fire_wv_depth_table(fire_ctx_t *c, const float *lams, float *depth_out) {
  if (!c || !depth_out) return FIRE_ERR_ARG;
  const double lo = lams ? lams[0] : 870.0, lc = lams ? lams[1] : 940.0, hi = lams ? lams[2] : 1010.0;
  const int nb = c->t.nb, nwv = c->t.nwv;
  const int blo = nearest_band(c->h_wl, lo), bc = nearest_band(c->h_wl, lc), bhi = nearest_band(c->h_wl, hi);
  if (!(blo < bc && bc < bhi)) return FIRE_ERR_ARG;
  const double f = ((double)c->h_wl[bc] - c->h_wl[blo]) / ((double)c->h_wl[bhi] - c->h_wl[blo]);
  for (int j = 0; j < nwv; j++) {
    double a[3];
    const int bb[3] = {blo, bc, bhi};
    for (int q = 0; q < 3; q++) {
      const int b = bb[q];
      a[q] = (double)c->h_e0[b] * (double)c->h_cos / M_PI * (double)c->h_td[(size_t)j * nb + b] *
             (double)c->h_tu[(size_t)j * nb + b];
    }
    depth_out[j] = (float)(1.0 - a[1] / (a[0] + (a[2] - a[0]) * f));
  }
  return FIRE_OK;
}

fire_status_t fire_wv_presolve(fire_ctx_t *c, const float *radiance, int64_t width, int64_t height,
                               int32_t block, const float *lams, uint16_t *wv_bin_out, float *depth_out,
                               fire_stream_t stream) {
  if (!c || width < 0 || height < 0 || block < 1 || block > 16) return FIRE_ERR_ARG;
  if (width * height > 0 && (!radiance || !wv_bin_out)) return FIRE_ERR_ARG;
  const double lo = lams ? lams[0] : 870.0, lc = lams ? lams[1] : 940.0, hi = lams ? lams[2] : 1010.0;
  const int blo = nearest_band(c->h_wl, lo), bc = nearest_band(c->h_wl, lc), bhi = nearest_band(c->h_wl, hi);
  WvLut lut;
  lut.n = c->t.nwv;
  fire_status_t s = fire_wv_depth_table(c, lams, lut.D);
  if (s != FIRE_OK) return s;
  for (int j = 1; j < lut.n; j++)
    if (!(lut.D[j] > lut.D[j - 1])) return FIRE_ERR_ARG;   // the depths must increase with water
  const float cf = (float)(((double)c->h_wl[bc] - c->h_wl[blo]) / ((double)c->h_wl[bhi] - c->h_wl[blo]));
  return cuda_status(launch_wv_presolve(radiance, c->t.nb, (long long)width, (long long)height, block, blo, bc,
                                        bhi, cf, c->d_sat, lut, wv_bin_out, depth_out,
                                        (cudaStream_t)stream));
}

fire_status_t fire_hfdi(fire_ctx_t *c, const float *radiance, int64_t n_pix, float *hfdi_out,
                        fire_stream_t stream) {
  if (!c || n_pix < 0) return FIRE_ERR_ARG;
  if (n_pix == 0) return FIRE_OK;
  if (!radiance || !hfdi_out) return FIRE_ERR_ARG;
  return cuda_status(launch_hfdi(radiance, c->t.nb, (long long)n_pix, c->t.bh, c->t.bl, hfdi_out,
                                 (cudaStream_t)stream));
}

fire_status_t fire_inject(fire_ctx_t *c, const float *radiance_bg, const uint16_t *wv_bin, const float *alpha,
                          const float *T, int64_t n_pix, float *radiance_out, fire_stream_t stream) {
  if (!c || n_pix < 0) return FIRE_ERR_ARG;
  if (n_pix == 0) return FIRE_OK;
  if (!radiance_bg || !wv_bin || !alpha || !T || !radiance_out) return FIRE_ERR_ARG;
  return cuda_status(launch_inject(c->t, c->d_wl, radiance_bg, wv_bin, alpha, T, (long long)n_pix,
                                   radiance_out, (cudaStream_t)stream));
}

fire_status_t fire_block_mean(const float *src, int32_t w, int32_t h, int32_t nb, int32_t blk,
                              float *dst, fire_stream_t stream) {
  if (!src || !dst || w < 0 || h < 0 || nb < 1 || blk < 1) return FIRE_ERR_ARG;
  return cuda_status(launch_block_mean(src, w, h, nb, blk, dst, (cudaStream_t)stream));
}

}  // extern "C"
