// noalloc.cu — fire_retrieve_static: the plain-LM fit of a device scene
// whose stage hand-over scratch, work counters and statistics live in one
// file-scope device array, so that the call allocates nothing.
#include <string.h>

#include <mutex>

#include "ctx_internal.h"

using namespace firert;

namespace {

// largest scene the static scratch holds
constexpr long long kStaticMaxPix = FIRE_STATIC_MAX_PIX;

// per-pixel scratch of the stage kernels: stage-1 state [K+2] (K <= kMaxK),
// stage-1 status word, stage-2 hand-over [32] and gradient [6]
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kS1x = al256((size_t)kStaticMaxPix * (kMaxK + 2) * 4);
constexpr size_t kS1m = al256((size_t)kStaticMaxPix * 4);
constexpr size_t kS2x = al256((size_t)kStaticMaxPix * 32 * 4);
constexpr size_t kS2g = al256((size_t)kStaticMaxPix * 6 * 4);
constexpr size_t kWork = al256((size_t)(2 + ST_COUNT) * 8);
constexpr size_t kStaticBytes = kS1x + kS1m + kS2x + kS2g + kWork;
static_assert(kStaticBytes <= FIRE_STATIC_SCRATCH_BYTES,
              "the static scratch outgrew the size the header documents");

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

// device address of g_scratch on each device, looked up on the first call
// (under a lock, so that two threads' first calls do not race on it)
constexpr int kMaxDevices = 64;
unsigned char *g_base[kMaxDevices] = {};
std::mutex g_base_mu;

}  // namespace

extern "C" fire_status_t fire_retrieve_static(fire_ctx_t *c, const fire_scene_t *sc,
                                              const fire_priors_t *pri, const fire_outputs_t *out,
                                              fire_stream_t stream) {
  if (!c || !sc || !out) return FIRE_ERR_ARG;
  if (sc->n_pix < 0 || sc->mem != FIRE_MEM_DEVICE) return FIRE_ERR_ARG;
  if (sc->gate_mode != FIRE_FIT_ALL && sc->gate_mode != FIRE_FIT_HFDI) return FIRE_ERR_ARG;
  if (sc->n_pix > kStaticMaxPix) return FIRE_ERR_SHAPE;
  fire_priors_t pd;
  if (!pri) {
    fire_default_priors(&pd, c->t.K, c->t.nt, c->t.tglo, c->t.tglo + c->t.tgstep * (c->t.nt - 1));
    pri = &pd;
  }
  if (!priors_valid(*pri, c->t.K) || !noise_sd_valid(*pri, c->t.nb)) return FIRE_ERR_ARG;
  if (pri->init_mode == FIRE_INIT_MLP) return FIRE_ERR_ARG;   // the learned start allocates
  if (pri->init_mode == FIRE_INIT_GIVEN && !pri->init_state) return FIRE_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FIRE_ERR_CUDA;
  unsigned char *b = nullptr;
  {
    // set-up, once per device (do this first call outside any stream capture)
    std::lock_guard<std::mutex> lk(g_base_mu);
    if (!g_base[dev]) {
      void *a = nullptr;
      if (cudaGetSymbolAddress(&a, g_scratch) != cudaSuccess) return FIRE_ERR_CUDA;
      g_base[dev] = (unsigned char *)a;
    }
    b = g_base[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *work = (unsigned long long *)(b + kS1x + kS1m + kS2x + kS2g);
  // the claim counters, the statistics and the context's error word start
  // at zero; a bounded wait that gives up sets that word, which the next
  // fire_get_stats on the context reports as FIRE_ERR_TIMEOUT
  if (cudaMemsetAsync(work, 0, (size_t)(2 + ST_COUNT) * 8, st) != cudaSuccess ||
      cudaMemsetAsync(c->d_err, 0, sizeof(int), st) != cudaSuccess)
    return FIRE_ERR_CUDA;
  c->last_launches = 0;
  if (sc->n_pix == 0) return FIRE_OK;
  if (!sc->radiance || !sc->wv_bin) return FIRE_ERR_ARG;
  LMLaunch p;
  fire_status_t e = prepare_launch(c, pri, sc->n_pix, sc->gate_mode == FIRE_FIT_HFDI, p, false);
  if (e != FIRE_OK) return e;
  p.w.s1x = (float *)b;
  p.w.s1meta = (int *)(b + kS1x);
  p.w.s2x = (float *)(b + kS1x + kS1m);
  p.w.s2g = (float *)(b + kS1x + kS1m + kS2x);
  p.w.counter = work;
  p.w.stats = work + 2;
  p.w.err = c->d_err;
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
  int blocks = 0;
  if (launch_lm(p, c->num_sms, st, &blocks, c->tune_variant) != cudaSuccess) return FIRE_ERR_CUDA;
  c->last_launches = 3;
  return FIRE_OK;
}
