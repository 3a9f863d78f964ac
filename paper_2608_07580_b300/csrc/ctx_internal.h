// ctx_internal.h — the context behind fire_ctx_t (host side).
#pragma once
#include <vector>

#include "../../include/firert.h"
#include "internal.cuh"

struct fire_ctx {
  int device = 0;
  int num_sms = 0;
  fire_config_t cfg;
  firert::KTables t;
  // device buffers
  float *d_image = nullptr;
  float *d_wl = nullptr;             // [nb] band centres (nm), for Eq. (inject)
  float *d_planck_full = nullptr;    // [nt][nb] Planck grid over every band (residual spectrum)
  double *d_planck64 = nullptr;      // [nt][n2] FP64 Planck grid of the stage-2 bands (posterior)
  unsigned char *d_plop = nullptr;   // stage-2 Planck grid as the tensor-core operand
  float4 *d_wvtab = nullptr;
  float *d_sat = nullptr;
  unsigned long long *d_work = nullptr;  // [0] counter, [1..] stats
  int *d_err = nullptr;
  // host staging for FIRE_MEM_HOST scenes
  void *d_stage = nullptr;
  size_t stage_bytes = 0;
  // stage-1 -> stage-2 hand-over, grown on demand
  float *d_s1x = nullptr;
  int *d_s1meta = nullptr;
  float *d_s2x = nullptr;
  float *d_s2g = nullptr;
  int64_t s1_cap = 0;
  // learned start: network, per-pixel starts, fallback list and re-fit outputs
  fire_mlp_t *mlp = nullptr;
  float *d_mlp_init = nullptr;
  long long *d_fb_idx = nullptr;
  float *d_fb_cost = nullptr;
  unsigned long long *d_fb_count = nullptr;
  int64_t mlp_cap = 0;
  void *d_cmp = nullptr;
  int64_t cmp_cap = 0;
  int last_launches = 0;
  // launch shape (autotuned): variant = 3 * stage-2 shape + stage-1 shape
  // (set at creation to the tensor-core stage 2 with 16 lanes per pixel in
  // stage 1 where the tables fit it) and pixels per claim
  int tune_variant = 3;
  int tune_claim = 1;
  // batched calls: scene descriptors on the device
  firert::SceneItem *d_items = nullptr;
  long long *d_prefix = nullptr;
  int items_cap = 0;
  // per-kernel timing: 4 events per fit launch, summed on request
  bool timing = false;
  std::vector<cudaEvent_t> tev;
  // host scenes: a copy stream and per-chunk events, so that the copies of
  // one chunk overlap the fit of another (created on first use)
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> chunk_ev;
  // ... and a second compute stream with claim counters per chunk, so that
  // one chunk's fit can start on the SMs that another chunk's tail frees
  cudaStream_t fit_st2 = nullptr;
  unsigned long long *d_ctr = nullptr;
  size_t tev_used = 0;
  // host copies of the tables the water-vapour presolve's depth table needs
  std::vector<float> h_wl, h_e0, h_td, h_tu;
  float h_cos = 0.f;
};

namespace firert {
// bounds, prior and start-rule checks of a priors block
bool priors_valid(const fire_priors_t &p, int K);
// per-band noise sd (host array) positive and finite, when given
bool noise_sd_valid(const fire_priors_t &p, int nb);
// the next 4 timing events of the context (nullptr when timing is off)
cudaEvent_t *timing_events(fire_ctx *c);
fire_status_t run_fit(fire_ctx *c, LMLaunch &p, bool learned, cudaStream_t st);
// ctx_scratch false: the caller provides the stage hand-over buffers
fire_status_t prepare_launch(fire_ctx *c, const fire_priors_t *pri, int64_t n, int gate, LMLaunch &p,
                             bool ctx_scratch = true);
}  // namespace firert
