/* firert.h — C ABI of the B300 (sm_103a) per-pixel wildfire-temperature
 * retrieval: the forward model of Eq. (fm) = Eq. (solar) + Eq. (thermal),
 * fitted to every pixel of a VSWIR scene by the two-stage windowed
 * least-squares inversion of Sec. 2.6 (Eq. loss, Eq. affine), here solved
 * with a damped Gauss-Newton (Levenberg-Marquardt) iteration.
 *
 * Conventions (all entry points):
 *  - Plain C types only. Every array is caller-owned unless stated; the
 *    context owns its device tables and workspace.
 *  - Device pointers are CUDA global-memory pointers on the context's device;
 *    host pointers are ordinary (ideally pinned) host memory.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream) unless stated. Per-pixel failures are reported in the per-pixel
 *    status byte, never in the return code, which only reports argument,
 *    shape, memory and CUDA errors. No exceptions cross the ABI.
 *  - A context is not thread-safe: use one per host thread.
 */
#ifndef FIRERT_H
#define FIRERT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fire_stream_t; /* == cudaStream_t */

typedef enum {
  FIRE_OK = 0,
  FIRE_ERR_ARG = 1,        /* NULL pointer or out-of-range scalar */
  FIRE_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  FIRE_ERR_NOMEM = 3,      /* device or pinned allocation failed */
  FIRE_ERR_SHAPE = 4,      /* sizes outside what the kernels support */
  FIRE_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
  FIRE_ERR_CHECKPOINT = 6, /* bad or corrupt MLP checkpoint */
  FIRE_ERR_STATE = 7,      /* call not valid in the context's state */
  FIRE_ERR_BOUNDS = 8      /* bounds-checked builds only (FIRERT_DEBUG): an index check
                              in a fit kernel failed and its access was skipped; the
                              site is in fire_debug_word */
} fire_status_t;

/* Per-pixel status byte: low 3 bits are the outcome, upper bits are flags. */
enum {
  FIRE_PX_CONVERGED = 0,     /* stage 2 met a convergence test */
  FIRE_PX_MAXITER = 1,       /* stage 2 hit its iteration cap */
  FIRE_PX_NONFINITE = 2,     /* a radiance value is NaN or Inf: not fitted */
  FIRE_PX_ALL_MASKED = 3,    /* too few unmasked bands in a window */
  FIRE_PX_CHOL_FAIL = 4,     /* damped normal matrix never factorised */
  FIRE_PX_NOT_CANDIDATE = 5, /* below the HFDI gate (Sec. 2.1): not fitted */
  FIRE_PX_F_FP64 = 8,        /* an ill-conditioned step was solved in FP64 */
  FIRE_PX_F_NOT_IDENT = 16,  /* Laplace sd(E[T]) or alpha SNR outside limits */
  FIRE_PX_F_MLP_FALLBACK = 32, /* MLP-initialised fit replaced by plain LM */
  FIRE_PX_F_S1_MAXITER = 64  /* stage 1 hit its iteration cap */
};

enum { FIRE_MEM_DEVICE = 0, FIRE_MEM_HOST = 1 };
enum { FIRE_INIT_DEFAULT = 0, FIRE_INIT_GIVEN = 1, FIRE_INIT_MLP = 2 };
enum { FIRE_FIT_ALL = 0, FIRE_FIT_HFDI = 1 };
enum { FIRE_MAX_ENDM = 8, FIRE_MAX_BANDS = 512, FIRE_MAX_TGRID = 128, FIRE_MAX_WV = 256 };

/* Scene tables (Sec. 2.3): HOST pointers, copied into the context by
 * fire_ctx_create; the caller may free them afterwards.
 *   wavelength_nm [n_bands]  band centres, strictly increasing (nm)
 *   solar_irr     [n_bands]  E_sun(lambda), W m^-2 nm^-1 (Eq. solar)
 *   cos_sza                   cos(theta_s)
 *   tau_down, tau_up, rho_atm, sph_alb [n_wv][n_bands]: the per-scene LUT
 *                             evaluated at each quantised water-vapour bin
 *                             (Sec. 2.5-2.6); rho_atm / sph_alb may be NULL (0)
 *   endmembers    [n_endm][n_bands] surface reflectance library (Sec. 2.4)
 *   sat_level     [n_bands] or NULL: a band with L >= sat_level is masked,
 *                             m(lambda) = 0 in Eq. (loss)
 *   tgrid_lo/hi, n_tgrid      temperature grid of Eq. (thermal), [350, 2200] K */
typedef struct {
  int32_t n_bands, n_wv, n_endm, n_tgrid;
  const float *wavelength_nm;
  const float *solar_irr;
  float cos_sza;
  const float *tau_down, *tau_up, *rho_atm, *sph_alb;
  const float *endmembers;
  const float *sat_level;
  float tgrid_lo, tgrid_hi;
} fire_tables_t;

/* Solver constants. Windows follow Sec. 2.3/2.6; everything else is this
 * library's stated choice (the paper gives no LM constants). The iteration
 * caps (100 / 600 trial steps) are set well above what the damped iteration
 * needs (stage 2 of the near-degenerate mixture: median ~70, up to ~300 on
 * flaming pixels in FP64, more in FP32 where the normal matrix resolves its
 * flat directions less well), so that a fit stops on a convergence test
 * rather than on the cap. Fill with fire_default_config and edit. */
typedef struct {
  float win1_lo, win1_hi;           /* Omega_1 (nm) */
  float win2h_lo, win2h_hi;         /* Omega_2^hot */
  float win2s_lo, win2s_hi;         /* Omega_2^smol; stage 2 fits the union */
  int32_t max_it1, max_it2;         /* trial steps per stage */
  float tau0;                       /* initial damping: the damped matrix is
                                       H + lambda diag(H), lambda starts at tau0 */
  float tol_g;                      /* |g_i| <= tol_g sqrt(H_ii cost) */
  float tol_x;                      /* max |step| in z below tol_x */
  float tol_f;                      /* relative cost decrease below tol_f */
  float kappa_max;                  /* condition estimate (max L_ii / min
                                       L_ii)^2 of the Jacobi-scaled damped
                                       matrix above which the step is
                                       re-solved in FP64 (default 1e6: the
                                       FP32 solve's relative error bound
                                       kappa 2^-24 stays below 6 %) */
  float dfloor;                     /* damping diagonal floor (relative) */
  float noise_rel, noise_abs;       /* noise model sd^2 = (rel L)^2 + abs^2 */
  int32_t weighted;                 /* 0: Eq. (loss) as printed; 1: 1/sd^2 */
  float hfdi_thresh;                /* Sec. 2.1: HFDI >= -0.1 */
  float hfdi_lambda_hi, hfdi_lambda_lo; /* 2430 nm, 2061 nm */
  float ident_sd_et;                /* identifiable: Laplace sd(E[T]) <= this */
  float ident_alpha_snr;            /* ... and alpha >= snr * sd(alpha) */
  int64_t wait_spins;               /* polls of a bounded device-side wait (table
                                       staging, tensor-core product) before it gives
                                       up and the call reports FIRE_ERR_TIMEOUT;
                                       0 = the default 2^26 */
  int32_t solver;                   /* FIRE_SOLVER_LM (default) or FIRE_SOLVER_ADAM */
  int32_t adam_steps1, adam_steps2; /* Adam steps per stage (Sec. 2.6: 30, 100) */
  double adam_lr1, adam_lr2;        /* Adam learning rates (Sec. 2.6: 0.03, 0.015) */
  double adam_clip;                 /* global-norm clip of the z gradient (1.0; the
                                       paper's value is not legible) */
  double adam_beta1, adam_beta2, adam_eps;  /* Eq. (adam): 0.9, 0.999, 1e-8 (double, so
                                       that 1 - beta is exact) */
} fire_config_t;

/* Solvers. FIRE_SOLVER_LM: damped Gauss-Newton with the convergence tests
 * and caps above, Eq. (loss) plus the weak prior of fire_priors_t.
 * FIRE_SOLVER_ADAM: the paper's optimiser (Sec. 2.6, Eq. adam): a fixed
 * adam_steps1 / adam_steps2 Adam steps per stage on Eq. (loss) as printed
 * (the prior precisions are ignored), every variable on its own z
 * coordinate of Eq. (affine), the gradient clipped to a global norm of
 * adam_clip, z clipped to [-1, 1] and the surface fractions projected onto
 * the unit simplex after each step; the result is the state after the last
 * step (status CONVERGED, iterations = the step counts), its posterior formed
 * there as after an LM fit. The launch shape's stage-1 lane count is 16
 * under Adam; stage 2 runs on the tensor cores (shapes 6-8) or in FP32. */
#define FIRE_SOLVER_LM 0
#define FIRE_SOLVER_ADAM 1

/* Priors: bounds of Eq. (affine), a weak diagonal Gaussian prior in z
 * (precision counted in units of one band's noise variance), the start rule.
 * Stage-1 layout [x_surf(K), alpha1, T1]; stage-2 layout
 * [mu_h, sigma_h, mu_s, sigma_s, eta, alpha]. A variable with lo == hi is
 * held fixed. The surface fractions must all have bounds [0, 1]. */
typedef struct {
  float lo1[FIRE_MAX_ENDM + 2], hi1[FIRE_MAX_ENDM + 2];
  float pm1[FIRE_MAX_ENDM + 2], pp1[FIRE_MAX_ENDM + 2];
  float lo2[6], hi2[6], pm2[6], pp2[6];
  float init_alpha1, init_T1, init_sigma, init_mu_h_floor, init_mu_s_ceil;
  float init_eta_lo, init_eta_hi;
  int32_t init_mode;                /* FIRE_INIT_* */
  const float *init_state;          /* [n_pix][n_endm + 8] when GIVEN, same
                                       memory kind as the scene */
  const float *noise_sd;            /* HOST [n_bands] per-band noise sd (> 0), or
                                       NULL. Given, the loss of Eq. (loss) is
                                       weighted by 1 / noise_sd_b^2 (and the
                                       covariance is not rescaled); NULL leaves
                                       fire_config_t.weighted in charge. */
} fire_priors_t;

/* One scene: BIP radiance [n_pix][n_bands] fp32 (W m^-2 sr^-1 nm^-1) and
 * the water-vapour bin of each pixel [n_pix] (< n_wv; a pixel whose bin is out
 * of range is not fitted and gets status FIRE_PX_NONFINITE). mem: FIRE_MEM_DEVICE
 * or FIRE_MEM_HOST (host buffers are staged through device memory inside
 * the call, which then synchronises the stream before returning). */
typedef struct {
  int64_t n_pix;
  const float *radiance;
  const uint16_t *wv_bin;
  int32_t mem;
  int32_t gate_mode;                /* FIRE_FIT_ALL or FIRE_FIT_HFDI */
} fire_scene_t;

/* Per-pixel outputs, same memory kind as the scene; any may be NULL.
 *   state  [n_pix][n_endm+8]  [x_surf, alpha1, T1, mu_h, s_h, mu_s, s_s, eta, alpha]
 *   ET, sdT                   moment-matched E[T], sigma[T] (Sec. 2.3), K
 *   alpha                     stage-2 thermal scaling
 *   cov    [n_pix][21]        Laplace covariance of the stage-2 state, packed
 *                             upper triangle, physical units, FP64-computed
 *   var_ET                    delta-method variance of E[T]
 *   cost                      final stage-2 cost; rms: unweighted residual rms
 *   hfdi                      HFDI of the pixel
 *   status, iters [n_pix][2]  status byte; trial steps of stage 1 and 2
 *   resid_spec                optional residual spectrum (below) */
typedef struct {
  float *state, *ET, *sdT, *alpha, *cov, *var_ET, *cost, *rms, *hfdi;
  uint8_t *status;
  uint16_t *iters;
  float *resid_spec;                /* [n_pix][n_bands]: L_b - M_b(x) of the full
                                       forward model Eq. (fm) at the final state,
                                       every band (Sec. 3.2's spectral residuals);
                                       NaN rows for pixels not fitted */
} fire_outputs_t;

/* Counters of the last retrieve call (read after the stream synchronises). */
typedef struct {
  uint64_t n_pixels, sum_it1, sum_it2, n_fp64_pixels;
  uint64_t band_evals1, band_evals2, node_band_evals2;  /* work units: full evaluations */
  uint64_t solves64_1, solves64_2;  /* FP64 re-solves of ill-conditioned steps, per stage */
  uint64_t mma_rounds2;             /* tensor-core stage 2: evaluation rounds (one product each) */
  uint64_t status_counts[8];
  double flops;                     /* algorithmic flops of the fit */
  double flops1, flops2;            /* ... of which stage 1 and stage 2 */
  int32_t kernel_launches;
  uint64_t n_post64;                /* pixels whose posterior normal matrix was
                                       formed in FP64 (alpha clear of noise) */
} fire_stats_t;

typedef struct fire_ctx fire_ctx_t;

/* Fill the documented defaults. */
void fire_default_config(fire_config_t *cfg);
void fire_default_priors(fire_priors_t *pri, int32_t n_endm, int32_t n_tgrid,
                         float tgrid_lo, float tgrid_hi);

/* Create a context on the current CUDA device: validates and uploads the
 * tables, builds the Planck grid B(lambda_b, T_j) and the per-band constants
 * on the device (Eq. thermal; synchronous). cfg NULL = defaults.
 * Errors: FIRE_ERR_ARG (NULL/invalid), FIRE_ERR_SHAPE (n_bands > 512,
 * n_endm not in 1..8, n_tgrid not in 2..128, empty window), FIRE_ERR_NOMEM,
 * FIRE_ERR_CUDA. On error *out is NULL. */
fire_status_t fire_ctx_create(fire_ctx_t **out, const fire_tables_t *tables,
                              const fire_config_t *cfg);
void fire_ctx_destroy(fire_ctx_t *ctx);

/* Retrieve every pixel of one scene (Sec. 2.6 stage 1 then stage 2, per
 * pixel, on the GPU). pri NULL = defaults. n_pix == 0 is a no-op.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_SHAPE, FIRE_ERR_NOMEM (scratch, host
 * staging), FIRE_ERR_CUDA, FIRE_ERR_TIMEOUT (a bounded device wait gave up;
 * the outputs are then incomplete). A host scene's call synchronises and
 * returns the timeout itself; a device scene's call returns before the fit
 * runs, and the timeout is reported by the next fire_get_stats. */
fire_status_t fire_retrieve(fire_ctx_t *ctx, const fire_scene_t *scene,
                            const fire_priors_t *pri, const fire_outputs_t *out,
                            fire_stream_t stream);

/* Forward model Eq. (fm) for n states (device pointers):
 *   mode 1: state [n][K+2] = [x_surf, alpha1, T1] (single temperature);
 *   mode 2: state [n][K+6] = [x_surf, mu_h, s_h, mu_s, s_s, eta, alpha]
 *           (two-component Gaussian p(T) on the grid).
 * L_out [n][n_bands] fp32. If noise_rel or noise_abs > 0, adds
 * sd * N(0,1) with sd^2 = (rel L)^2 + abs^2, the normal drawn by Box-Muller
 * from the counter-based SplitMix64 stream (seed, stream_id, pixel_offset + i,
 * 2b / 2b+1). A state whose water-vapour bin is out of range gets NaN radiance. */
fire_status_t fire_forward(fire_ctx_t *ctx, int32_t mode, const float *state,
                           const uint16_t *wv_bin, int64_t n, float noise_rel,
                           float noise_abs, uint64_t seed, uint64_t stream_id,
                           int64_t pixel_offset, float *L_out, fire_stream_t stream);

/* 12x12-style block mean of a BIP cube (Sec. 2.9): src [height][width][n_bands]
 * -> dst [height/block][width/block][n_bands], edge remainder dropped.
 * Device pointers. */
fire_status_t fire_block_mean(const float *src, int32_t width, int32_t height,
                              int32_t n_bands, int32_t block, float *dst,
                              fire_stream_t stream);

/* Normal equations of one stage at given states, for verification: the
 * model, Jacobian, J^T W J + P, J^T W r - P (z - pm) and the cost of Eq. (loss)
 * plus the prior, exactly as one iteration of the fit forms them, in the
 * fit's z coordinates (Eq. affine); stage 1 uses the reduced simplex basis
 * (fractions k != m, m = largest fraction, then alpha1, T1).
 * Device pointers: radiance [n][n_bands], wv_bin [n], states [n][K+2]
 * (stage 1: x_surf, alpha1, T1) or [n][K+6] (stage 2: x_surf, mu_h, s_h,
 * mu_s, s_s, eta, alpha); outputs H [n][P][P], g [n][P], cost [n] with
 * P = K+1 (stage 1) or 6. pri NULL = defaults. */
fire_status_t fire_normal_equations(fire_ctx_t *ctx, int32_t stage, const float *radiance,
                                    const uint16_t *wv_bin, const float *states, int64_t n,
                                    const fire_priors_t *pri, float *H, float *g, float *cost,
                                    fire_stream_t stream);

/* BF16 tensor-core GEMM used by the learned initial-state proposal:
 * C[M][N] = A[M][K] * B[N][K]^T (A, B bf16, K contiguous, rows 16-byte
 * aligned: K, lda, ldb multiples of 8), FP32 accumulation, fused epilogue.
 * epi: 0 = fp32 out (+bias), 1 = relu(acc + bias), 2 = tanh(acc + bias),
 * 3 = acc * (mask > 0) (ReLU gradient). Outputs (any may be NULL): Cf fp32
 * [M][ldc] (accumulate != 0 adds into it), Cb bf16 [M][ldcb], CbT bf16
 * transposed [N][ldcbT]. err: device int set to 1 if a bounded wait gave up
 * (may be NULL). All pointers are device pointers; asynchronous. */
typedef struct {
  const void *A;
  int64_t lda;
  const void *B;
  int64_t ldb;
  int32_t M, N, K, epi;
  const float *bias;
  const void *mask;
  int64_t ldm;
  float *Cf;
  int64_t ldc;
  void *Cb;
  int64_t ldcb;
  void *CbT;
  int64_t ldcbT;
  int32_t accumulate;
  int32_t *err;
} fire_gemm_t;
fire_status_t fire_gemm_bf16(const fire_gemm_t *g, fire_stream_t stream);

/* ---- Learned initial-state proposal (the task's extension; the paper has
 * no network). z = tanh(W3 relu(W2 relu(W1 x + b1) + b2) + b3), x = per-band
 * standardised radiance (bands padded to Din = n_bands rounded up to 16),
 * hidden width H, 16 outputs of which K + 6 are used: the surface fractions
 * and the five mixture-shape parameters in the z coordinates of Eq. (affine)
 * (stage-2 default bounds) and log10(alpha) in [-4, 0] mapped to [-1, 1].
 * BF16 tensor-core products with FP32 accumulation; FP32 master weights and
 * Adam (beta 0.9 / 0.999, eps 1e-8). Training spectra are drawn on the GPU
 * from the forward model (counter-based streams: the same seed and sample
 * indices give the same batch). */
typedef struct fire_mlp fire_mlp_t;
typedef struct {
  int64_t steps;          /* optimiser steps */
  int32_t batch;          /* spectra per step, a multiple of 128 */
  float lr;               /* Adam learning rate */
  float pfire;            /* share of training spectra with a fire */
  float noise_rel, noise_abs;  /* noise model of the spectra */
  uint64_t seed;          /* stream key */
  int64_t sample0;        /* index of the first sample (resume from fire_mlp_next_sample) */
} fire_mlp_train_cfg_t;

/* Create a network for the context's tables (weights He-uniform from seed).
 * Errors: FIRE_ERR_ARG, FIRE_ERR_SHAPE (hidden not a multiple of 16 in
 * 16..1024), FIRE_ERR_NOMEM, FIRE_ERR_CUDA. Synchronous. */
fire_status_t fire_mlp_create(fire_mlp_t **out, fire_ctx_t *ctx, int32_t hidden, uint64_t seed);
void fire_mlp_destroy(fire_mlp_t *m);
/* Train: cfg->steps Adam steps on fresh synthetic batches; the first call
 * also gathers the input standardisation from one batch. loss_host [steps]
 * (host, optional) receives the masked-MSE loss of each step (the call then
 * synchronises the stream). */
fire_status_t fire_mlp_train(fire_mlp_t *m, const fire_mlp_train_cfg_t *cfg, float *loss_host,
                             fire_stream_t stream);
/* Inference on device radiance [n][n_bands]: z_out [n][16] (optional) and
 * init_out [n][K+8] (optional), a starting state in the layout of
 * fire_outputs_t.state, usable as fire_priors_t.init_state. */
fire_status_t fire_mlp_infer(fire_mlp_t *m, const float *radiance, int64_t n, float *z_out,
                             float *init_out, fire_stream_t stream);
/* Forward + backward on given standardised inputs x [B][Din], targets and
 * masks [B][16] (device fp32): grads (device) packed as dW1 [H][Din], db1 [H],
 * dW2 [H][H], db2 [H], dW3^T [H][16], db3 [16]; loss (device, 1 float).
 * B must be a multiple of 8 (FIRE_ERR_SHAPE otherwise). Synchronous; for
 * verification against a reference. */
fire_status_t fire_mlp_gradients(fire_mlp_t *m, const float *x, const float *tgt, const float *msk,
                                 int64_t B, float *grads, float *loss, fire_stream_t stream);
/* Parameter count of the packed layout W1, b1, W2, b2, W3 [16][H], b3,
 * mean [Din], inv_std [Din]; fire_mlp_params copies them out (get) and/or in
 * (set), host pointers. */
int64_t fire_mlp_param_count(const fire_mlp_t *m);
fire_status_t fire_mlp_params(fire_mlp_t *m, float *get, const float *set);
/* Checkpoint (parameters, Adam moments, step and sample counters, FNV-1a
 * checksum); load rejects a corrupt or mismatched file with
 * FIRE_ERR_CHECKPOINT. */
fire_status_t fire_mlp_save(fire_mlp_t *m, const char *path);
fire_status_t fire_mlp_load(fire_mlp_t *m, const char *path);
int64_t fire_mlp_next_sample(const fire_mlp_t *m);
/* Attach a trained network to a context: fire_retrieve with init_mode
 * FIRE_INIT_MLP then starts every pixel from the network's proposal. A pixel
 * whose learned-start fit ends unconverged, or with a cost above three times
 * the expected chi-square (n_used - 6) x noise variance, is re-fitted from the
 * default start; the lower-cost fit is kept and the pixel is flagged
 * FIRE_PX_F_MLP_FALLBACK. The call synchronises the stream once (to size the
 * re-fit). m = NULL detaches. */
fire_status_t fire_ctx_set_mlp(fire_ctx_t *ctx, fire_mlp_t *m);

/* ---- Batched uneven scenes (one persistent launch over all pixels of all
 * scenes; device pointers; default start only). Scenes of any size share the
 * context's tables; each has its own outputs (any may be NULL). */
typedef struct {
  int64_t n_pix;
  const float *radiance;     /* [n_pix][n_bands] */
  const uint16_t *wv_bin;    /* [n_pix] */
  fire_outputs_t out;
} fire_batch_item_t;
/* Errors: FIRE_ERR_ARG (bad item, init_mode not DEFAULT), FIRE_ERR_NOMEM,
 * FIRE_ERR_CUDA. Synchronises the stream once to upload the scene table. */
fire_status_t fire_retrieve_batch(fire_ctx_t *ctx, const fire_batch_item_t *items, int32_t n_items,
                                  const fire_priors_t *pri, int32_t gate_mode,
                                  fire_stream_t stream);
/* CUDA graph of the whole batched fit (scene-table upload, counter resets,
 * the three kernels) over the given buffers; replay it with
 * fire_graph_launch after refilling those buffers with new scenes of the
 * same sizes. The graph owns its scratch (stage hand-over, counters), so
 * later calls on the context leave it valid, but two replays of one graph
 * must not overlap; fire_get_stats does not see graph replays. The context
 * must outlive the graph (its tables are read by the replays). */
typedef struct fire_graph fire_graph_t;
fire_status_t fire_graph_capture(fire_ctx_t *ctx, const fire_batch_item_t *items, int32_t n_items,
                                 const fire_priors_t *pri, int32_t gate_mode, fire_graph_t **out);
fire_status_t fire_graph_launch(fire_graph_t *g, fire_stream_t stream);
void fire_graph_destroy(fire_graph_t *g);
/* Autotuner: times each launch shape on the n given device pixels and keeps
 * the fastest for the context. variant = 3 * s2 + s1: s1 picks the lanes
 * per pixel of stage 1 (0 = 16 lanes, two pixels per warp; 1 = 8 lanes,
 * four per warp; 2 = 32 lanes, one per warp), s2 the stage-2 evaluation
 * (0 = FP32 with 32 lanes per pixel; 1 = FP32 with 16; 2 = 16 lanes per
 * pixel, 24 pixels per CTA in three 4-warp cohorts, with the grid-node sums
 * of a cohort's 8 pixels as one bf16x3 tensor-core product per round; tables
 * with more than 64 grid nodes or more stage-2 bands than its shared memory
 * holds (about 225), and the weighted loss, take 1 instead). claim: pixels
 * per work claim (1, 2, 4, 8). Each stage runs one persistent CTA per SM with
 * as many warps as its shared memory allows (at most 12 for stage 1, 8 for
 * the FP32 stage 2, 12 for the tensor-core stage 2). A new context starts at
 * variant 6 where the tables allow it, else 3.
 * fire_set_tuning sets a shape directly (variant 0..8, claim 1..64); the
 * stage-2 evaluation of the set shape is also the one that
 * fire_normal_equations uses. */
typedef struct {
  int32_t variant, claim;
  float ms;
} fire_tune_t;
fire_status_t fire_autotune(fire_ctx_t *ctx, const float *radiance, const uint16_t *wv_bin, int64_t n,
                            fire_tune_t *best, fire_stream_t stream);
fire_status_t fire_set_tuning(fire_ctx_t *ctx, int32_t variant, int32_t claim);

/* ---- Fit without allocation (an addition of this library; the paper has
 * no counterpart). The plain-LM fit of a device scene of at most
 * FIRE_STATIC_MAX_PIX pixels whose scratch (stage hand-over, work counters
 * and statistics; at most FIRE_STATIC_SCRATCH_BYTES) is one file-scope
 * device array of the library: the call makes no cudaMalloc/cudaFree and
 * calls no allocating routine; it clears the counters that must start at
 * zero on the stream and launches the fit kernels with the context's launch
 * shape, so its results equal fire_retrieve's.
 * - The first call on each device looks up the array's address
 *   (cudaGetSymbolAddress): make it before capturing the call in a graph.
 *   The address is kept for the life of the process; a cudaDeviceReset
 *   (which drops the device's copy of the array) invalidates it.
 * - All calls share the one array: two calls whose executions overlap (on
 *   different streams, threads or contexts) race and corrupt each other.
 * - Scene and outputs must be device memory; init_mode DEFAULT or GIVEN.
 * - Errors: FIRE_ERR_SHAPE if n_pix > FIRE_STATIC_MAX_PIX; FIRE_ERR_ARG
 *   for a host scene, the learned start or bad priors; FIRE_ERR_CUDA. The
 *   call returns before the fit runs: a bounded device wait that gives up
 *   during it is recorded in the context's error word and reported as
 *   FIRE_ERR_TIMEOUT by the next fire_get_stats on the context (whose
 *   counters do not include these calls). */
#define FIRE_STATIC_MAX_PIX 16384
#define FIRE_STATIC_SCRATCH_BYTES (3u * 1024u * 1024u + 256u * 1024u)
fire_status_t fire_retrieve_static(fire_ctx_t *ctx, const fire_scene_t *scene,
                                   const fire_priors_t *priors, const fire_outputs_t *out,
                                   fire_stream_t stream);

/* HFDI (Sec. 2.1): (L_hi - L_lo) / (L_hi + L_lo) of every pixel at the bands
 * nearest to the config's hfdi_lambda_hi / hfdi_lambda_lo (2430 / 2061 nm),
 * the index the fit's gate tests; NaN where either band is not finite.
 * DEVICE radiance [n_pix][n_bands], hfdi_out [n_pix]. For the threshold
 * studies of the paper's appendix. Errors: FIRE_ERR_ARG, FIRE_ERR_CUDA.
 * Asynchronous on the stream. */
fire_status_t fire_hfdi(fire_ctx_t *ctx, const float *radiance, int64_t n_pix, float *hfdi_out,
                        fire_stream_t stream);

/* Thermal injection, Eq. (inject) (Sec. 2.8): radiance_out = radiance_bg +
 * alpha tau_up(lambda) B(lambda, T) for every band of every pixel, tau_up of
 * the pixel's water-vapour bin (an out-of-range bin gives a NaN row), the
 * Planck term in FP64. All pointers DEVICE: radiance_bg, radiance_out
 * [n_pix][n_bands] (may alias), wv_bin, alpha, T [n_pix]. The injection
 * experiment's input generator. Errors: FIRE_ERR_ARG, FIRE_ERR_CUDA.
 * Asynchronous on the stream. */
fire_status_t fire_inject(fire_ctx_t *ctx, const float *radiance_bg, const uint16_t *wv_bin,
                          const float *alpha, const float *T, int64_t n_pix, float *radiance_out,
                          fire_stream_t stream);

/* Water-vapour presolve (Sec. 2.5, "pre-solved water vapor"): the bins that
 * fire_retrieve's scene takes, from the radiance itself.
 * - radiance: DEVICE [height * width][n_bands] fp32, pixels in row-major
 *   image order (x fastest); wv_bin_out: DEVICE [height * width];
 *   depth_out: DEVICE [height * width] or NULL (the per-pixel depth).
 * - For every pixel the depth of the 940 nm water feature against a
 *   continuum interpolated linearly across its shoulders,
 *   D = 1 - L(lc) / (L(lo) + (L(hi) - L(lo)) (lc - lo) / (hi - lo)), at the
 *   bands nearest to lams = {lo, lc, hi} nm (NULL: {870, 940, 1010}); a pixel
 *   with a non-finite or saturated one of the three bands, or a
 *   non-positive continuum, has no depth (NaN). Each pixel then gets the
 *   lower median (rank (n - 1) / 2) of the n depths of its block x block
 *   super-pixel (blocks from the image origin; edge blocks are smaller),
 *   quantised to the table: the fractional bin index by linear
 *   interpolation between the bracketing depths of fire_wv_depth_table,
 *   rounded to the nearest bin, clamped to [0, n_wv - 1]. A block without
 *   any depth gets 0xFFFF (an invalid bin: fire_retrieve reports its pixels
 *   NONFINITE). Depths, interpolation and rounding are single precision.
 * - Errors: FIRE_ERR_ARG (block outside 1..16, null pointers with pixels,
 *   shoulder / centre bands not in order, table depths not increasing with
 *   the bin); FIRE_ERR_CUDA. Asynchronous on the stream. */
fire_status_t fire_wv_presolve(fire_ctx_t *ctx, const float *radiance, int64_t width, int64_t height,
                               int32_t block, const float *lams, uint16_t *wv_bin_out,
                               float *depth_out, fire_stream_t stream);
/* The flat-surface depth of the 940 nm feature of every water-vapour bin of
 * the context's tables, D_j from the same formula applied to the two-way
 * direct path E0 cos(theta_s) / pi tau_down tau_up (in double, rounded once
 * to float): HOST depth_out [n_wv]. lams as for fire_wv_presolve.
 * Synchronous; errors FIRE_ERR_ARG. */
fire_status_t fire_wv_depth_table(fire_ctx_t *ctx, const float *lams, float *depth_out);

/* Per-kernel timing. With timing on, every fit launch records CUDA events
 * on its stream around the stage-1, stage-2 and finalize kernels (no
 * synchronisation). fire_get_kernel_times waits for the last one and
 * returns the summed milliseconds of each kernel [3] over the fits since
 * the last call (or since timing was switched on), and their number. */
fire_status_t fire_set_kernel_timing(fire_ctx_t *ctx, int32_t on);
fire_status_t fire_get_kernel_times(fire_ctx_t *ctx, float *ms, int32_t *n_fits);

/* Counters of the last fire_retrieve on this context (synchronises it). */
fire_status_t fire_get_stats(fire_ctx_t *ctx, fire_stats_t *stats);

/* Band index ranges of the two fitting windows (for tests and reporting). */
fire_status_t fire_window_bands(fire_ctx_t *ctx, int32_t *b1_lo, int32_t *n1,
                                int32_t *b2_lo, int32_t *n2);

/* Measured issue rate of an arithmetic unit the retrieval's kernels are
 * bound by, for roofline denominators (synchronous, ~0.1 s): every SM
 * loaded with independent dependency chains, timed with CUDA events on the
 * stream. kind 0: FP32 FMA (flop/s, an FMA counted as 2); 1: the packed
 * two-lane FP32 FMA (flop/s); 2: the SFU's ex2.approx (operations/s); 3:
 * FP64 FMA (flop/s). seconds (optional) receives the timed duration.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_NOMEM, FIRE_ERR_CUDA. */
fire_status_t fire_measure_peak(int32_t kind, double *rate, double *seconds, fire_stream_t stream);

/* Device allocator hook. The library's device allocations (context tables
 * and workspace, host-scene staging, learned-start and batch buffers, the
 * network's weights) go through alloc(bytes, user) while a hook is set, and
 * each such block is later returned through the free function that was set
 * when it was made (so the hook may change at any time). alloc returning
 * NULL makes the call that needed the memory return FIRE_ERR_NOMEM. alloc
 * NULL restores cudaMalloc / cudaFree for later allocations. Process-wide;
 * the functions must be callable from any thread that calls the library.
 * Pinned host memory (graph scene tables) does not use the hook. */
typedef void *(*fire_alloc_fn)(size_t bytes, void *user);
typedef void (*fire_free_fn)(void *ptr, void *user);
void fire_set_allocator(fire_alloc_fn alloc, fire_free_fn free_fn, void *user);

const char *fire_status_str(fire_status_t s);

/* Build flags of the loaded library: bit 0 set when it was compiled with
 * FIRERT_DEBUG, the bounds-checked build (libfirert_debug.so), in which the
 * fit kernels (stage 1, both stage 2s, finalize) check their per-pixel
 * indices, band indices and shared-memory regions before the access; a
 * failed check records its site in the fit's device error word (the first
 * failure wins), skips the access and never traps. The release build
 * compiles the checks out. */
int32_t fire_build_flags(void);
/* The context's device error word after its last fit (synchronises the
 * device): 0, 1 (a bounded wait gave up: FIRE_ERR_TIMEOUT) or 0x100 | site
 * (a failed index check of a bounds-checked build: FIRE_ERR_BOUNDS). Errors:
 * FIRE_ERR_ARG, FIRE_ERR_CUDA. */
fire_status_t fire_debug_word(fire_ctx_t *ctx, int32_t *word);

#ifdef __cplusplus
}
#endif
#endif /* FIRERT_H */
