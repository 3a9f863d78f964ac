// internal.cuh — device-side data structures shared by the kernels and the
// C-ABI implementation of the per-pixel wildfire-temperature retrieval.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cuda_bf16.h>

namespace firert {

constexpr int kWarp = 32;
constexpr int kMaxK = 8;
constexpr int kMaxTgrid = 128;
constexpr int kMaxBands = 512;
constexpr int kScratchPerNode = 8;   // floats per grid node in the warp scratch

// Device error word of a fit: 1 when a bounded wait gave up; kErrBounds |
// site when an index check of a bounds-checked build failed.
constexpr int kErrBounds = 0x100;

// Index checks of the bounds-checked build (compiled with FIRERT_DEBUG):
// fr_ok(ok, err, site) is ok; a false check records kErrBounds | site in the
// error word (the first failure wins) and the caller skips the access. Never
// traps. In the release build the check is the constant true and the
// condition is not evaluated.
#ifdef FIRERT_DEBUG
__device__ __forceinline__ bool fr_check(bool ok, int *err, int site) {
  if (!ok && err) atomicCAS(err, 0, kErrBounds | site);
  return ok;
}
#define fr_ok(ok, err, site) ::firert::fr_check((ok), (err), (site))
#else
#define fr_ok(ok, err, site) true
#endif

// bytes of dynamic shared memory the running kernel was launched with
__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// per-pixel status codes (mirrors the header)
enum : int {
  PX_CONVERGED = 0, PX_MAXITER = 1, PX_NONFINITE = 2, PX_ALL_MASKED = 3, PX_CHOL_FAIL = 4,
  PX_NOT_CANDIDATE = 5, PX_F_FP64 = 8, PX_F_NOT_IDENT = 16, PX_F_MLP_FALLBACK = 32,
  PX_F_S1_MAXITER = 64
};

// Layout of the per-CTA shared-memory table image (floats). The image is
// built once per context in global memory and bulk-copied into every CTA.
struct ImageLayout {
  int off_c2l;     // [nb]  c2 / lambda_b (K): Planck exponent numerator
  int off_c1l5;    // [nb]  c1 lambda_b^-5 (W m^-2 sr^-1 nm^-1)
  int off_endm;    // [K][nb] endmember reflectances
  int off_win1;    // [nb]  1 if band in Omega_1 else 0
  int off_win2;    // [nb]  1 if band in Omega_2^hot U Omega_2^smol else 0
  int off_planck;  // [nt][n2s] B(lambda_b, T_j) for b in the stage-2 range
  int n2s;         // stage-2 range padded to a multiple of 32
  int total;       // floats, multiple of 4 (16-byte bulk copies)
};

struct KTables {
  int nb, nwv, K, nt;
  int b1lo, n1;            // stage-1 band range [b1lo, b1lo + n1)
  int b2lo, n2;            // stage-2 band range [b2lo, b2lo + n2)
  int bh, bl;              // HFDI band indices (2430 nm, 2061 nm)
  float tglo, tgstep;      // temperature grid T_j = tglo + j * tgstep
  const float4 *wvtab;     // [nwv][nb] (A tau_d tau_u, A rho_atm, S, tau_u), A = E0 cos/pi
  const float *sat;        // [nb] or nullptr
  const float *image;      // per-CTA table image in global memory
  ImageLayout lay;
  // stage-2 Planck grid as the bf16 tensor-core operand: three parts
  // (hi, mid, lo), each plrows x 64 nodes, K-major 128-byte-swizzled rows
  const unsigned char *plop;
  int plrows;              // n2 rounded up to a multiple of 8
  const float *planck_full;  // [nt][nb] B(lambda_b, T_j) over every band (residual spectrum)
  const double *planck64;    // [nt][n2] B(lambda_b, T_j) in FP64 over the stage-2 bands (posterior)
};

// KConfig::solver values (the public FIRE_SOLVER_LM / FIRE_SOLVER_ADAM)
constexpr int kSolverLM = 0, kSolverAdam = 1;

struct KConfig {
  float lo1[kMaxK + 2], hi1[kMaxK + 2], pm1[kMaxK + 2], pp1[kMaxK + 2];
  float lo2[6], hi2[6], pm2[6], pp2[6];
  float zk1[kMaxK + 2], zk2[6];   // 2 / (hi - lo), the z scale of Eq. (affine); 0 if hi = lo
  float init_alpha1, init_T1, init_sigma, init_mu_h_floor, init_mu_s_ceil;
  float init_eta_lo, init_eta_hi;
  int max_it1, max_it2;
  float tau0, tol_g, tol_x, tol_f, kappa_max, dfloor;
  float noise_rel, noise_abs;
  int weighted;             // 1: weights 1 / variance (noise model, or per-band sd)
  float hfdi_thresh;
  float ident_sd_et, ident_alpha_snr;
  long long wait_spins;     // polls of a bounded wait before it gives up
  int has_nsd;              // 1: the caller's per-band noise sd weight the loss
  int solver;               // kSolverLM / kSolverAdam
  int adam_steps1, adam_steps2;
  float adam_lr1, adam_lr2, adam_clip, adam_eps;
  float adam_b1, adam_b2, adam_omb1, adam_omb2;   // beta and 1 - beta, each rounded once
  double adam_b1d, adam_b2d;                      // beta for the bias corrections 1 - beta^t
  float nsd[kMaxBands];     // noise_sd_b (weights 1 / noise_sd_b^2)
};

// one scene of a batched call: device pointers, its own outputs
struct SceneItem {
  const float *rad;        // [n][nb]
  const uint16_t *wv;      // [n]
  long long n;
  struct KOutItem {
    float *state, *ET, *sdT, *alpha, *cov, *var_ET, *cost, *rms, *hfdi;
    uint8_t *status;
    uint16_t *iters;
    float *resid;
  } out;
};

struct KScene {
  int64_t n_pix;
  const float *rad;        // [n_pix][nb]
  const uint16_t *wv;      // [n_pix]
  const float *init;       // [n_pix][K+8] or nullptr (indexed like rad)
  const long long *idx;    // optional: fitted pixel i reads source row idx[i]
  const SceneItem *items;  // optional: batched scenes (global pixel index over all)
  const long long *prefix; // [n_items + 1] first global pixel of each scene
  int n_items;
  int claim;               // pixels claimed per atomic (autotuned)
  int gate;                // 1: HFDI gate
  int init_best;           // 1: stage 2 starts from the lower-cost of the given
                           //    start and the stage-1-derived one (learned start)
  int want_resid;          // 1: some output asks for the residual spectrum
};

struct KOut {
  float *state, *ET, *sdT, *alpha, *cov, *var_ET, *cost, *rms, *hfdi;
  uint8_t *status;
  uint16_t *iters;
  float *resid;            // [n][nb] or nullptr
};

// device counters, indices into KWork::stats
enum : int {
  ST_NPIX = 0, ST_IT1, ST_IT2, ST_FP64, ST_BAND1, ST_BAND2, ST_NODEBAND2, ST_S64_1, ST_S64_2, ST_MMA2,
  ST_POST64, ST_STATUS0,
  ST_COUNT = ST_STATUS0 + 8
};

struct KWork {
  unsigned long long *counter;  // [2] work-claim counters of the two stage kernels (zeroed)
  unsigned long long *stats;    // [ST_COUNT]
  int *err;                     // bounded-wait failure flag
  float *s1x;                   // [n_pix][K+2] stage-1 result handed to stage 2
  int *s1meta;                  // [n_pix] status bits | 256 if the pixel goes on to stage 2
  float *s2x;                   // [n_pix][31] stage-2 state, J^T W J + P, costs, counts
  float *s2g;                   // [n_pix][6] stage-2 gradient at the final state
  long long *fb_idx;            // learned-start fallback list (nullptr: no check)
  float *fb_cost;               // cost of each listed pixel's first fit
  unsigned long long *fb_count; // list length
};

struct LMLaunch {
  KTables t;
  KConfig c;
  KScene s;
  KOut o;
  KWork w;
};
// passed by value as a kernel parameter: within the 4 KB parameter space
static_assert(sizeof(LMLaunch) <= 4096, "LMLaunch exceeds the kernel parameter space");

// BF16 tensor-core GEMM C = A B^T (kernels_gemm.cu)
enum : int { EPI_F32 = 0, EPI_BIAS_RELU = 1, EPI_BIAS_TANH = 2, EPI_RELU_MASK = 3 };
struct GemmArgs {
  const __nv_bfloat16 *A, *B;   // [M][lda], [N][ldb], K-major
  long long lda, ldb;
  int M, N, K;
  int epi;
  const float *bias;            // [N] or nullptr
  const __nv_bfloat16 *mask;    // [M][ldm] (EPI_RELU_MASK)
  long long ldm;
  float *Cf;                    // [M][ldc] fp32 or nullptr
  long long ldc;
  __nv_bfloat16 *Cb;            // [M][ldcb] bf16 or nullptr
  long long ldcb;
  __nv_bfloat16 *CbT;           // [N][ldcbT] bf16 transposed or nullptr
  long long ldcbT;
  int accumulate;               // Cf += result
  int *err;                     // bounded-wait failure flag or nullptr
};
cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st);

// host-side launchers (kernels_*.cu)
cudaError_t launch_build_tables(const KTables &t, const float *wl, const float *e0, float cos_sza,
                                const float *td, const float *tu, const float *ra, const float *sa,
                                const float *endm, float *image, float4 *wvtab,
                                const float win[6], cudaStream_t st);
// ev: optional 4 events recorded before stage 1, after stage 1, after
// stage 2 and after the finalize kernel (per-kernel timing)
cudaError_t launch_lm(const LMLaunch &p, int num_sms, cudaStream_t st, int *blocks_used,
                      int variant = 0, cudaEvent_t *ev = nullptr);
size_t lm_smem_bytes(const KTables &t, int warps_per_cta = 8);
cudaError_t launch_merge_fallback(const long long *idx, const float *cost_first, long long nfb,
                                  const KOut &compact, const KOut &out, int K, int nb,
                                  cudaStream_t st);
// B(lambda_b, T_j) for every band and grid node, [nt][nb] (FP64, stored fp32)
cudaError_t launch_planck_full(const KTables &t, const float *wl, float *out, cudaStream_t st);
// B(lambda_b, T_j) over the stage-2 bands, [nt][n2], kept in FP64
cudaError_t launch_planck64(const KTables &t, const float *wl, double *out, cudaStream_t st);
// device allocations of the library: through the caller's allocator when
// one is installed (fire_set_allocator), else cudaMalloc / cudaFree
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
// variant: the launch shape whose stage-2 evaluation is used (as launch_lm)
cudaError_t launch_normal_eq(const LMLaunch &p, int stage, const float *states, float *H, float *g,
                             float *cost, cudaStream_t st, int variant = 0);
// stage-2 tensor-core path: operand size, its construction from the table
// image, and whether the tables fit the path (grid nodes <= 64, stage-2
// bands <= 256, shared memory)
size_t planck_operand_bytes(const KTables &t);
cudaError_t launch_planck_operand(const KTables &t, unsigned char *out, cudaStream_t st);
bool lm_tc_ok(const KTables &t);
cudaError_t launch_forward(const KTables &t, int mode, const float *state, const uint16_t *wv,
                           int64_t n, float noise_rel, float noise_abs, uint64_t seed,
                           uint64_t stream_id, int64_t pix0, float *out, cudaStream_t st);
// water-vapour presolve: the 940 nm depths of the table's bins (increasing)
struct WvLut {
  float D[256];
  int n;
};
cudaError_t launch_wv_presolve(const float *rad, int nb, long long W, long long H, int B, int blo,
                               int bc, int bhi, float cf, const float *sat, const WvLut &lut,
                               uint16_t *bins, float *depth, cudaStream_t st);
cudaError_t launch_inject(const KTables &t, const float *wl, const float *bg, const uint16_t *wv,
                          const float *alpha, const float *T, long long n, float *out, cudaStream_t st);
cudaError_t launch_hfdi(const float *rad, int nb, long long n, int bhi, int blo, float *out,
                        cudaStream_t st);
cudaError_t launch_block_mean(const float *src, int w, int h, int nb, int blk, float *dst,
                              cudaStream_t st);

}  // namespace firert
