/* oracle.h — plain FP64 CPU oracle of the per-pixel wildfire-temperature
 * retrieval (forward model Eq. fm/solar/thermal, loss Eq. loss, bounds
 * Eq. affine, two-stage fit of Sec. 2.6, moment matching Sec. 2.3).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links or calls
 * this code; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code, header or table with the CUDA
 * path.
 */
#ifndef FIRE_ORACLE_H
#define FIRE_ORACLE_H
#include <stdint.h>

#define ORC_MAXB 512      /* bands */
#define ORC_MAXK 8        /* endmembers */
#define ORC_MAXT 256      /* temperature-grid nodes */
#define ORC_NS1 (ORC_MAXK + 2)
#define ORC_NS2 6
#define ORC_NSTATE (ORC_MAXK + 8)
#define ORC_MAXWV 256     /* water-vapour bins */

/* per-pixel status: low 3 bits = outcome, upper bits = flags */
enum {
  ORC_CONVERGED = 0, ORC_MAXITER = 1, ORC_NONFINITE = 2, ORC_ALL_MASKED = 3,
  ORC_CHOL_FAIL = 4, ORC_NOT_CANDIDATE = 5,
  ORC_F_FP64 = 8, ORC_F_NOT_IDENT = 16, ORC_F_MLP_FALLBACK = 32, ORC_F_S1_MAXITER = 64
};

typedef struct {
  int32_t n_bands, n_wv, n_endm, n_tgrid;
  const float *wavelength_nm;   /* [n_bands] nm */
  const float *solar_irr;       /* [n_bands] W m^-2 nm^-1 */
  double cos_sza;
  const float *tau_down, *tau_up, *rho_atm, *sph_alb;  /* [n_wv][n_bands] */
  const float *endmembers;      /* [n_endm][n_bands] */
  const float *sat_level;       /* [n_bands] or NULL */
  double tgrid_lo, tgrid_hi;
} orc_tables_t;

typedef struct {
  double win1_lo, win1_hi;            /* Omega_1 (nm) */
  double win2h_lo, win2h_hi;          /* Omega_2 hot */
  double win2s_lo, win2s_hi;          /* Omega_2 smouldering */
  double lo1[ORC_NS1], hi1[ORC_NS1];  /* stage-1 bounds, layout [x_surf(K), a1, T1] */
  double lo2[ORC_NS2], hi2[ORC_NS2];  /* stage-2 bounds [mu_h, s_h, mu_s, s_s, eta, a] */
  double pm1[ORC_NS1], pp1[ORC_NS1];  /* prior mean / precision in z (0 = off) */
  double pm2[ORC_NS2], pp2[ORC_NS2];
  double init_alpha1, init_T1, init_sigma, init_mu_h_floor, init_mu_s_ceil;
  double init_eta_lo, init_eta_hi;
  int32_t max_it1, max_it2;
  double tau0, tol_g, tol_x, tol_f, kappa_max, dfloor;
  double noise_rel, noise_abs;        /* noise model sd^2 = (rel L)^2 + abs^2 */
  int32_t weighted;                   /* 0: Eq. (loss) as printed; 1: weights 1/sd^2 */
  int32_t gate_hfdi;
  double hfdi_thresh, hfdi_lambda_hi, hfdi_lambda_lo;
  double ident_sd_et, ident_alpha_snr;
  const float *noise_sd;              /* [n_bands] per-band noise sd, or NULL; when given
                                         the loss is weighted by 1 / sd_b^2 */
  int32_t solver;                     /* ORC_SOLVER_LM or ORC_SOLVER_ADAM */
  int32_t adam_steps1, adam_steps2;   /* Adam steps per stage (Sec. 2.6: 30, 100) */
  double adam_lr1, adam_lr2;          /* learning rates (Sec. 2.6: 0.03, 0.015) */
  double adam_clip;                   /* global-norm gradient clip */
  double adam_beta1, adam_beta2, adam_eps;   /* Eq. (adam): 0.9, 0.999, 1e-8 */
  /* Sensitivity probe for tests, not part of the method (0 = off): at each
   * Adam step the gradient is formed as if every band's model value were
   * off by a relative adam_gnoise times a standard normal drawn from
   * SplitMix64 keyed by (adam_gseed, pixel, stage, step, band): the size of
   * the rounding of a single-precision evaluation of the model. */
  double adam_gnoise;
  uint64_t adam_gseed;
} orc_config_t;

enum { ORC_SOLVER_LM = 0, ORC_SOLVER_ADAM = 1 };

typedef struct {
  double *state;     /* [n][K+8] = [x_surf, a1, T1, mu_h, s_h, mu_s, s_s, eta, a] */
  double *ET, *sdT, *alpha, *var_ET, *cost, *rms, *hfdi, *cost1, *kappa;
  double *cov;       /* [n][21] packed upper, physical units, stage-2 order */
  int32_t *status, *it1, *it2, *n_used;
} orc_outputs_t;

double orc_planck(double lambda_nm, double T);
double orc_planck_dT(double lambda_nm, double T);
void orc_moments(const double *x2, double *E, double *Var);
void orc_simplex_project(double *v, int K);
int orc_cholesky(double *A, int n);
void orc_chol_solve(const double *L, int n, double *b);
void orc_forward(const orc_tables_t *t, int mode, const double *state,
                 const uint16_t *wv_bin, int64_t n, double *L_out);
void orc_stage_jacobian(const orc_tables_t *t, int stage, const double *xs,
                        const double *x, int wv_bin, double *L, double *J);
double orc_hfdi(const orc_tables_t *t, const orc_config_t *c, const float *L);
void orc_retrieve(const orc_tables_t *t, const orc_config_t *c, const float *radiance,
                  const uint16_t *wv_bin, int64_t n, const double *init_state,
                  orc_outputs_t *o, int n_threads);
void orc_synth_radiance(const orc_tables_t *t, int mode, const double *state,
                        const uint16_t *wv_bin, const double *normals, int64_t n,
                        double noise_rel, double noise_abs, float *L_out);
void orc_planck_array(int64_t n, const double *lambda_nm, const double *T, double *out);
void orc_mlp_forward(int B, int Din, int H, int Dout, const double *W1, const double *b1,
                     const double *W2, const double *b2, const double *W3, const double *b3,
                     const double *x, double *a1, double *a2, double *z);
double orc_mlp_backward(int B, int Din, int H, int Dout, int n_out, const double *W1,
                        const double *W2, const double *W3, const double *x, const double *a1,
                        const double *a2, const double *z, const double *t, const double *mask,
                        double *gW1, double *gb1, double *gW2, double *gb2, double *gW3,
                        double *gb3);
void orc_adam(int64_t n, double *w, const double *g, double *m, double *v, int t, double lr,
              double b1, double b2, double eps);
void orc_posterior_at(const orc_tables_t *t, const orc_config_t *c, const float *Lrow, int w,
                      const double *state, double *ET, double *sdT, double *cost, double *rms,
                      double *cov21, double *var_ET, int *ident);
void orc_inject(const orc_tables_t *t, const float *L_bg, const uint16_t *wv_bin, const double *alpha,
                const double *T, int64_t n, float *L_out);
void orc_wv_depth_table(const orc_tables_t *t, double lam_lo, double lam_c, double lam_hi,
                        float *D);
void orc_wv_presolve(const orc_tables_t *t, const float *radiance, int64_t width, int64_t height,
                     int block, double lam_lo, double lam_c, double lam_hi, uint16_t *bin_out,
                     float *depth_out);
void orc_normal_equations(const orc_tables_t *t, const orc_config_t *c, int stage,
                          const float *Lrow, int w, const double *x, double *Hout, double *gout,
                          double *cost_out);
#endif
