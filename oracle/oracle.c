/* oracle.c — plain FP64 CPU oracle of the per-pixel wildfire-temperature
 * retrieval of Keely et al., "Real-time physics inversion for retrieval of
 * sub-pixel wildfire temperatures from VSWIR imaging spectroscopy".
 *
 * TEST INFRASTRUCTURE ONLY: the product library never links or calls this
 * file. It is deliberately slow and direct: every band, every temperature
 * node and every matrix entry is computed from its definition in double
 * precision, with no blocking, fusion or reordering.
 *
 * What each part follows:
 *   Planck radiance B(lambda, T)          Eq. (thermal), Sec. 2.3 (formula
 *                                         not printed; CODATA SI constants,
 *                                         per-nm radiance)
 *   solar term                            Eq. (solar), Sec. 2.3
 *   surface mixture on the simplex        Sec. 2.3 (reflectance mixture)
 *   thermal term on the temperature grid  Eq. (thermal), grid [350, 2200] K
 *   two-component mixture, moments        Sec. 2.3 (E[T], Var[T])
 *   windowed masked loss                  Eq. (loss), Sec. 2.6
 *   affine bound map and clipping         Eq. (affine), Sec. 2.6
 *   simplex projection                    Sec. 2.6 (Euclidean projection,
 *                                         sort-based, Duchi et al. 2008)
 *   stage 1 / stage 2 structure           Sec. 2.6
 *   HFDI gate                             Sec. 2.1
 * Two optimisers: a damped Gauss-Newton (Levenberg-Marquardt) iteration,
 * whose rules and constants are a stated reading (Nielsen's damping update;
 * active-set handling of bounds; simplex handled in a reduced basis), and the
 * paper's own Adam (Sec. 2.6, Eq. adam: fixed step counts and learning rates
 * per stage, global-norm clip, z clip, simplex projection after each step).
 *
 * Parity unpinned: the per-pixel fit values themselves have no worked
 * example in the paper; the pieces are pinned by closed forms, brute force,
 * finite differences and noise-free recovery.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact SI values */
#define ORC_HPLANCK 6.62607015e-34
#define ORC_CLIGHT 299792458.0
#define ORC_KBOLTZ 1.380649e-23

/* ------------------------------------------------------------ Planck --- */
/* Blackbody spectral radiance in W m^-2 sr^-1 nm^-1 at wavelength
 * lambda_nm and temperature T (K): 2 h c^2 / lambda^5 / (exp(hc/(lambda k T)) - 1),
 * evaluated with lambda in metres, then scaled from per-metre to per-nm. */
double orc_planck(double lambda_nm, double T) {
  double lam = lambda_nm * 1e-9;
  double x = ORC_HPLANCK * ORC_CLIGHT / (lam * ORC_KBOLTZ * T);
  double c1 = 2.0 * ORC_HPLANCK * ORC_CLIGHT * ORC_CLIGHT;
  return c1 / pow(lam, 5) / expm1(x) * 1e-9;
}

/* dB/dT = B * (x/T) * e^x / (e^x - 1) = B * (x/T) / (1 - e^-x) */
double orc_planck_dT(double lambda_nm, double T) {
  double lam = lambda_nm * 1e-9;
  double x = ORC_HPLANCK * ORC_CLIGHT / (lam * ORC_KBOLTZ * T);
  return orc_planck(lambda_nm, T) * (x / T) / (-expm1(-x));
}

/* --------------------------------------------------- moment matching --- */
/* Sec. 2.3: E[T] = eta mu_h + (1-eta) mu_s,
 * Var[T] = eta s_h^2 + (1-eta) s_s^2 + eta (1-eta) (mu_h - mu_s)^2 */
void orc_moments(const double *x2, double *E, double *Var) {
  double mh = x2[0], sh = x2[1], ms = x2[2], ss = x2[3], eta = x2[4];
  *E = eta * mh + (1.0 - eta) * ms;
  *Var = eta * sh * sh + (1.0 - eta) * ss * ss + eta * (1.0 - eta) * (mh - ms) * (mh - ms);
}

/* ---------------------------------------------- simplex projection ---- */
/* Euclidean projection onto {v >= 0, sum v = 1} (Duchi et al. 2008): sort
 * descending, find the largest j with u_j > (sum_{i<=j} u_i - 1)/j, shift
 * by that threshold and clip at zero. */
static int cmp_desc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x < y) - (x > y);
}
void orc_simplex_project(double *v, int K) {
  double u[ORC_MAXK];
  memcpy(u, v, sizeof(double) * K);
  qsort(u, K, sizeof(double), cmp_desc);
  double cs = 0.0, theta = 0.0;
  for (int j = 0; j < K; j++) {
    cs += u[j];
    double t = (cs - 1.0) / (j + 1);
    if (u[j] - t > 0) theta = t;
  }
  for (int k = 0; k < K; k++) v[k] = v[k] - theta > 0 ? v[k] - theta : 0.0;
}

/* --------------------------------------------------------- Cholesky --- */
/* In-place lower Cholesky of an n x n row-major SPD matrix; -1 on a
 * non-positive pivot. */
int orc_cholesky(double *A, int n) {
  for (int j = 0; j < n; j++) {
    double d = A[j * n + j];
    for (int k = 0; k < j; k++) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double s = A[i * n + j];
      for (int k = 0; k < j; k++) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
    for (int i = 0; i < j; i++) A[i * n + j] = 0.0;
  }
  return 0;
}

/* Solve L L^T y = b in place. */
void orc_chol_solve(const double *L, int n, double *b) {
  for (int i = 0; i < n; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= L[i * n + k] * b[k];
    b[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = b[i];
    for (int k = i + 1; k < n; k++) s -= L[k * n + i] * b[k];
    b[i] = s / L[i * n + i];
  }
}

/* ------------------------------------------------------ pixel context --- */
typedef struct {
  const orc_tables_t *t;
  int nb, K, w;
  double A[ORC_MAXB];                    /* E0 cos(theta_s) / pi */
  double td[ORC_MAXB], tu[ORC_MAXB], ra[ORC_MAXB], S[ORC_MAXB];
  double lam[ORC_MAXB];
  double Lobs[ORC_MAXB];
  double wgt[ORC_MAXB];                  /* noise weight, 0 = masked band */
  double Ls[ORC_MAXB];                   /* solar term, fixed in stage 2 */
  double Tg[ORC_MAXT];
  int nt;
  const double *Bt;                      /* B(lambda_b, T_j), [nt][nb] */
} pix_t;

/* B(lambda_b, T_j) for every band and grid node, computed once per call */
static double *planck_table(const orc_tables_t *t) {
  int nb = t->n_bands, nt = t->n_tgrid;
  double *Bt = (double *)malloc(sizeof(double) * nb * nt);
  for (int j = 0; j < nt; j++) {
    double T = t->tgrid_lo + j * (t->tgrid_hi - t->tgrid_lo) / (nt - 1);
    for (int b = 0; b < nb; b++) Bt[j * nb + b] = orc_planck(t->wavelength_nm[b], T);
  }
  return Bt;
}

static void pix_tables(pix_t *P, const orc_tables_t *t, int w, const double *Bt) {
  P->t = t;
  P->Bt = Bt;
  P->nb = t->n_bands;
  P->K = t->n_endm;
  P->w = w;
  P->nt = t->n_tgrid;
  for (int b = 0; b < P->nb; b++) {
    P->A[b] = (double)t->solar_irr[b] * t->cos_sza / M_PI;
    P->td[b] = t->tau_down[(size_t)w * P->nb + b];
    P->tu[b] = t->tau_up[(size_t)w * P->nb + b];
    P->ra[b] = t->rho_atm ? t->rho_atm[(size_t)w * P->nb + b] : 0.0;
    P->S[b] = t->sph_alb ? t->sph_alb[(size_t)w * P->nb + b] : 0.0;
    P->lam[b] = t->wavelength_nm[b];
  }
  for (int j = 0; j < P->nt; j++)
    P->Tg[j] = t->tgrid_lo + j * (t->tgrid_hi - t->tgrid_lo) / (P->nt - 1);
}

/* Eq. (solar) with rho = sum_k x_k rho_k; also dLs/dx_k if dLs != NULL. */
static double solar_term(const pix_t *P, int b, const double *xs, double *dLs) {
  const orc_tables_t *t = P->t;
  double rho = 0.0;
  for (int k = 0; k < P->K; k++) rho += xs[k] * t->endmembers[(size_t)k * P->nb + b];
  double den = 1.0 - P->S[b] * rho;
  if (dLs)
    for (int k = 0; k < P->K; k++)
      dLs[k] = P->A[b] * P->td[b] * P->tu[b] * t->endmembers[(size_t)k * P->nb + b] / (den * den);
  return P->A[b] * (P->ra[b] + P->td[b] * P->tu[b] * rho / den);
}

/* Normalised Gaussian weights on the grid: w_j = u_j / sum u,
 * u_j = exp(-(T_j - mu)^2 / (2 s^2)) — the discrete p(T) of Eq. (thermal). */
static void grid_weights(const pix_t *P, double mu, double s, double *wj) {
  double U = 0.0;
  for (int j = 0; j < P->nt; j++) {
    double d = P->Tg[j] - mu;
    wj[j] = exp(-d * d / (2.0 * s * s));
    U += wj[j];
  }
  for (int j = 0; j < P->nt; j++) wj[j] /= U;
}

/* One mixture component at band b: Bbar = sum_j w_j B(lambda_b, T_j) and its
 * derivatives with respect to mu and s. With d_j = T_j - mu,
 *   dw_j/dmu = w_j (d_j - dbar) / s^2,  dw_j/ds = w_j (d_j^2 - m2) / s^3,
 * dbar = sum w_j d_j, m2 = sum w_j d_j^2. */
static void component(const pix_t *P, int b, double mu, double s, const double *wj,
                      double *Bbar, double *dmu, double *ds) {
  double S0 = 0, S1 = 0, S2 = 0, dbar = 0, m2 = 0;
  for (int j = 0; j < P->nt; j++) {
    double d = P->Tg[j] - mu;
    double B = P->Bt[j * P->nb + b];
    S0 += wj[j] * B;
    S1 += wj[j] * d * B;
    S2 += wj[j] * d * d * B;
    dbar += wj[j] * d;
    m2 += wj[j] * d * d;
  }
  *Bbar = S0;
  if (dmu) *dmu = (S1 - dbar * S0) / (s * s);
  if (ds) *ds = (S2 - m2 * S0) / (s * s * s);
}

/* Stage-1 model (Sec. 2.6): x = [x_surf(K), a1, T1], single-temperature
 * thermal term a1 tau_up B(lambda, T1). Fills L[b] for every band and
 * J[b*p + i] = dL_b/dx_i (physical units). */
static void eval_stage1(const pix_t *P, const double *x, const double *use, double *L, double *J) {
  int K = P->K, p = K + 2;
  double a1 = x[K], T1 = x[K + 1];
  double dLs[ORC_MAXK];
  for (int b = 0; b < P->nb; b++) {
    if (use && !(use[b] > 0)) continue;
    double Ls = solar_term(P, b, x, J ? dLs : NULL);
    double B = orc_planck(P->lam[b], T1);
    L[b] = Ls + a1 * P->tu[b] * B;
    if (J) {
      for (int k = 0; k < K; k++) J[b * p + k] = dLs[k];
      J[b * p + K] = P->tu[b] * B;
      J[b * p + K + 1] = a1 * P->tu[b] * orc_planck_dT(P->lam[b], T1);
    }
  }
}

/* Stage-2 model (Sec. 2.6, reading: the model's p(T) is the two-component
 * mixture eta N(mu_h, s_h) + (1-eta) N(mu_s, s_s) on the grid; the moment-
 * matched Gaussian is the reported summary). x = [mu_h, s_h, mu_s, s_s, eta, a];
 * the solar term P->Ls is fixed from stage 1. */
static void eval_stage2(const pix_t *P, const double *x, const double *use, double *L, double *J) {
  double mh = x[0], sh = x[1], ms = x[2], ss = x[3], eta = x[4], a = x[5];
  double wh[ORC_MAXT], ws[ORC_MAXT];
  grid_weights(P, mh, sh, wh);
  grid_weights(P, ms, ss, ws);
  for (int b = 0; b < P->nb; b++) {
    if (use && !(use[b] > 0)) continue;
    double Bh, dmh, dsh, Bs, dms, dss;
    component(P, b, mh, sh, wh, &Bh, J ? &dmh : NULL, J ? &dsh : NULL);
    component(P, b, ms, ss, ws, &Bs, J ? &dms : NULL, J ? &dss : NULL);
    double tu = P->tu[b];
    L[b] = P->Ls[b] + a * tu * (eta * Bh + (1.0 - eta) * Bs);
    if (J) {
      J[b * 6 + 0] = a * tu * eta * dmh;
      J[b * 6 + 1] = a * tu * eta * dsh;
      J[b * 6 + 2] = a * tu * (1.0 - eta) * dms;
      J[b * 6 + 3] = a * tu * (1.0 - eta) * dss;
      J[b * 6 + 4] = a * tu * (Bh - Bs);
      J[b * 6 + 5] = tu * (eta * Bh + (1.0 - eta) * Bs);
    }
  }
}

/* ------------------------------------------------------------- LM ------ */
typedef struct {
  int stage, p, nsimp;       /* nsimp: leading variables constrained to the simplex */
  const double *lo, *hi, *pm, *pp;
  const double *wst;         /* per-band weight for this stage (0 = not used) */
  int max_it;
  double psc;                /* prior scale: mean noise variance of the used bands
                                (unweighted loss) or 1 (noise-weighted loss) */
  int64_t pix;               /* pixel index (keys the Adam sensitivity probe) */
} lm_prob_t;

typedef struct {
  int iters, status, used64, n_used;
  double cost, kappa;
  int active[ORC_NS1];       /* final active set (full coordinates) */
  double H[ORC_NS1 * ORC_NS1];  /* final J^T W J + P in full z coordinates */
} lm_res_t;

/* Eq. (affine): z = 2 (x - lo) / (hi - lo) - 1; a variable with lo == hi is
 * held fixed (its z is 0 and its Jacobian column is zero). */
static double zcoord(const lm_prob_t *q, const double *x, int i) {
  return q->hi[i] > q->lo[i] ? 2.0 * (x[i] - q->lo[i]) / (q->hi[i] - q->lo[i]) - 1.0 : 0.0;
}

static void evaluate(const pix_t *P, const lm_prob_t *q, const double *x, double *L, double *J) {
  if (q->stage == 1) eval_stage1(P, x, q->wst, L, J);
  else eval_stage2(P, x, q->wst, L, J);
}

/* cost = sum_b w_b (Lobs - L)^2 + psc sum_i pp_i (z_i - pm_i)^2: Eq. (loss)
 * plus a weak diagonal Gaussian prior in z whose precision pp is counted in
 * units of one band's noise variance psc, so it stays dimensionless. */
static double cost_of(const pix_t *P, const lm_prob_t *q, const double *x, const double *L) {
  double c = 0.0;
  for (int b = 0; b < P->nb; b++)
    if (q->wst[b] > 0) {
      double r = P->Lobs[b] - L[b];
      c += q->wst[b] * r * r;
    }
  for (int i = 0; i < q->p; i++) {
    double z = zcoord(q, x, i);
    c += q->psc * q->pp[i] * (z - q->pm[i]) * (z - q->pm[i]);
  }
  return c;
}

/* Full-coordinate gradient g = Jz^T W r - psc P (z - pm), H = Jz^T W Jz + psc P,
 * with Jz = Jx * s, s_i = (hi_i - lo_i)/2 (Eq. affine). */
static void normal_eq(const pix_t *P, const lm_prob_t *q, const double *x, const double *L,
                      const double *J, double *H, double *g) {
  int p = q->p;
  double s[ORC_NS1];
  for (int i = 0; i < p; i++) s[i] = 0.5 * (q->hi[i] - q->lo[i]);
  memset(H, 0, sizeof(double) * p * p);
  memset(g, 0, sizeof(double) * p);
  for (int b = 0; b < P->nb; b++) {
    if (!(q->wst[b] > 0)) continue;
    double r = P->Lobs[b] - L[b];
    for (int i = 0; i < p; i++) {
      g[i] += q->wst[b] * J[b * p + i] * s[i] * r;
      for (int k = 0; k < p; k++) H[i * p + k] += q->wst[b] * J[b * p + i] * s[i] * J[b * p + k] * s[k];
    }
  }
  for (int i = 0; i < p; i++) {
    double z = zcoord(q, x, i);
    g[i] -= q->psc * q->pp[i] * (z - q->pm[i]);
    H[i * p + i] += q->psc * q->pp[i];
  }
}

/* Reduced basis E (p x pr): the simplex group keeps sum x = 1 by pairing
 * each fraction k != m with the largest fraction m (column e_k - e_m);
 * every other variable is its own column. Returns pr. */
static int reduced_basis(const lm_prob_t *q, const double *x, double *E, int *m_out) {
  int p = q->p, col = 0, m = -1;
  memset(E, 0, sizeof(double) * p * p);
  if (q->nsimp > 0) {
    m = 0;
    for (int k = 1; k < q->nsimp; k++)
      if (x[k] > x[m]) m = k;
    for (int k = 0; k < q->nsimp; k++) {
      if (k == m) continue;
      E[k * p + col] = 1.0;
      E[m * p + col] = -1.0;
      col++;
    }
  }
  for (int i = q->nsimp; i < p; i++) E[i * p + col++] = 1.0;
  *m_out = m;
  return col;
}

/* Apply a z-step to x: a variable pinned on a bound by the step solve is set
 * exactly to that bound (pdir -1 = lo, +1 = hi, 0 = free), box variables
 * are clipped to [lo, hi], the simplex group is projected onto the unit
 * simplex (Sec. 2.6). */
static void step_project(const lm_prob_t *q, const double *x, const double *dz, const int *pdir,
                         double *xt) {
  for (int i = 0; i < q->p; i++) {
    double s = 0.5 * (q->hi[i] - q->lo[i]);
    xt[i] = x[i] + s * dz[i];
    if (pdir[i] < 0) xt[i] = q->lo[i];
    if (pdir[i] > 0) xt[i] = q->hi[i];
    if (i >= q->nsimp) {
      if (xt[i] < q->lo[i]) xt[i] = q->lo[i];
      if (xt[i] > q->hi[i]) xt[i] = q->hi[i];
    }
  }
  if (q->nsimp > 0) orc_simplex_project(xt, q->nsimp);
}

static int lm_fit(const pix_t *P, const lm_prob_t *q, const orc_config_t *c, double *x, lm_res_t *res) {
  int p = q->p, nb = P->nb;
  double L[ORC_MAXB], Lt[ORC_MAXB];
  double *J = (double *)malloc(sizeof(double) * nb * p);
  double H[ORC_NS1 * ORC_NS1], g[ORC_NS1], E[ORC_NS1 * ORC_NS1];
  double Hr[ORC_NS1 * ORC_NS1], gr[ORC_NS1], xt[ORC_NS1], dz[ORC_NS1];
  double lam = -1.0, nu = 2.0;
  int it = 0, status = ORC_MAXITER, fresh = 1, pr = 0, m = -1;
  int act[ORC_NS1];
  res->used64 = 0;
  res->kappa = 0.0;
  res->n_used = 0;
  for (int b = 0; b < nb; b++) res->n_used += q->wst[b] > 0;

  evaluate(P, q, x, L, J);
  double cost = cost_of(P, q, x, L);
  for (it = 0; it < q->max_it;) {
    if (fresh) {
      normal_eq(P, q, x, L, J, H, g);
      pr = reduced_basis(q, x, E, &m);
      /* reduced system Hr = E^T H E, gr = E^T g */
      for (int a = 0; a < pr; a++) {
        gr[a] = 0;
        for (int i = 0; i < p; i++) gr[a] += E[i * p + a] * g[i];
        for (int bb = 0; bb < pr; bb++) {
          double s = 0;
          for (int i = 0; i < p; i++)
            for (int k = 0; k < p; k++) s += E[i * p + a] * H[i * p + k] * E[k * p + bb];
          Hr[a * pr + bb] = s;
        }
      }
      /* active set: a reduced variable sits on a bound and the Gauss-Newton
       * direction points outwards */
      for (int a = 0; a < pr; a++) {
        int i = -1;
        for (int k = 0; k < p; k++)
          if (E[k * p + a] == 1.0) { i = k; break; }
        int lo_hit = x[i] <= q->lo[i], hi_hit = i >= q->nsimp && x[i] >= q->hi[i];
        act[a] = (lo_hit && gr[a] <= 0) || (hi_hit && gr[a] >= 0);
      }
      /* convergence on the scaled gradient of the free variables */
      int small = 1;
      for (int a = 0; a < pr; a++)
        if (!act[a] && fabs(gr[a]) > c->tol_g * sqrt(Hr[a * pr + a] * cost)) small = 0;
      if (small) { status = ORC_CONVERGED; break; }
      /* initial damping: D = diag(Hr) below, so lam is the relative damping
       * of each diagonal and starts at tau0 */
      if (lam < 0) lam = c->tau0;
      fresh = 0;
    }
    /* damped solve (Hr_FF + lam D) d = gr_F, D = diag(Hr) floored, on the
     * diagonally scaled matrix. A free variable whose step would leave its
     * bound is pinned at that bound and the rest re-solved with the pinned
     * displacement moved to the right-hand side (projected Newton step). */
    double mxd = 0, Dg[ORC_NS1];
    for (int a = 0; a < pr; a++)
      if (!act[a] && Hr[a * pr + a] > mxd) mxd = Hr[a * pr + a];
    for (int a = 0; a < pr; a++) Dg[a] = Hr[a * pr + a] < c->dfloor * mxd ? c->dfloor * mxd : Hr[a * pr + a];
    int pin[ORC_NS1], pdir[ORC_NS1];
    double dr[ORC_NS1];
    for (int a = 0; a < pr; a++) { pin[a] = act[a]; dr[a] = 0.0; pdir[a] = 0; }
    int ok = 0;
    for (int pass = 0; pass <= pr; pass++) {
      int F[ORC_NS1], nf = 0;
      for (int a = 0; a < pr; a++)
        if (!pin[a]) F[nf++] = a;
      if (nf == 0) break;
      double M[ORC_NS1 * ORC_NS1], d[ORC_NS1], y[ORC_NS1];
      for (int u = 0; u < nf; u++) {
        for (int v = 0; v < nf; v++) M[u * nf + v] = Hr[F[u] * pr + F[v]];
        M[u * nf + u] += lam * Dg[F[u]];
        double rhs = gr[F[u]];
        for (int a = 0; a < pr; a++)
          if (pin[a]) rhs -= Hr[F[u] * pr + a] * dr[a];
        y[u] = rhs;
      }
      for (int u = 0; u < nf; u++) d[u] = sqrt(M[u * nf + u]);
      for (int u = 0; u < nf; u++) {
        for (int v = 0; v < nf; v++) M[u * nf + v] /= (d[u] * d[v]);
        y[u] /= d[u];
      }
      ok = orc_cholesky(M, nf);
      if (ok != 0) break;
      double lmax = 0, lmin = 1e300;
      for (int u = 0; u < nf; u++) {
        if (M[u * nf + u] > lmax) lmax = M[u * nf + u];
        if (M[u * nf + u] < lmin) lmin = M[u * nf + u];
      }
      double kap = (lmax / lmin) * (lmax / lmin);
      if (kap > res->kappa) res->kappa = kap;
      if (kap > c->kappa_max) res->used64 = 1;
      orc_chol_solve(M, nf, y);
      for (int u = 0; u < nf; u++) dr[F[u]] = y[u] / d[u];
      /* bound violations of the free variables (reduced variable a moves full
       * variable i by s_i * dr[a] in physical units) */
      int viol = 0;
      for (int u = 0; u < nf; u++) {
        int a = F[u], i = -1;
        for (int k = 0; k < p; k++)
          if (E[k * p + a] == 1.0) { i = k; break; }
        double s = 0.5 * (q->hi[i] - q->lo[i]);
        double xn = x[i] + s * dr[a];
        if (!(s > 0)) { pin[a] = 1; dr[a] = 0.0; viol = 1; }
        else if (xn < q->lo[i]) { pin[a] = 1; pdir[a] = -1; dr[a] = (q->lo[i] - x[i]) / s; viol = 1; }
        else if (i >= q->nsimp && xn > q->hi[i]) {
          pin[a] = 1; pdir[a] = 1; dr[a] = (q->hi[i] - x[i]) / s; viol = 1;
        }
      }
      if (!viol) break;
    }
    if (ok != 0) {
      /* damped matrix not positive definite: treat as a rejected step */
      lam *= nu; nu *= 2.0; it++;
      if (!(lam < 1e300)) { status = ORC_CHOL_FAIL; break; }
      continue;
    }
    int pfull[ORC_NS1];
    for (int i = 0; i < p; i++) {
      dz[i] = 0;
      pfull[i] = 0;
      for (int a = 0; a < pr; a++) {
        dz[i] += E[i * p + a] * dr[a];
        if (E[i * p + a] == 1.0) pfull[i] = pdir[a];
      }
    }
    step_project(q, x, dz, pfull, xt);
    /* actual step in z and its reduced coordinates */
    double Dz[ORC_NS1], Dr[ORC_NS1], dmax = 0;
    for (int i = 0; i < p; i++) {
      Dz[i] = q->hi[i] > q->lo[i] ? (xt[i] - x[i]) / (0.5 * (q->hi[i] - q->lo[i])) : 0.0;
      if (fabs(Dz[i]) > dmax) dmax = fabs(Dz[i]);
    }
    if (dmax < c->tol_x) { status = ORC_CONVERGED; break; }
    {
      int col = 0;
      if (q->nsimp > 0)
        for (int k = 0; k < q->nsimp; k++)
          if (k != m) Dr[col++] = Dz[k];
      for (int i = q->nsimp; i < p; i++) Dr[col++] = Dz[i];
    }
    it++;
    evaluate(P, q, xt, Lt, NULL);
    double ct = cost_of(P, q, xt, Lt);
    /* predicted decrease of the Gauss-Newton model: 2 gr.D - D.Hr.D */
    double pred = 0;
    for (int a = 0; a < pr; a++) {
      pred += 2.0 * gr[a] * Dr[a];
      for (int bb = 0; bb < pr; bb++) pred -= Dr[a] * Hr[a * pr + bb] * Dr[bb];
    }
    double rho = pred > 0 ? (cost - ct) / pred : -1.0;
    if (rho > 0) {
      double rel = (cost - ct) / cost;
      memcpy(x, xt, sizeof(double) * p);
      cost = ct;
      double f = 1.0 - pow(2.0 * rho - 1.0, 3);
      lam *= f > 1.0 / 3.0 ? f : 1.0 / 3.0;
      nu = 2.0;
      evaluate(P, q, x, L, J);
      fresh = 1;
      if (rel < c->tol_f) { status = ORC_CONVERGED; break; }
    } else {
      lam *= nu;
      nu *= 2.0;
    }
  }
  normal_eq(P, q, x, L, J, H, g); /* L, J are at the final x */
  /* final active set in full coordinates: box variables on a bound whose
   * gradient points outwards */
  for (int i = 0; i < p; i++) {
    res->active[i] = (x[i] <= q->lo[i] && g[i] <= 0) || (x[i] >= q->hi[i] && g[i] >= 0);
  }
  memcpy(res->H, H, sizeof(double) * p * p);
  res->iters = it;
  res->status = status;
  res->cost = cost;
  free(J);
  return status;
}

/* ------------------------------------------------------------ Adam ---- */
/* The paper's optimiser (Sec. 2.6, Eq. adam): a fixed number of Adam steps
 * in the z coordinates of Eq. (affine) on Eq. (loss). At each step t =
 * 1..steps:
 *   g_t   = grad_z L(x(z_{t-1})) = -2 Jz^T W r  (no prior: Eq. loss as printed),
 *   g_t  <- g_t min(1, clip / ||g_t||_2)         (global-norm clip),
 *   m_t   = beta1 m_{t-1} + (1 - beta1) g_t,  v_t = beta2 v_{t-1} + (1 - beta2) g_t^2,
 *   z_t   = z_{t-1} - lr mhat_t / (sqrt(vhat_t) + eps),
 *           mhat_t = m_t / (1 - beta1^t), vhat_t = v_t / (1 - beta2^t),
 * then z_t is clipped to [-1, 1] and the surface fractions (the simplex
 * group) are projected onto the unit simplex. Every variable, the fractions
 * included, moves on its own z coordinate. The result is the state after the
 * last step; its cost, normal matrix and active set are formed there for the
 * posterior, as after an LM fit. */
/* SplitMix64 (Steele, Lea and Flood 2014) and a Box-Muller normal from two
 * of its outputs: the counter-based draws of the Adam sensitivity probe. */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static double probe_normal(uint64_t seed, int64_t pix, int stage, int step, int i) {
  uint64_t k = splitmix64(seed ^ splitmix64((uint64_t)pix * 4096u + (uint64_t)stage * 1024u + (uint64_t)i));
  uint64_t a = splitmix64(k + 2u * (uint64_t)step), b = splitmix64(k + 2u * (uint64_t)step + 1u);
  double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* The probe's perturbation of the Adam gradient: each band's model value
 * M_b moved by a relative adam_gnoise times a standard normal (fresh per
 * pixel, stage, step and band), i.e. g_i -= adam_gnoise sum_b w_b Jz_bi M_b n_b,
 * the size of the rounding of an FP32 evaluation of the model. */
static void probe_gradient(const pix_t *P, const lm_prob_t *q, const orc_config_t *c,
                           const double *L, const double *J, int step, double *g) {
  int p = q->p;
  for (int b = 0; b < P->nb; b++) {
    if (!(q->wst[b] > 0)) continue;
    double d = c->adam_gnoise * L[b] * probe_normal(c->adam_gseed, q->pix, q->stage, step, b);
    for (int i = 0; i < p; i++) g[i] -= q->wst[b] * J[b * p + i] * 0.5 * (q->hi[i] - q->lo[i]) * d;
  }
}

static int adam_fit(const pix_t *P, const lm_prob_t *q, const orc_config_t *c, double *x,
                    int steps, double lr, lm_res_t *res) {
  int p = q->p, nb = P->nb;
  double L[ORC_MAXB];
  double *J = (double *)malloc(sizeof(double) * nb * p);
  double H[ORC_NS1 * ORC_NS1], g[ORC_NS1], m[ORC_NS1], v[ORC_NS1], gz[ORC_NS1];
  res->used64 = 0;
  res->kappa = 0.0;
  res->n_used = 0;
  for (int b = 0; b < nb; b++) res->n_used += q->wst[b] > 0;
  for (int i = 0; i < p; i++) m[i] = v[i] = 0.0;
  evaluate(P, q, x, L, J);
  for (int t = 1; t <= steps; t++) {
    normal_eq(P, q, x, L, J, H, g);      /* g = Jz^T W r (the prior is off) */
    if (c->adam_gnoise > 0.0) probe_gradient(P, q, c, L, J, t, g);   /* tests only; off by default */
    double nrm = 0.0;
    for (int i = 0; i < p; i++) {
      gz[i] = -2.0 * g[i];
      nrm += gz[i] * gz[i];
    }
    nrm = sqrt(nrm);
    double f = nrm > c->adam_clip ? c->adam_clip / nrm : 1.0;
    double bc1 = 1.0 - pow(c->adam_beta1, t), bc2 = 1.0 - pow(c->adam_beta2, t);
    for (int i = 0; i < p; i++) {
      if (!(q->hi[i] > q->lo[i])) continue;      /* a fixed variable does not move */
      double gi = gz[i] * f;
      m[i] = c->adam_beta1 * m[i] + (1.0 - c->adam_beta1) * gi;
      v[i] = c->adam_beta2 * v[i] + (1.0 - c->adam_beta2) * gi * gi;
      double z = zcoord(q, x, i) - lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + c->adam_eps);
      if (z < -1.0) z = -1.0;
      if (z > 1.0) z = 1.0;
      x[i] = q->lo[i] + 0.5 * (q->hi[i] - q->lo[i]) * (z + 1.0);
    }
    if (q->nsimp > 0) orc_simplex_project(x, q->nsimp);
    evaluate(P, q, x, L, J);
  }
  normal_eq(P, q, x, L, J, H, g);
  for (int i = 0; i < p; i++)
    res->active[i] = (x[i] <= q->lo[i] && g[i] <= 0) || (x[i] >= q->hi[i] && g[i] >= 0);
  memcpy(res->H, H, sizeof(double) * p * p);
  res->iters = steps;
  res->status = ORC_CONVERGED;
  res->cost = cost_of(P, q, x, L);
  free(J);
  return ORC_CONVERGED;
}

/* ---------------------------------------------------------- HFDI ------ */
static int nearest_band(const orc_tables_t *t, double lam) {
  int best = 0;
  for (int b = 1; b < t->n_bands; b++)
    if (fabs(t->wavelength_nm[b] - lam) < fabs(t->wavelength_nm[best] - lam)) best = b;
  return best;
}

/* Sec. 2.1: HFDI = (L(2430) - L(2061)) / (L(2430) + L(2061)) */
double orc_hfdi(const orc_tables_t *t, const orc_config_t *c, const float *L) {
  double a = L[nearest_band(t, c->hfdi_lambda_hi)], b = L[nearest_band(t, c->hfdi_lambda_lo)];
  return (a - b) / (a + b);
}

/* ------------------------------------------------ thermal injection ---- */
/* Eq. (inject), Sec. 2.8: a single-temperature thermal term added to a
 * background spectrum, L_inj = L_bg + alpha tau_up(lambda) B(lambda, T), with
 * the background pixel's water-vapour bin for tau_up; in double, rounded
 * once to single precision. */
void orc_inject(const orc_tables_t *t, const float *L_bg, const uint16_t *wv_bin, const double *alpha,
                const double *T, int64_t n, float *L_out) {
  int nb = t->n_bands;
  for (int64_t i = 0; i < n; i++)
    for (int b = 0; b < nb; b++) {
      double tu = t->tau_up[(int64_t)wv_bin[i] * nb + b];
      L_out[i * nb + b] = (float)((double)L_bg[i * nb + b] + alpha[i] * tu * orc_planck(t->wavelength_nm[b], T[i]));
    }
}

/* ---------------------------------------------- water-vapour presolve -- */
/* Sec. 2.5 (pre-solved water vapour): the depth of the 940 nm water
 * feature against a continuum interpolated linearly across its shoulders,
 *   D = 1 - L(lc) / (L(lo) + (L(hi) - L(lo)) (lc - lo) / (hi - lo)),
 * for every pixel; each pixel is then given the median of its 12 x 12
 * super-pixel (the block of the image it falls in; edge blocks are smaller;
 * the lower median, the element of rank (n - 1) / 2 of the n finite
 * depths), and that median is quantised to a bin of the scene's water-vapour
 * table. The table side: each bin's depth D_j from the same formula applied
 * to the two-way direct path A tau_down tau_up of a flat surface
 * (A = E0 cos(theta_s) / pi), in double and then rounded once to single
 * precision; the median's fractional bin index is found by linear
 * interpolation between the bins whose depths bracket it and rounded to the
 * nearest bin (below the first depth: bin 0; above the last: the last).
 * The depth, the interpolation and the rounding decide an integer, so they
 * are taken in single precision (the library's precision), with fmaf for
 * the continuum; a pixel with a non-finite or saturated shoulder or centre
 * band, or a non-positive continuum, is left out of its block's median; a
 * block without any depth gets the invalid bin 0xFFFF. */
static int cmp_float(const void *a, const void *b) {
  float x = *(const float *)a, y = *(const float *)b;
  return (x > y) - (x < y);
}

void orc_wv_depth_table(const orc_tables_t *t, double lam_lo, double lam_c, double lam_hi,
                        float *D) {
  int blo = nearest_band(t, lam_lo), bc = nearest_band(t, lam_c), bhi = nearest_band(t, lam_hi);
  double f = ((double)t->wavelength_nm[bc] - t->wavelength_nm[blo]) /
             ((double)t->wavelength_nm[bhi] - t->wavelength_nm[blo]);
  for (int j = 0; j < t->n_wv; j++) {
    double a[3];
    int bb[3] = {blo, bc, bhi};
    for (int q = 0; q < 3; q++) {
      int b = bb[q];
      a[q] = (double)t->solar_irr[b] * t->cos_sza / M_PI * (double)t->tau_down[j * t->n_bands + b] *
             (double)t->tau_up[j * t->n_bands + b];
    }
    D[j] = (float)(1.0 - a[1] / (a[0] + (a[2] - a[0]) * f));
  }
}

void orc_wv_presolve(const orc_tables_t *t, const float *radiance, int64_t width, int64_t height,
                     int block, double lam_lo, double lam_c, double lam_hi, uint16_t *bin_out,
                     float *depth_out) {
  int nb = t->n_bands;
  int blo = nearest_band(t, lam_lo), bc = nearest_band(t, lam_c), bhi = nearest_band(t, lam_hi);
  float cf = (float)(((double)t->wavelength_nm[bc] - t->wavelength_nm[blo]) /
                     ((double)t->wavelength_nm[bhi] - t->wavelength_nm[blo]));
  float Dj[ORC_MAXWV];
  orc_wv_depth_table(t, lam_lo, lam_c, lam_hi, Dj);
  int64_t n = width * height;
  float *D = (float *)malloc(sizeof(float) * (n > 0 ? n : 1));
  for (int64_t p = 0; p < n; p++) {
    const float *L = radiance + p * nb;
    float lo = L[blo], c = L[bc], hi = L[bhi];
    int ok = isfinite(lo) && isfinite(c) && isfinite(hi);
    if (t->sat_level)
      ok = ok && lo < t->sat_level[blo] && c < t->sat_level[bc] && hi < t->sat_level[bhi];
    float cont = fmaf(hi - lo, cf, lo);
    D[p] = ok && cont > 0.0f ? 1.0f - c / cont : NAN;
    if (depth_out) depth_out[p] = D[p];
  }
  float *v = (float *)malloc(sizeof(float) * block * block);
  for (int64_t by = 0; by * block < height; by++)
    for (int64_t bx = 0; bx * block < width; bx++) {
      int m = 0;
      for (int64_t y = by * block; y < height && y < (by + 1) * block; y++)
        for (int64_t x = bx * block; x < width && x < (bx + 1) * block; x++)
          if (isfinite(D[y * width + x])) v[m++] = D[y * width + x];
      uint16_t bin = 0xFFFF;
      if (m > 0) {
        qsort(v, m, sizeof(float), cmp_float);
        float med = v[(m - 1) / 2];
        float fi;
        int J = t->n_wv;
        if (!(med > Dj[0])) fi = 0.0f;
        else if (!(med < Dj[J - 1])) fi = (float)(J - 1);
        else {
          int j = 0;
          while (!(med < Dj[j + 1])) j++;   /* Dj[j] <= med < Dj[j + 1] */
          fi = (float)j + (med - Dj[j]) / (Dj[j + 1] - Dj[j]);
        }
        int b = (int)floorf(fi + 0.5f);
        bin = (uint16_t)(b < 0 ? 0 : (b > J - 1 ? J - 1 : b));
      }
      for (int64_t y = by * block; y < height && y < (by + 1) * block; y++)
        for (int64_t x = bx * block; x < width && x < (bx + 1) * block; x++) bin_out[y * width + x] = bin;
    }
  free(v);
  free(D);
}

/* ------------------------------------------------------- forward ------ */
/* mode 1: state [x_surf(K), a1, T1]; mode 2: [x_surf(K), mu_h, s_h, mu_s, s_s, eta, a] */
void orc_forward(const orc_tables_t *t, int mode, const double *state, const uint16_t *wv_bin,
                 int64_t n, double *L_out) {
  int K = t->n_endm, ns = mode == 1 ? K + 2 : K + 6;
  double *Bt = planck_table(t);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) {
    pix_t *P = (pix_t *)malloc(sizeof(pix_t));
    pix_tables(P, t, wv_bin[i], Bt);
    const double *s = state + i * ns;
    double *L = L_out + i * t->n_bands;
    if (mode == 1) {
      eval_stage1(P, s, NULL, L, NULL);
    } else {
      for (int b = 0; b < P->nb; b++) P->Ls[b] = solar_term(P, b, s, NULL);
      if (s[K + 5] != 0.0) eval_stage2(P, s + K, NULL, L, NULL);
      else memcpy(L, P->Ls, sizeof(double) * P->nb);
    }
    free(P);
  }
  free(Bt);
}

/* Model and analytic Jacobian (physical units) of one stage at one pixel.
 * stage 1: x = [x_surf(K), a1, T1], J is [n_bands][K+2];
 * stage 2: xs = surface fractions, x = [mu_h, s_h, mu_s, s_s, eta, a], J [n_bands][6]. */
void orc_stage_jacobian(const orc_tables_t *t, int stage, const double *xs, const double *x,
                        int wv_bin, double *L, double *J) {
  pix_t *P = (pix_t *)malloc(sizeof(pix_t));
  double *Bt = planck_table(t);
  pix_tables(P, t, wv_bin, Bt);
  if (stage == 1) {
    eval_stage1(P, x, NULL, L, J);
  } else {
    for (int b = 0; b < P->nb; b++) P->Ls[b] = solar_term(P, b, xs, NULL);
    eval_stage2(P, x, NULL, L, J);
  }
  free(Bt);
  free(P);
}

void orc_synth_radiance(const orc_tables_t *t, int mode, const double *state,
                        const uint16_t *wv_bin, const double *normals, int64_t n,
                        double noise_rel, double noise_abs, float *L_out) {
  int nb = t->n_bands;
  const int64_t chunk = 4096;
  double *L = (double *)malloc(sizeof(double) * chunk * nb);
  int K = t->n_endm, ns = mode == 1 ? K + 2 : K + 6;
  for (int64_t i0 = 0; i0 < n; i0 += chunk) {
    int64_t m = n - i0 < chunk ? n - i0 : chunk;
    orc_forward(t, mode, state + i0 * ns, wv_bin + i0, m, L);
    for (int64_t i = 0; i < m * nb; i++) {
      double sd = sqrt(noise_rel * noise_rel * L[i] * L[i] + noise_abs * noise_abs);
      double v = L[i] + (normals ? sd * normals[i0 * nb + i] : 0.0);
      L_out[i0 * nb + i] = (float)v;
    }
  }
  free(L);
}

/* ------------------------------------------------------ retrieval ----- */
/* Noise variance of band b at radiance L: the caller's per-band sd when
 * given, else the noise model (rel L)^2 + abs^2. */
static double noise_var(const orc_config_t *c, int b, double L) {
  if (c->noise_sd) return (double)c->noise_sd[b] * c->noise_sd[b];
  return c->noise_rel * c->noise_rel * L * L + c->noise_abs * c->noise_abs;
}

/* The loss is noise-weighted (w_b = 1 / variance) when the caller gives
 * per-band sd or asks for the noise model's weights; otherwise it is
 * Eq. (loss) as printed (w_b = 1 on unmasked bands). */
static int loss_weighted(const orc_config_t *c) { return c->weighted || c->noise_sd != NULL; }

/* Per-pixel set-up shared by the fit and the posterior: observed radiance,
 * mask m(lambda) (saturation, Eq. loss), band weights, the two windows'
 * weights w1 / w2 and used-band counts, and the prior scales (mean noise
 * variance of each window's used bands under the unweighted loss, 1 under
 * a weighted one). */
static void pixel_setup(pix_t *P, const orc_tables_t *t, const orc_config_t *c, const float *Lrow,
                        double *w1, double *w2, int *n1, int *n2, double *psc1, double *psc2) {
  int nb = t->n_bands;
  double s1 = 0, s2 = 0;
  *n1 = *n2 = 0;
  for (int b = 0; b < nb; b++) {
    P->Lobs[b] = Lrow[b];
    int ok = !(t->sat_level && Lrow[b] >= t->sat_level[b]);   /* m(lambda), Eq. (loss) */
    double var = noise_var(c, b, P->Lobs[b]);
    P->wgt[b] = ok ? (loss_weighted(c) ? 1.0 / var : 1.0) : 0.0;
    double l = P->lam[b];
    int in1 = l >= c->win1_lo && l <= c->win1_hi;
    int in2 = (l >= c->win2h_lo && l <= c->win2h_hi) || (l >= c->win2s_lo && l <= c->win2s_hi);
    w1[b] = in1 ? P->wgt[b] : 0.0;
    w2[b] = in2 ? P->wgt[b] : 0.0;
    if (w1[b] > 0) { (*n1)++; s1 += var; }
    if (w2[b] > 0) { (*n2)++; s2 += var; }
  }
  *psc1 = loss_weighted(c) || *n1 == 0 ? 1.0 : s1 / *n1;
  *psc2 = loss_weighted(c) || *n2 == 0 ? 1.0 : s2 / *n2;
}

/* Posterior at the final stage-2 state x2 (the outputs of Sec. 2.3 and the
 * Laplace covariance): from the normal matrix H = J^T W J + P at x2 in the z
 * coordinates of Eq. (affine), its active set, the cost and the used-band
 * count. C = s2 (H_FF)^-1 over the free variables, in FP64, in physical
 * units (s_i s_j); fixed (active) variables get zero rows; a free variable
 * with a zero column has infinite variance. var(E[T]) = gE^T C gE with gE =
 * dE/dx2. With alpha held on its lower bound there is no thermal signal:
 * E[T] and its posterior are undefined (covariance NaN, var(E[T]) = inf).
 * Identifiable: Laplace sd(E[T]) <= ident_sd_et and alpha >= snr sd(alpha),
 * alpha free and positive. Writes cv[21] (packed upper) and var(E[T]);
 * returns 1 if identifiable. */
static int posterior(const orc_config_t *c, const double *x2, const double *H, const int *active,
                     double cost, int n_used, double *cv, double *var_ET) {
  const double *lo2 = c->lo2, *hi2 = c->hi2;
  int F[6], nf = 0, zero_col[6] = {0};
  for (int k = 0; k < 6; k++) {
    if (active[k]) continue;
    if (!(H[k * 6 + k] > 0)) { zero_col[k] = 1; continue; }
    F[nf++] = k;
  }
  double s2 = loss_weighted(c) ? 1.0 : cost / (double)(n_used - nf);
  double Cz[36];
  memset(Cz, 0, sizeof(Cz));
  int cov_ok = 1;
  int no_signal = active[5] && x2[5] <= lo2[5];
  if (no_signal) cov_ok = 0;
  if (nf > 0 && !no_signal) {
    double A[36], dsc[6];
    for (int u = 0; u < nf; u++) dsc[u] = sqrt(H[F[u] * 6 + F[u]]);
    for (int u = 0; u < nf; u++)
      for (int v = 0; v < nf; v++) A[u * nf + v] = H[F[u] * 6 + F[v]] / (dsc[u] * dsc[v]);
    if (orc_cholesky(A, nf) != 0) cov_ok = 0;
    else {
      for (int v = 0; v < nf; v++) {
        double e[6] = {0};
        e[v] = 1.0;
        orc_chol_solve(A, nf, e);
        for (int u = 0; u < nf; u++) Cz[F[u] * 6 + F[v]] = s2 * e[u] / (dsc[u] * dsc[v]);
      }
    }
  }
  double sc[6];
  for (int k = 0; k < 6; k++) sc[k] = 0.5 * (hi2[k] - lo2[k]);
  double Cx[36];
  for (int a = 0; a < 6; a++)
    for (int b = 0; b < 6; b++) {
      Cx[a * 6 + b] = cov_ok ? Cz[a * 6 + b] * sc[a] * sc[b] : NAN;
      if (a == b && zero_col[a]) Cx[a * 6 + b] = INFINITY;
    }
  int q = 0;
  for (int a = 0; a < 6; a++)
    for (int b = a; b < 6; b++) cv[q++] = Cx[a * 6 + b];
  double gE[6] = {x2[4], 0, 1.0 - x2[4], 0, x2[0] - x2[2], 0};
  double vE = 0;
  for (int a = 0; a < 6; a++) {
    if (gE[a] == 0) continue;
    if (zero_col[a]) { vE = INFINITY; break; }
    for (int b = 0; b < 6; b++)
      if (gE[b] != 0) vE += gE[a] * Cx[a * 6 + b] * gE[b];
  }
  if (no_signal) vE = INFINITY;
  *var_ET = vE;
  double sdE = sqrt(vE), sda = sqrt(Cx[35]);
  return cov_ok && isfinite(sdE) && sdE <= c->ident_sd_et && x2[5] >= c->ident_alpha_snr * sda &&
         !active[5] && x2[5] > 0;
}

/* unweighted residual rms of the stage-2 model over the used bands */
static double stage2_rms(const pix_t *P, const double *x2, const double *w2, int n_used) {
  double L[ORC_MAXB], cdata = 0;
  eval_stage2(P, x2, w2, L, NULL);
  for (int b = 0; b < P->nb; b++)
    if (w2[b] > 0) cdata += (P->Lobs[b] - L[b]) * (P->Lobs[b] - L[b]);
  return sqrt(cdata / n_used);
}

static void retrieve_pixel(const orc_tables_t *t, const orc_config_t *c, const double *Bt,
                           const float *Lrow, int w, const double *init, orc_outputs_t *o,
                           int64_t i) {
  int K = t->n_endm, nb = t->n_bands, NS = K + 8;
  double *st = o->state + i * NS;
  double *cv = o->cov + i * 21;
  for (int k = 0; k < NS; k++) st[k] = NAN;
  for (int k = 0; k < 21; k++) cv[k] = NAN;
  o->ET[i] = o->sdT[i] = o->alpha[i] = o->var_ET[i] = o->cost[i] = o->rms[i] = NAN;
  o->cost1[i] = NAN;
  o->kappa[i] = 0;
  o->it1[i] = o->it2[i] = 0;
  o->n_used[i] = 0;
  o->hfdi[i] = NAN;
  for (int b = 0; b < nb; b++)
    if (!isfinite(Lrow[b])) { o->status[i] = ORC_NONFINITE; return; }
  o->hfdi[i] = orc_hfdi(t, c, Lrow);
  if (c->gate_hfdi && !(o->hfdi[i] >= c->hfdi_thresh)) { o->status[i] = ORC_NOT_CANDIDATE; return; }

  pix_t *P = (pix_t *)malloc(sizeof(pix_t));
  pix_tables(P, t, w, Bt);
  double w1[ORC_MAXB], w2[ORC_MAXB], psc1, psc2;
  int n1, n2;
  pixel_setup(P, t, c, Lrow, w1, w2, &n1, &n2, &psc1, &psc2);
  int status = 0;
  if (n1 <= K + 2 || n2 <= 6) { o->status[i] = ORC_ALL_MASKED; free(P); return; }

  /* stage 1: x1 = [x_surf, a1, T1] */
  double x1[ORC_NS1];
  if (init) {
    for (int k = 0; k < K + 2; k++) x1[k] = init[k];
    orc_simplex_project(x1, K);
    for (int k = K; k < K + 2; k++) {
      if (x1[k] < c->lo1[k]) x1[k] = c->lo1[k];
      if (x1[k] > c->hi1[k]) x1[k] = c->hi1[k];
    }
  } else {
    for (int k = 0; k < K; k++) x1[k] = 1.0 / K;
    x1[K] = c->init_alpha1;
    x1[K + 1] = c->init_T1;
  }
  /* the Adam solver minimises Eq. (loss) as printed: no prior term */
  static const double no_prior[ORC_NS1] = {0};
  const int adam = c->solver == ORC_SOLVER_ADAM;
  lm_prob_t q1 = {1, K + 2, K, c->lo1, c->hi1, c->pm1, adam ? no_prior : c->pp1, w1, c->max_it1, psc1, i};
  lm_res_t r1;
  if (adam) adam_fit(P, &q1, c, x1, c->adam_steps1, c->adam_lr1, &r1);
  else lm_fit(P, &q1, c, x1, &r1);
  if (r1.status == ORC_MAXITER) status |= ORC_F_S1_MAXITER;
  if (r1.used64) status |= ORC_F_FP64;
  o->it1[i] = r1.iters;
  o->cost1[i] = r1.cost;
  for (int b = 0; b < nb; b++) P->Ls[b] = solar_term(P, b, x1, NULL);

  /* stage 2: x2 = [mu_h, s_h, mu_s, s_s, eta, a], surface fixed */
  double x2[ORC_NS2];
  const double *lo2 = c->lo2, *hi2 = c->hi2;
  if (init) {
    for (int k = 0; k < 6; k++) x2[k] = init[K + 2 + k];
  } else {
    double T1 = x1[K + 1];
    x2[0] = T1 > c->init_mu_h_floor ? T1 : c->init_mu_h_floor;
    x2[2] = T1 < c->init_mu_s_ceil ? T1 : c->init_mu_s_ceil;
    x2[1] = x2[3] = c->init_sigma;
    x2[5] = x1[K];
  }
  for (int k = 0; k < 6; k++) {
    if (k == 4) continue;
    if (x2[k] < lo2[k]) x2[k] = lo2[k];
    if (x2[k] > hi2[k]) x2[k] = hi2[k];
  }
  if (!init) {
    double T1 = x1[K + 1];
    double e = (x2[0] > x2[2]) ? (T1 - x2[2]) / (x2[0] - x2[2]) : 0.5;
    x2[4] = e < c->init_eta_lo ? c->init_eta_lo : (e > c->init_eta_hi ? c->init_eta_hi : e);
    /* stage 1 found no thermal signal (alpha1 on its lower bound, so T1
     * says nothing): the mixture shape starts at the prior's means, where
     * its fit ends while the data give alpha no signal either */
    if (x1[K] <= c->lo1[K])
      for (int k = 0; k < 5; k++) x2[k] = lo2[k] + 0.5 * (hi2[k] - lo2[k]) * (c->pm2[k] + 1.0);
  } else {
    if (x2[4] < lo2[4]) x2[4] = lo2[4];
    if (x2[4] > hi2[4]) x2[4] = hi2[4];
  }
  lm_prob_t q2 = {2, 6, 0, lo2, hi2, c->pm2, adam ? no_prior : c->pp2, w2, c->max_it2, psc2, i};
  lm_res_t r2;
  if (adam) adam_fit(P, &q2, c, x2, c->adam_steps2, c->adam_lr2, &r2);
  else lm_fit(P, &q2, c, x2, &r2);
  if (r2.used64) status |= ORC_F_FP64;
  status |= r2.status;
  o->it2[i] = r2.iters;

  for (int k = 0; k < K + 2; k++) st[k] = x1[k];
  for (int k = 0; k < 6; k++) st[K + 2 + k] = x2[k];
  double E, V;
  orc_moments(x2, &E, &V);
  o->ET[i] = E;
  o->sdT[i] = sqrt(V);
  o->alpha[i] = x2[5];
  o->cost[i] = r2.cost;
  o->kappa[i] = r1.kappa > r2.kappa ? r1.kappa : r2.kappa;
  o->n_used[i] = r2.n_used;
  o->rms[i] = stage2_rms(P, x2, w2, r2.n_used);
  if (!posterior(c, x2, r2.H, r2.active, r2.cost, r2.n_used, cv, &o->var_ET[i])) status |= ORC_F_NOT_IDENT;
  o->status[i] = status;
  free(P);
}

/* The outputs that follow from a given final state alone (the posterior
 * step of the retrieval, for checking it apart from the fit): at state
 * [x_surf(K), a1, T1, mu_h, s_h, mu_s, s_s, eta, a] the stage-2 cost of
 * Eq. (loss) plus the prior, its normal matrix and active set, then E[T],
 * sigma[T] (Sec. 2.3), the Laplace covariance, var(E[T]), the unweighted
 * residual rms and the identifiability flag, exactly as the fit's last step
 * forms them. The surface fractions fix the solar term of stage 2. */
void orc_posterior_at(const orc_tables_t *t, const orc_config_t *c, const float *Lrow, int w,
                      const double *state, double *ET, double *sdT, double *cost, double *rms,
                      double *cov21, double *var_ET, int *ident) {
  int K = t->n_endm, nb = t->n_bands;
  double *Bt = planck_table(t);
  pix_t *P = (pix_t *)malloc(sizeof(pix_t));
  pix_tables(P, t, w, Bt);
  double w1[ORC_MAXB], w2[ORC_MAXB], psc1, psc2;
  int n1, n2;
  pixel_setup(P, t, c, Lrow, w1, w2, &n1, &n2, &psc1, &psc2);
  for (int b = 0; b < nb; b++) P->Ls[b] = solar_term(P, b, state, NULL);
  const double *x2 = state + K + 2;
  static const double no_prior[6] = {0};
  const double *pp2 = c->solver == ORC_SOLVER_ADAM ? no_prior : c->pp2;   /* Adam: Eq. (loss) only */
  lm_prob_t q2 = {2, 6, 0, c->lo2, c->hi2, c->pm2, pp2, w2, 0, psc2};
  double L[ORC_MAXB], H[36], g[6];
  double *J = (double *)malloc(sizeof(double) * nb * 6);
  evaluate(P, &q2, x2, L, J);
  *cost = cost_of(P, &q2, x2, L);
  normal_eq(P, &q2, x2, L, J, H, g);
  int active[6];
  for (int k = 0; k < 6; k++)
    active[k] = (x2[k] <= c->lo2[k] && g[k] <= 0) || (x2[k] >= c->hi2[k] && g[k] >= 0);
  double V;
  orc_moments(x2, ET, &V);
  *sdT = sqrt(V);
  *rms = stage2_rms(P, x2, w2, n2);
  *ident = posterior(c, x2, H, active, *cost, n2, cov21, var_ET);
  free(J);
  free(P);
  free(Bt);
}

void orc_retrieve(const orc_tables_t *t, const orc_config_t *c, const float *radiance,
                  const uint16_t *wv_bin, int64_t n, const double *init_state, orc_outputs_t *o,
                  int n_threads) {
  /* n_threads > 0 bounds this call's threads only (a num_threads clause, not
   * the process-wide setting, so a later call with 0 gets every core) */
#ifdef _OPENMP
  const int nt = n_threads > 0 ? n_threads : omp_get_num_procs();
#else
  const int nt = 1;
  (void)n_threads;
#endif
  int NS = t->n_endm + 8;
  double *Bt = planck_table(t);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t i = 0; i < n; i++)
    retrieve_pixel(t, c, Bt, radiance + i * t->n_bands, wv_bin[i], init_state ? init_state + i * NS : NULL,
                   o, i);
  free(Bt);
}

/* array helper for tests: out[i] = B(lambda[i], T[i]) */
void orc_planck_array(int64_t n, const double *lambda_nm, const double *T, double *out) {
  for (int64_t i = 0; i < n; i++) out[i] = orc_planck(lambda_nm[i], T[i]);
}

/* ------------------------------------------------ MLP proposal (a7) --- */
/* Learned initial-state proposal (the task's learned extension; the paper
 * has no network): z = tanh(W3 relu(W2 relu(W1 x + b1) + b2) + b3), weights
 * row-major [out][in]. Plain FP64 definition, one sample at a time. */
void orc_mlp_forward(int B, int Din, int H, int Dout, const double *W1, const double *b1,
                     const double *W2, const double *b2, const double *W3, const double *b3,
                     const double *x, double *a1, double *a2, double *z) {
  for (int s = 0; s < B; s++) {
    const double *xs = x + (size_t)s * Din;
    double *A1 = a1 + (size_t)s * H, *A2 = a2 + (size_t)s * H, *Z = z + (size_t)s * Dout;
    for (int o = 0; o < H; o++) {
      double v = b1[o];
      for (int i = 0; i < Din; i++) v += W1[(size_t)o * Din + i] * xs[i];
      A1[o] = v;
    }
    for (int o = 0; o < H; o++) {
      double v = b2[o];
      for (int i = 0; i < H; i++) v += W2[(size_t)o * H + i] * (A1[i] > 0 ? A1[i] : 0.0);
      A2[o] = v;
    }
    for (int o = 0; o < Dout; o++) {
      double v = b3[o];
      for (int i = 0; i < H; i++) v += W3[(size_t)o * H + i] * (A2[i] > 0 ? A2[i] : 0.0);
      Z[o] = tanh(v);
    }
  }
}

/* Masked mean-squared error over B samples and its gradients (chain rule
 * through tanh and the two ReLUs): loss = sum_{s,o} mask[s][o] (z - t)^2 /
 * (B * n_out). Returns the loss. */
double orc_mlp_backward(int B, int Din, int H, int Dout, int n_out, const double *W1,
                        const double *W2, const double *W3, const double *x, const double *a1,
                        const double *a2, const double *z, const double *t, const double *mask,
                        double *gW1, double *gb1, double *gW2, double *gb2, double *gW3,
                        double *gb3) {
  double norm = 1.0 / ((double)B * n_out), loss = 0;
  memset(gW1, 0, sizeof(double) * H * Din);
  memset(gb1, 0, sizeof(double) * H);
  memset(gW2, 0, sizeof(double) * H * H);
  memset(gb2, 0, sizeof(double) * H);
  memset(gW3, 0, sizeof(double) * Dout * H);
  memset(gb3, 0, sizeof(double) * Dout);
  double *dy = (double *)malloc(sizeof(double) * Dout);
  double *d2 = (double *)malloc(sizeof(double) * H), *d1 = (double *)malloc(sizeof(double) * H);
  for (int s = 0; s < B; s++) {
    const double *xs = x + (size_t)s * Din, *A1 = a1 + (size_t)s * H, *A2 = a2 + (size_t)s * H;
    const double *Z = z + (size_t)s * Dout, *T = t + (size_t)s * Dout;
    const double *Mk = mask + (size_t)s * Dout;
    for (int o = 0; o < Dout; o++) {
      double e = (Z[o] - T[o]) * Mk[o];
      loss += e * e * norm;
      dy[o] = 2.0 * e * norm * (1.0 - Z[o] * Z[o]);
    }
    for (int i = 0; i < H; i++) {
      double v = 0;
      for (int o = 0; o < Dout; o++) v += dy[o] * W3[(size_t)o * H + i];
      d2[i] = A2[i] > 0 ? v : 0.0;
    }
    for (int i = 0; i < H; i++) {
      double v = 0;
      for (int o = 0; o < H; o++) v += d2[o] * W2[(size_t)o * H + i];
      d1[i] = A1[i] > 0 ? v : 0.0;
    }
    for (int o = 0; o < Dout; o++) {
      gb3[o] += dy[o];
      for (int i = 0; i < H; i++) gW3[(size_t)o * H + i] += dy[o] * (A2[i] > 0 ? A2[i] : 0.0);
    }
    for (int o = 0; o < H; o++) {
      gb2[o] += d2[o];
      for (int i = 0; i < H; i++) gW2[(size_t)o * H + i] += d2[o] * (A1[i] > 0 ? A1[i] : 0.0);
    }
    for (int o = 0; o < H; o++) {
      gb1[o] += d1[o];
      for (int i = 0; i < Din; i++) gW1[(size_t)o * Din + i] += d1[o] * xs[i];
    }
  }
  free(dy);
  free(d2);
  free(d1);
  return loss;
}

/* Adam (Kingma & Ba 2014) on a flat parameter vector, step t >= 1. */
void orc_adam(int64_t n, double *w, const double *g, double *m, double *v, int t, double lr,
              double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int64_t i = 0; i < n; i++) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* Normal equations of one stage at a given state (for parity tests of the
 * GPU's Jacobian and reductions): H = J^T W J + psc P and g = J^T W r - psc
 * P (z - pm) in the reduced z coordinates used by the fit (stage 1:
 * fractions k != m with m = the largest, then alpha1, T1), plus the cost.
 * x: stage 1 [x_surf(K), a1, T1]; stage 2 [x_surf(K), mu_h, s_h, mu_s,
 * s_s, eta, a]. H is [P][P] row-major, g [P]. */
void orc_normal_equations(const orc_tables_t *t, const orc_config_t *c, int stage,
                          const float *Lrow, int w, const double *x, double *Hout, double *gout,
                          double *cost_out) {
  int K = t->n_endm, nb = t->n_bands;
  double *Bt = planck_table(t);
  pix_t *P = (pix_t *)malloc(sizeof(pix_t));
  pix_tables(P, t, w, Bt);
  double ws[ORC_MAXB];
  int n = 0;
  double sv = 0;
  for (int b = 0; b < nb; b++) {
    P->Lobs[b] = Lrow[b];
    int ok = !(t->sat_level && Lrow[b] >= t->sat_level[b]);
    double l = P->lam[b];
    int in = stage == 1 ? (l >= c->win1_lo && l <= c->win1_hi)
                        : ((l >= c->win2h_lo && l <= c->win2h_hi) || (l >= c->win2s_lo && l <= c->win2s_hi));
    double var = noise_var(c, b, P->Lobs[b]);
    ws[b] = (ok && in) ? (loss_weighted(c) ? 1.0 / var : 1.0) : 0.0;
    if (ws[b] > 0) { n++; sv += var; }
  }
  double psc = loss_weighted(c) ? 1.0 : sv / n;
  static const double no_prior[ORC_NS1] = {0};
  const int adam = c->solver == ORC_SOLVER_ADAM;   /* Adam: Eq. (loss) only */
  lm_prob_t q1 = {1, K + 2, K, c->lo1, c->hi1, c->pm1, adam ? no_prior : c->pp1, ws, 0, psc};
  lm_prob_t q2 = {2, 6, 0, c->lo2, c->hi2, c->pm2, adam ? no_prior : c->pp2, ws, 0, psc};
  const lm_prob_t *q = stage == 1 ? &q1 : &q2;
  const double *xx = stage == 1 ? x : x + K;
  if (stage == 2)
    for (int b = 0; b < nb; b++) P->Ls[b] = solar_term(P, b, x, NULL);
  int p = q->p;
  double L[ORC_MAXB], H[ORC_NS1 * ORC_NS1], g[ORC_NS1], E[ORC_NS1 * ORC_NS1];
  double *J = (double *)malloc(sizeof(double) * nb * p);
  evaluate(P, q, xx, L, J);
  *cost_out = cost_of(P, q, xx, L);
  normal_eq(P, q, xx, L, J, H, g);
  int m, pr = reduced_basis(q, xx, E, &m);
  for (int a = 0; a < pr; a++) {
    gout[a] = 0;
    for (int i = 0; i < p; i++) gout[a] += E[i * p + a] * g[i];
    for (int bb = 0; bb < pr; bb++) {
      double sacc = 0;
      for (int i = 0; i < p; i++)
        for (int k = 0; k < p; k++) sacc += E[i * p + a] * H[i * p + k] * E[k * p + bb];
      Hout[a * pr + bb] = sacc;
    }
  }
  free(J);
  free(P);
  free(Bt);
}
