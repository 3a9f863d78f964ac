// kernels_lm.cu — the per-pixel two-stage retrieval on sm_103a.
//
// G lanes of a warp fit one pixel (32 / G pixels per warp; G = 8, 16 or 32
// by launch shape), in persistent CTAs whose groups claim pixels from a
// global counter. A group's lanes own band slots (sub + G s within each
// stage's window), so radiance and the shared Planck table are read
// band-coalesced; the normal equations J^T W J, J^T W r and the cost are
// reduced with shuffles inside the group, and every lane of the group then
// runs the same small solve on registers. Each round, every group with a
// pixel takes one LM step, so the groups of a warp evaluate the model in
// step; a pixel that converges hands over and its group takes the next.
//
// Stage 1 (Sec. 2.6): x1 = [x_surf(K), alpha1, T1] over Omega_1 with the
// single-temperature Planck term computed on the SFU in the overflow-safe
// form e^-x / (1 - e^-x). Stage 2: x2 = [mu_h, s_h, mu_s, s_s, eta, alpha]
// over Omega_2 with the solar term fixed; the thermal term sums the Planck
// grid (staged per CTA in shared memory by bulk copy) against normalised
// Gaussian weights (Eq. thermal), and its Jacobian uses the weight moments
// sum w (d - dbar) B and sum w (d^2 - m2) B.
//
// The iteration is Levenberg-Marquardt in the z coordinates of Eq. (affine):
// Nielsen's damping update, a projected-Newton step (a variable whose step
// leaves its bound is pinned there and the rest re-solved), the surface
// fractions moved in the basis e_k - e_m (m = largest fraction) and then
// projected onto the simplex (Sec. 2.6). Steps are solved in FP32 on the
// diagonally scaled damped matrix; an ill-conditioned one (condition
// estimate above kappa_max, or a failed pivot) is re-solved in FP64. The
// final Laplace covariance is FP64.
#include <cuda_bf16.h>
#include <float.h>

#include "internal.cuh"
#include "tc.cuh"


namespace firert {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Loop shapes of the stage kernels. The per-iteration code of an LM step runs
// once per round as straight-line code and is fetch-bound (ncu: instruction
// fetch stalls first), so the band and node loops stay rolled: measured on
// the flight-line chunk, unrolling them by 2 cost 17 % in stage 1 and 7 % in
// stage 2; rolling the Jacobian assembly over a chunk's slots saved another
// 2.5 % in stage 2.
constexpr int kBand1Unroll = 1, kNodeUnroll = 1;
constexpr int kSlotUnroll = 1;   // stage-2 Jacobian assembly over a chunk's band slots

constexpr int kClaim = 4;          // pixels claimed per atomic
constexpr size_t kMaxSmemPerCta = 227 * 1024;   // opt-in dynamic shared memory per CTA
// Stage-1 steps whose predicted decrease is below this fraction of the cost
// are judged by the increment-form decrease: the decrease from residual
// differences carries a rounding error of a few 1e-6 of the cost, which
// would decide the acceptance of smaller steps.
constexpr float kIncBelow = 1e-5f;
// FP32 rounding floor of the gradient: each residual carries the rounding of
// its model value M_b (a few units in the last place), so g_a = sum_b w_b
// J_ba r_b cannot be resolved below about kFloorC u sqrt(sum_b (w_b J_ba
// M_b)^2), u = 2^-24. Where the noise is low (block-averaged spectra) this
// floor exceeds the gradient tolerance and an FP32 fit cannot pass the test;
// such a fit runs to the iteration cap and is reported converged if its
// gradient is within the tolerance plus the floor there (and plus the
// gradient that the FP32 spacing of the state makes: see next_trial_t).
constexpr float kFloorC = 8.f * 5.9604645e-8f;

template <int I>
struct IC { static constexpr int value = I; };
template <int N, int I = 0, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (I < N) {
    f(IC<I>{});
    static_for<N, I + 1>(f);
  }
}

// packed upper-triangular index of (a, b), a <= b, for a P x P matrix
template <int P>
__device__ __forceinline__ constexpr int up(int a, int b) {
  return a <= b ? a * P - (a * (a - 1)) / 2 + (b - a) : b * P - (b * (b - 1)) / 2 + (a - b);
}

// Reciprocal square root in FP64 by the Newton-Raphson iteration for
// 1 / sqrt(x), y <- y (3 - x y^2) / 2, which squares the relative error at
// each step: from the FP32 SFU estimate (relative error near 2^-22) two steps
// leave only the rounding of the last one (about 1 ulp), with six FP64
// operations instead of a double square root and division (FP64 runs at
// 1/64 of the FP32 rate). A pivot outside the FP32 range (a near-singular
// matrix) takes the IEEE square root and division.
__device__ __forceinline__ double rsq(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// expm1(y) for |y| < 0.5 by its Taylor series to y^9 (truncation below
// |y|^10 / 10! e^|y| < 5e-10 |y|): nine FMAs, no branches
__device__ __forceinline__ float em1_mid(float y) {
  float p = fmaf(y, 1.f / 362880.f, 1.f / 40320.f);
  p = fmaf(y, p, 1.f / 5040.f);
  p = fmaf(y, p, 1.f / 720.f);
  p = fmaf(y, p, 1.f / 120.f);
  p = fmaf(y, p, 1.f / 24.f);
  p = fmaf(y, p, 1.f / 6.f);
  p = fmaf(y, p, 0.5f);
  p = fmaf(y, p, 1.f);
  return y * p;
}
// the same for a pair, with the packed FP32 FMA
__device__ __forceinline__ float2 em1_mid2(float2 y) {
  float2 p = __ffma2_rn(y, make_float2(1.f / 362880.f, 1.f / 362880.f),
                        make_float2(1.f / 40320.f, 1.f / 40320.f));
  p = __ffma2_rn(y, p, make_float2(1.f / 5040.f, 1.f / 5040.f));
  p = __ffma2_rn(y, p, make_float2(1.f / 720.f, 1.f / 720.f));
  p = __ffma2_rn(y, p, make_float2(1.f / 120.f, 1.f / 120.f));
  p = __ffma2_rn(y, p, make_float2(1.f / 24.f, 1.f / 24.f));
  p = __ffma2_rn(y, p, make_float2(1.f / 6.f, 1.f / 6.f));
  p = __ffma2_rn(y, p, make_float2(0.5f, 0.5f));
  p = __ffma2_rn(y, p, make_float2(1.f, 1.f));
  return __fmul2_rn(y, p);
}

// ------------------------------------------------------------- solve ----
// reciprocal square root for the step solve: the SFU in FP32; in FP64 (the
// cold path of ill-conditioned steps) the Newton-refined rsq above
__device__ __forceinline__ float rsq_step(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq_step(double x) { return rsq(x); }

// Solve (H + lam D) d = rhs over the free variables on the diagonally scaled
// matrix; pinned variables are identity rows with their displacement moved
// to the right-hand side. Returns false on a non-positive pivot. kap is the
// condition estimate (max L_ii / min L_ii)^2 over the free variables. T is
// the precision of the whole solve (FP32, or FP64 for an ill-conditioned
// matrix; the FP32 inputs convert to FP64 exactly).
template <int P, typename T>
__device__ __forceinline__ bool damped_solve(const float (&H)[P * (P + 1) / 2],
                                             const float (&g)[P], float lam,
                                             const float (&D)[P], const bool (&pin)[P],
                                             float (&dr)[P], float &kap) {
  T A[P * (P + 1) / 2];  // packed lower: (i, j), j <= i at i (i+1) / 2 + j
  T y[P], rd[P], il[P];
#pragma unroll
  for (int i = 0; i < P; i++) {
    T r = pin[i] ? T(0) : (T)g[i];
#pragma unroll
    for (int j = 0; j < P; j++)
      if (pin[j] && !pin[i]) r -= (T)H[up<P>(i, j)] * (T)dr[j];
    y[i] = r;
#pragma unroll
    for (int j = 0; j <= i; j++) {
      T m;
      if (!pin[i] && !pin[j]) m = (T)H[up<P>(i, j)];
      else m = (i == j) ? T(1) : T(0);
      if (i == j && !pin[i]) m += (T)lam * (T)D[i];
      A[i * (i + 1) / 2 + j] = m;
    }
  }
  // diagonal (Jacobi) scaling: unit diagonal, scaled right-hand side
#pragma unroll
  for (int i = 0; i < P; i++) rd[i] = rsq_step(A[i * (i + 1) / 2 + i]);
#pragma unroll
  for (int i = 0; i < P; i++) {
    y[i] *= rd[i];
#pragma unroll
    for (int j = 0; j <= i; j++) A[i * (i + 1) / 2 + j] *= rd[i] * rd[j];
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < P; j++) {
    T s = A[j * (j + 1) / 2 + j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
    ok = ok && (s > T(0));
    T r = rsq_step(s > T(0) ? s : T(1));
    il[j] = r;                               // 1 / L_jj
    A[j * (j + 1) / 2 + j] = (s > T(0) ? s : T(1)) * r;
#pragma unroll
    for (int i = j + 1; i < P; i++) {
      T t = A[i * (i + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
      A[i * (i + 1) / 2 + j] = t * r;
    }
  }
  if (!ok) return false;
  // the condition estimate needs no more than FP32
  float lmax = 0.f, lmin = 1e30f;
#pragma unroll
  for (int i = 0; i < P; i++)
    if (!pin[i]) {
      const float l = (float)A[i * (i + 1) / 2 + i];
      lmax = fmaxf(l, lmax);
      lmin = fminf(l, lmin);
    }
  kap = lmax > 0.f ? (lmax * lmax) / (lmin * lmin) : 1.f;
#pragma unroll
  for (int i = 0; i < P; i++) {
    T s = y[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= A[i * (i + 1) / 2 + k] * y[k];
    y[i] = s * il[i];
  }
#pragma unroll
  for (int i = P - 1; i >= 0; i--) {
    T s = y[i];
#pragma unroll
    for (int k = i + 1; k < P; k++) s -= A[k * (k + 1) / 2 + i] * y[k];
    y[i] = s * il[i];
  }
#pragma unroll
  for (int i = 0; i < P; i++)
    if (!pin[i]) dr[i] = (float)(y[i] * rd[i]);
  return true;
}

// The damped solve of damped_solve<P, double> (the same operations in the
// same order) in little code and few registers, for the cold FP64 path of the
// tensor-core stage 2, where a call to an out-of-line FP64 step cost the hot
// loop registers and instruction-cache room: the group's first lane solves
// on a shared-memory scratch w (8-byte aligned; (P (P + 1) / 2 + 3 P) doubles
// and 3 P + 2 floats) with rolled loops, and the group reads the step back.
template <int P, class GP>
__device__ __forceinline__ bool damped_solve_s64(const GP &gp, const float *H, const float *g, float lam,
                                                 const float (&D)[P], const bool (&pin)[P],
                                                 float (&dr)[P], float &kap, double *w) {
  constexpr int NA = P * (P + 1) / 2;
  double *A = w, *y = w + NA, *rd = y + P, *il = rd + P;
  float *fD = reinterpret_cast<float *>(il + P), *fdr = fD + P, *fpin = fdr + P, *fout = fpin + P;
  if (gp.sub == 0) {
#pragma unroll
    for (int i = 0; i < P; i++) {
      fD[i] = D[i];
      fdr[i] = dr[i];
      fpin[i] = pin[i] ? 1.f : 0.f;
    }
#pragma unroll 1
    for (int i = 0; i < P; i++) {
      const bool pi = fpin[i] != 0.f;
      double r = pi ? 0.0 : (double)g[i];
#pragma unroll 1
      for (int j = 0; j < P; j++)
        if (fpin[j] != 0.f && !pi) r -= (double)H[up<P>(i, j)] * (double)fdr[j];
      y[i] = r;
#pragma unroll 1
      for (int j = 0; j <= i; j++) {
        const bool pj = fpin[j] != 0.f;
        double m;
        if (!pi && !pj) m = (double)H[up<P>(i, j)];
        else m = (i == j) ? 1.0 : 0.0;
        if (i == j && !pi) m += (double)lam * (double)fD[i];
        A[i * (i + 1) / 2 + j] = m;
      }
    }
#pragma unroll 1
    for (int i = 0; i < P; i++) rd[i] = rsq_step(A[i * (i + 1) / 2 + i]);
#pragma unroll 1
    for (int i = 0; i < P; i++) {
      y[i] *= rd[i];
#pragma unroll 1
      for (int j = 0; j <= i; j++) A[i * (i + 1) / 2 + j] *= rd[i] * rd[j];
    }
    bool ok = true;
#pragma unroll 1
    for (int j = 0; j < P; j++) {
      double sj = A[j * (j + 1) / 2 + j];
#pragma unroll 1
      for (int k = 0; k < j; k++) sj -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
      ok = ok && (sj > 0.0);
      const double r = rsq_step(sj > 0.0 ? sj : 1.0);
      il[j] = r;
      A[j * (j + 1) / 2 + j] = (sj > 0.0 ? sj : 1.0) * r;
#pragma unroll 1
      for (int i = j + 1; i < P; i++) {
        double t = A[i * (i + 1) / 2 + j];
#pragma unroll 1
        for (int k = 0; k < j; k++) t -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
        A[i * (i + 1) / 2 + j] = t * r;
      }
    }
    float kp = 1.f;
    if (ok) {
      float lmax = 0.f, lmin = 1e30f;
#pragma unroll 1
      for (int i = 0; i < P; i++)
        if (fpin[i] == 0.f) {
          const float l = (float)A[i * (i + 1) / 2 + i];
          lmax = fmaxf(l, lmax);
          lmin = fminf(l, lmin);
        }
      kp = lmax > 0.f ? (lmax * lmax) / (lmin * lmin) : 1.f;
#pragma unroll 1
      for (int i = 0; i < P; i++) {
        double t = y[i];
#pragma unroll 1
        for (int k = 0; k < i; k++) t -= A[i * (i + 1) / 2 + k] * y[k];
        y[i] = t * il[i];
      }
#pragma unroll 1
      for (int i = P - 1; i >= 0; i--) {
        double t = y[i];
#pragma unroll 1
        for (int k = i + 1; k < P; k++) t -= A[k * (k + 1) / 2 + i] * y[k];
        y[i] = t * il[i];
      }
#pragma unroll 1
      for (int i = 0; i < P; i++)
        if (fpin[i] == 0.f) fdr[i] = (float)(y[i] * rd[i]);
    }
    fout[0] = ok ? 1.f : 0.f;
    fout[1] = kp;
  }
  gp.sync();
  const bool ok = fout[0] != 0.f;
  kap = fout[1];
  if (ok) {
#pragma unroll
    for (int i = 0; i < P; i++)
      if (!pin[i]) dr[i] = fdr[i];
  }
  gp.sync();
  return ok;
}

// -------------------------------------------------------- LM driver -----
template <int G>
struct Grp;
struct LMResult {
  int iters, full, status;   // trial steps; full model + Jacobian evaluations
  bool used64;
  float cost, cdata;
};

// State of the damped iteration shared by the two stage drivers.
template <int P>
struct LMIter {
  float lam = -1.f, nu = 2.f, pred = 0.f;
  int it = 0, status = PX_MAXITER, n64 = 0;   // n64: FP64 step solves
  bool fresh = true, used64 = false;
  bool act[P];
};

// From the normal equations (H, g) at the current state x: the convergence
// test (when they are fresh; gf is the FP32 rounding floor of g, see
// kFloorC), then the damped projected-Newton step and the
// trial point xt with its predicted decrease. Returns false when the fit
// stops (converged, step below tol_x, damping overflow, iteration cap).
// T is the precision of the step solve. In FP32 an ill-conditioned or
// indefinite damped matrix sets want64 and returns at once, leaving the
// iteration's state as it is, so that the FP64 instantiation (out of line:
// next_trial64) takes the whole step from there; keeping the rare FP64 path
// out of this function keeps the hot loop's registers free (with the FP64
// call inline the solve took 5,400 instead of 3,400 cycles per trial).
template <class St, typename T, bool SM64 = false>
__device__ __forceinline__ bool next_trial_t(const St &S, const Grp<St::GL> &gp, const KConfig &c,
                                             const float (&x)[St::NX], const float (&H)[St::NH],
                                             const float (&g)[St::P], const float (&gf)[St::P], int m,
                                             float cst, int max_it, LMIter<St::P> &L,
                                             float (&xt)[St::NX], bool &want64, double *s64 = nullptr) {
  constexpr int P = St::P, NX = St::NX;
  // SM64: an ill-conditioned or indefinite FP32 solve switches the rest of
  // this call to FP64 solves (damped_solve_s64 on the scratch s64) and
  // restarts its projected-Newton passes, instead of returning want64
  bool use64 = false;
#pragma unroll 1
  while (L.it < max_it) {
    if (L.fresh) {
      bool small = true;
      static_for<P>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        float xv = St::template rsel<a>(x, m);
        bool lo_hit = xv <= S.template lo_r<a>(c, m);
        bool hi_hit = St::template has_upper<a>() && xv >= S.template hi_r<a>(c, m);
        L.act[a] = (lo_hit && g[a] <= 0.f) || (hi_hit && g[a] >= 0.f);
        if (!L.act[a] && fabsf(g[a]) > c.tol_g * sqrtf(H[up<P>(a, a)] * cst)) small = false;
      });
      if (small) { L.status = PX_CONVERGED; return false; }
      // the damping matrix is diag H, so lambda is the relative damping of
      // every diagonal: it starts at tau0 whatever the units of H
      if (L.lam < 0.f) L.lam = c.tau0;
      L.fresh = false;
    }
    // damping diagonal, projected-Newton solve with re-solve on bound hits
    float D[P], dr[P];
    bool pin[P];
    signed char pd[P];   // -1 / +1: pinned on lo / hi by the step solve
    float mxd = 0.f;
#pragma unroll
    for (int a = 0; a < P; a++)
      if (!L.act[a]) mxd = fmaxf(mxd, H[up<P>(a, a)]);
#pragma unroll
    for (int a = 0; a < P; a++) {
      D[a] = fmaxf(H[up<P>(a, a)], c.dfloor * mxd);
      pin[a] = L.act[a];
      dr[a] = 0.f;
      pd[a] = 0;
    }
    bool ok = true;
#pragma unroll 1
    for (int pass = 0; pass <= P; pass++) {
      int nf = 0;
#pragma unroll
      for (int a = 0; a < P; a++) nf += !pin[a];
      if (nf == 0) break;
      float kap = 0.f;
      if (SM64 && use64) {
        ok = damped_solve_s64<P>(gp, H, g, L.lam, D, pin, dr, kap, s64);
        L.used64 = true;
        L.n64++;
      } else {
        ok = damped_solve<P, T>(H, g, L.lam, D, pin, dr, kap);
        if constexpr (sizeof(T) == sizeof(float)) {
          if (!ok || !(kap <= c.kappa_max)) {
            if constexpr (SM64) {
              use64 = true;
#pragma unroll
              for (int a = 0; a < P; a++) {
                pin[a] = L.act[a];
                dr[a] = 0.f;
                pd[a] = 0;
              }
              pass = -1;
              continue;
            } else {
              want64 = true;
              return false;
            }
          }
        } else {
          L.used64 = true;
          L.n64++;
        }
      }
      if (!ok) break;
      bool viol = false;
      static_for<P>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        if (!pin[a]) {
          float xv = St::template rsel<a>(x, m);
          float sc = S.template sc_r<a>(c, m);
          float lo = S.template lo_r<a>(c, m), hi = S.template hi_r<a>(c, m);
          float xn = xv + sc * dr[a];
          if (!(sc > 0.f)) { pin[a] = true; dr[a] = 0.f; viol = true; }
          else if (xn < lo) { pin[a] = true; pd[a] = -1; dr[a] = (lo - xv) / sc; viol = true; }
          else if (St::template has_upper<a>() && xn > hi) {
            pin[a] = true; pd[a] = 1; dr[a] = (hi - xv) / sc; viol = true;
          }
        }
      });
      if (!viol) break;
    }
    if (!ok) {
      L.lam *= L.nu; L.nu *= 2.f; L.it++;
      if (!(L.lam < 1e30f)) { L.status = PX_CHOL_FAIL; return false; }
      continue;
    }
    S.apply(c, x, dr, pd, m, xt);
    float Dz[NX], dmax = 0.f;
#pragma unroll
    for (int i = 0; i < NX; i++) {
      Dz[i] = (xt[i] - x[i]) * S.zk(c, i);   // 1 / scale, 0 for a fixed variable
      dmax = fmaxf(dmax, fabsf(Dz[i]));
    }
    if (dmax < c.tol_x) { L.status = PX_CONVERGED; return false; }
    float Dr[P];
    static_for<P>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      Dr[a] = St::template rsel<a>(Dz, m);
    });
    // predicted decrease of the Gauss-Newton model: 2 g.D - D.H.D, as
    // sum_a D_a (2 g_a - (H D)_a): P independent dot products, then one
    // short sum (the one long accumulation chain was a latency chain)
    float pred = 0.f;
#pragma unroll
    for (int a = 0; a < P; a++) {
      float hd = 0.f;
#pragma unroll
      for (int b = 0; b < P; b++) hd = fmaf(H[up<P>(a, b)], Dr[b], hd);
      pred = fmaf(Dr[a], fmaf(2.f, g[a], -hd), pred);
    }
    L.pred = pred;
    L.it++;
    return true;
  }
  // iteration cap: converged if the gradient of the free variables is within
  // the tolerance plus its FP32 floors: the rounding of its band sums (gf),
  // and the spacing of the FP32 state, the gradient that moves of the free
  // variables by two units in the last place make, sum_b |H_ab| u_b. Next to
  // a minimum sharper than that spacing no FP32 state meets the tolerance,
  // and the iteration cycles between neighbouring states up to the cap.
  float Uz[NX], u[P];
#pragma unroll
  for (int i = 0; i < NX; i++) Uz[i] = fabsf(x[i]) * 0x1p-22f * S.zk(c, i);
  static_for<P>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    u[a] = L.act[a] ? 0.f : St::template rsel<a>(Uz, m);
  });
  bool small = true;
  static_for<P>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    float q = gf[a];
#pragma unroll
    for (int b = 0; b < P; b++) q = fmaf(fabsf(H[up<P>(a, b)]), u[b], q);
    if (!L.act[a] && fabsf(g[a]) > fmaf(c.tol_g, sqrtf(H[up<P>(a, a)] * cst), q)) small = false;
  });
  if (small) L.status = PX_CONVERGED;
  return false;
}

// The LM step with its solves in FP64, out of line: inputs and outputs in
// one struct, so that the caller's arrays are not address-taken
template <class St>
struct Step64 {
  float x[St::NX], H[St::NH], g[St::P], gf[St::P], xt[St::NX];
  int m, max_it;
  float cst;
  LMIter<St::P> L;
};
template <class St>
__device__ __noinline__ bool next_trial64(const St &S, const Grp<St::GL> &gp, const KConfig &c,
                                          Step64<St> &q) {
  bool unused = false;
  return next_trial_t<St, double>(S, gp, c, q.x, q.H, q.g, q.gf, q.m, q.cst, q.max_it, q.L, q.xt, unused);
}

template <class St>
__device__ __forceinline__ bool next_trial(const St &S, const Grp<St::GL> &gp, const KConfig &c,
                                           const float (&x)[St::NX], const float (&H)[St::NH],
                                           const float (&g)[St::P], const float (&gf)[St::P], int m,
                                           float cst, int max_it, LMIter<St::P> &L,
                                           float (&xt)[St::NX]) {
  bool want64 = false;
  const bool go = next_trial_t<St, float>(S, gp, c, x, H, g, gf, m, cst, max_it, L, xt, want64);
  if (!want64) return go;
  Step64<St> q;
#pragma unroll
  for (int i = 0; i < St::NX; i++) { q.x[i] = x[i]; q.xt[i] = xt[i]; }
#pragma unroll
  for (int i = 0; i < St::NH; i++) q.H[i] = H[i];
#pragma unroll
  for (int a = 0; a < St::P; a++) { q.g[a] = g[a]; q.gf[a] = gf[a]; }
  q.m = m;
  q.max_it = max_it;
  q.cst = cst;
  q.L = L;
  const bool go64 = next_trial64<St>(S, gp, c, q);
  L = q.L;
#pragma unroll
  for (int i = 0; i < St::NX; i++) xt[i] = q.xt[i];
  return go64;
}

// Nielsen damping update after a step with gain ratio rho
template <int P>
__device__ __forceinline__ void damping_update(LMIter<P> &L, bool accept, float rho) {
  if (accept) {
    float f = 2.f * rho - 1.f;
    f = 1.f - f * f * f;
    L.lam *= fmaxf(f, 1.f / 3.f);
    L.nu = 2.f;
    L.fresh = true;
  } else {
    L.lam *= L.nu;
    L.nu *= 2.f;
  }
}

// ------------------------------------------------------------ Adam -----
// The paper's optimiser (Sec. 2.6, Eq. adam), the FIRE_SOLVER_ADAM path of
// the stage kernels: a fixed number of steps, each on every variable's own z
// coordinate of Eq. (affine). Its moments live in registers of the Adam
// instantiations only.
template <int NX>
struct AdamState {
  float m[NX], v[NX];
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int i = 0; i < NX; i++) m[i] = v[i] = 0.f;
  }
};

// One Adam step t (1-based) from x, given G = Jz^T W r of every coordinate
// (the z gradient of Eq. loss is -2 G): the gradient clipped to a global norm
// of adam_clip, the moment updates, the bias-corrected step
// lr mhat / (sqrt(vhat) + eps), z clipped to [-1, 1]. A fixed variable
// (zk = 0) keeps its value.
template <int NX>
__device__ __forceinline__ void adam_step(const KConfig &c, int t, float lr, const float *lo,
                                          const float *hi, const float *zk, const float (&x)[NX],
                                          const float (&G)[NX], AdamState<NX> &A, float (&xt)[NX]) {
  float gz[NX], n2 = 0.f;
#pragma unroll
  for (int i = 0; i < NX; i++) {
    gz[i] = zk[i] > 0.f ? -2.f * G[i] : 0.f;
    n2 = fmaf(gz[i], gz[i], n2);
  }
  const float nrm = sqrtf(n2);
  const float f = nrm > c.adam_clip ? c.adam_clip / nrm : 1.f;
  // bias corrections 1 - beta^t in FP64 (once per step): in FP32, 1 - 0.999^t
  // would lose its leading digits to cancellation for small t
  const float bc1 = (float)(1.0 - pow(c.adam_b1d, (double)t));
  const float bc2 = (float)(1.0 - pow(c.adam_b2d, (double)t));
#pragma unroll
  for (int i = 0; i < NX; i++) {
    if (!(zk[i] > 0.f)) { xt[i] = x[i]; continue; }
    const float gi = gz[i] * f;
    A.m[i] = fmaf(c.adam_b1, A.m[i], c.adam_omb1 * gi);
    A.v[i] = fmaf(c.adam_b2, A.v[i], c.adam_omb2 * gi * gi);
    float z = fmaf(x[i] - lo[i], zk[i], -1.f);
    z -= lr * (A.m[i] / bc1) / (sqrtf(A.v[i] / bc2) + c.adam_eps);
    z = fminf(fmaxf(z, -1.f), 1.f);
    xt[i] = fmaf(0.5f * (hi[i] - lo[i]), z + 1.f, lo[i]);
  }
}

// The next Adam trial point of stage 1 (false once adam_steps1 steps are
// taken): the full-coordinate gradient from the reduced one (pivot m) and
// the pivot's own sum gm, the step, then the simplex projection of the
// fractions (Sec. 2.6).
template <int K, class St>
__device__ __forceinline__ bool adam_next1(const KConfig &c, const float (&x)[K + 2],
                                           const float (&g)[K + 1], float gm, int m,
                                           AdamState<K + 2> &A, LMIter<K + 1> &L,
                                           float (&xt)[K + 2]) {
  if (L.it >= c.adam_steps1) { L.status = PX_CONVERGED; return false; }
  float Gf[K + 2];
#pragma unroll
  for (int k = 0; k < K; k++) {
    float gr = 0.f;
#pragma unroll
    for (int a = 0; a < K - 1; a++)
      if (a == (k < m ? k : k - 1)) gr = g[a];
    Gf[k] = k == m ? gm : gr + gm;
  }
  Gf[K] = g[K - 1];
  Gf[K + 1] = g[K];
  adam_step<K + 2>(c, L.it + 1, c.adam_lr1, c.lo1, c.hi1, c.zk1, x, Gf, A, xt);
  St::simplex_project(xt);
  L.it++;
  return true;
}

// The next Adam trial point of stage 2 (false once adam_steps2 steps are taken)
__device__ __forceinline__ bool adam_next2(const KConfig &c, const float (&x)[6], const float (&g)[6],
                                           AdamState<6> &A, LMIter<6> &L, float (&xt)[6]) {
  if (L.it >= c.adam_steps2) { L.status = PX_CONVERGED; return false; }
  adam_step<6>(c, L.it + 1, c.adam_lr2, c.lo2, c.hi2, c.zk2, x, g, A, xt);
  L.it++;
  return true;
}

// ------------------------------------------------------- pixel groups ---
// G consecutive lanes of a warp fit one pixel, so a warp carries 32 / G
// pixels. Reductions are xor shuffles restricted to the group's lanes, so a
// group needs no other group to make progress; the fit loop keeps the
// groups of a warp in step where the work is (every active group evaluates
// the model at the same point of each round).
template <int G>
struct Grp {
  int lane, sub;
  unsigned mask;
  __device__ __forceinline__ explicit Grp(int l)
      : lane(l), sub(l & (G - 1)),
        mask(G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (l & ~(G - 1)))) {}
  template <int N>
  __device__ __forceinline__ void sum(float (&v)[N]) const {
#pragma unroll
    for (int o = G / 2; o; o >>= 1)
#pragma unroll
      for (int i = 0; i < N; i++) v[i] += __shfl_xor_sync(mask, v[i], o);
  }
  __device__ __forceinline__ float sum1(float v) const {
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
  }
  __device__ __forceinline__ int isum(int v) const {
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
  }
  __device__ __forceinline__ bool all(bool p) const { return __all_sync(mask, p); }
  __device__ __forceinline__ long long bcast(long long v) const {
    return __shfl_sync(mask, v, lane & ~(G - 1));
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

// Per-pixel shared scratch of one group: stage 2 node weights [nt][8], then
// band buffers of nbs = G * ceil(n / G) slots each (slot i = sub + G s).
// The stride between groups is congruent to G modulo 32 floats, so that the
// groups of a warp, reading the same slot or node, hit different banks.
__host__ __device__ __forceinline__ int band_slots(int n, int G) { return G * ((n + G - 1) / G); }
__host__ __device__ __forceinline__ int pix_stride1(const KTables &t, int G) {
  int f = 4 * band_slots(t.n1, G);
  return f + ((G - f % 32) % 32 + 32) % 32;
}
constexpr int kNE2 = 48;   // stage-2 per-pixel slot: trial H[21], g[6], floor[6] at 30
__host__ __device__ __forceinline__ int pix_stride2(const KTables &t, int G) {
  int f = t.nt * kScratchPerNode + 5 * band_slots(t.n2, G) + kNE2;
  return f + ((G - f % 32) % 32 + 32) % 32;
}
// table-image floats a stage needs: stage 1 stops before the Planck grid
__host__ __device__ __forceinline__ int image_floats(const KTables &t, int stage) {
  return stage == 1 ? ((t.lay.off_planck + 3) & ~3) : t.lay.total;
}
// the water-vapour table [nwv][nb] float4, staged in shared memory by stage 1
// when it takes at most 96 KB (16 bins x 284 bands: 71 KB) and the shape has
// 16 or more lanes per pixel, else read from global memory: at 8 lanes the
// band buffers of four pixels per warp need the room (11 warps instead of 7
// per SM; measured 4 % faster than staging the table)
__host__ __device__ __forceinline__ int wvtab_floats(const KTables &t, int G) {
  return G >= 16 && t.nwv * t.nb * 16 <= 96 * 1024 ? t.nwv * t.nb * 4 : 0;
}

// ------------------------------------------------------- pixel context --
struct PixCtx {
  const KTables *t;
  const KConfig *c;
  const float *img;       // shared-memory table image
  float *node;            // this group's node scratch [nt][8] (stage 2)
  const float4 *wvrow;    // this pixel's water-vapour row of the atmosphere table
};

// ------------------------------------------------------------ stage 1 ---
template <int K, int G>
struct Stage1 {
  static constexpr int P = K + 1, NX = K + 2, NH = P * (P + 1) / 2, GL = G;
  // band buffers in shared memory, [4][nbs]: observed radiance, weight, and
  // the residuals of the current and the trial state (index rc, rc ^ 1)
  float *bb;
  int nbs;
  float psc;
  float sf, sa, sT;

  __device__ __forceinline__ float &Lo(int i) const { return bb[i]; }
  __device__ __forceinline__ float &W(int i) const { return bb[nbs + i]; }
  __device__ __forceinline__ float &R(int k, int i) const { return bb[(2 + k) * nbs + i]; }

  // reduced variable a: fractions k != m in order, then alpha1, T1. These
  // accessors select with compile-time indices (no local-memory indexing).
  template <int A>
  __device__ __forceinline__ static float rsel(const float (&v)[NX], int m) {
    if constexpr (A >= K - 1) return v[A + 1];
    else return A < m ? v[A] : v[A + 1];
  }
  template <int A>
  __device__ __forceinline__ float lo_r(const KConfig &c, int m) const {
    if constexpr (A >= K - 1) return c.lo1[A + 1];
    else return A < m ? c.lo1[A] : c.lo1[A + 1];
  }
  template <int A>
  __device__ __forceinline__ float hi_r(const KConfig &c, int m) const {
    if constexpr (A >= K - 1) return c.hi1[A + 1];
    else return A < m ? c.hi1[A] : c.hi1[A + 1];
  }
  template <int A>
  __device__ __forceinline__ float sc_r(const KConfig &c, int m) const {
    return 0.5f * (hi_r<A>(c, m) - lo_r<A>(c, m));
  }
  template <int A>
  __device__ __forceinline__ static constexpr bool has_upper() { return A >= K - 1; }
  __device__ __forceinline__ float scale(const KConfig &c, int i) const {
    return 0.5f * (c.hi1[i] - c.lo1[i]);
  }
  __device__ __forceinline__ float zk(const KConfig &c, int i) const { return c.zk1[i]; }

  __device__ __forceinline__ static int argmax_frac(const float (&x)[NX]) {
    int m = 0;
    float best = x[0];
#pragma unroll
    for (int k = 1; k < K; k++)
      if (x[k] > best) { m = k; best = x[k]; }
    return m;
  }

  // model, reduced Jacobian, normal equations and cost at x (all lanes of
  // the group get the totals); writes the residuals into set rn and returns
  // the data-cost decrease from the state xo, whose residuals are set 1 - rn. cd = unweighted data cost. The
  // decrease is formed from residual differences, or, with inc (small
  // steps, whose decrease the difference of two FP32 model values no longer
  // resolves), in increment form: dM_b = dLs_b + tu_b (d alpha B_o + alpha
  // dB_b) with
  //   dLs_b = A_b drho_b / ((1 - S_b rho_t)(1 - S_b rho_o)),
  //   dB_b = B_o expm1(-dx_b) / (1 - e^-x_t), dx_b = -(c2/lambda_b) dT / (T_t T_o)
  //   (expm1 by its Taylor series for |dx_b| < 0.5, else B_t - B_o),
  // each increment formed from the exact parameter differences; B_o and
  // 1 / (1 - S_b rho_o) are recomputed at xo with the instructions that
  // formed them when xo was evaluated.
  //
  // With GM (the Adam solver, which moves every fraction on its own z
  // coordinate) it also returns gm = sum_b w_b r_b dL_b/dz_m of the pivot
  // fraction m, from which the full-coordinate gradient follows:
  // G_k = g_(k) + gm for k != m, G_m = gm.
  template <bool GM = false>
  __device__ __forceinline__ void eval(const PixCtx &pc, const Grp<G> &gp, const float (&x)[NX],
                                       int rn, float (&H)[NH], float (&g)[P], float (&gf)[P],
                                       float &cst, float &cd, float &drop, int &m,
                                       const float (&xo)[NX], bool inc, float *gm = nullptr) const {
    constexpr int NA = NH + P + 5 + (GM ? 1 : 0);
    const KTables &t = *pc.t;
    const KConfig &c = *pc.c;
    m = argmax_frac(x);
    // Each lane takes its bands in consecutive pairs (i0, i0 + 1), i0 = 2 sub
    // + 2 G s, and forms both with the packed FP32 instructions (two
    // round-to-nearest operations per instruction); the pair's two partial
    // sums are added at the end. A masked band of a pair (weight 0) adds
    // exact zeros.
    float2 sm[NA];
#pragma unroll
    for (int i = 0; i < NA; i++) sm[i] = make_float2(0.f, 0.f);
    const float a1 = x[K], invT = 1.f / x[K + 1], invTo = 1.f / xo[K + 1];
    const float dTT = (x[K + 1] - xo[K + 1]) * invT / xo[K + 1];
    const float dal = a1 - xo[K];
    float dxs[K];
#pragma unroll
    for (int k = 0; k < K; k++) dxs[k] = x[k] - xo[k];
    const float *ro = bb + (3 - rn) * nbs;
    float *rw = bb + (2 + rn) * nbs;
    const float2 one = make_float2(1.f, 1.f), a1v = make_float2(a1, a1);
    const float2 invTv = make_float2(invT, invT);
#pragma unroll kBand1Unroll
    for (int i0 = 2 * gp.sub; i0 < t.n1; i0 += 2 * G) {
      const float2 wv = *reinterpret_cast<const float2 *>(&W(i0));
      if (!(wv.x > 0.f) && !(wv.y > 0.f)) continue;
      const int b0 = t.b1lo + i0, b1 = min(b0 + 1, t.nb - 1);
      const float4 qa = pc.wvrow[b0], qb = pc.wvrow[b1];
      const float2 qx = make_float2(qa.x, qb.x), qy = make_float2(qa.y, qb.y);
      const float2 nqz = make_float2(-qa.z, -qb.z), qw = make_float2(qa.w, qb.w);
      float2 E[K];
      float2 rho = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < K; k++) {
        const float *ek = pc.img + t.lay.off_endm + k * t.nb;
        E[k] = make_float2(ek[b0], ek[b1]);
        rho = __ffma2_rn(make_float2(x[k], x[k]), E[k], rho);
      }
      // fast reciprocals (within 2 ulp): both arguments lie well inside (0, 1]
      const float2 den = __ffma2_rn(nqz, rho, one);
      const float2 inv = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));
      const float2 Ls = __ffma2_rn(__fmul2_rn(qx, rho), inv, qy);
      const float2 c2l = make_float2(pc.img[t.lay.off_c2l + b0], pc.img[t.lay.off_c2l + b1]);
      const float2 c1l5 = make_float2(pc.img[t.lay.off_c1l5 + b0], pc.img[t.lay.off_c1l5 + b1]);
      const float2 xx = __fmul2_rn(c2l, invTv);
      const float2 e = make_float2(__expf(-xx.x), __expf(-xx.y));
      const float2 rom = make_float2(__fdividef(1.f, 1.f - e.x), __fdividef(1.f, 1.f - e.y));
      const float2 B = __fmul2_rn(__fmul2_rn(c1l5, e), rom);
      const float2 dB = __fmul2_rn(__fmul2_rn(__fmul2_rn(B, xx), invTv), rom);
      const float2 Lo2 = *reinterpret_cast<const float2 *>(&Lo(i0));
      const float2 mod = __ffma2_rn(__fmul2_rn(a1v, qw), B, Ls);
      // a masked band's residual is taken as 0, so that it adds nothing to
      // the unweighted data cost either
      const float2 r = make_float2(wv.x > 0.f ? Lo2.x - mod.x : 0.f, wv.y > 0.f ? Lo2.y - mod.y : 0.f);
      const float2 rold = *reinterpret_cast<const float2 *>(ro + i0);
      *reinterpret_cast<float2 *>(rw + i0) = r;
      if (inc) {
        float2 drho = make_float2(0.f, 0.f), rho_o = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; k++) {
          drho = __ffma2_rn(make_float2(dxs[k], dxs[k]), E[k], drho);
          rho_o = __ffma2_rn(make_float2(xo[k], xo[k]), E[k], rho_o);
        }
        const float2 den_o = __ffma2_rn(nqz, rho_o, one);
        const float2 inv_o = make_float2(__fdividef(1.f, den_o.x), __fdividef(1.f, den_o.y));
        const float2 xo2 = __fmul2_rn(c2l, make_float2(invTo, invTo));
        const float2 e_o = make_float2(__expf(-xo2.x), __expf(-xo2.y));
        const float2 Bo = __fmul2_rn(__fmul2_rn(c1l5, e_o),
                                     make_float2(__fdividef(1.f, 1.f - e_o.x), __fdividef(1.f, 1.f - e_o.y)));
        const float2 dLs = __fmul2_rn(__fmul2_rn(__fmul2_rn(qx, drho), inv), inv_o);
        const float2 dx = __fmul2_rn(c2l, make_float2(-dTT, -dTT));
        // dB = B_o expm1(-dx) / (1 - e^-x_t), equal to B - B_o, which has no
        // cancellation left once |dx| >= 0.5
        const float2 pm = __fmul2_rn(__fmul2_rn(Bo, em1_mid2(make_float2(-dx.x, -dx.y))), rom);
        float2 dBi;
        dBi.x = fabsf(dx.x) < 0.5f ? pm.x : B.x - Bo.x;
        dBi.y = fabsf(dx.y) < 0.5f ? pm.y : B.y - Bo.y;
        const float2 dM = __ffma2_rn(qw, __ffma2_rn(make_float2(dal, dal), Bo, __fmul2_rn(a1v, dBi)), dLs);
        const float2 t2 = __ffma2_rn(make_float2(2.f, 2.f), rold, make_float2(-dM.x, -dM.y));
        sm[NH + P + 2] = __ffma2_rn(__fmul2_rn(wv, dM), t2, sm[NH + P + 2]);
      } else {
        sm[NH + P + 2] = __ffma2_rn(__fmul2_rn(wv, make_float2(rold.x - r.x, rold.y - r.y)),
                                    __fadd2_rn(rold, r), sm[NH + P + 2]);
      }
      float2 dL[K], dEm = make_float2(0.f, 0.f);
      const float2 qi2 = __fmul2_rn(__fmul2_rn(__fmul2_rn(qx, inv), inv), make_float2(sf, sf));
#pragma unroll
      for (int k = 0; k < K; k++) {
        dL[k] = __fmul2_rn(qi2, E[k]);
        dEm = (k == m) ? dL[k] : dEm;
      }
      float2 J[P];
#pragma unroll
      for (int a = 0; a < K - 1; a++) {
        const float2 d = a < m ? dL[a] : dL[a + 1];
        J[a] = make_float2(d.x - dEm.x, d.y - dEm.y);
      }
      J[K - 1] = __fmul2_rn(__fmul2_rn(qw, B), make_float2(sa, sa));
      J[K] = __fmul2_rn(__fmul2_rn(__fmul2_rn(a1v, qw), dB), make_float2(sT, sT));
      const float2 wr = __fmul2_rn(wv, r);
      const float2 wM = __fmul2_rn(wv, make_float2(Lo2.x - r.x, Lo2.y - r.y));   // weight x model value
      sm[NH + P] = __ffma2_rn(wr, r, sm[NH + P]);
      sm[NH + P + 1] = __ffma2_rn(r, r, sm[NH + P + 1]);
      sm[NH + P + 3] = __ffma2_rn(wM, wM, sm[NH + P + 3]);
      sm[NH + P + 4] = __fadd2_rn(sm[NH + P + 4], wv);
      if constexpr (GM) sm[NA - 1] = __ffma2_rn(wr, dEm, sm[NA - 1]);
#pragma unroll
      for (int a = 0; a < P; a++) {
        sm[NH + a] = __ffma2_rn(J[a], wr, sm[NH + a]);
        const float2 wj = __fmul2_rn(wv, J[a]);
#pragma unroll
        for (int bb_ = a; bb_ < P; bb_++) sm[up<P>(a, bb_)] = __ffma2_rn(wj, J[bb_], sm[up<P>(a, bb_)]);
      }
    }
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; i++) acc[i] = sm[i].x + sm[i].y;
    gp.sum(acc);
    if constexpr (GM) *gm = acc[NA - 1];
#pragma unroll
    for (int i = 0; i < NH; i++) H[i] = acc[i];
    // FP32 floor of g_a: kFloorC sqrt(sum_b (w_b J_ba M_b)^2), estimated as
    // kFloorC sqrt(H_aa sum_b w_b^2 M_b^2 / sum_b w_b) (data part of H_aa)
    const float m2 = acc[NH + P + 3] / fmaxf(acc[NH + P + 4], 1e-30f);
#pragma unroll
    for (int a = 0; a < P; a++) {
      g[a] = acc[NH + a];
      gf[a] = kFloorC * sqrtf(acc[up<P>(a, a)] * m2);
    }
    cd = acc[NH + P + 1];
    cst = acc[NH + P];
    drop = acc[NH + P + 2];
    // weak Gaussian prior in z, pulled into the reduced basis (e_k - e_m)
    float zr[NX], ppm = 0.f, rm = 0.f;
#pragma unroll
    for (int i = 0; i < NX; i++) {
      zr[i] = c.zk1[i] > 0.f ? fmaf(x[i] - c.lo1[i], c.zk1[i], -1.f) : 0.f;
      zr[i] -= c.pm1[i];
      float ppi = psc * c.pp1[i];
      cst += ppi * zr[i] * zr[i];
      if (i < K && i == m) { ppm = ppi; rm = zr[i]; }
    }
#pragma unroll
    for (int a = 0; a < K - 1; a++) {
      float ppa = psc * (a < m ? c.pp1[a] : c.pp1[a + 1]);
      float ra = a < m ? zr[a] : zr[a + 1];
      g[a] -= ppa * ra - ppm * rm;
      H[up<P>(a, a)] += ppa + ppm;
#pragma unroll
      for (int bb_ = a + 1; bb_ < K - 1; bb_++) H[up<P>(a, bb_)] += ppm;
    }
#pragma unroll
    for (int a = K - 1; a < P; a++) {
      g[a] -= psc * c.pp1[a + 1] * zr[a + 1];
      H[up<P>(a, a)] += psc * c.pp1[a + 1];
    }
    gp.sync();
  }

  // prior(x_old) - prior(x_new), formed from differences of z
  __device__ __forceinline__ float prior_drop(const KConfig &c, const float (&xo)[NX],
                                              const float (&xn)[NX]) const {
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < NX; i++) {
      if (c.hi1[i] > c.lo1[i] && c.pp1[i] > 0.f) {
        const float k = c.zk1[i];
        float zo = k * (xo[i] - c.lo1[i]) - 1.f - c.pm1[i], zn = k * (xn[i] - c.lo1[i]) - 1.f - c.pm1[i];
        d += psc * c.pp1[i] * (k * (xo[i] - xn[i])) * (zo + zn);
      }
    }
    return d;
  }

  // x + step (z units, reduced basis) -> projected trial point
  __device__ __forceinline__ void apply(const KConfig &c, const float (&x)[NX], const float (&dr)[P],
                                        const signed char (&pd)[P], int m, float (&xt)[NX]) const {
    float sum = 0.f;
#pragma unroll
    for (int a = 0; a < K - 1; a++) sum += dr[a];
#pragma unroll
    for (int k = 0; k < K; k++) {
      float d = 0.f;
      bool at0 = false;   // pinned on its lower bound by the step solve
      if (k < K - 1 && k < m) { d = dr[k < K - 1 ? k : 0]; at0 = pd[k < K - 1 ? k : 0] < 0; }
      if (k > 0 && k > m) { d = dr[k > 0 ? k - 1 : 0]; at0 = pd[k > 0 ? k - 1 : 0] < 0; }
      xt[k] = (k == m) ? x[k] - sf * sum : (at0 ? c.lo1[k] : x[k] + sf * d);
    }
#pragma unroll
    for (int i = K; i < K + 2; i++) {
      float v = x[i] + scale(c, i) * dr[i - 1];
      if (pd[i - 1] < 0) v = c.lo1[i];
      if (pd[i - 1] > 0) v = c.hi1[i];
      xt[i] = fminf(fmaxf(v, c.lo1[i]), c.hi1[i]);
    }
    simplex_project(xt);
  }

  // Euclidean projection of the fractions onto the unit simplex (sort-based)
  __device__ __forceinline__ static void simplex_project(float (&x)[NX]) {
    float u[K];
#pragma unroll
    for (int k = 0; k < K; k++) u[k] = x[k];
#pragma unroll
    for (int i = 1; i < K; i++)
#pragma unroll
      for (int j = i; j > 0; j--)
        if (u[j] > u[j - 1]) {
          float tmp = u[j];
          u[j] = u[j - 1];
          u[j - 1] = tmp;
        }
    float cs = 0.f, theta = 0.f;
#pragma unroll
    for (int j = 0; j < K; j++) {
      cs += u[j];
      float th = (cs - 1.f) / (float)(j + 1);
      if (u[j] - th > 0.f) theta = th;
    }
#pragma unroll
    for (int k = 0; k < K; k++) x[k] = fmaxf(x[k] - theta, 0.f);
  }
};

// ------------------------------------------------------------ stage 2 ---
constexpr int kChunk2 = 7;   // stage-2 band slots per lane accumulated per node pass

template <int G>
struct Stage2 {
  static constexpr int P = 6, NX = 6, NH = 21, GL = G;
  // band buffers in shared memory, [5][nbs]: y (radiance minus the fixed
  // solar term), tau_up, weight, and the residuals of the current and of the
  // trial state (index rc, rc ^ 1)
  float *bb;
  int nbs;
  float psc;

  __device__ __forceinline__ float &Y(int i) const { return bb[i]; }
  __device__ __forceinline__ float &TU(int i) const { return bb[nbs + i]; }
  __device__ __forceinline__ float &W(int i) const { return bb[2 * nbs + i]; }
  __device__ __forceinline__ float &R(int k, int i) const { return bb[(3 + k) * nbs + i]; }

  template <int A>
  __device__ __forceinline__ static float rsel(const float (&v)[NX], int) { return v[A]; }
  template <int A>
  __device__ __forceinline__ float lo_r(const KConfig &c, int) const { return c.lo2[A]; }
  template <int A>
  __device__ __forceinline__ float hi_r(const KConfig &c, int) const { return c.hi2[A]; }
  template <int A>
  __device__ __forceinline__ float sc_r(const KConfig &c, int) const {
    return 0.5f * (c.hi2[A] - c.lo2[A]);
  }
  template <int A>
  __device__ __forceinline__ static constexpr bool has_upper() { return true; }
  __device__ __forceinline__ float scale(const KConfig &c, int i) const {
    return 0.5f * (c.hi2[i] - c.lo2[i]);
  }
  __device__ __forceinline__ float zk(const KConfig &c, int i) const { return c.zk2[i]; }

  // Gaussian weight u_o = exp(-a_o^2/2), a = (T - mu)/sigma, of one node at
  // the current state and its change du under the step to (mut, sgt): the
  // exponent change is formed from the parameter differences,
  //   a_t - a_o = -(dmu sigma_o + (T - mu_o) dsig) / (sigma_t sigma_o),
  // and du = u_o expm1(-dq), so du is resolved relative to itself.
  __device__ __forceinline__ static void node_step(float T, float mu, float isg, float mut, float isgt,
                                                   float dmu, float dsg, float &u, float &du) {
    const float ao = (T - mu) * isg, at = (T - mut) * isgt;
    const float da = -fmaf((T - mu) * dsg, isg, dmu) * isgt;
    const float dq = 0.5f * da * (at + ao);
    u = expf(-0.5f * ao * ao);
    du = fabsf(dq) < 0.5f ? u * em1_mid(-dq) : expf(-0.5f * at * at) - u;
  }

  // Model, Jacobian (z-scaled), normal equations and cost at the trial
  // state xt, with the residuals written into buffer rn; and the data-cost
  // decrease from the current state x (residuals in buffer 1 - rn) in
  // increment form: sum_b w_b dM_b (2 r_b - dM_b) with dM_b = tu_b (a_t
  // dBm_b + (a_t - a) (Bm_b - dBm_b)), where dBm is the node sum of the
  // mixture-weight increments, formed node by node from the exact parameter
  // differences. The decrease is then accurate relative to itself, where
  // the difference of two FP32 model values would be lost below their
  // rounding. 7 FMA per band and node.
  // H, g and the gradient's FP32 floor go to the shared slot ne ([21] packed
  // upper H, [6] g at 21, [6] floor at 30), so that they need no registers
  // until the step is accepted.
  __device__ __forceinline__ void eval(const PixCtx &pc, const Grp<G> &gp, const float (&x)[NX],
                                       const float (&xt)[NX], int rn, float *ne, float &cst,
                                       float &cd, float &drop) const {
    const KTables &t = *pc.t;
    const KConfig &c = *pc.c;
    const float mh = xt[0], sh = xt[1], ms = xt[2], ss = xt[3], eta = xt[4], al = xt[5];
    const float eo = x[4], ao = x[5];
    // node pass 1: weights at xt from the weights at x and their increments
    float mom[10];   // U_h, M1_h, M2_h, U_s, M1_s, M2_s at xt; U_h, dU_h, U_s, dU_s at x
#pragma unroll
    for (int k = 0; k < 10; k++) mom[k] = 0.f;
    {
      const float ih = 1.f / x[1], iht = 1.f / sh, is = 1.f / x[3], ist = 1.f / ss;
      const float dmh = mh - x[0], dsh = sh - x[1], dms = ms - x[2], dss = ss - x[3];
      float4 *nd = reinterpret_cast<float4 *>(pc.node);
      for (int j = gp.sub; j < t.nt; j += G) {
        const float T = t.tglo + (float)j * t.tgstep;
        float uh, duh, us, dus;
        node_step(T, x[0], ih, mh, iht, dmh, dsh, uh, duh);
        node_step(T, x[2], is, ms, ist, dms, dss, us, dus);
        const float uth = uh + duh, uts = us + dus, dh = T - mh, ds = T - ms;
        mom[0] += uth;
        mom[1] += uth * dh;
        mom[2] += uth * dh * dh;
        mom[3] += uts;
        mom[4] += uts * ds;
        mom[5] += uts * ds * ds;
        mom[6] += uh;
        mom[7] += duh;
        mom[8] += us;
        mom[9] += dus;
        nd[2 * j] = make_float4(uh, duh, us, dus);
      }
    }
    gp.sum(mom);
    {
      // node pass 2: normalised weights, their moment-weighted forms and
      // the increment of the mixture weight
      const float rUh = 1.f / mom[0], rUs = 1.f / mom[3];
      const float dbh = mom[1] * rUh, m2h = mom[2] * rUh, dbs = mom[4] * rUs, m2s = mom[5] * rUs;
      const float rUho = 1.f / mom[6], rUso = 1.f / mom[8];
      const float kh = mom[7] * rUho, ks = mom[9] * rUso;
      float4 *nd = reinterpret_cast<float4 *>(pc.node);
      for (int j = gp.sub; j < t.nt; j += G) {
        const float T = t.tglo + (float)j * t.tgstep;
        const float4 u = nd[2 * j];
        const float dh = T - mh, ds = T - ms;
        const float wh = (u.x + u.y) * rUh, ws = (u.z + u.w) * rUs;
        const float dwh = (u.y - u.x * kh) * rUh, dws = (u.w - u.z * ks) * rUs;
        const float dW = eta * dwh + (1.f - eta) * dws + (eta - eo) * (u.x * rUho - u.z * rUso);
        nd[2 * j] = make_float4(wh, wh * (dh - dbh), wh * (dh * dh - m2h), ws);
        nd[2 * j + 1] = make_float4(ws * (ds - dbs), ws * (ds * ds - m2s), dW, 0.f);
      }
    }
    gp.sync();
    float acc[NH + P + 5];
#pragma unroll
    for (int i = 0; i < NH + P + 5; i++) acc[i] = 0.f;
    const float ish2 = 1.f / (sh * sh), iss2 = 1.f / (ss * ss);
    const float ish3 = ish2 / sh, iss3 = iss2 / ss;
    const float sc0 = scale(c, 0), sc1 = scale(c, 1), sc2 = scale(c, 2), sc3 = scale(c, 3);
    const float sc4 = scale(c, 4), sc5 = scale(c, 5);
    const float da_ = al - ao;
    const float *ro = bb + (4 - rn) * nbs;
    float *rw = bb + (3 + rn) * nbs;
    const float4 *nd = reinterpret_cast<const float4 *>(pc.node);
    const float *pl = pc.img + t.lay.off_planck + gp.sub;
    const int ns = nbs / G;
#pragma unroll 1
    for (int s0 = 0; s0 < ns; s0 += kChunk2) {
      // moment sums over the grid nodes for kChunk2 band slots of this lane,
      // in pairs with the packed FP32 FMA (two round-to-nearest FMAs per
      // instruction, the same results as one at a time): (S0, S1), (S2, S3),
      // (S4, S5), (S6, -)
      float2 S2v[kChunk2][4];
#pragma unroll
      for (int k = 0; k < kChunk2; k++)
#pragma unroll
        for (int q = 0; q < 4; q++) S2v[k][q] = make_float2(0.f, 0.f);
      const float *pls = pl + G * s0;
#pragma unroll kNodeUnroll
      for (int j = 0; j < t.nt; j++) {
        const float4 A = nd[2 * j], B = nd[2 * j + 1];
        const float2 a01 = make_float2(A.x, A.y), a23 = make_float2(A.z, A.w);
        const float2 b01 = make_float2(B.x, B.y), b23 = make_float2(B.z, B.w);
        const float *row = pls + j * t.lay.n2s;
#pragma unroll
        for (int k = 0; k < kChunk2; k++) {
          const float Bv = (s0 + k < ns) ? row[G * k] : 0.f;
          const float2 bb2 = make_float2(Bv, Bv);
          S2v[k][0] = __ffma2_rn(a01, bb2, S2v[k][0]);
          S2v[k][1] = __ffma2_rn(a23, bb2, S2v[k][1]);
          S2v[k][2] = __ffma2_rn(b01, bb2, S2v[k][2]);
          S2v[k][3] = __ffma2_rn(b23, bb2, S2v[k][3]);
        }
      }
      float S[kChunk2][7];
#pragma unroll
      for (int k = 0; k < kChunk2; k++) {
        S[k][0] = S2v[k][0].x;
        S[k][1] = S2v[k][0].y;
        S[k][2] = S2v[k][1].x;
        S[k][3] = S2v[k][1].y;
        S[k][4] = S2v[k][2].x;
        S[k][5] = S2v[k][2].y;
        S[k][6] = S2v[k][3].x;
      }
#pragma unroll kSlotUnroll
      for (int k = 0; k < kChunk2; k++) {
        const int i = gp.sub + G * (s0 + k);
        if (s0 + k < ns && i < t.n2) {
          const float wv = W(i);
          if (wv > 0.f) {
            const float Bh = S[k][0], Bs = S[k][3];
            const float Bm = eta * Bh + (1.f - eta) * Bs;
            const float tuv = TU(i);
            const float atu = al * tuv;
            const float r = Y(i) - atu * Bm;
            rw[i] = r;
            const float dM = tuv * fmaf(al, S[k][6], da_ * (Bm - S[k][6]));
            acc[NH + P + 2] = fmaf(wv * dM, 2.f * ro[i] - dM, acc[NH + P + 2]);
            float J[6];
            J[0] = atu * eta * S[k][1] * ish2 * sc0;
            J[1] = atu * eta * S[k][2] * ish3 * sc1;
            J[2] = atu * (1.f - eta) * S[k][4] * iss2 * sc2;
            J[3] = atu * (1.f - eta) * S[k][5] * iss3 * sc3;
            J[4] = atu * (Bh - Bs) * sc4;
            J[5] = tuv * Bm * sc5;
            const float wr = wv * r;
            const float wM = wv * atu * Bm;     // weight x thermal model value
            acc[NH + P] = fmaf(wr, r, acc[NH + P]);
            acc[NH + P + 1] = fmaf(r, r, acc[NH + P + 1]);
            acc[NH + P + 3] = fmaf(wM, wM, acc[NH + P + 3]);
            acc[NH + P + 4] += wv;
#pragma unroll
            for (int a = 0; a < P; a++) {
              acc[NH + a] = fmaf(J[a], wr, acc[NH + a]);
              const float wj = wv * J[a];
#pragma unroll
              for (int bb_ = a; bb_ < P; bb_++) acc[up<P>(a, bb_)] = fmaf(wj, J[bb_], acc[up<P>(a, bb_)]);
            }
          }
        }
      }
    }
    gp.sum(acc);
    cst = acc[NH + P];
    cd = acc[NH + P + 1];
    drop = acc[NH + P + 2];
    // FP32 floor of g_a (as in stage 1), from the data part of H_aa
    float gfl[P];
    const float m2 = acc[NH + P + 3] / fmaxf(acc[NH + P + 4], 1e-30f);
#pragma unroll
    for (int a = 0; a < P; a++) gfl[a] = kFloorC * sqrtf(acc[up<P>(a, a)] * m2);
#pragma unroll
    for (int i = 0; i < 6; i++) {
      float z = c.zk2[i] > 0.f ? fmaf(xt[i] - c.lo2[i], c.zk2[i], -1.f) : 0.f;
      float pp = psc * c.pp2[i];
      cst += pp * (z - c.pm2[i]) * (z - c.pm2[i]);
      acc[NH + i] -= pp * (z - c.pm2[i]);
      acc[up<P>(i, i)] += pp;
    }
    // lane sub stores entries sub, sub + G, ... of [H | g], then the floor at 30
#pragma unroll
    for (int k = 0; k < NH + P; k++)
      if ((k & (G - 1)) == gp.sub) ne[k] = acc[k];
#pragma unroll
    for (int a = 0; a < P; a++)
      if (((30 + a) & (G - 1)) == gp.sub) ne[30 + a] = gfl[a];
    gp.sync();
  }

  __device__ __forceinline__ float prior_drop(const KConfig &c, const float (&xo)[NX],
                                              const float (&xn)[NX]) const {
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) {
      if (c.hi2[i] > c.lo2[i] && c.pp2[i] > 0.f) {
        const float k = c.zk2[i];
        float zo = k * (xo[i] - c.lo2[i]) - 1.f - c.pm2[i], zn = k * (xn[i] - c.lo2[i]) - 1.f - c.pm2[i];
        d += psc * c.pp2[i] * (k * (xo[i] - xn[i])) * (zo + zn);
      }
    }
    return d;
  }

  __device__ __forceinline__ void apply(const KConfig &c, const float (&x)[NX], const float (&dr)[P],
                                        const signed char (&pd)[P], int, float (&xt)[NX]) const {
#pragma unroll
    for (int i = 0; i < 6; i++) {
      float v = x[i] + scale(c, i) * dr[i];
      if (pd[i] < 0) v = c.lo2[i];
      if (pd[i] > 0) v = c.hi2[i];
      xt[i] = fminf(fmaxf(v, c.lo2[i]), c.hi2[i]);
    }
  }
};

// -------------------------------------------- final covariance (FP64) ---
// C = s2 (H_FF)^-1 over the free stage-2 variables (not on an outward-
// pressed bound, non-zero diagonal), in physical units; writes the packed
// upper triangle and returns var(E[T]) and var(alpha). FP64 throughout,
// division-free: Jacobi scaling and the Cholesky pivots use Newton-refined
// reciprocal square roots, and C = L^-T L^-1 from the triangular inverse.
struct CovIO {
  float x[6], g[6], s2;
  double H[21];
  float cov[21];
  bool cov_ok;
  double vE, va;
};

__device__ __noinline__ void laplace_cov(const KConfig &c, CovIO &io) {
  const float (&x)[6] = io.x;
  const double (&H)[21] = io.H;
  const float (&g)[6] = io.g;
  const float s2 = io.s2;
  float (&cov)[21] = io.cov;
  bool &cov_ok = io.cov_ok;
  double &vE = io.vE;
  double &va = io.va;
  bool fix[6], zc[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    bool act = (x[k] <= c.lo2[k] && g[k] <= 0.f) || (x[k] >= c.hi2[k] && g[k] >= 0.f);
    zc[k] = !act && !(H[up<6>(k, k)] > 0.0);
    fix[k] = act || zc[k];
  }
  double A[21], rd[6], il[6];
#pragma unroll
  for (int i = 0; i < 6; i++) rd[i] = fix[i] ? 1.0 : rsq(H[up<6>(i, i)]);
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = 0; j <= i; j++)
      A[i * (i + 1) / 2 + j] = (fix[i] || fix[j]) ? (i == j ? 1.0 : 0.0)
                                                   : H[up<6>(i, j)] * rd[i] * rd[j];
  cov_ok = true;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    double s = A[j * (j + 1) / 2 + j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
    cov_ok = cov_ok && s > 0.0;
    double r = rsq(s > 0.0 ? s : 1.0);
    il[j] = r;
#pragma unroll
    for (int i = j + 1; i < 6; i++) {
      double t = A[i * (i + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
      A[i * (i + 1) / 2 + j] = t * r;
    }
  }
  // W = L^-1 (lower), by forward substitution of the unit vectors
  double W[21];
#pragma unroll
  for (int v = 0; v < 6; v++)
#pragma unroll
    for (int i = v; i < 6; i++) {
      double t = (i == v) ? 1.0 : 0.0;
#pragma unroll
      for (int k = v; k < i; k++) t -= A[i * (i + 1) / 2 + k] * W[k * (k + 1) / 2 + v];
      W[i * (i + 1) / 2 + v] = t * il[i];
    }
  double Cx[21];   // packed upper, physical units
  double sc[6];
#pragma unroll
  for (int i = 0; i < 6; i++) sc[i] = 0.5 * ((double)c.hi2[i] - c.lo2[i]) * rd[i];
  int q = 0;
#pragma unroll
  for (int a = 0; a < 6; a++)
#pragma unroll
    for (int b = a; b < 6; b++) {
      double t = 0.0;
#pragma unroll
      for (int k = b; k < 6; k++) t += W[k * (k + 1) / 2 + a] * W[k * (k + 1) / 2 + b];
      double v = (fix[a] || fix[b]) ? 0.0 : (double)s2 * t * sc[a] * sc[b];
      if (a == b && zc[a]) v = __longlong_as_double(0x7ff0000000000000ll);
      Cx[q] = v;
      cov[q] = cov_ok ? (float)v : __int_as_float(0x7fc00000);
      q++;
    }
  double gE[6] = {x[4], 0.0, 1.0 - x[4], 0.0, (double)x[0] - x[2], 0.0};
  vE = 0.0;
  bool inf = false;
#pragma unroll
  for (int a = 0; a < 6; a++) {
    if (gE[a] == 0.0) continue;
    if (zc[a]) inf = true;
#pragma unroll
    for (int b = 0; b < 6; b++)
      if (gE[b] != 0.0 && !zc[a] && !zc[b]) vE += gE[a] * Cx[up<6>(a, b)] * gE[b];
  }
  if (inf) vE = __longlong_as_double(0x7ff0000000000000ll);
  if (!cov_ok) vE = __longlong_as_double(0x7ff8000000000000ll);
  va = Cx[up<6>(5, 5)];
}

// A lower bound of the Laplace variance of alpha over every active set the
// final state admits, from the FP32 normal matrix: every variable on a bound
// held (holding more variables can only lower alpha's marginal variance),
// in z units of the Jacobi-scaled matrix A = D^-1/2 H D^-1/2. Returns false
// when the bound cannot be trusted: the scaled matrix not positive definite,
// or trace(A^-1) so large that the FP32 matrix's error (a relative 5e-5 of
// the diagonal scale, six times the measured 8.5e-6) could move A^-1 by more
// than a quarter (6 x 5e-5 x trace(A^-1) >= 0.25).
__device__ __noinline__ bool alpha_var_floor(const KConfig &c, const CovIO &io, double &va_min) {
  bool fix[6];
#pragma unroll
  for (int k = 0; k < 6; k++)
    fix[k] = io.x[k] <= c.lo2[k] || io.x[k] >= c.hi2[k] || !(io.H[up<6>(k, k)] > 0.0);
  if (fix[5]) return false;
  double A[21], rd[6];
#pragma unroll
  for (int i = 0; i < 6; i++) rd[i] = fix[i] ? 1.0 : rsq(io.H[up<6>(i, i)]);
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = 0; j <= i; j++)
      A[i * (i + 1) / 2 + j] = (fix[i] || fix[j]) ? (i == j ? 1.0 : 0.0) : io.H[up<6>(i, j)] * rd[i] * rd[j];
  double il[6];
#pragma unroll
  for (int j = 0; j < 6; j++) {
    double s = A[j * (j + 1) / 2 + j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
    if (!(s > 0.0)) return false;
    const double r = rsq(s);
    il[j] = r;
#pragma unroll
    for (int i = j + 1; i < 6; i++) {
      double t = A[i * (i + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
      A[i * (i + 1) / 2 + j] = t * r;
    }
  }
  // W = L^-1: trace(A^-1) = sum of W's squares, (A^-1)_55 = sum_k W_k5^2 = W_55^2
  double W[21], tr = 0.0;
#pragma unroll
  for (int v = 0; v < 6; v++)
#pragma unroll
    for (int i = v; i < 6; i++) {
      double t = (i == v) ? 1.0 : 0.0;
#pragma unroll
      for (int k = v; k < i; k++) t -= A[i * (i + 1) / 2 + k] * W[k * (k + 1) / 2 + v];
      W[i * (i + 1) / 2 + v] = t * il[i];
      if (!fix[i] && !fix[v]) tr += W[i * (i + 1) / 2 + v] * W[i * (i + 1) / 2 + v];
    }
  if (!(6.0 * 5e-5 * tr < 0.25)) return false;
  va_min = W[20] * W[20] * rd[5] * rd[5];   // z units squared
  return true;
}

// ------------------------------------------------------------ kernels ---
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// true in every thread of the CTA if a kernel of this fit has set the error
// word (a bounded wait gave up): the later kernels of the fit then leave at
// once. Called by all threads of the CTA at the same point.
__device__ __forceinline__ bool cta_err(const int *err) {
  return __syncthreads_or(threadIdx.x == 0 && *(volatile const int *)err != 0) != 0;
}

// Stage the first nfloats of the per-CTA table image into shared memory with 1D bulk copies
// completing on one mbarrier. The wait is bounded (spins polls): on timeout
// the error flag is set, the copies still in flight are waited for (bounded
// again, by 2^26 polls, so the CTA never leaves with a copy landing in its
// shared memory) and the CTA leaves (returns false).
// The table image (its first nfloats floats) goes to the start of the
// dynamic shared memory; an optional second region (bytes2 bytes from src2 to
// dst2, both 16-byte aligned, bytes2 a multiple of 16) rides on the same
// mbarrier.
__device__ __forceinline__ bool stage_tables(const KTables &t, float *smem, int nfloats,
                                             unsigned long long *bar, int *err, long long spins,
                                             void *dst2 = nullptr, const void *src2 = nullptr,
                                             unsigned bytes2 = 0) {
  const unsigned bytes = (unsigned)nfloats * 4u;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes + bytes2) : "memory");
    const unsigned chunk = 32768u;
    for (unsigned off = 0; off < bytes; off += chunk) {
      unsigned n = bytes - off < chunk ? bytes - off : chunk;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(smem_u32(reinterpret_cast<char *>(smem) + off)),
          "l"(reinterpret_cast<const char *>(t.image) + off), "r"(n), "r"(smem_u32(bar))
          : "memory");
    }
    for (unsigned off = 0; off < bytes2; off += chunk) {
      unsigned n = bytes2 - off < chunk ? bytes2 - off : chunk;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(smem_u32(reinterpret_cast<char *>(dst2) + off)),
          "l"(reinterpret_cast<const char *>(src2) + off), "r"(n), "r"(smem_u32(bar))
          : "memory");
    }
  }
  __syncthreads();
  // the bounded wait polls with the non-blocking test (each poll returns at
  // once, so `spins` counts polls, not the hardware's suspend intervals)
  unsigned done = 0;
  for (long long spin = 0; spin < spins && !done; spin++)
    asm volatile(
        "{ .reg .pred P; mbarrier.test_wait.parity.shared::cta.b64 P, [%1], 0; selp.u32 %0, 1, 0, P; }"
        : "=r"(done) : "r"(smem_u32(bar)) : "memory");
  if (__syncthreads_and(done)) return true;
  if (threadIdx.x == 0) atomicExch(err, 1);
  for (long long spin = 0; spin < (1ll << 26) && !done; spin++)
    asm volatile(
        "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0; selp.u32 %0, 1, 0, P; }"
        : "=r"(done) : "r"(smem_u32(bar)) : "memory");
  return false;
}

// pixel-claim helper: the group's first lane takes n pixels from a global
// counter and shares the first index with the group
template <int G>
__device__ __forceinline__ long long claim(unsigned long long *ctr, const Grp<G> &gp, int n) {
  unsigned long long base = 0;
  if (gp.sub == 0) base = atomicAdd(ctr, (unsigned long long)n);
  return gp.bcast((long long)base);
}

// stage-1 per-pixel setup: radiance, mask m(lambda) (saturation) x window,
// weights and the prior scale (mean noise variance of the used bands)
template <int K, int G>
__device__ __forceinline__ int setup1(Stage1<K, G> &s1, const PixCtx &pc, const Grp<G> &gp,
                                      const float *row) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0;
  for (int i = gp.sub; i < s1.nbs; i += G) {
    float Lv = 0.f, wv = 0.f;
    if (i < t.n1) {
      int b = t.b1lo + i;
      float L = __ldg(row + b);
      bool ok = pc.img[t.lay.off_win1 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      Lv = L;
      wv = ok ? (c.weighted ? 1.f / (c.has_nsd ? c.nsd[b] * c.nsd[b] : var) : 1.f) : 0.f;
      if (ok) { nv += var; nu++; }
    }
    s1.Lo(i) = Lv;
    s1.W(i) = wv;
#pragma unroll
    for (int k = 2; k < 4; k++) s1.bb[k * s1.nbs + i] = 0.f;
  }
  nv = gp.sum1(nv);
  nu = gp.isum(nu);
  s1.psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  s1.sf = 0.5f * (c.hi1[0] - c.lo1[0]);
  s1.sa = 0.5f * (c.hi1[K] - c.lo1[K]);
  s1.sT = 0.5f * (c.hi1[K + 1] - c.lo1[K + 1]);
  gp.sync();
  return nu;
}

// A warp-wide loop over a pixel's bands (lane l takes band i0 + l of each
// block of 32) that sums like the pixel's G-lane group would: class_add adds,
// in band order, the values of this lane's class (lane mod G) in the block,
// so that every lane holds its group lane's running sum; class_total then
// reduces the G classes with Grp<G>::sum1's butterfly. The results are the
// group loop's to the bit.
template <int G>
__device__ __forceinline__ float class_add(float acc, float v, int lane) {
#pragma unroll
  for (int q = 0; q < 32 / G; q++) acc += __shfl_sync(kFull, v, (lane & (G - 1)) + q * G);
  return acc;
}
template <int G>
__device__ __forceinline__ float class_total(float acc) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  return acc;
}

// The ungated intake of one pixel in one pass over its radiance row, by a
// whole warp (32 lanes over the row: at 8 lanes a pixel a quarter of the
// dependent loads per lane): the finiteness of every band, the stage-1
// buffers as setup1 builds them (bb, the pixel's band buffers) and the
// stage-2 band count as count2 forms it (the stage-2 bands lie inside the
// stage-1 range). fin, n1u, n2u and the prior scale are warp totals, the
// prior scale summed in the order of the pixel's G-lane group.
template <int G>
__device__ __forceinline__ void setup1_warp(const PixCtx &pc, int lane, const float *row, float *bb, int nbs,
                                            bool &fin, int &n1u, int &n2u, float &psc, int *err) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0, nu2 = 0;
  bool f = true;
#pragma unroll 1
  for (int i0 = 0; i0 < nbs; i0 += 32) {
    const int i = i0 + lane;
    float Lv = 0.f, wv = 0.f, vv = 0.f;
    if (i < t.n1 && fr_ok(t.b1lo + i < t.nb, err, 13)) {   // site 13: band inside the row
      const int b = t.b1lo + i;
      const float L = __ldg(row + b);
      f = f && isfinite(L);
      const bool unsat = !(t.sat && L >= __ldg(t.sat + b));
      const bool ok = pc.img[t.lay.off_win1 + b] > 0.f && unsat;
      const float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      Lv = L;
      wv = ok ? (c.weighted ? 1.f / (c.has_nsd ? c.nsd[b] * c.nsd[b] : var) : 1.f) : 0.f;
      if (ok) { vv = var; nu++; }
      if (b >= t.b2lo && b < t.b2lo + t.n2) nu2 += (pc.img[t.lay.off_win2 + b] > 0.f && unsat) ? 1 : 0;
    }
    nv = class_add<G>(nv, vv, lane);
    if (i < nbs) {
      bb[i] = Lv;
      bb[nbs + i] = wv;
      bb[2 * nbs + i] = 0.f;
      bb[3 * nbs + i] = 0.f;
    }
  }
#pragma unroll 1
  for (int b = lane; b < t.b1lo; b += 32) f = f && isfinite(__ldg(row + b));
#pragma unroll 1
  for (int b = t.b1lo + t.n1 + lane; b < t.nb; b += 32) f = f && isfinite(__ldg(row + b));
  fin = __all_sync(kFull, f);
  nv = class_total<G>(nv);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    nu += __shfl_xor_sync(kFull, nu, o);
    nu2 += __shfl_xor_sync(kFull, nu2, o);
  }
  n1u = nu;
  n2u = nu2;
  psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  __syncwarp();
}

// stage-2 band count (mask x window) without building the stage state
template <int G>
__device__ __forceinline__ int count2(const PixCtx &pc, const Grp<G> &gp, const float *row) {
  const KTables &t = *pc.t;
  int nu = 0;
  for (int bi = gp.sub; bi < t.n2; bi += G) {
    int b = t.b2lo + bi;
    float L = __ldg(row + b);
    nu += (pc.img[t.lay.off_win2 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b))) ? 1 : 0;
  }
  return gp.isum(nu);
}

// stage-2 per-pixel setup: y = L - Ls(x_surf) (solar term fixed, Eq. solar),
// tau_up, weights, prior scale
template <int K, int G>
__device__ __forceinline__ int setup2(Stage2<G> &s2, const PixCtx &pc, const Grp<G> &gp,
                                      const float *row, const float (&xs)[K]) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0;
  for (int i = gp.sub; i < s2.nbs; i += G) {
    float yv = 0.f, tv = 0.f, wv = 0.f;
    if (i < t.n2) {
      int b = t.b2lo + i;
      float L = __ldg(row + b);
      bool ok = pc.img[t.lay.off_win2 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      float4 q = __ldg(pc.wvrow + b);
      float rho = 0.f;
#pragma unroll
      for (int k = 0; k < K; k++) rho = fmaf(xs[k], pc.img[t.lay.off_endm + k * t.nb + b], rho);
      yv = L - (q.y + q.x * rho / (1.f - q.z * rho));
      tv = q.w;
      wv = ok ? (c.weighted ? 1.f / (c.has_nsd ? c.nsd[b] * c.nsd[b] : var) : 1.f) : 0.f;
      if (ok) { nv += var; nu++; }
    }
    s2.Y(i) = yv;
    s2.TU(i) = tv;
    s2.W(i) = wv;
    s2.R(0, i) = yv;
    s2.R(1, i) = yv;
  }
  nv = gp.sum1(nv);
  nu = gp.isum(nu);
  s2.psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  gp.sync();
  return nu;
}

// setup2 of one pixel by a whole warp (32 lanes over its bands; bb is the
// pixel's band buffers, [5][nbs] as Stage2 lays them out); returns the
// used-band count, psc the prior scale (warp totals)
template <int K, int G>
__device__ __forceinline__ int setup2_warp(const PixCtx &pc, int lane, const float4 *wvrow, const float *row,
                                           const float (&xs)[K], float *bb, int nbs, float &psc, int *err) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < nbs; i0 += 32) {
    const int i = i0 + lane;
    float yv = 0.f, tv = 0.f, wv = 0.f, vv = 0.f;
    if (i < t.n2 && fr_ok(t.b2lo + i < t.nb, err, 33)) {   // site 33: band inside the row
      const int b = t.b2lo + i;
      const float L = __ldg(row + b);
      const bool ok = pc.img[t.lay.off_win2 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      const float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      const float4 q = __ldg(wvrow + b);
      float rho = 0.f;
#pragma unroll
      for (int k = 0; k < K; k++) rho = fmaf(xs[k], pc.img[t.lay.off_endm + k * t.nb + b], rho);
      yv = L - (q.y + q.x * rho / (1.f - q.z * rho));
      tv = q.w;
      wv = ok ? (c.weighted ? 1.f / (c.has_nsd ? c.nsd[b] * c.nsd[b] : var) : 1.f) : 0.f;
      if (ok) { vv = var; nu++; }
    }
    nv = class_add<G>(nv, vv, lane);
    if (i < nbs) {
      bb[i] = yv;
      bb[nbs + i] = tv;
      bb[2 * nbs + i] = wv;
      bb[3 * nbs + i] = yv;
      bb[4 * nbs + i] = yv;
    }
  }
  nv = class_total<G>(nv);
#pragma unroll
  for (int o = 16; o; o >>= 1) nu += __shfl_xor_sync(kFull, nu, o);
  psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  __syncwarp();
  return nu;
}

// Where pixel pix reads its inputs and writes its outputs: the single scene
// (optionally through a subset index), or the scene of a batch that holds
// global pixel pix (binary search over the scenes' first pixels).
struct PixRef {
  const float *row;
  int wv;
  const float *init;
  KOut o;
  long long opix;
};

__device__ __forceinline__ PixRef resolve(const LMLaunch &p, long long pix, int K) {
  PixRef r;
  const int nb = p.t.nb;
  if (!p.s.items) {
    const long long src = p.s.idx ? p.s.idx[pix] : pix;
    r.row = p.s.rad + src * nb;
    r.wv = p.s.wv[src];
    r.init = p.s.init ? p.s.init + src * (K + 8) : nullptr;
    r.o = p.o;
    r.opix = pix;
    return r;
  }
  int lo = 0, hi = p.s.n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (p.s.prefix[mid] <= pix) lo = mid;
    else hi = mid - 1;
  }
  const SceneItem &it = p.s.items[lo];
  const long long loc = pix - p.s.prefix[lo];
  r.row = it.rad + loc * nb;
  r.wv = it.wv[loc];
  r.init = nullptr;
  r.o.state = it.out.state;
  r.o.ET = it.out.ET;
  r.o.sdT = it.out.sdT;
  r.o.alpha = it.out.alpha;
  r.o.cov = it.out.cov;
  r.o.var_ET = it.out.var_ET;
  r.o.cost = it.out.cost;
  r.o.rms = it.out.rms;
  r.o.hfdi = it.out.hfdi;
  r.o.status = it.out.status;
  r.o.iters = it.out.iters;
  r.o.resid = it.out.resid;
  r.opix = loc;
  return r;
}

constexpr int kFitted = 256;   // scratch flag: pixel goes on to stage 2
constexpr int kS2Hand = 32;    // floats handed from stage 2 to finalize per pixel

// value k of a compile-time-indexed list, chosen by a runtime k (select
// chain: no local-memory indexing)
template <int N>
__device__ __forceinline__ float pick(const float (&v)[N], int k) {
  float r = v[0];
#pragma unroll
  for (int i = 1; i < N; i++) r = (k == i) ? v[i] : r;
  return r;
}

// Each round of the two stage kernels: groups without a pixel take the next
// one (and settle at once the pixels that are not fitted); then every group
// with a pixel runs one LM step: the damped step from the current normal
// equations, the evaluation at the trial point, and its acceptance. The
// evaluation is the same code at the same point of the round for every
// group, so the groups of a warp evaluate in step. A warp leaves when all
// its groups have run out of pixels.

// ---- stage 1: checks, HFDI gate, stage-1 fit -> scratch
template <int K, int G, int MAXW, bool ADAM = false>
__global__ void __launch_bounds__(MAXW * 32, 1) lm_stage1_kernel(const __grid_constant__ LMLaunch p) {
  constexpr int P = K + 1, NX = K + 2, NH = P * (P + 1) / 2;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned long long cstat[ST_COUNT];
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  // the table head, then the whole water-vapour table, then the pixels'
  // band buffers
  const int img_f = image_floats(t, 1), wv_f = wvtab_floats(t, G);
  const float4 *wvs = wv_f ? reinterpret_cast<const float4 *>(smem + img_f) : t.wvtab;
  if (!stage_tables(t, smem, img_f, &bar, p.w.err, c.wait_spins, smem + img_f, t.wvtab,
                    (unsigned)wv_f * 4u))
    return;
  const Grp<G> gp(lane);
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  pc.node = nullptr;
  pc.wvrow = wvs;
  Stage1<K, G> S;
  S.nbs = band_slots(t.n1, G);
  S.bb = smem + img_f + wv_f + (threadIdx.x / G) * pix_stride1(t, G);
#ifdef FIRERT_DEBUG
  // site 11: this group's band buffers end inside the launch's shared memory
  if (!__syncthreads_and(fr_ok(reinterpret_cast<unsigned char *>(S.bb + 4 * S.nbs) <=
                                   reinterpret_cast<unsigned char *>(smem) + dyn_smem_bytes(), p.w.err, 11)))
    return;
#endif
  const int NSx = K + 8;
  const long long n = p.s.n_pix;
  const int nclaim = p.s.claim > 0 ? p.s.claim : kClaim;
  long long next = 0, end = 0, pix = 0, opix = 0;
  uint16_t *iters_out = nullptr;
  bool active = false, done = false, first = false;
  float x[NX], xt[NX], H[NH], g[P], gf[P], cst = 0.f, gm = 0.f;
  int m = 0, rc = 0, nfull = 0, status = 0;
  LMIter<P> L;
  AdamState<NX> A;
  S.sf = 0.5f * (c.hi1[0] - c.lo1[0]);
  S.sa = 0.5f * (c.hi1[K] - c.lo1[K]);
  S.sT = 0.5f * (c.hi1[K + 1] - c.lo1[K + 1]);
  // every pixel is fitted (no gate) and the stage-2 bands lie inside the
  // stage-1 range: one pass builds the stage-1 buffers with the finiteness
  // test, by the whole warp; gated, most pixels stop at the gate, so the
  // group's own finiteness pass comes first
  const bool fuse = !p.s.gate && t.b2lo >= t.b1lo && t.b2lo + t.n2 <= t.b1lo + t.n1;
  for (;;) {
    // ---- take pixels until one is to be fitted, for every group of the
    // warp without one
    while (__any_sync(kFull, !active && !done)) {
      bool have = false;
      PixRef ref{};
      if (!active && !done) {
        if (next >= end) {
          const long long b = claim(p.w.counter, gp, nclaim);
          if (b >= n) {
            done = true;
          } else {
            next = b;
            end = min(b + (long long)nclaim, n);
          }
        }
        if (!done) {
          pix = next++;
          if (fr_ok(pix < n, p.w.err, 12)) {   // site 12: claimed pixel
            ref = resolve(p, pix, K);
            have = true;
          } else {
            done = true;
          }
        }
      }
      const float *row = ref.row;
      bool fin = true;
      int n1u = 0, n2u = 0;
      if (fuse) {
        unsigned need = __ballot_sync(kFull, have && gp.sub == 0);
        while (need) {
          const int src = __ffs(need) - 1;
          need &= need - 1;
          const float *rs = reinterpret_cast<const float *>(
              __shfl_sync(kFull, reinterpret_cast<unsigned long long>(row), src));
          bool fs;
          int a1, a2;
          float ps;
          float *bbs = smem + img_f + wv_f + ((threadIdx.x & ~31) + src) / G * pix_stride1(t, G);
          setup1_warp<G>(pc, lane, rs, bbs, S.nbs, fs, a1, a2, ps, p.w.err);
          if ((lane ^ src) < G) {
            fin = fs;
            n1u = a1;
            n2u = a2;
            S.psc = ps;
          }
        }
      }
      if (!have) continue;
      const int wvb = ref.wv;
      const bool wv_ok = wvb < t.nwv;   // an out-of-range bin is an invalid input
      pc.wvrow = wvs + (size_t)(wv_ok ? wvb : 0) * t.nb;
      if (!fuse)
        for (int b = gp.sub; b < t.nb; b += G) fin = fin && isfinite(__ldg(row + b));
      fin = gp.all(fin) && wv_ok;
      const float Lh = __ldg(row + t.bh), Ll = __ldg(row + t.bl);
      float hf = (Lh - Ll) / (Lh + Ll);
      status = 0;
      bool fit = false;
      if (!fin) {
        status = PX_NONFINITE;
        hf = __int_as_float(0x7fc00000);
      } else if (p.s.gate && !(hf >= c.hfdi_thresh)) {
        status = PX_NOT_CANDIDATE;
      } else {
        if (!fuse) {
          n1u = setup1(S, pc, gp, row);
          n2u = count2(pc, gp, row);
        }
        if (n1u <= K + 2 || n2u <= 6) status = PX_ALL_MASKED;
        else fit = true;
      }
      const KOut &o = ref.o;
      const long long op = ref.opix;
      if (gp.sub == 0 && o.hfdi) o.hfdi[op] = hf;
      if (fit) {
        const float *ini = ref.init;
        if (ini) {
#pragma unroll
          for (int i = 0; i < NX; i++) x[i] = ini[i];
          Stage1<K, G>::simplex_project(x);
#pragma unroll
          for (int i = K; i < NX; i++) x[i] = fminf(fmaxf(x[i], c.lo1[i]), c.hi1[i]);
        } else {
#pragma unroll
          for (int k = 0; k < K; k++) x[k] = 1.f / (float)K;
          x[K] = c.init_alpha1;
          x[K + 1] = c.init_T1;
        }
#pragma unroll
        for (int i = 0; i < NX; i++) xt[i] = x[i];
        L = LMIter<P>();
#pragma unroll
        for (int a = 0; a < P; a++) L.act[a] = false;
        if constexpr (ADAM) A.reset();
        first = true;
        rc = 0;
        nfull = 0;
        opix = op;
        iters_out = o.iters;
        active = true;
      } else {
        // settled without a fit: the outputs of the pixel are final here
        const float nan = __int_as_float(0x7fc00000);
        if (o.state)
          for (int i = gp.sub; i < NSx; i += G) o.state[op * NSx + i] = nan;
        if (o.cov)
          for (int i = gp.sub; i < 21; i += G) o.cov[op * 21 + i] = nan;
        if (gp.sub == 0) {
          p.w.s1meta[pix] = status;
          if (o.ET) o.ET[op] = nan;
          if (o.sdT) o.sdT[op] = nan;
          if (o.alpha) o.alpha[op] = nan;
          if (o.var_ET) o.var_ET[op] = nan;
          if (o.cost) o.cost[op] = nan;
          if (o.rms) o.rms[op] = nan;
          if (o.status) o.status[op] = (uint8_t)status;
          if (o.iters) {
            o.iters[2 * op] = 0;
            o.iters[2 * op + 1] = 0;
          }
          atomicAdd(&cstat[ST_STATUS0 + (status & 7)], 1ull);
          atomicAdd(&cstat[ST_NPIX], 1ull);
        }
      }
    }
    if (__all_sync(kFull, done)) break;
    // ---- one LM step of this group's pixel: the step, then (with every
    // lane of the warp reconverged) the evaluation
    bool go = false;
    if (active) {
      if constexpr (ADAM) go = first || adam_next1<K, Stage1<K, G>>(c, x, g, gm, m, A, L, xt);
      else go = first || next_trial(S, gp, c, x, H, g, gf, m, cst, c.max_it1, L, xt);
    }
    __syncwarp();
    if (go) {
      float Ht[NH], gt[P], gft[P], ct, cdt, drop, gmt = 0.f;
      int mt;
      // small steps: decrease in increment form (FP32 resolution)
      const bool inc = !ADAM && !first && L.pred < kIncBelow * cst;
      S.template eval<ADAM>(pc, gp, xt, rc ^ 1, Ht, gt, gft, ct, cdt, drop, mt, x, inc, &gmt);
      nfull++;
      bool accept = first || ADAM;   // an Adam step is always taken
      if (!first && !ADAM) {
        drop += S.prior_drop(c, x, xt);
        const float rho = L.pred > 0.f ? drop / L.pred : -1.f;
        accept = rho > 0.f;
        damping_update(L, accept, rho);
        if (accept && drop / cst < c.tol_f) { L.status = PX_CONVERGED; go = false; }
      }
      if (accept) {
#pragma unroll
        for (int i = 0; i < NX; i++) x[i] = xt[i];
#pragma unroll
        for (int i = 0; i < NH; i++) H[i] = Ht[i];
#pragma unroll
        for (int a = 0; a < P; a++) {
          g[a] = gt[a];
          gf[a] = gft[a];
        }
        cst = ct;
        m = mt;
        gm = gmt;
        rc ^= 1;
      }
      first = false;
    }
    __syncwarp();
    if (active && !go) {
      // ---- stage 1 done: hand the state to stage 2
      if (L.status == PX_MAXITER) status |= PX_F_S1_MAXITER;
      if (L.used64) status |= PX_F_FP64;
      if (gp.sub < NX) p.w.s1x[pix * NX + gp.sub] = pick(x, gp.sub);
      if (gp.sub == 0) {
        p.w.s1meta[pix] = status | kFitted;
        if (iters_out) iters_out[2 * opix] = (uint16_t)L.it;
        atomicAdd(&cstat[ST_BAND1], (unsigned long long)nfull * (unsigned long long)t.n1);
        atomicAdd(&cstat[ST_IT1], (unsigned long long)L.it);
        atomicAdd(&cstat[ST_S64_1], (unsigned long long)L.n64);
        atomicAdd(&cstat[ST_NPIX], 1ull);
      }
      active = false;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(p.w.stats + i, cstat[i]);
}

// ---- stage 2: mixture fit from the stage-1 hand-over -> finalize scratch
template <int K, int G, int MAXW, bool ADAM = false>
__global__ void __launch_bounds__(MAXW * 32, 1) lm_stage2_kernel(const __grid_constant__ LMLaunch p) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned long long cstat[ST_COUNT];
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  const int img_f = image_floats(t, 2);
  if (cta_err(p.w.err)) return;   // an earlier kernel of this fit gave up
  if (!stage_tables(t, smem, img_f, &bar, p.w.err, c.wait_spins)) return;
  const Grp<G> gp(lane);
  float *mine = smem + img_f + (threadIdx.x / G) * pix_stride2(t, G);
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  pc.node = mine;
  pc.wvrow = t.wvtab;
  Stage2<G> S;
  S.nbs = band_slots(t.n2, G);
  S.bb = mine + t.nt * kScratchPerNode;
  const long long n = p.s.n_pix;
  const int nclaim = p.s.claim > 0 ? p.s.claim : kClaim;
  long long next = 0, end = 0, pix = 0;
  bool active = false, done = false, first = false;
  float x[6], xt[6], H[21], g[6], gf[6], cst = 0.f, cd = 0.f;
  float *ne = S.bb + 5 * S.nbs;   // trial H, g, gradient floor
#ifdef FIRERT_DEBUG
  // site 31: this group's node scratch, band buffers and normal-equation
  // block end inside the launch's shared memory
  if (!__syncthreads_and(fr_ok(reinterpret_cast<unsigned char *>(ne + kNE2) <=
                                   reinterpret_cast<unsigned char *>(smem) + dyn_smem_bytes(), p.w.err, 31)))
    return;
#endif
  int rc = 0, nfull = 0, status = 0, n2u = 0;
  LMIter<6> L;
  AdamState<6> A;
  // a pixel taken this round whose set-up is pending (16-lane groups: the
  // warp sets it up): radiance row, stage-1 surface weights
  bool pend = false;
  const float *prow = nullptr;
  float xsp[K];
  for (;;) {
    while (!active && !done) {
      if (next >= end) {
        const long long b = claim(p.w.counter + 1, gp, nclaim);
        if (b >= n) { done = true; break; }
        next = b;
        end = min(b + (long long)nclaim, n);
      }
      pix = next++;
      if (!fr_ok(pix < n, p.w.err, 32)) { done = true; break; }   // site 32: claimed pixel
      const int meta = p.w.s1meta[pix];
      if (!(meta & kFitted)) continue;
      status = meta & 0xff;
      const PixRef ref = resolve(p, pix, K);
      pc.wvrow = t.wvtab + (size_t)ref.wv * t.nb;
      float x1[K + 2];
#pragma unroll
      for (int i = 0; i < K + 2; i++) x1[i] = p.w.s1x[pix * (K + 2) + i];
      float xs[K];
#pragma unroll
      for (int k = 0; k < K; k++) xs[k] = x1[k];
      if constexpr (G == 32) {
        n2u = setup2<K>(S, pc, gp, ref.row, xs);
      } else {
#pragma unroll
        for (int k = 0; k < K; k++) xsp[k] = xs[k];
        prow = ref.row;
        pend = true;
      }
      // the start derived from the stage-1 result
      const float T1 = x1[K + 1];
      x[0] = fminf(fmaxf(fmaxf(T1, c.init_mu_h_floor), c.lo2[0]), c.hi2[0]);
      x[2] = fminf(fmaxf(fminf(T1, c.init_mu_s_ceil), c.lo2[2]), c.hi2[2]);
      x[1] = fminf(fmaxf(c.init_sigma, c.lo2[1]), c.hi2[1]);
      x[3] = fminf(fmaxf(c.init_sigma, c.lo2[3]), c.hi2[3]);
      x[5] = fminf(fmaxf(x1[K], c.lo2[5]), c.hi2[5]);
      const float e = x[0] > x[2] ? (T1 - x[2]) / (x[0] - x[2]) : 0.5f;
      x[4] = fminf(fmaxf(e, c.init_eta_lo), c.init_eta_hi);
      // stage 1 found no thermal signal (alpha1 on its bound, T1 says
      // nothing): the mixture shape starts at the prior's means, where its
      // fit ends while the data give alpha no signal either
      if (x1[K] <= c.lo1[K]) {
#pragma unroll
        for (int k = 0; k < 5; k++) x[k] = fmaf(0.5f * (c.hi2[k] - c.lo2[k]), c.pm2[k] + 1.f, c.lo2[k]);
      }
      // a given start replaces the derived one; the learned start only
      // seeds stage 1, so that stage 2 starts where plain LM's does
      const float *ini = ref.init;
      if (ini && !p.s.init_best) {
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = fminf(fmaxf(ini[K + 2 + i], c.lo2[i]), c.hi2[i]);
      }
#pragma unroll
      for (int i = 0; i < 6; i++) xt[i] = x[i];
      L = LMIter<6>();
#pragma unroll
      for (int a = 0; a < 6; a++) L.act[a] = false;
      if constexpr (ADAM) A.reset();
      first = true;
      rc = 0;
      nfull = 0;
      active = true;
    }
    if constexpr (G < 32) {
      // the set-ups of the pixels the warp's groups just took, one after the
      // other, each by the whole warp (32 lanes over the bands instead of 16)
      unsigned need = __ballot_sync(kFull, pend && gp.sub == 0);
      while (need) {
        const int src = __ffs(need) - 1;
        need &= need - 1;
        const float *rs = reinterpret_cast<const float *>(
            __shfl_sync(kFull, reinterpret_cast<unsigned long long>(prow), src));
        const float4 *ws = reinterpret_cast<const float4 *>(
            __shfl_sync(kFull, reinterpret_cast<unsigned long long>(pc.wvrow), src));
        float xss[K];
#pragma unroll
        for (int k = 0; k < K; k++) xss[k] = __shfl_sync(kFull, xsp[k], src);
        float *bbs = smem + img_f + ((threadIdx.x & ~31) + src) / G * pix_stride2(t, G) +
                     t.nt * kScratchPerNode;
        float pss;
        const int nu = setup2_warp<K, G>(pc, lane, ws, rs, xss, bbs, S.nbs, pss, p.w.err);
        if ((lane ^ src) < G) {
          n2u = nu;
          S.psc = pss;
        }
      }
      pend = false;
    }
    if (__all_sync(kFull, done)) break;
    bool go = active;
    if (active && !first) {
      if constexpr (ADAM) go = adam_next2(c, x, g, A, L, xt);
      else go = next_trial(S, gp, c, x, H, g, gf, 0, cst, c.max_it2, L, xt);
    }
    __syncwarp();
    if (go) {
      float ct, cdt, drop;
      S.eval(pc, gp, x, xt, rc ^ 1, ne, ct, cdt, drop);
      nfull++;
      bool accept = first || ADAM;   // an Adam step is always taken
      if (!first && !ADAM) {
        drop += S.prior_drop(c, x, xt);
        const float rho = L.pred > 0.f ? drop / L.pred : -1.f;
        accept = rho > 0.f;
        damping_update(L, accept, rho);
        if (accept && drop / cst < c.tol_f) { L.status = PX_CONVERGED; go = false; }
      }
      if (accept) {
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = xt[i];
#pragma unroll
        for (int i = 0; i < 21; i++) H[i] = ne[i];
#pragma unroll
        for (int a = 0; a < 6; a++) {
          g[a] = ne[21 + a];
          gf[a] = ne[30 + a];
        }
        cst = ct;
        cd = cdt;
        rc ^= 1;
      }
      first = false;
    }
    __syncwarp();
    if (active && !go) {
      // ---- hand the final state and normal equations to the finalize kernel
      if (L.used64) status |= PX_F_FP64;
      status |= L.status;
      float* hand = p.w.s2x + pix * kS2Hand;
#pragma unroll
      for (int k = 0; k < 32; k++) {
        if ((k & (G - 1)) != gp.sub) continue;
        float v;
        if (k < 6) v = x[k];
        else if (k < 27) v = H[k - 6];
        else if (k == 27) v = cst;
        else if (k == 28) v = cd;
        else if (k == 29) v = __int_as_float(n2u);
        else if (k == 30) v = __int_as_float(status | (L.it << 8));
        else v = S.psc;
        hand[k] = v;
      }
      if (gp.sub < 6) p.w.s2g[pix * 6 + gp.sub] = pick(g, gp.sub);
      if (gp.sub == 0) {
        atomicAdd(&cstat[ST_IT2], (unsigned long long)L.it);
        atomicAdd(&cstat[ST_S64_2], (unsigned long long)L.n64);
        atomicAdd(&cstat[ST_BAND2], (unsigned long long)nfull * (unsigned long long)t.n2);
        atomicAdd(&cstat[ST_NODEBAND2],
                  (unsigned long long)nfull * (unsigned long long)t.nt * (unsigned long long)t.n2);
      }
      active = false;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(p.w.stats + i, cstat[i]);
}

// ------------------------------------------ stage 2 on the tensor cores ---
// The grid-node sums of the stage-2 evaluation, S_k(b) = sum_j c_kj
// B(lambda_b, T_j) for the seven node coefficients of a pixel (the weights
// of each component times 1, d - dbar and d^2 - m2, and the mixture-weight
// increment), are one dense product per CTA and round once the pixels of
// the CTA evaluate together:
//   D[band b][8 s + k'] = sum_j Bgrid[b][j] C[8 s + k'][j], k' = k (even s) or k ^ 4 (odd s),
// M = 128 bands per tile (two tiles cover up to 256 bands), N = 8 pixel
// slots of a cohort x 8 coefficients, K = 64 nodes. Both operands are split into three
// bf16 parts (x = x0 + x1 + x2, each part the bf16 rounding of what the
// previous ones leave, 27 significant bits together) and the six products
// of parts whose orders add up to at most 2 are accumulated in FP32 in
// tensor memory, smallest first: the dropped products are below 2^-26 of
// the sum, under FP32 rounding. The Planck operand is built once per
// context; the coefficient operand is written each round by the pixels'
// groups.
//
// A round: (1) every group with a trial point forms its node coefficients
// (two node passes, as in the FP32 evaluation) and writes their parts as its
// 8 rows of the coefficient operand; (2) one thread issues the MMAs and
// commits them to an mbarrier; (3) with the sums in tensor memory, warp w
// reads lane quarter w & 3 (32 bands of each tile) and forms, for the 8
// pixel slots of its cohort, each band's residual, Jacobian row and
// contributions to J^T J, J^T r, the cost and the increment-form decrease;
// a reduce-scatter across the warp leaves one of the 32 sums per lane,
// written as the quarter's partial; (4) each group adds its four quarters'
// partials.
//
// This path fits the unweighted loss (every used band weight 1): a pixel's
// slot holds only y (radiance minus the fixed solar term) and tau_up, both
// 0 on a band the window or saturation masks, so a masked band adds exact
// zeros and no weight buffer is needed; the weighted loss runs the FP32
// stage 2. With the two band buffers and no table image in shared memory,
// three cohorts fit one SM.
namespace tcs2 {
constexpr int G = 16, kWarps = 12, kSlots = kWarps * 32 / G;   // 24 pixels per CTA
// three cohorts of 4 warps (one per TMEM lane quarter) and 8 pixel slots
// each, with their own product, mbarrier and named barrier: a cohort waits
// only for its own 8 pixels, and the cohorts' CUDA-core work overlaps the
// others' products and step logic
constexpr int kCohorts = 3, kCoSlots = kSlots / kCohorts, kCoThreads = kWarps * 32 / kCohorts;
constexpr int kN = kSlots * 8;            // coefficient rows
constexpr int kNc = kCoSlots * 8;         // D columns of one cohort and band tile
constexpr int kCoPart = kN * 128;         // bytes of one part of the coefficient operand
constexpr int kPrm = 16;                  // per-slot parameters of the band phase
constexpr int kPartStride = 4 * 32 + 16;  // per-slot partial sums [4 quarters][32], padded
constexpr long long kSpinMMA = 1ll << 24;

// per-slot block: band buffers [2][nbs] (y, tau_up), two ne slots (the
// normal equations of the accepted state and of the trial, swapped on
// acceptance, so that they need no registers), the parameters; stride
// congruent to 16 modulo 32 floats so the two groups of a warp hit
// different banks
__host__ __device__ __forceinline__ int slot_floats(const KTables &t) {
  const int f = 2 * band_slots(t.n2, G) + 2 * kNE2 + kPrm;
  return f + ((16 - f % 32) % 32 + 32) % 32;
}
struct Lay {
  int pl_bytes, co_bytes;  // operands (offsets from the 1024-aligned base)
  int slots_off, parts_off, total;   // bytes from the aligned base; total dynamic bytes
};
__host__ __device__ __forceinline__ Lay layout(const KTables &t) {
  Lay L;
  L.pl_bytes = 3 * t.plrows * 128;
  L.co_bytes = 3 * kCoPart;
  L.slots_off = L.pl_bytes + L.co_bytes;
  L.parts_off = L.slots_off + kSlots * slot_floats(t) * 4;
  L.total = 1024 + L.parts_off + kSlots * kPartStride * 4;
  return L;
}

// slot set-up of a pixel: y = L - Ls(x_surf) (solar term fixed, Eq. solar)
// and tau_up on the used bands, 0 and 0 on the masked ones; the prior scale
// (mean noise variance of the used bands). The table image is read from
// global memory (once per pixel). Returns the used-band count.
template <int K>
__device__ __forceinline__ int setup_slot(const KTables &t, const KConfig &c, const Grp<G> &gp,
                                          const float4 *wvrow, const float *row, const float (&xs)[K],
                                          float *sb, int nbs, float &psc) {
  float nv = 0.f;
  int nu = 0;
#pragma unroll 1
  for (int i = gp.sub; i < nbs; i += G) {
    float yv = 0.f, tv = 0.f;
    if (i < t.n2) {
      const int b = t.b2lo + i;
      const float L = __ldg(row + b);
      const bool ok = __ldg(t.image + t.lay.off_win2 + b) > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      if (ok) {
        const float4 q = __ldg(wvrow + b);
        float rho = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) rho = fmaf(xs[k], __ldg(t.image + t.lay.off_endm + k * t.nb + b), rho);
        yv = L - (q.y + q.x * rho / (1.f - q.z * rho));
        tv = q.w;
        nv += c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
        nu++;
      }
    }
    sb[i] = yv;
    sb[nbs + i] = tv;
  }
  nv = gp.sum1(nv);
  nu = gp.isum(nu);
  psc = nv / (float)max(nu, 1);
  gp.sync();
  return nu;
}

// setup_slot of one pixel by a whole warp: 32 lanes over the bands, so half
// the dependent loads per lane, and the noise sum reduced over the warp
template <int K>
__device__ __forceinline__ int setup_slot_warp(const KTables &t, const KConfig &c, int lane,
                                               const float4 *wvrow, const float *row, const float (&xs)[K],
                                               float *sb, int nbs, float &psc, int *err) {
  float nv = 0.f;
  int nu = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < nbs; i0 += 32) {
    const int i = i0 + lane;
    float yv = 0.f, tv = 0.f, vv = 0.f;
    if (i < t.n2 && fr_ok(t.b2lo + i < t.nb, err, 23)) {   // site 23: band inside the row
      const int b = t.b2lo + i;
      const float L = __ldg(row + b);
      const bool ok = __ldg(t.image + t.lay.off_win2 + b) > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      if (ok) {
        const float4 q = __ldg(wvrow + b);
        float rho = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) rho = fmaf(xs[k], __ldg(t.image + t.lay.off_endm + k * t.nb + b), rho);
        yv = L - (q.y + q.x * rho / (1.f - q.z * rho));
        tv = q.w;
        vv = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
        nu++;
      }
    }
    nv = class_add<G>(nv, vv, lane);
    if (i < nbs) {
      sb[i] = yv;
      sb[nbs + i] = tv;
    }
  }
  nv = class_total<G>(nv);
#pragma unroll
  for (int o = 16; o; o >>= 1) nu += __shfl_xor_sync(kFull, nu, o);
  psc = nv / (float)max(nu, 1);
  __syncwarp();
  return nu;
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &p0, __nv_bfloat16 &p1,
                                       __nv_bfloat16 &p2) {
  p0 = __float2bfloat16_rn(v);
  float r = v - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r);
  r -= __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// (1) node coefficients of the slot's pixel at xt, with the mixture-weight
// increment from x, as rows 8 slot + k (k < 7) of the coefficient operand;
// lane sub holds nodes 2 sub, 2 sub + 1, 2 sub + 32, 2 sub + 33; then the
// band-phase parameters of the slot
__device__ __forceinline__ void coef(const KTables &t, const KConfig &c, const Grp<G> &gp,
                                     const float (&x)[6], const float (&xt)[6], unsigned char *co,
                                     int slot, float *prm) {
  const float mh = xt[0], sh = xt[1], ms = xt[2], ss = xt[3], eta = xt[4], al = xt[5];
  const float eo = x[4];
  const float ih = 1.f / x[1], iht = 1.f / sh, is = 1.f / x[3], ist = 1.f / ss;
  const float dmh = mh - x[0], dsh = sh - x[1], dms = ms - x[2], dss = ss - x[3];
  float uh[4], duh[4], us[4], dus[4];
  float mom[10];
#pragma unroll
  for (int k = 0; k < 10; k++) mom[k] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int j = 2 * gp.sub + (q & 1) + 32 * (q >> 1);
    uh[q] = duh[q] = us[q] = dus[q] = 0.f;
    if (j < t.nt) {
      const float T = t.tglo + (float)j * t.tgstep;
      Stage2<G>::node_step(T, x[0], ih, mh, iht, dmh, dsh, uh[q], duh[q]);
      Stage2<G>::node_step(T, x[2], is, ms, ist, dms, dss, us[q], dus[q]);
      const float uth = uh[q] + duh[q], uts = us[q] + dus[q], dh = T - mh, ds = T - ms;
      mom[0] += uth;
      mom[1] += uth * dh;
      mom[2] += uth * dh * dh;
      mom[3] += uts;
      mom[4] += uts * ds;
      mom[5] += uts * ds * ds;
      mom[6] += uh[q];
      mom[7] += duh[q];
      mom[8] += us[q];
      mom[9] += dus[q];
    }
  }
  gp.sum(mom);
  const float rUh = 1.f / mom[0], rUs = 1.f / mom[3];
  const float dbh = mom[1] * rUh, m2h = mom[2] * rUh, dbs = mom[4] * rUs, m2s = mom[5] * rUs;
  const float rUho = 1.f / mom[6], rUso = 1.f / mom[8];
  const float kh = mom[7] * rUho, ks = mom[9] * rUso;
  const unsigned cob = tc::su32(co);
#pragma unroll
  for (int pr = 0; pr < 2; pr++) {
    const int j0 = 2 * gp.sub + 32 * pr;
    if (j0 >= t.nt) continue;
    float cf[2][7];
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const int q = 2 * pr + e, j = j0 + e;
      const float T = t.tglo + (float)j * t.tgstep;
      const float dh = T - mh, ds = T - ms;
      const float wh = (uh[q] + duh[q]) * rUh, ws = (us[q] + dus[q]) * rUs;
      const float dwh = (duh[q] - uh[q] * kh) * rUh, dws = (dus[q] - us[q] * ks) * rUs;
      const bool in = j < t.nt;
      cf[e][0] = in ? wh : 0.f;
      cf[e][1] = in ? wh * (dh - dbh) : 0.f;
      cf[e][2] = in ? wh * (dh * dh - m2h) : 0.f;
      cf[e][3] = in ? ws : 0.f;
      cf[e][4] = in ? ws * (ds - dbs) : 0.f;
      cf[e][5] = in ? ws * (ds * ds - m2s) : 0.f;
      cf[e][6] = in ? eta * dwh + (1.f - eta) * dws + (eta - eo) * (uh[q] * rUho - us[q] * rUso) : 0.f;
    }
    const unsigned cc = (unsigned)(j0 & 7) * 2u;
    // coefficient k of an odd slot goes to row k ^ 4 of the slot's eight, so
    // that the two groups of a warp store to disjoint swizzled chunks
    const int kx = (slot & 1) << 2;
#pragma unroll
    for (int k = 0; k < 7; k++) {
      // the three parts of the node pair (j0, j0 + 1), two lanes per
      // conversion (node j0 in the low half, at the lower address)
      const float2 v = make_float2(cf[0][k], cf[1][k]);
      const __nv_bfloat162 h0 = __float22bfloat162_rn(v);
      const float2 f0 = __bfloat1622float2(h0);
      const float2 r1 = make_float2(v.x - f0.x, v.y - f0.y);
      const __nv_bfloat162 h1 = __float22bfloat162_rn(r1);
      const float2 f1 = __bfloat1622float2(h1);
      const __nv_bfloat162 h2 = __float22bfloat162_rn(make_float2(r1.x - f1.x, r1.y - f1.y));
      const unsigned off = cob + tc::swz(8 * slot + (k ^ kx), j0 >> 3) + cc;
      asm volatile("st.shared.b32 [%0], %1;" ::"r"(off), "r"(*reinterpret_cast<const uint32_t *>(&h0)) : "memory");
      asm volatile("st.shared.b32 [%0], %1;" ::"r"(off + kCoPart), "r"(*reinterpret_cast<const uint32_t *>(&h1)) : "memory");
      asm volatile("st.shared.b32 [%0], %1;" ::"r"(off + 2 * kCoPart), "r"(*reinterpret_cast<const uint32_t *>(&h2)) : "memory");
    }
  }
  // band-phase parameters: [1] eta, [2] alpha, [3] alpha - alpha_o, [4..7]
  // the Jacobian factors of mu_h, s_h, mu_s, s_s, [8] [9] z scales of eta and
  // alpha; [0] (the flag) is set by the caller
  // (the group's first lane writes them: less code than a per-lane choice)
  if (gp.sub == 0) {
    const float sc0 = 0.5f * (c.hi2[0] - c.lo2[0]), sc1 = 0.5f * (c.hi2[1] - c.lo2[1]);
    const float sc2 = 0.5f * (c.hi2[2] - c.lo2[2]), sc3 = 0.5f * (c.hi2[3] - c.lo2[3]);
    const float ish2 = 1.f / (sh * sh), iss2 = 1.f / (ss * ss);
    prm[1] = eta;
    prm[2] = al;
    prm[3] = al - x[5];
    prm[4] = eta * ish2 * sc0;
    prm[5] = eta * (ish2 / sh) * sc1;
    prm[6] = (1.f - eta) * iss2 * sc2;
    prm[7] = (1.f - eta) * (iss2 / ss) * sc3;
    prm[8] = 0.5f * (c.hi2[4] - c.lo2[4]);
    prm[9] = 0.5f * (c.hi2[5] - c.lo2[5]);
  }
}

// (2) the six part products of one cohort (its 64 coefficient rows),
// smallest first, for each band tile; D of tile m at column 64 m
__device__ __forceinline__ void mma(uint32_t tmem, unsigned pl, unsigned co, int plrows, int ntile,
                                    unsigned bar) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  constexpr uint32_t idesc = tc::idesc_bf16(128, kNc);
  constexpr int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
  // the descriptors of the 24 products of a tile are the base descriptors
  // plus fixed offsets (the start-address field counts 16-byte units and
  // shared addresses stay below its 256 KB range), so each costs one add
  const uint64_t b0 = tc::sdesc(co);
  const uint64_t apart = (uint64_t)(((unsigned)plrows * 128u) >> 4);
  for (int m = 0; m < ntile; m++) {
    const uint64_t am = tc::sdesc(pl + (unsigned)(m * 16384));
#pragma unroll
    for (int pr = 0; pr < 6; pr++)
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const uint64_t ad = am + (uint64_t)pa[pr] * apart + (uint64_t)(kk * 2);
        const uint64_t bd = b0 + (uint64_t)((pb[pr] * kCoPart + kk * 32) >> 4);
        const uint32_t acc = (pr > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
            ::"r"(tmem + (uint32_t)(kNc * m)), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// reduce-scatter of 32 values over the warp: lane l returns the warp total
// of value l
__device__ __forceinline__ float reduce_scatter(float (&v)[32], int l) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool hi = (l & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      const float send = hi ? v[i] : v[i + o];
      const float keep = hi ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// (3) band phase: warp w, lane quarter q = w & 3, slots 8 h .. 8 h + 7 of its
// cohort h = w >> 2
__device__ __forceinline__ void band(const KTables &t, uint32_t tmem, float *slots, int sstride,
                                     float *parts, int nbs) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, q = w & 3, h = w >> 2;
  const int ntile = (t.n2 + 127) >> 7;
  constexpr int NH = 21, P = 6;
#pragma unroll 1
  for (int s = 8 * h; s < 8 * h + 8; s++) {
    float *sb = slots + s * sstride;
    const float *prm = sb + 2 * nbs + 2 * kNE2;
    if (prm[0] == 0.f) continue;
    float v[2][8];
    // the cohort's columns start at h * 64 * ntile; tile m at + 64 m
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * kNc * ntile + 8 * (s - 8 * h));
    tmem_ld8(ta, v[0]);
    if (ntile > 1) tmem_ld8(ta + (uint32_t)kNc, v[1]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (s & 1) {   // odd slots hold coefficient k in column k ^ 4
#pragma unroll
      for (int m = 0; m < 2; m++)
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const float u = v[m][i];
          v[m][i] = v[m][i + 4];
          v[m][i + 4] = u;
        }
    }
    const float eta = prm[1], al = prm[2], da = prm[3];
    const float f0 = prm[4], f1 = prm[5], f2 = prm[6], f3 = prm[7], sc4 = prm[8], sc5 = prm[9];
    const float *Y = sb, *TU = sb + nbs;
    // [0, 21) J^T J, [21, 27) J^T r, 27 cost, 28 decrease, 29 sum of squared
    // thermal model values; 30, 31 unused
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; i++) acc[i] = 0.f;
#pragma unroll
    for (int m = 0; m < 2; m++) {
      const int b = 128 * m + 32 * q + l;
      if (m < ntile && b < t.n2) {
        const float tuv = TU[b];
        if (tuv > 0.f) {
          const float *S = v[m];
          const float Bh = S[0], Bs = S[3];
          const float Bm = eta * Bh + (1.f - eta) * Bs;
          const float atu = al * tuv;
          const float M = atu * Bm;
          const float r = Y[b] - M;
          // decrease from the current state in increment form:
          // dM (2 r + dM) = r_o^2 - r^2 with r_o = r + dM
          const float dM = tuv * fmaf(al, S[6], da * (Bm - S[6]));
          acc[NH + P + 1] = fmaf(dM, fmaf(2.f, r, dM), acc[NH + P + 1]);
          float J[6];
          J[0] = atu * S[1] * f0;
          J[1] = atu * S[2] * f1;
          J[2] = atu * S[4] * f2;
          J[3] = atu * S[5] * f3;
          J[4] = atu * (Bh - Bs) * sc4;
          J[5] = tuv * Bm * sc5;
          acc[NH + P] = fmaf(r, r, acc[NH + P]);
          acc[NH + P + 2] = fmaf(M, M, acc[NH + P + 2]);
#pragma unroll
          for (int a = 0; a < P; a++) {
            acc[NH + a] = fmaf(J[a], r, acc[NH + a]);
#pragma unroll
            for (int b2 = a; b2 < P; b2++) acc[up<P>(a, b2)] = fmaf(J[a], J[b2], acc[up<P>(a, b2)]);
          }
        }
      }
    }
    parts[s * kPartStride + q * 32 + l] = reduce_scatter(acc, l);
  }
}

// (4) the slot's totals: H, g and the floor to ne (as the FP32 evaluation),
// cost, data cost and decrease to the caller; nu is the used-band count
// (the sum of the unit weights). Lane sub adds the four quarters' partials
// of sums sub and sub + 16 and writes the ne entries they make, with the
// prior; the scalars come from their lanes by shuffle.
__device__ __forceinline__ void post(const KConfig &c, const Grp<G> &gp, const float *ps,
                                     const float (&xt)[6], float psc, int nu, float *ne, float &cst,
                                     float &cd, float &drop) {
  constexpr int NH = 21, P = 6;
  float a = 0.f, b = 0.f;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    a += ps[q * 32 + gp.sub];
    b += ps[q * 32 + gp.sub + 16];
  }
  const int base = gp.lane & ~(G - 1);
  const float cdat = __shfl_sync(gp.mask, b, base + NH + P - 16);   // sum 27: data cost
  drop = __shfl_sync(gp.mask, b, base + NH + P + 1 - 16);           // sum 28: decrease
  const float m2 = __shfl_sync(gp.mask, b, base + NH + P + 2 - 16) / fmaxf((float)nu, 1.f);
  // the prior of Eq. (affine)'s z: curvature psc pp, gradient -psc pp (z - pm)
  cst = cdat;
#pragma unroll
  for (int i = 0; i < P; i++) {
    const float z = c.zk2[i] > 0.f ? fmaf(xt[i] - c.lo2[i], c.zk2[i], -1.f) : 0.f;
    const float pp = psc * c.pp2[i];
    cst += pp * (z - c.pm2[i]) * (z - c.pm2[i]);
  }
  cd = cdat;
  // sum sub: an entry of H (diagonals 0, 6, 11, 15 of variables 0-3)
  const int s = gp.sub;
  const int d1 = s == 0 ? 0 : s == 6 ? 1 : s == 11 ? 2 : s == 15 ? 3 : -1;
  float va = a;
  if (d1 >= 0) {
    ne[30 + d1] = kFloorC * sqrtf(a * m2);
    va += psc * c.pp2[d1];
  }
  ne[s] = va;
  // sum sub + 16: an entry of H (diagonals 18, 20 of variables 4, 5), of g,
  // or a scalar
  const int k2 = s + 16;
  if (k2 < NH) {
    const int d2 = k2 == 18 ? 4 : k2 == 20 ? 5 : -1;
    float vb = b;
    if (d2 >= 0) {
      ne[30 + d2] = kFloorC * sqrtf(b * m2);
      vb += psc * c.pp2[d2];
    }
    ne[k2] = vb;
  } else if (k2 < NH + P) {
    const int i = k2 - NH;
    const float z = c.zk2[i] > 0.f ? fmaf(pick(xt, i) - c.lo2[i], c.zk2[i], -1.f) : 0.f;
    const float pp = psc * c.pp2[i];
    ne[k2] = b - pp * (z - c.pm2[i]);
  }
  gp.sync();
}

// CTA set-up: Planck operand staged, coefficient operand zeroed, the MMA
// mbarriers initialised, tensor memory allocated (64 columns per cohort and
// band tile). Returns false (nothing allocated) if the staging timed out.
struct Cta {
  unsigned char *base;      // 1024-aligned: Planck operand, coefficient operand, slots, parts
  float *slots, *parts;
  int sstride, nbs, ntile, cols;
  uint32_t tmem;
};

// named barrier of a cohort's 128 threads (barrier 0 is the CTA's)
__device__ __forceinline__ void co_sync(int h) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(kCoThreads) : "memory");
}
__device__ __forceinline__ bool co_and(int h, bool p) {
  int r;
  asm volatile(
      "{ .reg .pred pi, po; setp.ne.s32 pi, %1, 0; bar.red.and.pred po, %2, %3, pi; selp.s32 %0, 1, 0, po; }"
      : "=r"(r) : "r"((int)p), "r"(1 + h), "r"(kCoThreads) : "memory");
  return r != 0;
}

__device__ __forceinline__ bool setup(const LMLaunch &p, float *smem, unsigned long long *bar,
                                      unsigned long long *mbar, uint32_t *tslot, Cta &C) {
  // mbar: one per cohort
  const KTables &t = p.t;
  const Lay L = layout(t);
  const unsigned a = tc::su32(smem);
  C.base = reinterpret_cast<unsigned char *>(smem) + ((1024u - (a & 1023u)) & 1023u);
  C.slots = reinterpret_cast<float *>(C.base + L.slots_off);
  C.parts = reinterpret_cast<float *>(C.base + L.parts_off);
  C.sstride = slot_floats(t);
  C.nbs = band_slots(t.n2, G);
  C.ntile = (t.n2 + 127) >> 7;
  // tensor memory: 64 columns per cohort and band tile, allocated as a power of 2
  C.cols = 32;
  while (C.cols < kCohorts * kNc * C.ntile) C.cols <<= 1;
#ifdef FIRERT_DEBUG
  // site 21: the partial sums end inside the launch's shared memory; 22:
  // the cohorts' accumulators fit the 512 TMEM columns
  const bool in = fr_ok(reinterpret_cast<unsigned char *>(C.parts + kSlots * kPartStride) <=
                            reinterpret_cast<unsigned char *>(smem) + dyn_smem_bytes(), p.w.err, 21) &&
                  fr_ok(C.cols <= 512, p.w.err, 22);
  if (!__syncthreads_and(in)) return false;
#endif
  if (cta_err(p.w.err)) return false;
  // only the Planck operand is staged: the slot set-up reads the table image
  // from global memory
  if (!stage_tables(t, smem, 0, bar, p.w.err, p.c.wait_spins, C.base, t.plop, (unsigned)L.pl_bytes))
    return false;
  uint4 *co = reinterpret_cast<uint4 *>(C.base + L.pl_bytes);
  for (int i = threadIdx.x; i < L.co_bytes / 16; i += blockDim.x) co[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < kSlots; i += blockDim.x)
    C.slots[i * C.sstride + 2 * C.nbs + 2 * kNE2] = 0.f;
  if (threadIdx.x == 0) {
    for (int h = 0; h < kCohorts; h++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(mbar + h)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(tc::su32(tslot)), "r"(C.cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  C.tmem = *tslot;
  return true;
}

// one evaluation round of cohort h after its groups wrote their
// coefficients (flag prm[0] set by every group); mbar is the cohort's;
// false if the MMA wait timed out
__device__ __forceinline__ bool round(const KTables &t, Cta &C, int h, unsigned long long *mbar,
                                      unsigned &phase, long long spins) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  co_sync(h);
  if (threadIdx.x == kCoThreads * h)
    mma(C.tmem + (uint32_t)(h * kNc * C.ntile), tc::su32(C.base),
        tc::su32(C.base + 3 * t.plrows * 128 + h * kNc * 128), t.plrows, C.ntile, tc::su32(mbar));
  // each warp reads the product once its own wait has seen the commit (the
  // warp's lanes agree first, the band phase shuffles across all of them);
  // the cohort agrees on a timed-out wait at the one barrier after the band
  // phase (a warp whose wait gave up skips the phase, and the round is
  // dropped)
  const bool w = __all_sync(kFull, tc::mbar_wait(tc::su32(mbar), phase, spins));
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (w) band(t, C.tmem, C.slots, C.sstride, C.parts, C.nbs);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  return co_and(h, w);
}

// release (both cohorts): on a timed-out round, a bounded wait for the
// cohort's outstanding commit (mbar is the cohort's); then tensor memory is
// freed
__device__ __forceinline__ void release(const Cta &C, unsigned long long *mbar, unsigned phase,
                                        bool ok, int *err) {
  if (!ok) {
    if (threadIdx.x % kCoThreads == 0) atomicExch(err, 1);   // the cohort that gave up
    tc::mbar_wait(tc::su32(mbar), phase ^ 1u, kSpinMMA);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(C.tmem), "r"(C.cols));
}

// Planck operand: part p, row b (stage-2 band), node j at
// p * plrows * 128 + swz(b, j / 8) + 2 (j % 8); zero outside n2 x nt
__global__ void planck_operand_kernel(const KTables t, const float *image, unsigned char *out) {
  const int nchunk = t.plrows * 8;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nchunk; e += gridDim.x * blockDim.x) {
    const int b = e >> 3, c = e & 7;
    uint32_t w[3][4];
#pragma unroll
    for (int h = 0; h < 4; h++) {
      __nv_bfloat16 p[2][3];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int j = 8 * c + 2 * h + u;
        const float v = (b < t.n2 && j < t.nt) ? image[t.lay.off_planck + j * t.lay.n2s + b] : 0.f;
        split3(v, p[u][0], p[u][1], p[u][2]);
      }
#pragma unroll
      for (int q = 0; q < 3; q++) w[q][h] = pack2(p[0][q], p[1][q]);
    }
#pragma unroll
    for (int q = 0; q < 3; q++)
      *reinterpret_cast<uint4 *>(out + (size_t)q * t.plrows * 128 + tc::swz(b, c)) =
          make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
}
}  // namespace tcs2

// ---- stage 2 with the grid-node sums on the tensor cores: the fit of
// lm_stage2_kernel (16 lanes per pixel, 12 warps), with the evaluation a
// round of each 4-warp cohort (tcs2) so that a cohort's 8 pixels share one
// product; unweighted loss only
template <int K, bool ADAM = false>
__global__ void __launch_bounds__(tcs2::kWarps * 32, 1) lm_stage2_tc_kernel(const __grid_constant__ LMLaunch p) {
  constexpr int G = tcs2::G;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar, mbar[tcs2::kCohorts];
  __shared__ unsigned long long cstat[ST_COUNT];
  __shared__ uint32_t tslot;
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  tcs2::Cta C;
  if (!tcs2::setup(p, smem, &bar, mbar, &tslot, C)) return;
  const int hc = threadIdx.x / tcs2::kCoThreads;   // cohort
  const Grp<G> gp(lane);
  const int slot = threadIdx.x / G;
  float *mine = C.slots + slot * C.sstride;
  unsigned char *co = C.base + 3 * t.plrows * 128;
  Stage2<G> S;
  S.nbs = C.nbs;
  S.bb = mine;
  // two ne slots: cb holds H, g and the gradient floor of the accepted
  // state, cb ^ 1 receives the trial's
  float *ne2 = mine + 2 * S.nbs;
  float *prm = ne2 + 2 * kNE2;
  const long long n = p.s.n_pix;
  const int nclaim = p.s.claim > 0 ? p.s.claim : kClaim;
  long long next = 0, end = 0, pix = 0;
  bool active = false, done = false, first = false, ok = true;
  float x[6], xt[6], cst = 0.f, cd = 0.f;
  int nfull = 0, status = 0, n2u = 0, cb = 0;
  unsigned phase = 0;
  LMIter<6> L;
  AdamState<6> A;
  // claim ahead: while a pixel is fitted, the group's first lane takes the
  // group's next claim (its result is first read a round later), and the
  // round after that the claimed pixels' inputs are prefetched into L2, so
  // that the next set-up waits on neither the atomic nor HBM
  unsigned long long pfb = 0;   // first lane: base index of the claim held in reserve
  int pfs = 0;                  // 0: none held, 1: claimed, 2: prefetched
  unsigned long long nround = 0;
  // a pixel taken this round whose slot set-up is pending: radiance row,
  // WV bin, stage-1 surface weights
  bool pend = false;
  const float *prow = nullptr;
  int pwv = 0;
  float xsp[K];
  for (;;) {
    while (!active && !done) {
      if (next >= end) {
        long long b;
        if (pfs) {
          b = gp.bcast((long long)pfb);
          pfs = 0;
        } else {
          b = claim(p.w.counter + 1, gp, nclaim);
        }
        if (b >= n) { done = true; break; }
        next = b;
        end = min(b + (long long)nclaim, n);
      }
      pix = next++;
      if (!fr_ok(pix < n, p.w.err, 24)) { done = true; break; }   // site 24: claimed pixel
      const int meta = p.w.s1meta[pix];
      if (!(meta & kFitted)) continue;
      status = meta & 0xff;
      const PixRef ref = resolve(p, pix, K);
      float x1[K + 2];
#pragma unroll
      for (int i = 0; i < K + 2; i++) x1[i] = p.w.s1x[pix * (K + 2) + i];
#pragma unroll
      for (int k = 0; k < K; k++) xsp[k] = x1[k];
      prow = ref.row;
      pwv = ref.wv;
      pend = true;
      const float T1 = x1[K + 1];
      x[0] = fminf(fmaxf(fmaxf(T1, c.init_mu_h_floor), c.lo2[0]), c.hi2[0]);
      x[2] = fminf(fmaxf(fminf(T1, c.init_mu_s_ceil), c.lo2[2]), c.hi2[2]);
      x[1] = fminf(fmaxf(c.init_sigma, c.lo2[1]), c.hi2[1]);
      x[3] = fminf(fmaxf(c.init_sigma, c.lo2[3]), c.hi2[3]);
      x[5] = fminf(fmaxf(x1[K], c.lo2[5]), c.hi2[5]);
      const float e = x[0] > x[2] ? (T1 - x[2]) / (x[0] - x[2]) : 0.5f;
      x[4] = fminf(fmaxf(e, c.init_eta_lo), c.init_eta_hi);
      // stage 1 found no thermal signal (alpha1 on its bound, T1 says
      // nothing): the mixture shape starts at the prior's means, where its
      // fit ends while the data give alpha no signal either
      if (x1[K] <= c.lo1[K]) {
#pragma unroll
        for (int k = 0; k < 5; k++) x[k] = fmaf(0.5f * (c.hi2[k] - c.lo2[k]), c.pm2[k] + 1.f, c.lo2[k]);
      }
      const float *ini = ref.init;
      if (ini && !p.s.init_best) {
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = fminf(fmaxf(ini[K + 2 + i], c.lo2[i]), c.hi2[i]);
      }
#pragma unroll
      for (int i = 0; i < 6; i++) xt[i] = x[i];
      L = LMIter<6>();
#pragma unroll
      for (int a = 0; a < 6; a++) L.act[a] = false;
      if constexpr (ADAM) A.reset();
      first = true;
      nfull = 0;
      active = true;
    }
    {
      // the set-ups of the pixels the warp's two groups just took, one after
      // the other, each by the whole warp
      unsigned need = __ballot_sync(kFull, pend && gp.sub == 0);
      while (need) {
        const int src = __ffs(need) - 1;
        need &= need - 1;
        const float *rs = reinterpret_cast<const float *>(
            __shfl_sync(kFull, reinterpret_cast<unsigned long long>(prow), src));
        const int ws = __shfl_sync(kFull, pwv, src);
        float xss[K];
#pragma unroll
        for (int k = 0; k < K; k++) xss[k] = __shfl_sync(kFull, xsp[k], src);
        float pss;
        const int nu = tcs2::setup_slot_warp<K>(t, c, lane, t.wvtab + (size_t)ws * t.nb, rs, xss,
                                                C.slots + (((threadIdx.x & ~31) + src) / G) * C.sstride,
                                                S.nbs, pss, p.w.err);
        if ((lane ^ src) < G) {
          n2u = nu;
          S.psc = pss;
        }
      }
      pend = false;
    }
    if (active && next >= end) {
      if (pfs == 0) {
        if (gp.sub == 0) pfb = atomicAdd(p.w.counter + 1, (unsigned long long)nclaim);
        pfs = 1;
      } else if (pfs == 1) {
        const long long b = gp.bcast((long long)pfb);
        if (b < n && !p.s.items && !p.s.idx) {
          // 11 lines per pixel: 8 of the stage-2 radiance window, the
          // stage-1 status word, the stage-1 state and the WV bin
          const long long e_end = min((long long)nclaim, n - b) * 11;
#pragma unroll 1
          for (long long e = gp.sub; e < e_end; e += G) {
            const long long q = b + e / 11;
            const int l = (int)(e % 11);
            const void *a;
            if (l < 8) a = p.s.rad + q * t.nb + min(t.b2lo + 32 * l, t.nb - 1);
            else if (l == 8) a = p.w.s1meta + q;
            else if (l == 9) a = p.w.s1x + q * (K + 2);
            else a = p.s.wv + q;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
          }
        }
        pfs = 2;
      }
    }
    if (tcs2::co_and(hc, done)) break;
    bool go = active;
    const float *cur = ne2 + cb * kNE2;
    const float(&H)[21] = *reinterpret_cast<const float(*)[21]>(cur);
    const float(&g)[6] = *reinterpret_cast<const float(*)[6]>(cur + 21);
    const float(&gf)[6] = *reinterpret_cast<const float(*)[6]>(cur + 30);
    if (active && !first) {
      if constexpr (ADAM) go = adam_next2(c, x, g, A, L, xt);
      else {
        // the FP64 solves of ill-conditioned steps on the slot's partial-sum
        // block, free until the band phase of this round
        bool unused = false;
        go = next_trial_t<Stage2<G>, float, true>(S, gp, c, x, H, g, gf, 0, cst, c.max_it2, L, xt, unused,
                                                  reinterpret_cast<double *>(C.parts + slot * tcs2::kPartStride));
      }
    }
    if (go) tcs2::coef(t, c, gp, x, xt, co, slot, prm);
    if (gp.sub == 0) prm[0] = go ? 1.f : 0.f;
    if (!tcs2::round(t, C, hc, &mbar[hc], phase, c.wait_spins)) { ok = false; break; }
    nround++;
    if (go) {
      float ct, cdt, drop;
      tcs2::post(c, gp, C.parts + slot * tcs2::kPartStride, xt, S.psc, n2u, ne2 + (cb ^ 1) * kNE2,
                 ct, cdt, drop);
      nfull++;
      bool accept = first || ADAM;   // an Adam step is always taken
      if (!first && !ADAM) {
        drop += S.prior_drop(c, x, xt);
        const float rho = L.pred > 0.f ? drop / L.pred : -1.f;
        accept = rho > 0.f;
        damping_update(L, accept, rho);
        if (accept && drop / cst < c.tol_f) { L.status = PX_CONVERGED; go = false; }
      }
      if (accept) {
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = xt[i];
        cb ^= 1;
        cst = ct;
        cd = cdt;
      }
      first = false;
    }
    if (active && !go) {
      const float *fin = ne2 + cb * kNE2;   // the accepted state's H and g
      // ---- hand the final state and normal equations to the finalize kernel
      if (L.used64) status |= PX_F_FP64;
      status |= L.status;
      float *hand = p.w.s2x + pix * kS2Hand;
      // lane sub writes entries sub and sub + 16: the state, H, then the scalars
      const int hs = gp.sub, hk = gp.sub + 16;
      hand[hs] = hs < 6 ? pick(x, hs) : fin[max(hs - 6, 0)];
      float hv;
      if (hk < 27) hv = fin[hk - 6];
      else if (hk == 27) hv = cst;
      else if (hk == 28) hv = cd;
      else if (hk == 29) hv = __int_as_float(n2u);
      else if (hk == 30) hv = __int_as_float(status | (L.it << 8));
      else hv = S.psc;
      hand[hk] = hv;
      if (gp.sub < 6) p.w.s2g[pix * 6 + gp.sub] = fin[21 + gp.sub];
      if (gp.sub == 0) {
        atomicAdd(&cstat[ST_IT2], (unsigned long long)L.it);
        atomicAdd(&cstat[ST_S64_2], (unsigned long long)L.n64);
        atomicAdd(&cstat[ST_BAND2], (unsigned long long)nfull * (unsigned long long)t.n2);
        atomicAdd(&cstat[ST_NODEBAND2],
                  (unsigned long long)nfull * (unsigned long long)t.nt * (unsigned long long)t.n2);
      }
      active = false;
    }
  }
  tcs2::release(C, &mbar[hc], phase, ok, p.w.err);
  if (threadIdx.x % tcs2::kCoThreads == 0) atomicAdd(&cstat[ST_MMA2], nround);
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(p.w.stats + i, cstat[i]);
}

// ---- one stage-2 evaluation per state through the tensor-core round (test
// hook of the normal equations): 16 states per CTA and round
template <int K>
__global__ void __launch_bounds__(tcs2::kWarps * 32, 1) normal_eq_tc_kernel(const __grid_constant__ LMLaunch p,
                                                              const float *states, float *Hout,
                                                              float *gout, float *cost_out) {
  constexpr int G = tcs2::G;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar, mbar[tcs2::kCohorts];
  __shared__ uint32_t tslot;
  const KTables &t = p.t;
  const KConfig &c = p.c;
  tcs2::Cta C;
  if (!tcs2::setup(p, smem, &bar, mbar, &tslot, C)) return;
  const int hc = threadIdx.x / tcs2::kCoThreads;   // cohort
  const Grp<G> gp(threadIdx.x & 31);
  const int slot = threadIdx.x / G;
  float *mine = C.slots + slot * C.sstride;
  unsigned char *co = C.base + 3 * t.plrows * 128;
  Stage2<G> S;
  S.nbs = C.nbs;
  S.bb = mine;
  float *ne = mine + 2 * S.nbs;
  float *prm = ne + 2 * kNE2;
  unsigned phase = 0;
  bool ok = true;
  for (long long b0 = (long long)blockIdx.x * tcs2::kSlots; b0 < p.s.n_pix;
       b0 += (long long)gridDim.x * tcs2::kSlots) {
    const long long pix = b0 + slot;
    const bool has = pix < p.s.n_pix;
    float x[6];
    int nu = 0;
    if (has) {
      float xs[K];
#pragma unroll
      for (int k = 0; k < K; k++) xs[k] = states[pix * (K + 6) + k];
#pragma unroll
      for (int i = 0; i < 6; i++) x[i] = states[pix * (K + 6) + K + i];
      nu = tcs2::setup_slot<K>(t, c, gp, t.wvtab + (size_t)min((int)p.s.wv[pix], t.nwv - 1) * t.nb,
                               p.s.rad + pix * t.nb, xs, mine, S.nbs, S.psc);
      tcs2::coef(t, c, gp, x, x, co, slot, prm);
    }
    if (gp.sub == 0) prm[0] = has ? 1.f : 0.f;
    if (!tcs2::round(t, C, hc, &mbar[hc], phase, c.wait_spins)) { ok = false; break; }
    if (has) {
      float cst, cd, drop;
      tcs2::post(c, gp, C.parts + slot * tcs2::kPartStride, x, S.psc, nu, ne, cst, cd, drop);
      if (gp.sub == 0) {
        for (int a = 0; a < 6; a++) {
          gout[pix * 6 + a] = ne[21 + a];
          for (int b = 0; b < 6; b++) Hout[pix * 36 + a * 6 + b] = ne[up<6>(a, b)];
        }
        cost_out[pix] = cst;
      }
    }
    tcs2::co_sync(hc);
  }
  tcs2::release(C, &mbar[hc], phase, ok, p.w.err);
}

// ---- the FP64 normal equations of stage 2 at a pixel's final state, for the
// Laplace posterior: J^T W J + psc P and J^T W r - psc P (z - pm) in the z
// coordinates of Eq. (affine) (the gradient decides which variables sit on
// an outward-pressed bound, so it must not carry FP32 rounding either),
// with the Jacobian of the thermal term (Eq. thermal, the two-component
// mixture on the grid) formed in FP64 from the FP64 Planck grid. The
// covariance inverts this matrix, whose condition number reaches 1e7 and
// more for the near-degenerate mixture, so an FP32-formed matrix would give
// variances of no precision. One warp per pixel: the node coefficients go
// to shared memory (cf [6][kMaxTgrid]), the lanes take the stage-2 bands,
// and the 21 sums are reduced across the warp (every lane gets them).
__device__ __noinline__ void normal_matrix64(const LMLaunch &p, const float *row, int wv,
                                             const float *xs, const double (&x2)[6], double psc,
                                             double *cf, double (&H)[21], double (&g)[6]) {
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31;
  const double mh = x2[0], sh = x2[1], ms = x2[2], ss = x2[3], eta = x2[4], al = x2[5];
  double Uh = 0.0, Us = 0.0;
  for (int j = lane; j < t.nt; j += 32) {
    const double T = (double)t.tglo + j * (double)t.tgstep;
    const double dh = (T - mh) / sh, ds = (T - ms) / ss;
    cf[j] = exp(-0.5 * dh * dh);
    cf[3 * kMaxTgrid + j] = exp(-0.5 * ds * ds);
    Uh += cf[j];
    Us += cf[3 * kMaxTgrid + j];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    Uh += __shfl_xor_sync(kFull, Uh, o);
    Us += __shfl_xor_sync(kFull, Us, o);
  }
  double dbh = 0.0, m2h = 0.0, dbs = 0.0, m2s = 0.0;
  for (int j = lane; j < t.nt; j += 32) {
    const double T = (double)t.tglo + j * (double)t.tgstep;
    const double wh = cf[j] / Uh, ws = cf[3 * kMaxTgrid + j] / Us;
    cf[j] = wh;
    cf[3 * kMaxTgrid + j] = ws;
    dbh += wh * (T - mh);
    m2h += wh * (T - mh) * (T - mh);
    dbs += ws * (T - ms);
    m2s += ws * (T - ms) * (T - ms);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    dbh += __shfl_xor_sync(kFull, dbh, o);
    m2h += __shfl_xor_sync(kFull, m2h, o);
    dbs += __shfl_xor_sync(kFull, dbs, o);
    m2s += __shfl_xor_sync(kFull, m2s, o);
  }
  for (int j = lane; j < t.nt; j += 32) {
    const double T = (double)t.tglo + j * (double)t.tgstep;
    const double dh = T - mh, ds = T - ms;
    const double wh = cf[j], ws = cf[3 * kMaxTgrid + j];
    cf[kMaxTgrid + j] = wh * (dh - dbh);
    cf[2 * kMaxTgrid + j] = wh * (dh * dh - m2h);
    cf[4 * kMaxTgrid + j] = ws * (ds - dbs);
    cf[5 * kMaxTgrid + j] = ws * (ds * ds - m2s);
  }
  __syncwarp();
  double sc[6];
#pragma unroll
  for (int i = 0; i < 6; i++) sc[i] = 0.5 * ((double)c.hi2[i] - (double)c.lo2[i]);
  const double fh2 = al * eta / (sh * sh), fs2 = al * (1.0 - eta) / (ss * ss);
  double acc[27];   // J^T W J (21), then J^T W r (6)
#pragma unroll
  for (int i = 0; i < 27; i++) acc[i] = 0.0;
  const float4 *wvrow = t.wvtab + (size_t)wv * t.nb;
  const float *endm = t.image + t.lay.off_endm;
  for (int i = lane; i < t.n2; i += 32) {
    const int b = t.b2lo + i;
    const float L = __ldg(row + b);
    if (!(t.image[t.lay.off_win2 + b] > 0.f) || (t.sat && L >= __ldg(t.sat + b))) continue;
    double w = 1.0;
    if (c.weighted) {
      const double var = c.has_nsd ? (double)c.nsd[b] * (double)c.nsd[b]
                                   : (double)c.noise_rel * c.noise_rel * (double)L * L +
                                         (double)c.noise_abs * c.noise_abs;
      w = 1.0 / var;
    }
    const float4 q = __ldg(&wvrow[b]);
    const double tu = (double)q.w;
    double rho = 0.0;
    for (int k = 0; k < t.K; k++) rho = fma((double)xs[k], (double)__ldg(endm + k * t.nb + b), rho);
    const double Ls = (double)q.y + (double)q.x * rho / (1.0 - (double)q.z * rho);   // Eq. (solar)
    double S[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double *Bp = t.planck64 + i;
    for (int j = 0; j < t.nt; j++) {
      const double Bj = __ldg(Bp + (size_t)j * t.n2);
#pragma unroll
      for (int k = 0; k < 6; k++) S[k] = fma(cf[k * kMaxTgrid + j], Bj, S[k]);
    }
    double J[6];
    J[0] = tu * fh2 * S[1] * sc[0];
    J[1] = tu * fh2 * S[2] / sh * sc[1];
    J[2] = tu * fs2 * S[4] * sc[2];
    J[3] = tu * fs2 * S[5] / ss * sc[3];
    J[4] = tu * al * (S[0] - S[3]) * sc[4];
    J[5] = tu * (eta * S[0] + (1.0 - eta) * S[3]) * sc[5];
    const double r = (double)L - (Ls + al * tu * (eta * S[0] + (1.0 - eta) * S[3]));
#pragma unroll
    for (int a2 = 0; a2 < 6; a2++) {
      acc[21 + a2] = fma(w * J[a2], r, acc[21 + a2]);
#pragma unroll
      for (int b2 = a2; b2 < 6; b2++) acc[up<6>(a2, b2)] = fma(w * J[a2], J[b2], acc[up<6>(a2, b2)]);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1)
#pragma unroll
    for (int i = 0; i < 27; i++) acc[i] += __shfl_xor_sync(kFull, acc[i], o);
#pragma unroll
  for (int i = 0; i < 21; i++) H[i] = acc[i];
  // the prior of Eq. (affine)'s z: curvature psc pp, gradient -psc pp (z - pm)
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const double zk = (double)c.zk2[i] > 0.0 ? (x2[i] - (double)c.lo2[i]) / sc[i] - 1.0 : 0.0;
    H[up<6>(i, i)] += psc * (double)c.pp2[i];
    g[i] = acc[21 + i] - psc * (double)c.pp2[i] * (zk - (double)c.pm2[i]);
  }
  __syncwarp();
}

// ---- finalize: moment matching (Sec. 2.3), FP64 Laplace covariance,
// identifiability and the outputs of every fitted pixel; one thread per
// pixel, so the FP64 work is not repeated across the lanes of a warp. The
// covariance first inverts the fit's last FP32 normal matrix; a pixel that
// may be identifiable (alpha free, and alpha above 0.9 of its threshold
// times a lower bound of sd(alpha)) is then given the FP64 normal equations
// of its final state (normal_matrix64, the warp working on one such pixel at
// a time) and its covariance, var(E[T]) and identifiability come from those.
// The warps loop over 32 consecutive pixels at a time, so every lane of a
// warp runs the same iterations. Four CTAs per SM (128 registers; the FP64
// temporaries partly spill to L1-resident local memory): at 249 registers
// and two CTAs the kernel took 28.4 ms on the flight line, at four 21.3 ms.
constexpr int kFinWarps = 4;
__global__ void __launch_bounds__(kFinWarps * 32, 4) finalize_kernel(const __grid_constant__ LMLaunch p,
                                                                     int K) {
  __shared__ unsigned long long cstat[ST_COUNT];
  __shared__ double cfs[kFinWarps][6 * kMaxTgrid];
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  if (cta_err(p.w.err)) return;
  const KConfig &c = p.c;
  const int NSx = K + 8, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned long long st_fp64 = 0, st_post = 0, st_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long n = p.s.n_pix, step = (long long)gridDim.x * kFinWarps * 32;
  for (long long base = ((long long)blockIdx.x * kFinWarps + wib) * 32; base < n; base += step) {
    const long long pix = base + lane;
    const bool fitted = pix < n && (p.w.s1meta[pix] & kFitted);
    CovIO io;
    float cost = 0.f, cdata = 0.f, psc = 0.f;
    int n2u = 1, status = 0, it2 = 0, nf = 0;
    bool act_a = false;
    if (fitted) {
      const float *hand = p.w.s2x + pix * kS2Hand;
#pragma unroll
      for (int k = 0; k < 6; k++) { io.x[k] = hand[k]; io.g[k] = p.w.s2g[pix * 6 + k]; }
#pragma unroll
      for (int k = 0; k < 21; k++) io.H[k] = hand[6 + k];
      cost = hand[27];
      cdata = hand[28];
      n2u = __float_as_int(hand[29]);
      const int sw = __float_as_int(hand[30]);
      status = sw & 0xff;
      it2 = sw >> 8;
      psc = hand[31];
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const bool act = (io.x[k] <= c.lo2[k] && io.g[k] <= 0.f) || (io.x[k] >= c.hi2[k] && io.g[k] >= 0.f);
        nf += (!act && io.H[up<6>(k, k)] > 0.0);
      }
      io.s2 = c.weighted ? 1.f : cost / (float)(n2u - nf);
      act_a = (io.x[5] <= c.lo2[5] && io.g[5] <= 0.f) || (io.x[5] >= c.hi2[5] && io.g[5] >= 0.f);
      if (act_a && io.x[5] <= c.lo2[5]) {
        // no thermal signal: E[T] is undefined, so is its posterior
        io.cov_ok = false;
        io.vE = __longlong_as_double(0x7ff0000000000000ll);
        io.va = 0.0;
#pragma unroll
        for (int i = 0; i < 21; i++) io.cov[i] = __int_as_float(0x7fc00000);
      } else if (nf > 0) {
        laplace_cov(c, io);
      } else {
        io.cov_ok = true;
        io.vE = io.va = 0.0;
#pragma unroll
        for (int i = 0; i < 21; i++) io.cov[i] = 0.f;
      }
    }
    // the FP64 posterior for pixels that may be identifiable: alpha free and
    // alpha / sd(alpha) possibly above its threshold. sd(alpha) is at least
    // sc5 sqrt(s2 / H_55) (the marginal variance of a variable is at least
    // the inverse of its own curvature), a bound the FP32 matrix gives
    // without an inversion; 0.9 of the threshold leaves room for rounding
    const double sd_min = 0.5 * ((double)c.hi2[5] - (double)c.lo2[5]) *
                          sqrt((double)io.s2 / fmax(io.H[up<6>(5, 5)], 1e-300));
    bool cand = fitted && !act_a && nf > 0 &&
                (double)io.x[5] >= 0.9 * (double)c.ident_alpha_snr * sd_min;
    // ... and not surely unidentifiable: alpha below half its threshold
    // against the floor of sd(alpha) over every admissible active set (with
    // the matrix error allowed for, sd(alpha) stays above 0.86 of that
    // floor, so alpha / sd(alpha) < 0.58 of the threshold whatever the FP64
    // matrix gives); s2 moves by under 3 % with the free count
    double va_min;
    if (cand && alpha_var_floor(c, io, va_min)) {
      const double sda_min = 0.5 * ((double)c.hi2[5] - (double)c.lo2[5]) * sqrt((double)io.s2 * 0.97 * va_min);
      if ((double)io.x[5] < 0.5 * (double)c.ident_alpha_snr * sda_min) cand = false;
    }
    unsigned m = __ballot_sync(kFull, cand);
    bool mine = false;
    double H64[21], g64[6];
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const long long sp = __shfl_sync(kFull, pix, src);
      double xs[6];
#pragma unroll
      for (int k = 0; k < 6; k++) xs[k] = (double)__shfl_sync(kFull, io.x[k], src);
      const double ps = (double)__shfl_sync(kFull, psc, src);
      const PixRef ref = resolve(p, sp, K);
      double Hs[21], gs[6];
      normal_matrix64(p, ref.row, ref.wv, p.w.s1x + sp * (K + 2), xs, ps, cfs[wib], Hs, gs);
      if (lane == src) {
        mine = true;
#pragma unroll
        for (int i = 0; i < 21; i++) H64[i] = Hs[i];
#pragma unroll
        for (int i = 0; i < 6; i++) g64[i] = gs[i];
      }
    }
    if (mine) {
      // the active set and the free count from the FP64 gradient, then the
      // covariance from the FP64 matrix
#pragma unroll
      for (int i = 0; i < 21; i++) io.H[i] = H64[i];
      nf = 0;
#pragma unroll
      for (int k = 0; k < 6; k++) {
        io.g[k] = g64[k] > 0.0 ? 1.f : (g64[k] < 0.0 ? -1.f : 0.f);
        const bool act = (io.x[k] <= c.lo2[k] && io.g[k] <= 0.f) || (io.x[k] >= c.hi2[k] && io.g[k] >= 0.f);
        nf += (!act && io.H[up<6>(k, k)] > 0.0);
      }
      io.s2 = c.weighted ? 1.f : cost / (float)(n2u - nf);
      act_a = (io.x[5] <= c.lo2[5] && io.g[5] <= 0.f) || (io.x[5] >= c.hi2[5] && io.g[5] >= 0.f);
      laplace_cov(c, io);
      st_post++;
    }
    if (fitted) {
      const float *x2 = io.x;
      const float ET = x2[4] * x2[0] + (1.f - x2[4]) * x2[2];
      const float dmu = x2[0] - x2[2];
      const float sdT = sqrtf(x2[4] * x2[1] * x2[1] + (1.f - x2[4]) * x2[3] * x2[3] +
                              x2[4] * (1.f - x2[4]) * dmu * dmu);
      const float rms = sqrtf(cdata / (float)n2u);
      const double sdE = sqrt(io.vE), sda = sqrt(io.va);
      const bool ident = io.cov_ok && isfinite(sdE) && sdE <= (double)c.ident_sd_et &&
                         (double)x2[5] >= (double)c.ident_alpha_snr * sda && !act_a && x2[5] > 0.f;
      if (!ident) status |= PX_F_NOT_IDENT;
      if (p.w.fb_idx) {
        // fallback rule of the learned start: the fit did not converge, or its
        // cost exceeds three times the expected chi-square (n_used - 6) psc
        const float expect = (float)(n2u - 6) * (c.weighted ? 1.f : psc);
        if ((status & 7) != PX_CONVERGED || cost > 3.f * expect) {
          unsigned long long j = atomicAdd(p.w.fb_count, 1ull);
          p.w.fb_idx[j] = pix;
          p.w.fb_cost[j] = cost;
        }
      }
      const PixRef ref = resolve(p, pix, K);
      const KOut &o = ref.o;
      const long long op = ref.opix;
      if (o.state) {
        for (int k = 0; k < K + 2; k++) o.state[op * NSx + k] = p.w.s1x[pix * (K + 2) + k];
        for (int k = 0; k < 6; k++) o.state[op * NSx + K + 2 + k] = x2[k];
      }
      if (o.cov)
        for (int k = 0; k < 21; k++) o.cov[op * 21 + k] = io.cov[k];
      if (o.ET) o.ET[op] = ET;
      if (o.sdT) o.sdT[op] = sdT;
      if (o.alpha) o.alpha[op] = x2[5];
      if (o.var_ET) o.var_ET[op] = (float)io.vE;
      if (o.cost) o.cost[op] = cost;
      if (o.rms) o.rms[op] = rms;
      if (o.status) o.status[op] = (uint8_t)status;
      if (o.iters) o.iters[2 * op + 1] = (uint16_t)it2;
      st_fp64 += (status & PX_F_FP64) ? 1ull : 0ull;
#pragma unroll
      for (int k = 0; k < 8; k++) st_s[k] += ((status & 7) == k) ? 1ull : 0ull;
    }
  }
  // warp-aggregate, then one shared atomic per warp and counter
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    st_fp64 += __shfl_xor_sync(kFull, st_fp64, o);
    st_post += __shfl_xor_sync(kFull, st_post, o);
#pragma unroll
    for (int k = 0; k < 8; k++) st_s[k] += __shfl_xor_sync(kFull, st_s[k], o);
  }
  if (lane == 0) {
    if (st_fp64) atomicAdd(&cstat[ST_FP64], st_fp64);
    if (st_post) atomicAdd(&cstat[ST_POST64], st_post);
    for (int k = 0; k < 8; k++)
      if (st_s[k]) atomicAdd(&cstat[ST_STATUS0 + k], st_s[k]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(p.w.stats + i, cstat[i]);
}

// ---- residual spectrum (Sec. 3.2's spectral residuals): r_b = L_b - M_b(x)
// of the full forward model Eq. (fm) at each fitted pixel's final state, for
// every band, one warp per pixel: the normalised grid weights of the two
// mixture components (Eq. thermal) in shared memory, then per band the
// solar term (Eq. solar) at the stage-1 surface and the thermal grid sum
// against the context's Planck table [nt][nb]. Pixels not fitted get NaN.
__global__ void __launch_bounds__(256) resid_kernel(const __grid_constant__ LMLaunch p) {
  __shared__ float wsh[8][kMaxTgrid];
  if (cta_err(p.w.err)) return;
  const KTables &t = p.t;
  const int K = t.K, nb = t.nb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *wj = wsh[warp];
  const long long nw = (long long)gridDim.x * 8;
  for (long long pix = (long long)blockIdx.x * 8 + warp; pix < p.s.n_pix; pix += nw) {
    const PixRef ref = resolve(p, pix, K);
    if (!ref.o.resid) continue;
    float *r = ref.o.resid + ref.opix * nb;
    if (!(p.w.s1meta[pix] & kFitted)) {
      for (int b = lane; b < nb; b += 32) r[b] = __int_as_float(0x7fc00000);
      continue;
    }
    const float *x1 = p.w.s1x + pix * (K + 2);
    const float *x2 = p.w.s2x + pix * kS2Hand;
    const float mh = x2[0], sh = x2[1], ms = x2[2], ss = x2[3], eta = x2[4], al = x2[5];
    float uh[kMaxTgrid / 32], us[kMaxTgrid / 32], Uh = 0.f, Us = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxTgrid / 32; q++) {
      const int j = lane + 32 * q;
      uh[q] = us[q] = 0.f;
      if (j < t.nt) {
        const float T = t.tglo + (float)j * t.tgstep;
        const float dh = (T - mh) / sh, ds = (T - ms) / ss;
        uh[q] = expf(-0.5f * dh * dh);
        us[q] = expf(-0.5f * ds * ds);
      }
      Uh += uh[q];
      Us += us[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      Uh += __shfl_xor_sync(kFull, Uh, o);
      Us += __shfl_xor_sync(kFull, Us, o);
    }
#pragma unroll
    for (int q = 0; q < kMaxTgrid / 32; q++) {
      const int j = lane + 32 * q;
      if (j < t.nt) wj[j] = eta * uh[q] / Uh + (1.f - eta) * us[q] / Us;
    }
    __syncwarp();
    const float4 *row = t.wvtab + (size_t)ref.wv * nb;
    const float *endm = t.image + t.lay.off_endm;
    for (int b = lane; b < nb; b += 32) {
      const float4 q = __ldg(row + b);
      float rho = 0.f;
      for (int k = 0; k < K; k++) rho = fmaf(x1[k], __ldg(endm + k * nb + b), rho);
      float acc = 0.f;
      for (int j = 0; j < t.nt; j++) acc = fmaf(wj[j], __ldg(t.planck_full + (size_t)j * nb + b), acc);
      const float M = q.y + q.x * rho / (1.f - q.z * rho) + al * q.w * acc;
      r[b] = __ldg(ref.row + b) - M;
    }
    __syncwarp();
  }
}

// ---- keep the lower-cost of the learned-start fit and the default-start
// re-fit of each flagged pixel; both get the MLP_FALLBACK flag
__global__ void merge_fallback_kernel(const long long *idx, const float *cost_first, long long nfb,
                                      KOut compact, KOut out, int K, int nb) {
  const int NSx = K + 8;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nfb;
       j += (long long)gridDim.x * blockDim.x) {
    const long long pix = idx[j];
    const float c2 = compact.cost[j];
    const bool take = c2 < cost_first[j] || isnan(cost_first[j]);
    if (take) {
      if (out.state) for (int k = 0; k < NSx; k++) out.state[pix * NSx + k] = compact.state[j * NSx + k];
      if (out.cov) for (int k = 0; k < 21; k++) out.cov[pix * 21 + k] = compact.cov[j * 21 + k];
      if (out.ET) out.ET[pix] = compact.ET[j];
      if (out.sdT) out.sdT[pix] = compact.sdT[j];
      if (out.alpha) out.alpha[pix] = compact.alpha[j];
      if (out.var_ET) out.var_ET[pix] = compact.var_ET[j];
      if (out.cost) out.cost[pix] = c2;
      if (out.rms) out.rms[pix] = compact.rms[j];
      if (out.iters) {
        out.iters[2 * pix] = compact.iters[2 * j];
        out.iters[2 * pix + 1] = compact.iters[2 * j + 1];
      }
      if (out.resid && compact.resid)
        for (int b = 0; b < nb; b++) out.resid[pix * nb + b] = compact.resid[j * nb + b];
    }
    if (out.status)
      out.status[pix] = (uint8_t)((take ? compact.status[j] : out.status[pix]) | PX_F_MLP_FALLBACK);
  }
}

// ---- one evaluation of a stage's normal equations per state (test hook),
// through the same evaluation code as the fit, one pixel per group
template <int K, int G, int MAXW>
__global__ void __launch_bounds__(MAXW * 32, 1) normal_eq_kernel(const __grid_constant__ LMLaunch p,
                                                                 int stage, const float *states,
                                                                 float *Hout, float *gout,
                                                                 float *cost_out) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31;
  const int img_f = image_floats(t, stage);
  if (!stage_tables(t, smem, img_f, &bar, p.w.err, c.wait_spins)) return;
  const Grp<G> gp(lane);
  const int gid = threadIdx.x / G, groups = blockDim.x / G;
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  const long long ng = (long long)gridDim.x * groups;
  for (long long pix = (long long)blockIdx.x * groups + gid; pix < p.s.n_pix; pix += ng) {
    const float *row = p.s.rad + pix * t.nb;
    pc.wvrow = t.wvtab + (size_t)min((int)p.s.wv[pix], t.nwv - 1) * t.nb;
    if (stage == 1) {
      constexpr int P = K + 1;
      Stage1<K, G> s1;
      s1.nbs = band_slots(t.n1, G);
      s1.bb = smem + img_f + gid * pix_stride1(t, G);
      pc.node = nullptr;
      setup1(s1, pc, gp, row);
      float x[K + 2], H[P * (P + 1) / 2], g[P], gf[P], cst, cd, drop;
      int m;
#pragma unroll
      for (int i = 0; i < K + 2; i++) x[i] = states[pix * (K + 2) + i];
      s1.eval(pc, gp, x, 1, H, g, gf, cst, cd, drop, m, x, false);
      if (gp.sub == 0) {
        for (int a = 0; a < P; a++) {
          gout[pix * P + a] = g[a];
          for (int b = 0; b < P; b++) Hout[pix * P * P + a * P + b] = H[up<P>(a, b)];
        }
        cost_out[pix] = cst;
      }
    } else {
      float *mine = smem + img_f + gid * pix_stride2(t, G);
      pc.node = mine;
      Stage2<G> s2;
      s2.nbs = band_slots(t.n2, G);
      s2.bb = mine + t.nt * kScratchPerNode;
      float xs[K], x[6];
#pragma unroll
      for (int k = 0; k < K; k++) xs[k] = states[pix * (K + 6) + k];
#pragma unroll
      for (int i = 0; i < 6; i++) x[i] = states[pix * (K + 6) + K + i];
      setup2<K>(s2, pc, gp, row, xs);
      float cst, cd, drop;
      float *ne = s2.bb + 5 * s2.nbs;
      s2.eval(pc, gp, x, x, 1, ne, cst, cd, drop);
      if (gp.sub == 0) {
        for (int a = 0; a < 6; a++) {
          gout[pix * 6 + a] = ne[21 + a];
          for (int b = 0; b < 6; b++) Hout[pix * 36 + a * 6 + b] = ne[up<6>(a, b)];
        }
        cost_out[pix] = cst;
      }
    }
  }
}

// Launch shapes. A stage kernel runs as one persistent CTA per SM of up to
// MAXW warps (the register budget follows from MAXW: 65536 / (32 MAXW)),
// with G lanes per pixel; the warps actually launched are as many as the
// shared memory of the table image plus one scratch block per pixel allows.
struct Shape { int G, maxw; };
constexpr Shape kShape1[3] = {{16, 12}, {8, 12}, {32, 8}};
constexpr Shape kShape2[2] = {{32, 8}, {16, 8}};

size_t stage_smem(const KTables &t, int stage, int G, int wpb) {
  const int per = stage == 1 ? pix_stride1(t, G) : pix_stride2(t, G);
  const size_t head = (size_t)image_floats(t, stage) + (stage == 1 ? (size_t)wvtab_floats(t, G) : 0);
  return (head + (size_t)wpb * (32 / G) * per) * 4;
}

int fit_warps(const KTables &t, int stage, int G, int maxw) {
  int w = maxw;
  while (w > 1 && stage_smem(t, stage, G, w) > kMaxSmemPerCta) w--;
  return stage_smem(t, stage, G, w) <= kMaxSmemPerCta ? w : 0;
}

template <class Kern>
cudaError_t launch_persistent(Kern kern, const LMLaunch &p, int num_sms, cudaStream_t st,
                              int *blocks_used, int stage, int G, int maxw) {
  const int wpb = fit_warps(p.t, stage, G, maxw);
  if (wpb < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = stage_smem(p.t, stage, G, wpb);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int cl = p.s.claim > 0 ? p.s.claim : kClaim;
  const long long per_cta = (long long)wpb * (32 / G) * cl;
  long long need = (p.s.n_pix + per_cta - 1) / per_cta;
  long long blocks = (long long)num_sms * occ;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  kern<<<(int)blocks, wpb * 32, smem, st>>>(p);
  if (blocks_used) *blocks_used += (int)blocks;
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_stage1(const LMLaunch &p, int num_sms, cudaStream_t st, int *bu, int v) {
  if (p.c.solver == kSolverAdam) {
    // the Adam solver runs on the 16-lane shape
    const Shape s = kShape1[0];
    return launch_persistent(lm_stage1_kernel<K, 16, 12, true>, p, num_sms, st, bu, 1, s.G, s.maxw);
  }
  const Shape s = kShape1[v];
  switch (v) {
    case 1: return launch_persistent(lm_stage1_kernel<K, 8, 12>, p, num_sms, st, bu, 1, s.G, s.maxw);
    case 2: return launch_persistent(lm_stage1_kernel<K, 32, 8>, p, num_sms, st, bu, 1, s.G, s.maxw);
    default: return launch_persistent(lm_stage1_kernel<K, 16, 12>, p, num_sms, st, bu, 1, s.G, s.maxw);
  }
}

template <int K, bool ADAM>
cudaError_t launch_stage2_tc(const LMLaunch &p, int num_sms, cudaStream_t st, int *bu) {
  const size_t smem = (size_t)tcs2::layout(p.t).total;
  cudaError_t e = cudaFuncSetAttribute(lm_stage2_tc_kernel<K, ADAM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int cl = p.s.claim > 0 ? p.s.claim : kClaim;
  const long long per_cta = (long long)tcs2::kSlots * cl;
  long long blocks = (p.s.n_pix + per_cta - 1) / per_cta;
  if (blocks > num_sms) blocks = num_sms;
  if (blocks < 1) blocks = 1;
  lm_stage2_tc_kernel<K, ADAM><<<(int)blocks, tcs2::kWarps * 32, smem, st>>>(p);
  if (bu) *bu += (int)blocks;
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_stage2(const LMLaunch &p, int num_sms, cudaStream_t st, int *bu, int v) {
  const bool adam = p.c.solver == kSolverAdam;
  if (v == 2) {
    if (lm_tc_ok(p.t) && !p.c.weighted)
      return adam ? launch_stage2_tc<K, true>(p, num_sms, st, bu)
                  : launch_stage2_tc<K, false>(p, num_sms, st, bu);
    v = 1;   // tables outside the tensor-core path, or a weighted loss: the FP32 shape of 16 lanes
  }
  if (adam) {
    // the Adam solver's FP32 stage 2 runs on the 16-lane shape
    const Shape s = kShape2[1];
    return launch_persistent(lm_stage2_kernel<K, 16, 8, true>, p, num_sms, st, bu, 2, s.G, s.maxw);
  }
  const Shape s = kShape2[v];
  if (v == 1) return launch_persistent(lm_stage2_kernel<K, 16, 8>, p, num_sms, st, bu, 2, s.G, s.maxw);
  return launch_persistent(lm_stage2_kernel<K, 32, 8>, p, num_sms, st, bu, 2, s.G, s.maxw);
}

template <int K>
cudaError_t launch_k(const LMLaunch &p, int num_sms, cudaStream_t st, int *blocks_used, int variant,
                     cudaEvent_t *ev) {
  // variant = 3 * (stage-2 shape) + (stage-1 shape); stage-2 shape 2 is the
  // tensor-core evaluation
  const int v1 = variant % 3, v2 = (variant / 3) % 3;
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  if ((e = launch_stage1<K>(p, num_sms, st, blocks_used, v1)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  if ((e = launch_stage2<K>(p, num_sms, st, blocks_used, v2)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  long long blocks = (p.s.n_pix + kFinWarps * 32 - 1) / (kFinWarps * 32);
  if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
  finalize_kernel<<<(int)blocks, kFinWarps * 32, 0, st>>>(p, K);
  if (blocks_used) *blocks_used += (int)blocks;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  if (p.s.want_resid) {
    long long rb = (p.s.n_pix + 7) / 8;
    if (rb > (long long)num_sms * 16) rb = (long long)num_sms * 16;
    resid_kernel<<<(int)rb, 256, 0, st>>>(p);
    if (blocks_used) *blocks_used += (int)rb;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int K>
cudaError_t launch_ne_k(const LMLaunch &p, int stage, const float *states, float *H, float *g,
                        float *cost, cudaStream_t st, int variant) {
  if (stage == 2 && (variant / 3) % 3 == 2 && lm_tc_ok(p.t) && !p.c.weighted) {
    const size_t smem = (size_t)tcs2::layout(p.t).total;
    cudaError_t e = cudaFuncSetAttribute(normal_eq_tc_kernel<K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long long blocks = (p.s.n_pix + tcs2::kSlots - 1) / tcs2::kSlots;
    if (blocks > 1024) blocks = 1024;
    normal_eq_tc_kernel<K><<<(int)blocks, tcs2::kWarps * 32, smem, st>>>(p, states, H, g, cost);
    return cudaGetLastError();
  }
  // the lanes per pixel of the default fit shapes
  auto go = [&](auto kern, int G, int maxw) {
    const int wpb = fit_warps(p.t, stage, G, maxw);
    if (wpb < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = stage_smem(p.t, stage, G, wpb);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per = wpb * (32 / G);
    int blocks = (int)((p.s.n_pix + per - 1) / per);
    if (blocks > 1024) blocks = 1024;
    kern<<<blocks, wpb * 32, smem, st>>>(p, stage, states, H, g, cost);
    return cudaGetLastError();
  };
  if (stage == 1) return go(normal_eq_kernel<K, 16, 8>, 16, 8);
  return go(normal_eq_kernel<K, 32, 8>, 32, 8);
}

}  // namespace

size_t planck_operand_bytes(const KTables &t) { return (size_t)3 * t.plrows * 128; }

cudaError_t launch_planck_operand(const KTables &t, unsigned char *out, cudaStream_t st) {
  const int n = t.plrows * 8;
  tcs2::planck_operand_kernel<<<(n + 255) / 256, 256, 0, st>>>(t, t.image, out);
  return cudaGetLastError();
}

bool lm_tc_ok(const KTables &t) {
  return t.plop && t.nt <= 64 && t.n2 <= 256 &&
         (size_t)tcs2::layout(t).total <= kMaxSmemPerCta;
}

size_t lm_smem_bytes(const KTables &t, int) {
  // the smallest launch: one warp of the widest-group stage-2 shape
  return stage_smem(t, 2, 32, 1);
}

cudaError_t launch_lm(const LMLaunch &p, int num_sms, cudaStream_t st, int *blocks_used, int variant,
                      cudaEvent_t *ev) {
  switch (p.t.K) {
    case 3: return launch_k<3>(p, num_sms, st, blocks_used, variant, ev);
    case 5: return launch_k<5>(p, num_sms, st, blocks_used, variant, ev);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_fallback(const long long *idx, const float *cost_first, long long nfb,
                                  const KOut &compact, const KOut &out, int K, int nb,
                                  cudaStream_t st) {
  if (nfb <= 0) return cudaSuccess;
  long long blocks = (nfb + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  merge_fallback_kernel<<<(int)blocks, 128, 0, st>>>(idx, cost_first, nfb, compact, out, K, nb);
  return cudaGetLastError();
}

cudaError_t launch_normal_eq(const LMLaunch &p, int stage, const float *states, float *H, float *g,
                             float *cost, cudaStream_t st, int variant) {
  if (p.s.n_pix <= 0) return cudaSuccess;
  switch (p.t.K) {
    case 3: return launch_ne_k<3>(p, stage, states, H, g, cost, st, variant);
    case 5: return launch_ne_k<5>(p, stage, states, H, g, cost, st, variant);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace firert
