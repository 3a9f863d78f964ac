// kernels_lm.cu — the per-pixel two-stage retrieval on sm_103a.
//
// One warp per pixel, persistent CTAs claiming pixels from a global counter.
// Lanes own bands (lane + 32 i within each stage's window), so radiance and
// the shared Planck table are read band-coalesced; the normal equations
// J^T W J, J^T W r and the cost are reduced with warp shuffles, and every
// lane then runs the same small solve on registers (uniform control flow).
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
#include <float.h>

#include "internal.cuh"

namespace firert {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kClaim = 4;          // pixels claimed per atomic
constexpr size_t kMaxSmemPerCta = 227 * 1024;   // opt-in dynamic shared memory per CTA

template <int N>
__device__ __forceinline__ void warp_sum(float (&v)[N]) {
#pragma unroll
  for (int o = 16; o; o >>= 1)
#pragma unroll
    for (int i = 0; i < N; i++) v[i] += __shfl_xor_sync(kFull, v[i], o);
}

__device__ __forceinline__ float warp_sum1(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

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

// Reciprocal square root without division: FP32 uses the SFU; FP64 refines an
// FP32 seed with two Newton-Raphson steps y <- y (3 - x y^2) / 2 (quadratic
// convergence: 2^-23 -> 2^-46 -> full precision).
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}

// ------------------------------------------------------------- solve ----
// Solve (H + lam D) d = rhs over the free variables on the diagonally scaled
// matrix; pinned variables are identity rows with their displacement moved
// to the right-hand side. Returns false on a non-positive pivot. kap is the
// condition estimate (max L_ii / min L_ii)^2 over the free variables.
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
  for (int i = 0; i < P; i++) rd[i] = rsq(A[i * (i + 1) / 2 + i]);
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
    T r = rsq(s > T(0) ? s : T(1));
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
  T lmax = T(0), lmin = T(1e30);
#pragma unroll
  for (int i = 0; i < P; i++)
    if (!pin[i]) {
      T l = A[i * (i + 1) / 2 + i];
      lmax = l > lmax ? l : lmax;
      lmin = l < lmin ? l : lmin;
    }
  kap = lmax > T(0) ? (float)(lmax * lmax) / (float)(lmin * lmin) : 1.f;
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

// per-warp shared scratch: node weights [nt][8], then (stage 2) the band
// buffers [4][S2 * 32] of the band-slot count the kernel is instantiated for
__host__ __device__ __forceinline__ int s2_slots(int n2) {
  const int s2 = (n2 + 31) / 32;
  return s2 <= 7 ? 7 : (s2 <= 9 ? 9 : 16);
}
__host__ __device__ __forceinline__ int warp_scratch_floats(const KTables &t) {
  return t.nt * kScratchPerNode + 4 * 32 * s2_slots(t.n2);
}

// ------------------------------------------------------- pixel context --
struct PixCtx {
  const KTables *t;
  const KConfig *c;
  const float *img;       // shared-memory table image
  float *wsc;             // this warp's node scratch [nt][8]
  const float4 *wvrow;    // this pixel's water-vapour row of the atmosphere table
  int lane;
  int node_evals;         // sum over stage-2 full evaluations of active nodes
  int trial_nodes;        // sum over stage-2 trial (decrease-only) evaluations
};

// ------------------------------------------------------------ stage 1 ---
template <int K, int S1>
struct Stage1 {
  static constexpr int P = K + 1, NX = K + 2, NH = P * (P + 1) / 2, NS = S1;
  float Lobs[S1], w[S1];
  float psc;
  float sf, sa, sT;

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

  __device__ __forceinline__ static int argmax_frac(const float (&x)[NX]) {
    int m = 0;
    float best = x[0];
#pragma unroll
    for (int k = 1; k < K; k++)
      if (x[k] > best) { m = k; best = x[k]; }
    return m;
  }

  // model, reduced Jacobian, normal equations and cost at x (all lanes get
  // the warp totals). cd = unweighted data cost.
  __device__ __forceinline__ void eval(PixCtx &pc, const float (&x)[NX], float (&H)[NH],
                                       float (&g)[P], float &cst, float &cd, int &m,
                                       const float (&rold)[NS], float (&rnew)[NS],
                                       float &dcd) const {
    const KTables &t = *pc.t;
    const KConfig &c = *pc.c;
    m = argmax_frac(x);
    float acc[NH + P + 3];
#pragma unroll
    for (int i = 0; i < NH + P + 3; i++) acc[i] = 0.f;
    const float a1 = x[K], invT = 1.f / x[K + 1];
#pragma unroll
    for (int s = 0; s < S1; s++) {
      int bi = pc.lane + 32 * s;
      if (bi < t.n1 && w[s] > 0.f) {
        int b = t.b1lo + bi;
        float4 q = __ldg(pc.wvrow + b);
        float E[K];
        float rho = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) {
          E[k] = pc.img[t.lay.off_endm + k * t.nb + b];
          rho = fmaf(x[k], E[k], rho);
        }
        float inv = __frcp_rn(1.f - q.z * rho);
        float Ls = fmaf(q.x * rho, inv, q.y);
        float xx = pc.img[t.lay.off_c2l + b] * invT;
        float e = __expf(-xx);
        float rom = __frcp_rn(1.f - e);
        float B = pc.img[t.lay.off_c1l5 + b] * e * rom;
        float dB = B * xx * invT * rom;
        float r = Lobs[s] - fmaf(a1 * q.w, B, Ls);
        rnew[s] = r;
        acc[NH + P + 2] = fmaf(w[s] * (rold[s] - r), rold[s] + r, acc[NH + P + 2]);
        float dL[K], dEm = 0.f;
        const float qi2 = q.x * inv * inv * sf;
#pragma unroll
        for (int k = 0; k < K; k++) {
          dL[k] = qi2 * E[k];
          dEm = (k == m) ? dL[k] : dEm;
        }
        float J[P];
#pragma unroll
        for (int a = 0; a < K - 1; a++) J[a] = (a < m ? dL[a] : dL[a + 1]) - dEm;
        J[K - 1] = q.w * B * sa;
        J[K] = a1 * q.w * dB * sT;
        float wr = w[s] * r;
        acc[NH + P] = fmaf(wr, r, acc[NH + P]);
        acc[NH + P + 1] = fmaf(r, r, acc[NH + P + 1]);
#pragma unroll
        for (int a = 0; a < P; a++) {
          acc[NH + a] = fmaf(J[a], wr, acc[NH + a]);
          float wj = w[s] * J[a];
#pragma unroll
          for (int bb = a; bb < P; bb++) acc[up<P>(a, bb)] = fmaf(wj, J[bb], acc[up<P>(a, bb)]);
        }
      }
    }
    warp_sum(acc);
#pragma unroll
    for (int i = 0; i < NH; i++) H[i] = acc[i];
#pragma unroll
    for (int a = 0; a < P; a++) g[a] = acc[NH + a];
    cd = acc[NH + P + 1];
    cst = acc[NH + P];
    dcd = acc[NH + P + 2];
    // weak Gaussian prior in z, pulled into the reduced basis (e_k - e_m)
    float zr[NX], ppm = 0.f, rm = 0.f;
#pragma unroll
    for (int i = 0; i < NX; i++) {
      zr[i] = c.hi1[i] > c.lo1[i] ? 2.f * (x[i] - c.lo1[i]) / (c.hi1[i] - c.lo1[i]) - 1.f : 0.f;
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
      for (int bb = a + 1; bb < K - 1; bb++) H[up<P>(a, bb)] += ppm;
    }
#pragma unroll
    for (int a = K - 1; a < P; a++) {
      g[a] -= psc * c.pp1[a + 1] * zr[a + 1];
      H[up<P>(a, a)] += psc * c.pp1[a + 1];
    }
  }

  // prior(x_old) - prior(x_new), formed from differences of z
  __device__ __forceinline__ float prior_drop(const KConfig &c, const float (&xo)[NX],
                                              const float (&xn)[NX]) const {
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < NX; i++) {
      if (c.hi1[i] > c.lo1[i] && c.pp1[i] > 0.f) {
        float k = 2.f / (c.hi1[i] - c.lo1[i]);
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
template <int S2>
struct Stage2 {
  static constexpr int P = 6, NX = 6, NH = 21, NS = S2;
  static constexpr int NB = S2 * 32;   // band slots per buffer
  // this warp's band buffers in shared memory, [4][NB]: y (radiance minus
  // the fixed solar term), tu (tau_up), w (loss weight), r (residual at the
  // current state); lane l owns slots l + 32 s
  float *bb;
  float psc;

  __device__ __forceinline__ float &yb(int i) const { return bb[i]; }
  __device__ __forceinline__ float &tub(int i) const { return bb[NB + i]; }
  __device__ __forceinline__ float &wb(int i) const { return bb[2 * NB + i]; }
  __device__ __forceinline__ float &rb(int i) const { return bb[3 * NB + i]; }

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

  // model, Jacobian (z-scaled), normal equations and cost at x; writes the
  // residuals into the r buffer. All lanes get the warp totals.
  __device__ __forceinline__ void eval(PixCtx &pc, const float (&x)[NX], float (&H)[NH],
                                       float (&g)[P], float &cst, float &cd) const {
    const KTables &t = *pc.t;
    const KConfig &c = *pc.c;
    const float mh = x[0], sh = x[1], ms = x[2], ss = x[3], eta = x[4], al = x[5];
    // grid weights of the two components: lanes own nodes j = lane + 32 q
    float uh[4], us[4], dh[4], ds[4];
    float mom[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float ih = 0.5f / (sh * sh), is = 0.5f / (ss * ss);
    unsigned act[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j = pc.lane + 32 * q;
      uh[q] = us[q] = dh[q] = ds[q] = 0.f;
      if (j < t.nt) {
        float T = t.tglo + (float)j * t.tgstep;
        dh[q] = T - mh;
        ds[q] = T - ms;
        uh[q] = expf(-dh[q] * dh[q] * ih);
        us[q] = expf(-ds[q] * ds[q] * is);
      }
      mom[0] += uh[q];
      mom[1] += uh[q] * dh[q];
      mom[2] += uh[q] * dh[q] * dh[q];
      mom[3] += us[q];
      mom[4] += us[q] * ds[q];
      mom[5] += us[q] * ds[q] * ds[q];
      act[q] = __ballot_sync(kFull, uh[q] > 1e-30f || us[q] > 1e-30f);
    }
    warp_sum(mom);
    const float rUh = 1.f / mom[0], rUs = 1.f / mom[3];
    const float dbh = mom[1] * rUh, m2h = mom[2] * rUh, dbs = mom[4] * rUs, m2s = mom[5] * rUs;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j = pc.lane + 32 * q;
      if (j < t.nt) {
        float wh = uh[q] * rUh, ws = us[q] * rUs;
        float4 A = make_float4(wh, wh * (dh[q] - dbh), wh * (dh[q] * dh[q] - m2h), ws);
        float4 B = make_float4(ws * (ds[q] - dbs), ws * (ds[q] * ds[q] - m2s), 0.f, 0.f);
        reinterpret_cast<float4 *>(pc.wsc)[2 * j] = A;
        reinterpret_cast<float4 *>(pc.wsc)[2 * j + 1] = B;
      }
    }
    int jlo = t.nt, jhi = -1;
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (act[q]) {
        jlo = min(jlo, 32 * q + __ffs(act[q]) - 1);
        jhi = max(jhi, 32 * q + 31 - __clz(act[q]));
      }
    __syncwarp();
    // moment sums over the active nodes: 6 FMA per band and node
    float S[S2][6];
#pragma unroll
    for (int s2 = 0; s2 < S2; s2++)
#pragma unroll
      for (int k = 0; k < 6; k++) S[s2][k] = 0.f;
    const float *pl = pc.img + t.lay.off_planck + pc.lane;
    const float4 *wv4 = reinterpret_cast<const float4 *>(pc.wsc);
    for (int j = jlo; j <= jhi; j++) {
      float4 A = wv4[2 * j], B = wv4[2 * j + 1];
      const float *row = pl + j * t.lay.n2s;
#pragma unroll
      for (int s2 = 0; s2 < S2; s2++) {
        float Bv = row[32 * s2];
        S[s2][0] = fmaf(A.x, Bv, S[s2][0]);
        S[s2][1] = fmaf(A.y, Bv, S[s2][1]);
        S[s2][2] = fmaf(A.z, Bv, S[s2][2]);
        S[s2][3] = fmaf(A.w, Bv, S[s2][3]);
        S[s2][4] = fmaf(B.x, Bv, S[s2][4]);
        S[s2][5] = fmaf(B.y, Bv, S[s2][5]);
      }
    }
    pc.node_evals += (jhi >= jlo) ? (jhi - jlo + 1) : 0;
    float acc[NH + P + 2];
#pragma unroll
    for (int i = 0; i < NH + P + 2; i++) acc[i] = 0.f;
    const float ish2 = 1.f / (sh * sh), iss2 = 1.f / (ss * ss);
    const float ish3 = ish2 / sh, iss3 = iss2 / ss;
    const float sc0 = scale(c, 0), sc1 = scale(c, 1), sc2 = scale(c, 2), sc3 = scale(c, 3);
    const float sc4 = scale(c, 4), sc5 = scale(c, 5);
#pragma unroll
    for (int s2 = 0; s2 < S2; s2++) {
      const int i = pc.lane + 32 * s2;
      const float wv = wb(i);
      if (wv > 0.f) {
        float Bh = S[s2][0], Bs = S[s2][3];
        float Bm = eta * Bh + (1.f - eta) * Bs;
        float tuv = tub(i);
        float atu = al * tuv;
        float r = yb(i) - atu * Bm;
        rb(i) = r;
        float J[6];
        J[0] = atu * eta * S[s2][1] * ish2 * sc0;
        J[1] = atu * eta * S[s2][2] * ish3 * sc1;
        J[2] = atu * (1.f - eta) * S[s2][4] * iss2 * sc2;
        J[3] = atu * (1.f - eta) * S[s2][5] * iss3 * sc3;
        J[4] = atu * (Bh - Bs) * sc4;
        J[5] = tuv * Bm * sc5;
        float wr = wv * r;
        acc[NH + P] = fmaf(wr, r, acc[NH + P]);
        acc[NH + P + 1] = fmaf(r, r, acc[NH + P + 1]);
#pragma unroll
        for (int a = 0; a < P; a++) {
          acc[NH + a] = fmaf(J[a], wr, acc[NH + a]);
          float wj = wv * J[a];
#pragma unroll
          for (int bb_ = a; bb_ < P; bb_++) acc[up<P>(a, bb_)] = fmaf(wj, J[bb_], acc[up<P>(a, bb_)]);
        }
      } else {
        rb(i) = 0.f;
      }
    }
    warp_sum(acc);
#pragma unroll
    for (int i = 0; i < NH; i++) H[i] = acc[i];
#pragma unroll
    for (int a = 0; a < P; a++) g[a] = acc[NH + a];
    cst = acc[NH + P];
    cd = acc[NH + P + 1];
#pragma unroll
    for (int i = 0; i < 6; i++) {
      float z = c.hi2[i] > c.lo2[i] ? 2.f * (x[i] - c.lo2[i]) / (c.hi2[i] - c.lo2[i]) - 1.f : 0.f;
      float pp = psc * c.pp2[i];
      cst += pp * (z - c.pm2[i]) * (z - c.pm2[i]);
      g[i] -= pp * (z - c.pm2[i]);
      H[up<P>(i, i)] += pp;
    }
    __syncwarp();
  }

  // Gaussian weight u_o = exp(-a_o^2/2), a = (T - mu)/sigma, of one node at
  // the current state and its change du under the step (dmu, dsig): the
  // exponent change is formed from the parameter differences,
  //   a_t - a_o = -(dmu sigma_o + (T - mu_o) dsig) / (sigma_t sigma_o),
  // and du = u_o expm1(-dq), so du is resolved relative to itself.
  __device__ __forceinline__ static void node_step(float T, float mu, float isg, float mut, float isgt,
                                                   float dmu, float dsg, float &u, float &du) {
    const float ao = (T - mu) * isg, at = (T - mut) * isgt;
    const float da = -fmaf((T - mu) * dsg, isg, dmu) * isgt;
    const float dq = 0.5f * da * (at + ao);
    u = expf(-0.5f * ao * ao);
    du = fabsf(dq) < 0.5f ? u * expm1f(-dq) : expf(-0.5f * at * at) - u;
  }

  // Data-term decrease of the trial step x -> xt, sum_b w_b dM_b (2 r_b -
  // dM_b) with r the residuals at x and dM_b = tu_b (a_t dBm_b + (a_t - a)
  // Bm_b) the model increment: Bm and dBm are the node sums of the current
  // mixture weights and of their increments (the weight differences formed
  // node by node from the exact parameter differences). The decrease is then
  // accurate relative to itself, where the difference of two FP32 costs (or
  // of two FP32 model values) would be lost below the model's rounding.
  // 2 FMA per band and node.
  __device__ __forceinline__ float trial_drop(PixCtx &pc, const float (&x)[NX],
                                              const float (&xt)[NX], bool r_is_y = false) const {
    const KTables &t = *pc.t;
    const float eo = x[4], ao = x[5], et = xt[4], at = xt[5];
    float uho[4], uso[4], duh[4], dus[4];
    float U[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned act[4];
    const float ih = 1.f / x[1], iht = 1.f / xt[1], is = 1.f / x[3], ist = 1.f / xt[3];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j = pc.lane + 32 * q;
      uho[q] = uso[q] = duh[q] = dus[q] = 0.f;
      if (j < t.nt) {
        float T = t.tglo + (float)j * t.tgstep;
        node_step(T, x[0], ih, xt[0], iht, xt[0] - x[0], xt[1] - x[1], uho[q], duh[q]);
        node_step(T, x[2], is, xt[2], ist, xt[2] - x[2], xt[3] - x[3], uso[q], dus[q]);
      }
      U[0] += uho[q];
      U[1] += duh[q];
      U[2] += uso[q];
      U[3] += dus[q];
      act[q] = __ballot_sync(kFull, uho[q] > 1e-30f || uso[q] > 1e-30f || uho[q] + duh[q] > 1e-30f ||
                                        uso[q] + dus[q] > 1e-30f);
    }
    warp_sum(U);
    const float rho_ = 1.f / U[0], rso = 1.f / U[2];
    const float rht = 1.f / (U[0] + U[1]), rst = 1.f / (U[2] + U[3]);
    const float kh = U[1] * rho_, ks = U[3] * rso;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j = pc.lane + 32 * q;
      if (j < t.nt) {
        // w_t - w_o = (du - u_o dU/U_o) / U_t per component
        float who = uho[q] * rho_, wso = uso[q] * rso;
        float dwh = (duh[q] - uho[q] * kh) * rht, dws = (dus[q] - uso[q] * ks) * rst;
        float Wo = eo * who + (1.f - eo) * wso;
        float dW = et * dwh + (1.f - et) * dws + (et - eo) * (who - wso);
        reinterpret_cast<float2 *>(pc.wsc)[4 * j] = make_float2(Wo, dW);
      }
    }
    int jlo = t.nt, jhi = -1;
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (act[q]) {
        jlo = min(jlo, 32 * q + __ffs(act[q]) - 1);
        jhi = max(jhi, 32 * q + 31 - __clz(act[q]));
      }
    __syncwarp();
    float Bo[S2], dB[S2];
#pragma unroll
    for (int s2 = 0; s2 < S2; s2++) Bo[s2] = dB[s2] = 0.f;
    const float *pl = pc.img + t.lay.off_planck + pc.lane;
    const float2 *wv2 = reinterpret_cast<const float2 *>(pc.wsc);
    for (int j = jlo; j <= jhi; j++) {
      float2 A = wv2[4 * j];
      const float *row = pl + j * t.lay.n2s;
#pragma unroll
      for (int s2 = 0; s2 < S2; s2++) {
        float Bv = row[32 * s2];
        Bo[s2] = fmaf(A.x, Bv, Bo[s2]);
        dB[s2] = fmaf(A.y, Bv, dB[s2]);
      }
    }
    pc.trial_nodes += (jhi >= jlo) ? (jhi - jlo + 1) : 0;
    float d = 0.f;
    const float da_ = at - ao;
#pragma unroll
    for (int s2 = 0; s2 < S2; s2++) {
      const int i = pc.lane + 32 * s2;
      const float wv = wb(i);
      if (wv > 0.f) {
        float dM = tub(i) * fmaf(at, dB[s2], da_ * Bo[s2]);
        float r = r_is_y ? yb(i) : rb(i);
        d = fmaf(wv * dM, 2.f * r - dM, d);
      }
    }
    __syncwarp();
    return warp_sum1(d);
  }

  __device__ __forceinline__ float prior_drop(const KConfig &c, const float (&xo)[NX],
                                              const float (&xn)[NX]) const {
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) {
      if (c.hi2[i] > c.lo2[i] && c.pp2[i] > 0.f) {
        float k = 2.f / (c.hi2[i] - c.lo2[i]);
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

// -------------------------------------------------------- LM driver -----
struct LMResult {
  int iters, full, status;   // trial steps; full model + Jacobian evaluations
  bool used64;
  float cost, cdata;
};

// FP64 re-solve of an ill-conditioned step, kept out of line (cold path) so
// the hot loop stays small in the instruction cache.
template <int P>
struct Solve64 {
  float H[P * (P + 1) / 2], g[P], D[P], dr[P];
  bool pin[P];
  float lam, kap;
};

template <int P>
__device__ __noinline__ bool solve_fp64(Solve64<P> &q) {
  return damped_solve<P, double>(q.H, q.g, q.lam, q.D, q.pin, q.dr, q.kap);
}

// One stage of the fit. The model is evaluated at a single call site per
// stage (start point, then every trial point) to keep the code compact.
// State of the damped iteration shared by the two stage drivers.
template <int P>
struct LMIter {
  float lam = -1.f, nu = 2.f, pred = 0.f;
  int it = 0, status = PX_MAXITER;
  bool fresh = true, used64 = false;
  bool act[P];
};

// From the normal equations (H, g) at the current state x: the convergence
// test (when they are fresh), then the damped projected-Newton step and the
// trial point xt with its predicted decrease. Returns false when the fit
// stops (converged, step below tol_x, damping overflow, iteration cap).
template <class St>
__device__ __forceinline__ bool next_trial(const St &S, const KConfig &c, const float (&x)[St::NX],
                                           const float (&H)[St::NH], const float (&g)[St::P], int m,
                                           float cst, int max_it, LMIter<St::P> &L,
                                           float (&xt)[St::NX]) {
  constexpr int P = St::P, NX = St::NX;
#pragma unroll 1
  while (L.it < max_it) {
    if (L.fresh) {
      bool small = true;
      float mx = 0.f;
      static_for<P>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        float xv = St::template rsel<a>(x, m);
        bool lo_hit = xv <= S.template lo_r<a>(c, m);
        bool hi_hit = St::template has_upper<a>() && xv >= S.template hi_r<a>(c, m);
        L.act[a] = (lo_hit && g[a] <= 0.f) || (hi_hit && g[a] >= 0.f);
        float haa = H[up<P>(a, a)];
        if (!L.act[a]) {
          if (fabsf(g[a]) > c.tol_g * sqrtf(haa * cst)) small = false;
          mx = fmaxf(mx, haa);
        }
      });
      if (small) { L.status = PX_CONVERGED; return false; }
      if (L.lam < 0.f) L.lam = c.tau0 * mx;
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
      ok = damped_solve<P, float>(H, g, L.lam, D, pin, dr, kap);
      if (!ok || !(kap <= c.kappa_max)) {
        Solve64<P> q;
#pragma unroll
        for (int i = 0; i < St::NH; i++) q.H[i] = H[i];
#pragma unroll
        for (int a = 0; a < P; a++) {
          q.g[a] = g[a];
          q.D[a] = D[a];
          q.pin[a] = pin[a];
          q.dr[a] = dr[a];
        }
        q.lam = L.lam;
        ok = solve_fp64<P>(q);
#pragma unroll
        for (int a = 0; a < P; a++) dr[a] = q.dr[a];
        L.used64 = true;
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
      float sc = S.scale(c, i);
      Dz[i] = sc > 0.f ? (xt[i] - x[i]) / sc : 0.f;
      dmax = fmaxf(dmax, fabsf(Dz[i]));
    }
    if (dmax < c.tol_x) { L.status = PX_CONVERGED; return false; }
    float Dr[P];
    static_for<P>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      Dr[a] = St::template rsel<a>(Dz, m);
    });
    // predicted decrease of the Gauss-Newton model: 2 g.D - D.H.D
    float pred = 0.f;
#pragma unroll
    for (int a = 0; a < P; a++) {
      pred += 2.f * g[a] * Dr[a];
#pragma unroll
      for (int b = 0; b < P; b++) pred -= Dr[a] * H[up<P>(a, b)] * Dr[b];
    }
    L.pred = pred;
    L.it++;
    return true;
  }
  return false;
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

// Stage-1 driver: every trial point is evaluated in full (model, Jacobian,
// normal equations); the decrease comes from residual differences.
template <class St>
__device__ __forceinline__ void lm_fit(const St &S, PixCtx &pc, float (&x)[St::NX], int max_it,
                                       float (&H)[St::NH], float (&g)[St::P], int &m,
                                       LMResult &res) {
  constexpr int P = St::P, NX = St::NX, NH = St::NH, NS = St::NS;
  const KConfig &c = *pc.c;
  float cst = 0.f, cd = 0.f;
  float r[NS], rt[NS], xt[NX];
#pragma unroll
  for (int i = 0; i < NS; i++) r[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NX; i++) xt[i] = x[i];
  LMIter<P> L;
  int nfull = 0;
  bool first = true;
#pragma unroll
  for (int a = 0; a < P; a++) L.act[a] = false;
#pragma unroll 1
  for (;;) {
    float Ht[NH], gt[P], ct, cdt, dct;
    int mt;
    S.eval(pc, xt, Ht, gt, ct, cdt, mt, r, rt, dct);
    nfull++;
    bool accept = first, done = false;
    float rel = 1.f, rho = 1.f;
    if (!first) {
      // actual decrease from residual differences (accurate where cost - ct
      // would cancel in FP32) against the Gauss-Newton prediction
      const float drop = dct + S.prior_drop(c, x, xt);
      rho = L.pred > 0.f ? drop / L.pred : -1.f;
      accept = rho > 0.f;
      rel = drop / cst;
    }
    if (accept) {
#pragma unroll
      for (int i = 0; i < NS; i++) r[i] = rt[i];
#pragma unroll
      for (int i = 0; i < NX; i++) x[i] = xt[i];
#pragma unroll
      for (int i = 0; i < NH; i++) H[i] = Ht[i];
#pragma unroll
      for (int a = 0; a < P; a++) g[a] = gt[a];
      cst = ct;
      cd = cdt;
      m = mt;
      if (!first && rel < c.tol_f) { L.status = PX_CONVERGED; done = true; }
    }
    if (!first) damping_update(L, accept, rho);
    first = false;
    if (done) break;
    if (!next_trial(S, c, x, H, g, m, cst, max_it, L, xt)) break;
  }
  res.iters = L.it;
  res.full = nfull;
  res.status = L.status;
  res.used64 = L.used64;
  res.cost = cst;
  res.cdata = cd;
}

// Stage-2 driver: a trial point is judged by the decrease-only evaluation
// in increment form; the full evaluation runs only at accepted points and
// writes the new state's normal equations and residuals in place.
template <class St>
__device__ __forceinline__ void lm_fit2(const St &S, PixCtx &pc, float (&x)[St::NX], int max_it,
                                        float (&H)[St::NH], float (&g)[St::P], LMResult &res) {
  constexpr int P = St::P, NX = St::NX;
  const KConfig &c = *pc.c;
  float cst = 0.f, cd = 0.f, xt[NX];
  LMIter<P> L;
#pragma unroll
  for (int a = 0; a < P; a++) L.act[a] = false;
  S.eval(pc, x, H, g, cst, cd);
  int nfull = 1;
#pragma unroll 1
  while (next_trial(S, c, x, H, g, 0, cst, max_it, L, xt)) {
    const float drop = S.trial_drop(pc, x, xt) + S.prior_drop(c, x, xt);
    const float rho = L.pred > 0.f ? drop / L.pred : -1.f;
    const bool accept = rho > 0.f;
    damping_update(L, accept, rho);
    if (accept) {
      const float rel = drop / cst;   // relative to the cost before the step
#pragma unroll
      for (int i = 0; i < NX; i++) x[i] = xt[i];
      S.eval(pc, x, H, g, cst, cd);
      nfull++;
      if (rel < c.tol_f) { L.status = PX_CONVERGED; break; }
    }
  }
  res.iters = L.it;
  res.full = nfull;
  res.status = L.status;
  res.used64 = L.used64;
  res.cost = cst;
  res.cdata = cd;
}

// -------------------------------------------- final covariance (FP64) ---
// C = s2 (H_FF)^-1 over the free stage-2 variables (not on an outward-
// pressed bound, non-zero diagonal), in physical units; writes the packed
// upper triangle and returns var(E[T]) and var(alpha). FP64 throughout,
// division-free: Jacobi scaling and the Cholesky pivots use Newton-refined
// reciprocal square roots, and C = L^-T L^-1 from the triangular inverse.
struct CovIO {
  float x[6], H[21], g[6], s2;
  float cov[21];
  bool cov_ok;
  double vE, va;
};

__device__ __noinline__ void laplace_cov(const KConfig &c, CovIO &io) {
  const float (&x)[6] = io.x;
  const float (&H)[21] = io.H;
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
    zc[k] = !act && !(H[up<6>(k, k)] > 0.f);
    fix[k] = act || zc[k];
  }
  double A[21], rd[6], il[6];
#pragma unroll
  for (int i = 0; i < 6; i++) rd[i] = fix[i] ? 1.0 : rsq((double)H[up<6>(i, i)]);
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = 0; j <= i; j++)
      A[i * (i + 1) / 2 + j] = (fix[i] || fix[j]) ? (i == j ? 1.0 : 0.0)
                                                   : (double)H[up<6>(i, j)] * rd[i] * rd[j];
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

// ------------------------------------------------------------ kernels ---
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Stage the per-CTA table image into shared memory with 1D bulk copies
// completing on one mbarrier. The wait is bounded: on timeout the error flag
// is set, the copies still in flight are waited for (bounded again) and the
// CTA leaves (returns false).
__device__ __forceinline__ bool stage_tables(const KTables &t, float *smem, unsigned long long *bar,
                                             int *err) {
  const unsigned bytes = (unsigned)t.lay.total * 4u;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    const unsigned chunk = 32768u;
    for (unsigned off = 0; off < bytes; off += chunk) {
      unsigned n = bytes - off < chunk ? bytes - off : chunk;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(smem_u32(reinterpret_cast<char *>(smem) + off)),
          "l"(reinterpret_cast<const char *>(t.image) + off), "r"(n), "r"(smem_u32(bar))
          : "memory");
    }
  }
  __syncthreads();
  unsigned done = 0;
  for (long long spin = 0; spin < (1ll << 26) && !done; spin++)
    asm volatile(
        "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0; selp.u32 %0, 1, 0, P; }"
        : "=r"(done) : "r"(smem_u32(bar)) : "memory");
  if (__syncthreads_and(done)) return true;
  if (threadIdx.x == 0) atomicExch(err, 1);
  for (long long spin = 0; spin < (1ll << 26) && !done; spin++)
    asm volatile(
        "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0; selp.u32 %0, 1, 0, P; }"
        : "=r"(done) : "r"(smem_u32(bar)) : "memory");
  return false;
}

// pixel-claim helper: lane 0 takes n pixels from a global counter
__device__ __forceinline__ long long claim(unsigned long long *ctr, int lane, int n) {
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(ctr, (unsigned long long)n);
  return (long long)__shfl_sync(kFull, base, 0);
}

// stage-1 per-pixel setup: radiance, mask m(lambda) (saturation) x window,
// weights and the prior scale (mean noise variance of the used bands)
template <int K, int S1>
__device__ __forceinline__ int setup1(Stage1<K, S1> &s1, const PixCtx &pc, const float *row) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0;
#pragma unroll
  for (int s = 0; s < S1; s++) {
    int bi = pc.lane + 32 * s;
    s1.Lobs[s] = 0.f;
    s1.w[s] = 0.f;
    if (bi < t.n1) {
      int b = t.b1lo + bi;
      float L = __ldg(row + b);
      bool ok = pc.img[t.lay.off_win1 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      s1.Lobs[s] = L;
      s1.w[s] = ok ? (c.weighted ? 1.f / var : 1.f) : 0.f;
      if (ok) { nv += var; nu++; }
    }
  }
  nv = warp_sum1(nv);
  nu = __reduce_add_sync(kFull, nu);
  s1.psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  s1.sf = 0.5f * (c.hi1[0] - c.lo1[0]);
  s1.sa = 0.5f * (c.hi1[K] - c.lo1[K]);
  s1.sT = 0.5f * (c.hi1[K + 1] - c.lo1[K + 1]);
  return nu;
}

// stage-2 band count (mask x window) without building the stage state
__device__ __forceinline__ int count2(const PixCtx &pc, const float *row) {
  const KTables &t = *pc.t;
  int nu = 0;
  for (int bi = pc.lane; bi < t.n2; bi += 32) {
    int b = t.b2lo + bi;
    float L = __ldg(row + b);
    nu += (pc.img[t.lay.off_win2 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b))) ? 1 : 0;
  }
  return __reduce_add_sync(kFull, nu);
}

// stage-2 per-pixel setup: y = L - Ls(x_surf) (solar term fixed, Eq. solar),
// tau_up, weights, prior scale
template <int K, int S2>
__device__ __forceinline__ int setup2(Stage2<S2> &s2, const PixCtx &pc, const float *row,
                                      const float (&xs)[K]) {
  const KTables &t = *pc.t;
  const KConfig &c = *pc.c;
  float nv = 0.f;
  int nu = 0;
#pragma unroll
  for (int s = 0; s < S2; s++) {
    int bi = pc.lane + 32 * s;
    float yv = 0.f, tv = 0.f, wv = 0.f;
    if (bi < t.n2) {
      int b = t.b2lo + bi;
      float L = __ldg(row + b);
      bool ok = pc.img[t.lay.off_win2 + b] > 0.f && !(t.sat && L >= __ldg(t.sat + b));
      float var = c.noise_rel * c.noise_rel * L * L + c.noise_abs * c.noise_abs;
      float4 q = __ldg(pc.wvrow + b);
      float rho = 0.f;
#pragma unroll
      for (int k = 0; k < K; k++) rho = fmaf(xs[k], pc.img[t.lay.off_endm + k * t.nb + b], rho);
      yv = L - (q.y + q.x * rho / (1.f - q.z * rho));
      tv = q.w;
      wv = ok ? (c.weighted ? 1.f / var : 1.f) : 0.f;
      if (ok) { nv += var; nu++; }
    }
    s2.yb(bi) = yv;
    s2.tub(bi) = tv;
    s2.wb(bi) = wv;
    s2.rb(bi) = yv;
  }
  __syncwarp();
  nv = warp_sum1(nv);
  nu = __reduce_add_sync(kFull, nu);
  s2.psc = c.weighted ? 1.f : nv / (float)max(nu, 1);
  return nu;
}

__device__ __forceinline__ void flush_stats(unsigned long long *cstat, const unsigned long long *mine,
                                            unsigned long long *gstats, int lane) {
  if (lane == 0)
    for (int i = 0; i < ST_COUNT; i++)
      if (mine[i]) atomicAdd(&cstat[i], mine[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(gstats + i, cstat[i]);
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
  r.opix = loc;
  return r;
}

constexpr int kFitted = 256;   // scratch flag: pixel goes on to stage 2
constexpr int kS2Hand = 32;    // floats handed from stage 2 to finalize per pixel

// ---- stage 1: checks, HFDI gate, stage-1 fit -> scratch
template <int K, int S1, int WPB, int MINB>
__global__ void __launch_bounds__(WPB * 32, MINB) lm_stage1_kernel(const __grid_constant__ LMLaunch p) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned long long cstat[ST_COUNT];
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  if (!stage_tables(t, smem, &bar, p.w.err)) return;
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  pc.wsc = smem + t.lay.total + warp * warp_scratch_floats(t);
  pc.lane = lane;
  const int NSx = K + 8;
  unsigned long long mine[ST_COUNT];
#pragma unroll
  for (int i = 0; i < ST_COUNT; i++) mine[i] = 0ull;
  const int nclaim = p.s.claim > 0 ? p.s.claim : kClaim;
  for (;;) {
    const long long base = claim(p.w.counter, lane, nclaim);
    if (base >= p.s.n_pix) break;
    for (int ci = 0; ci < nclaim; ci++) {
      const long long pix = base + ci;
      if (pix >= p.s.n_pix) break;
      const PixRef ref = resolve(p, pix, K);
      const float *row = ref.row;
      const int wvb = ref.wv;
      const bool wv_ok = wvb < t.nwv;   // an out-of-range bin is an invalid input
      pc.wvrow = t.wvtab + (size_t)(wv_ok ? wvb : 0) * t.nb;
      bool fin = true;
      for (int b = lane; b < t.nb; b += 32) fin = fin && isfinite(__ldg(row + b));
      fin = __all_sync(kFull, fin) && wv_ok;
      const float Lh = __ldg(row + t.bh), Ll = __ldg(row + t.bl);
      float hf = (Lh - Ll) / (Lh + Ll);
      int status = 0, it1 = 0;
      bool fitted = false;
      float x1[K + 2];
      if (!fin) {
        status = PX_NONFINITE;
        hf = __int_as_float(0x7fc00000);
      } else if (p.s.gate && !(hf >= c.hfdi_thresh)) {
        status = PX_NOT_CANDIDATE;
      } else {
        Stage1<K, S1> s1;
        const int n1u = setup1(s1, pc, row);
        const int n2u = count2(pc, row);
        if (n1u <= K + 2 || n2u <= 6) {
          status = PX_ALL_MASKED;
        } else {
          const float *ini = ref.init;
          if (ini) {
#pragma unroll
            for (int i = 0; i < K + 2; i++) x1[i] = ini[i];
            Stage1<K, S1>::simplex_project(x1);
#pragma unroll
            for (int i = K; i < K + 2; i++) x1[i] = fminf(fmaxf(x1[i], c.lo1[i]), c.hi1[i]);
          } else {
#pragma unroll
            for (int k = 0; k < K; k++) x1[k] = 1.f / (float)K;
            x1[K] = c.init_alpha1;
            x1[K + 1] = c.init_T1;
          }
          float H1[Stage1<K, S1>::NH], g1[K + 1];
          int m1;
          LMResult r1;
          lm_fit(s1, pc, x1, c.max_it1, H1, g1, m1, r1);
          it1 = r1.iters;
          if (r1.status == PX_MAXITER) status |= PX_F_S1_MAXITER;
          if (r1.used64) status |= PX_F_FP64;
          mine[ST_BAND1] += (unsigned long long)r1.full * (unsigned long long)t.n1;
          mine[ST_IT1] += it1;
          fitted = true;
        }
      }
      // hand-over to stage 2, or the final outputs of a pixel that is not fitted
      const KOut &o = ref.o;
      const long long op = ref.opix;
      if (lane == 0) {
        p.w.s1meta[pix] = status | (fitted ? kFitted : 0);
        if (o.hfdi) o.hfdi[op] = hf;
        if (o.iters) o.iters[2 * op] = (uint16_t)it1;
      }
      if (fitted) {
        if (lane < K + 2) {
          float v = x1[0];
#pragma unroll
          for (int k = 0; k < K + 2; k++) v = (k == lane) ? x1[k] : v;
          p.w.s1x[pix * (K + 2) + lane] = v;
        }
      } else {
        const float nan = __int_as_float(0x7fc00000);
        if (o.state)
          for (int i = lane; i < NSx; i += 32) o.state[op * NSx + i] = nan;
        if (o.cov && lane < 21) o.cov[op * 21 + lane] = nan;
        if (lane == 0) {
          if (o.ET) o.ET[op] = nan;
          if (o.sdT) o.sdT[op] = nan;
          if (o.alpha) o.alpha[op] = nan;
          if (o.var_ET) o.var_ET[op] = nan;
          if (o.cost) o.cost[op] = nan;
          if (o.rms) o.rms[op] = nan;
          if (o.status) o.status[op] = (uint8_t)status;
          if (o.iters) o.iters[2 * op + 1] = 0;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) mine[ST_STATUS0 + k] += ((status & 7) == k) ? 1ull : 0ull;
      }
      mine[ST_NPIX] += 1;
    }
  }
  flush_stats(cstat, mine, p.w.stats, lane);
}

// ---- stage 2: mixture fit from the stage-1 hand-over, covariance, outputs
template <int K, int S2, int WPB>
__global__ void __launch_bounds__(WPB * 32, 1) lm_stage2_kernel(const __grid_constant__ LMLaunch p) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned long long cstat[ST_COUNT];
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  if (!stage_tables(t, smem, &bar, p.w.err)) return;
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  pc.wsc = smem + t.lay.total + warp * warp_scratch_floats(t);
  pc.lane = lane;
  unsigned long long mine[ST_COUNT];
#pragma unroll
  for (int i = 0; i < ST_COUNT; i++) mine[i] = 0ull;
  const int nclaim = p.s.claim > 0 ? p.s.claim : kClaim;
  for (;;) {
    const long long base = claim(p.w.counter + 1, lane, nclaim);
    if (base >= p.s.n_pix) break;
    for (int ci = 0; ci < nclaim; ci++) {
      const long long pix = base + ci;
      if (pix >= p.s.n_pix) break;
      const int meta = p.w.s1meta[pix];
      if (!(meta & kFitted)) continue;
      int status = meta & 0xff;
      const PixRef ref = resolve(p, pix, K);
      const float *row = ref.row;
      pc.wvrow = t.wvtab + (size_t)ref.wv * t.nb;
      pc.node_evals = 0;
      pc.trial_nodes = 0;
      float x1[K + 2];
#pragma unroll
      for (int i = 0; i < K + 2; i++) x1[i] = p.w.s1x[pix * (K + 2) + i];
      float xs[K];
#pragma unroll
      for (int k = 0; k < K; k++) xs[k] = x1[k];
      Stage2<S2> s2;
      s2.bb = pc.wsc + t.nt * kScratchPerNode;
      const int n2u = setup2<K, S2>(s2, pc, row, xs);
      float x2[6];
      const float *ini = ref.init;
      if (ini) {
#pragma unroll
        for (int i = 0; i < 6; i++) x2[i] = fminf(fmaxf(ini[K + 2 + i], c.lo2[i]), c.hi2[i]);
      }
      if (!ini || p.s.init_best) {
        float xd[6];
        float T1 = x1[K + 1];
        xd[0] = fminf(fmaxf(fmaxf(T1, c.init_mu_h_floor), c.lo2[0]), c.hi2[0]);
        xd[2] = fminf(fmaxf(fminf(T1, c.init_mu_s_ceil), c.lo2[2]), c.hi2[2]);
        xd[1] = fminf(fmaxf(c.init_sigma, c.lo2[1]), c.hi2[1]);
        xd[3] = fminf(fmaxf(c.init_sigma, c.lo2[3]), c.hi2[3]);
        xd[5] = fminf(fmaxf(x1[K], c.lo2[5]), c.hi2[5]);
        float e = xd[0] > xd[2] ? (T1 - xd[2]) / (xd[0] - xd[2]) : 0.5f;
        xd[4] = fminf(fmaxf(e, c.init_eta_lo), c.init_eta_hi);
        bool take_d = !ini;
        if (ini) {
          // cost(xd) - cost(x2) from the data-term decreases of both starts
          // against the thermal-free model (residuals y), plus the prior
          float z2[6], zd[6];
#pragma unroll
          for (int i = 0; i < 6; i++) {
            z2[i] = x2[i];
            zd[i] = xd[i];
          }
          z2[5] = 0.f;
          zd[5] = 0.f;
          const float Dp = s2.trial_drop(pc, z2, x2, true), Dd = s2.trial_drop(pc, zd, xd, true);
          take_d = !(Dp - Dd + s2.prior_drop(c, xd, x2) > 0.f);
        }
        if (take_d) {
#pragma unroll
          for (int i = 0; i < 6; i++) x2[i] = xd[i];
        }
      }
      float H2[21], g2[6];
      LMResult r2;
      lm_fit2(s2, pc, x2, c.max_it2, H2, g2, r2);
      if (r2.used64) status |= PX_F_FP64;
      status |= r2.status;
      mine[ST_IT2] += r2.iters;
      mine[ST_BAND2] += (unsigned long long)r2.full * (unsigned long long)t.n2;
      mine[ST_NODEBAND2] += (unsigned long long)pc.node_evals * (unsigned long long)t.n2;
      mine[ST_TRIAL2] += (unsigned long long)r2.iters * (unsigned long long)t.n2;
      mine[ST_TRIALNODE2] += (unsigned long long)pc.trial_nodes * (unsigned long long)t.n2;
      // hand the final state and normal equations to the finalize kernel
      float* hand = p.w.s2x + pix * kS2Hand;
      {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < 6; k++) v = (lane == k) ? x2[k] : v;
#pragma unroll
        for (int k = 0; k < 21; k++) v = (lane == 6 + k) ? H2[k] : v;
        v = (lane == 27) ? r2.cost : v;
        v = (lane == 28) ? r2.cdata : v;
        v = (lane == 29) ? __int_as_float(n2u) : v;
        v = (lane == 30) ? __int_as_float(status | (r2.iters << 8)) : v;
        v = (lane == 31) ? s2.psc : v;
        hand[lane] = v;
      }
      if (lane < 6) {
        float v = g2[0];
#pragma unroll
        for (int k = 0; k < 6; k++) v = (lane == k) ? g2[k] : v;
        p.w.s2g[pix * 6 + lane] = v;
      }
    }
  }
  flush_stats(cstat, mine, p.w.stats, lane);
}

// ---- finalize: moment matching (Sec. 2.3), FP64 Laplace covariance,
// identifiability and the outputs of every fitted pixel; one thread per
// pixel, so the FP64 work is not repeated across the lanes of a warp
__global__ void __launch_bounds__(128) finalize_kernel(const __grid_constant__ LMLaunch p, int K) {
  __shared__ unsigned long long cstat[ST_COUNT];
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) cstat[i] = 0ull;
  __syncthreads();
  const KConfig &c = p.c;
  const int NSx = K + 8;
  unsigned long long st_fp64 = 0, st_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < p.s.n_pix;
       pix += (long long)gridDim.x * blockDim.x) {
    if (!(p.w.s1meta[pix] & kFitted)) continue;
    const float *hand = p.w.s2x + pix * kS2Hand;
    CovIO io;
#pragma unroll
    for (int k = 0; k < 6; k++) { io.x[k] = hand[k]; io.g[k] = p.w.s2g[pix * 6 + k]; }
#pragma unroll
    for (int k = 0; k < 21; k++) io.H[k] = hand[6 + k];
    const float cost = hand[27], cdata = hand[28];
    const int n2u = __float_as_int(hand[29]), sw = __float_as_int(hand[30]);
    int status = sw & 0xff;
    const int it2 = sw >> 8;
    const float *x2 = io.x;
    const float ET = x2[4] * x2[0] + (1.f - x2[4]) * x2[2];
    const float dmu = x2[0] - x2[2];
    const float sdT = sqrtf(x2[4] * x2[1] * x2[1] + (1.f - x2[4]) * x2[3] * x2[3] +
                            x2[4] * (1.f - x2[4]) * dmu * dmu);
    const float rms = sqrtf(cdata / (float)n2u);
    int nf = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      bool act = (x2[k] <= c.lo2[k] && io.g[k] <= 0.f) || (x2[k] >= c.hi2[k] && io.g[k] >= 0.f);
      nf += (!act && io.H[up<6>(k, k)] > 0.f);
    }
    io.s2 = c.weighted ? 1.f : cost / (float)(n2u - nf);
    const bool act_a = (x2[5] <= c.lo2[5] && io.g[5] <= 0.f) || (x2[5] >= c.hi2[5] && io.g[5] >= 0.f);
    if (act_a && x2[5] <= c.lo2[5]) {
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
    const double sdE = sqrt(io.vE), sda = sqrt(io.va);
    const bool ident = io.cov_ok && isfinite(sdE) && sdE <= (double)c.ident_sd_et &&
                       (double)x2[5] >= (double)c.ident_alpha_snr * sda && !act_a && x2[5] > 0.f;
    if (!ident) status |= PX_F_NOT_IDENT;
    if (p.w.fb_idx) {
      // fallback rule of the learned start: the fit did not converge, or its
      // cost exceeds three times the expected chi-square (n_used - 6) psc
      const float psc = hand[31];
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
  // warp-aggregate, then one shared atomic per warp and counter
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    st_fp64 += __shfl_xor_sync(kFull, st_fp64, o);
#pragma unroll
    for (int k = 0; k < 8; k++) st_s[k] += __shfl_xor_sync(kFull, st_s[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (st_fp64) atomicAdd(&cstat[ST_FP64], st_fp64);
    for (int k = 0; k < 8; k++)
      if (st_s[k]) atomicAdd(&cstat[ST_STATUS0 + k], st_s[k]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
    if (cstat[i]) atomicAdd(p.w.stats + i, cstat[i]);
}

// ---- keep the lower-cost of the learned-start fit and the default-start
// re-fit of each flagged pixel; both get the MLP_FALLBACK flag
__global__ void merge_fallback_kernel(const long long *idx, const float *cost_first, long long nfb,
                                      KOut compact, KOut out, int K) {
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
    }
    if (out.status)
      out.status[pix] = (uint8_t)((take ? compact.status[j] : out.status[pix]) | PX_F_MLP_FALLBACK);
  }
}

// ---- one evaluation of a stage's normal equations per state (test hook)
template <int K, int S1, int S2, int WPB>
__global__ void __launch_bounds__(WPB * 32, 1) normal_eq_kernel(const __grid_constant__ LMLaunch p,
                                                                int stage, const float *states,
                                                                float *Hout, float *gout,
                                                                float *cost_out) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  const KTables &t = p.t;
  const KConfig &c = p.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (!stage_tables(t, smem, &bar, p.w.err)) return;
  PixCtx pc;
  pc.t = &t;
  pc.c = &c;
  pc.img = smem;
  pc.wsc = smem + t.lay.total + warp * warp_scratch_floats(t);
  pc.lane = lane;
  const long long nw = (long long)gridDim.x * WPB;
  for (long long pix = (long long)blockIdx.x * WPB + warp; pix < p.s.n_pix; pix += nw) {
    const float *row = p.s.rad + pix * t.nb;
    pc.wvrow = t.wvtab + (size_t)min((int)p.s.wv[pix], t.nwv - 1) * t.nb;
    if (stage == 1) {
      Stage1<K, S1> s1;
      setup1(s1, pc, row);
      constexpr int P = K + 1, NS = S1;
      float x[K + 2], H[P * (P + 1) / 2], g[P], cst, cd, dcd, r0[NS], r1[NS];
      int m;
#pragma unroll
      for (int i = 0; i < K + 2; i++) x[i] = states[pix * (K + 2) + i];
#pragma unroll
      for (int i = 0; i < NS; i++) r0[i] = 0.f;
      s1.eval(pc, x, H, g, cst, cd, m, r0, r1, dcd);
      if (lane == 0) {
        for (int a = 0; a < P; a++) {
          gout[pix * P + a] = g[a];
          for (int b = 0; b < P; b++) Hout[pix * P * P + a * P + b] = H[up<P>(a, b)];
        }
        cost_out[pix] = cst;
      }
    } else {
      float xs[K], x[6];
#pragma unroll
      for (int k = 0; k < K; k++) xs[k] = states[pix * (K + 6) + k];
#pragma unroll
      for (int i = 0; i < 6; i++) x[i] = states[pix * (K + 6) + K + i];
      Stage2<S2> s2;
      s2.bb = pc.wsc + t.nt * kScratchPerNode;
      setup2<K, S2>(s2, pc, row, xs);
      float H[21], g[6], cst, cd;
      s2.eval(pc, x, H, g, cst, cd);
      if (lane == 0) {
        for (int a = 0; a < 6; a++) {
          gout[pix * 6 + a] = g[a];
          for (int b = 0; b < 6; b++) Hout[pix * 36 + a * 6 + b] = H[up<6>(a, b)];
        }
        cost_out[pix] = cst;
      }
    }
  }
}

constexpr int kWPB = 8;

template <int WPB, class Kern>
cudaError_t launch_persistent(Kern kern, const LMLaunch &p, int num_sms, cudaStream_t st,
                              int *blocks_used) {
  size_t smem = lm_smem_bytes(p.t, WPB);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WPB * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int cl = p.s.claim > 0 ? p.s.claim : kClaim;
  long long need = (p.s.n_pix + (long long)WPB * cl - 1) / ((long long)WPB * cl);
  long long blocks = (long long)num_sms * occ;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  kern<<<(int)blocks, WPB * 32, smem, st>>>(p);
  if (blocks_used) *blocks_used += (int)blocks;
  return cudaGetLastError();
}

template <int K, int S1, int S2>
cudaError_t launch_t(const LMLaunch &p, int num_sms, cudaStream_t st, int *blocks_used, int variant,
                     cudaEvent_t *ev) {
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  // variant bit 0: stage 1 with two CTAs per SM (128 registers) instead of one
  e = (variant & 1)
          ? launch_persistent<kWPB>(lm_stage1_kernel<K, S1, kWPB, 2>, p, num_sms, st, blocks_used)
          : launch_persistent<kWPB>(lm_stage1_kernel<K, S1, kWPB, 1>, p, num_sms, st, blocks_used);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  // variant bits 1-2: stage 2 with 8, 12 or 16 warps per CTA (one CTA per
  // SM; up to 255, 168 or 128 registers)
  int v2 = (variant >> 1) & 3;
  if (v2 == 2 && lm_smem_bytes(p.t, 16) > kMaxSmemPerCta) v2 = 1;   // too many band slots
  if (v2 == 1 && lm_smem_bytes(p.t, 12) > kMaxSmemPerCta) v2 = 0;
  switch (v2) {
    case 1: e = launch_persistent<12>(lm_stage2_kernel<K, S2, 12>, p, num_sms, st, blocks_used); break;
    case 2: e = launch_persistent<16>(lm_stage2_kernel<K, S2, 16>, p, num_sms, st, blocks_used); break;
    default: e = launch_persistent<kWPB>(lm_stage2_kernel<K, S2, kWPB>, p, num_sms, st, blocks_used);
  }
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  long long blocks = (p.s.n_pix + 127) / 128;
  if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
  finalize_kernel<<<(int)blocks, 128, 0, st>>>(p, K);
  if (blocks_used) *blocks_used += (int)blocks;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) return cudaEventRecord(ev[3], st);
  return cudaSuccess;
}

template <int K>
cudaError_t launch_k(const LMLaunch &p, int num_sms, cudaStream_t st, int *blocks_used, int variant,
                     cudaEvent_t *ev) {
  int s1 = (p.t.n1 + 31) / 32, s2 = (p.t.n2 + 31) / 32;
  if (s1 <= 9 && s2 <= 7) return launch_t<K, 9, 7>(p, num_sms, st, blocks_used, variant, ev);
  if (s1 <= 9 && s2 <= 9) return launch_t<K, 9, 9>(p, num_sms, st, blocks_used, variant, ev);
  if (s1 <= 16 && s2 <= 16) return launch_t<K, 16, 16>(p, num_sms, st, blocks_used, variant, ev);
  return cudaErrorInvalidValue;
}

template <int K>
cudaError_t launch_ne_k(const LMLaunch &p, int stage, const float *states, float *H, float *g,
                        float *cost, cudaStream_t st) {
  int s1 = (p.t.n1 + 31) / 32, s2 = (p.t.n2 + 31) / 32;
  size_t smem = lm_smem_bytes(p.t, kWPB);
  int blocks = (int)((p.s.n_pix + kWPB - 1) / kWPB);
  if (blocks > 1024) blocks = 1024;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kWPB * 32, smem, st>>>(p, stage, states, H, g, cost);
    return cudaGetLastError();
  };
  if (s1 <= 9 && s2 <= 7) return go(normal_eq_kernel<K, 9, 7, kWPB>);
  if (s1 <= 9 && s2 <= 9) return go(normal_eq_kernel<K, 9, 9, kWPB>);
  if (s1 <= 16 && s2 <= 16) return go(normal_eq_kernel<K, 16, 16, kWPB>);
  return cudaErrorInvalidValue;
}

}  // namespace

size_t lm_smem_bytes(const KTables &t, int wpb) {
  return (size_t)t.lay.total * 4 + (size_t)wpb * warp_scratch_floats(t) * 4;
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
                                  const KOut &compact, const KOut &out, int K, cudaStream_t st) {
  if (nfb <= 0) return cudaSuccess;
  long long blocks = (nfb + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  merge_fallback_kernel<<<(int)blocks, 128, 0, st>>>(idx, cost_first, nfb, compact, out, K);
  return cudaGetLastError();
}

cudaError_t launch_normal_eq(const LMLaunch &p, int stage, const float *states, float *H, float *g,
                             float *cost, cudaStream_t st) {
  if (p.s.n_pix <= 0) return cudaSuccess;
  switch (p.t.K) {
    case 3: return launch_ne_k<3>(p, stage, states, H, g, cost, st);
    case 5: return launch_ne_k<5>(p, stage, states, H, g, cost, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace firert
