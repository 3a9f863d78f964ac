// kernels_aux.cu — table construction, the forward model (with optional
// counter-based noise) and the block-mean coarsening kernel.
#include "internal.cuh"
#include "model.cuh"

namespace firert {

namespace {

// CODATA 2018 exact SI values
constexpr double kH = 6.62607015e-34;
constexpr double kC = 299792458.0;
constexpr double kKB = 1.380649e-23;

// Table build (once per context, FP64 inside the kernel, rounded to fp32):
//   c2l[b]  = h c / (k lambda_b)              Planck exponent numerator (K)
//   c1l5[b] = 2 h c^2 / lambda_b^5 * 1e-9      per-nm radiance prefactor
//   planck[j][b - b2lo] = c1l5 e^-x / (1 - e^-x), x = c2l / T_j   (Eq. thermal)
//   wvtab[w][b] = (A td tu, A rho_atm, S, tu), A = E0 cos(theta_s) / pi   (Eq. solar)
__global__ void build_tables_kernel(KTables t, const float *wl, const float *e0, float cos_sza,
                                    const float *td, const float *tu, const float *ra,
                                    const float *sa, const float *endm, float *img,
                                    float4 *wvtab, float w1lo, float w1hi, float w2hlo,
                                    float w2hhi, float w2slo, float w2shi) {
  const ImageLayout L = t.lay;
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nthr = gridDim.x * blockDim.x;
  for (int b = tid; b < t.nb; b += nthr) {
    double lam = (double)wl[b] * 1e-9;
    img[L.off_c2l + b] = (float)(kH * kC / (kKB * lam));
    img[L.off_c1l5 + b] = (float)(2.0 * kH * kC * kC / (lam * lam * lam * lam * lam) * 1e-9);
    float l = wl[b];
    img[L.off_win1 + b] = (l >= w1lo && l <= w1hi) ? 1.f : 0.f;
    img[L.off_win2 + b] = ((l >= w2hlo && l <= w2hhi) || (l >= w2slo && l <= w2shi)) ? 1.f : 0.f;
    for (int k = 0; k < t.K; k++) img[L.off_endm + k * t.nb + b] = endm[k * t.nb + b];
  }
  for (int e = tid; e < t.nt * L.n2s; e += nthr) {
    int j = e / L.n2s, bb = e % L.n2s, b = t.b2lo + bb;
    float v = 0.f;
    if (bb < t.n2) {
      double lam = (double)wl[b] * 1e-9;
      double T = (double)t.tglo + j * (double)t.tgstep;
      double x = kH * kC / (kKB * lam * T);
      double ex = exp(-x);
      v = (float)(2.0 * kH * kC * kC / (lam * lam * lam * lam * lam) * 1e-9 * ex / (1.0 - ex));
    }
    img[L.off_planck + e] = v;
  }
  for (int e = tid; e < t.nwv * t.nb; e += nthr) {
    int b = e % t.nb;
    double A = (double)e0[b] * cos_sza / 3.14159265358979323846;
    float4 q;
    q.x = (float)(A * td[e] * tu[e]);
    q.y = (float)(A * (ra ? ra[e] : 0.f));
    q.z = sa ? sa[e] : 0.f;
    q.w = tu[e];
    wvtab[e] = q;
  }
}

// B(lambda_b, T_j) for every band and grid node, [nt][nb] (Eq. thermal, the
// same FP64 formula as the stage-2 grid above, stored fp32)
__global__ void planck_full_kernel(KTables t, const float *wl, float *out) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nthr = gridDim.x * blockDim.x;
  for (int e = tid; e < t.nt * t.nb; e += nthr) {
    int j = e / t.nb, b = e % t.nb;
    double lam = (double)wl[b] * 1e-9;
    double T = (double)t.tglo + j * (double)t.tgstep;
    double ex = exp(-kH * kC / (kKB * lam * T));
    out[e] = (float)(2.0 * kH * kC * kC / (lam * lam * lam * lam * lam) * 1e-9 * ex / (1.0 - ex));
  }
}

// B(lambda_b, T_j) over the stage-2 bands, [nt][n2], kept in FP64 (the
// posterior's normal matrix at the final state)
__global__ void planck64_kernel(KTables t, const float *wl, double *out) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nthr = gridDim.x * blockDim.x;
  for (int e = tid; e < t.nt * t.n2; e += nthr) {
    int j = e / t.n2, b = t.b2lo + e % t.n2;
    double lam = (double)wl[b] * 1e-9;
    double T = (double)t.tglo + j * (double)t.tgstep;
    double ex = exp(-kH * kC / (kKB * lam * T));
    out[e] = 2.0 * kH * kC * kC / (lam * lam * lam * lam * lam) * 1e-9 * ex / (1.0 - ex);
  }
}

// Forward model, one warp per state (the model itself is warp_forward in
// model.cuh), with optional counter-based noise.
__global__ void __launch_bounds__(256) forward_kernel(KTables t, int mode, const float *state,
                                                      const uint16_t *wv, long long n,
                                                      float nrel, float nabs,
                                                      unsigned long long seed,
                                                      unsigned long long sid, long long pix0,
                                                      float *out) {
  extern __shared__ float sh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *wsc = sh + warp * 2 * kMaxTgrid;
  const int K = t.K, ns = mode == 1 ? K + 2 : K + 6;
  long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = gw; i < n; i += nw) {
    const float *s = state + i * ns;
    if (wv[i] >= t.nwv) {   // invalid water-vapour bin: NaN radiance, no table read
      for (int b = lane; b < t.nb; b += 32) out[i * t.nb + b] = __int_as_float(0x7fc00000);
      continue;
    }
    const bool noisy = nrel > 0.f || nabs > 0.f;
    const unsigned long long kpix = noisy ? sm_key(seed, sid, (unsigned long long)(pix0 + i)) : 0ull;
    float *o = out + i * t.nb;
    warp_forward(t, t.image, lane, mode, s, wv[i], wsc, [&](int b, float Lv) {
      if (noisy) Lv += sqrtf(nrel * nrel * Lv * Lv + nabs * nabs) * counter_normal(kpix, b);
      o[b] = Lv;
    });
  }
}

// dst[cy][cx][b] = mean of the blk x blk block of src (Sec. 2.9 coarsening)
__global__ void block_mean_kernel(const float *src, int w, int h, int nb, int blk, float *dst) {
  int cw = w / blk, ch = h / blk;
  long long total = (long long)cw * ch * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e % nb);
    long long c = e / nb;
    int cx = (int)(c % cw), cy = (int)(c / cw);
    float acc = 0.f;
    for (int dy = 0; dy < blk; dy++) {
      const float *r = src + ((long long)(cy * blk + dy) * w + (long long)cx * blk) * nb + b;
      for (int dx = 0; dx < blk; dx++) acc += r[(long long)dx * nb];
    }
    dst[e] = acc / (float)(blk * blk);
  }
}

}  // namespace

cudaError_t launch_build_tables(const KTables &t, const float *wl, const float *e0, float cos_sza,
                                  const float *td, const float *tu, const float *ra,
                                  const float *sa, const float *endm, float *image, float4 *wvtab,
                                  const float win[6], cudaStream_t st) {
  build_tables_kernel<<<64, 256, 0, st>>>(t, wl, e0, cos_sza, td, tu, ra, sa, endm, image, wvtab,
                                          win[0], win[1], win[2], win[3], win[4], win[5]);
  return cudaGetLastError();
}

cudaError_t launch_planck_full(const KTables &t, const float *wl, float *out, cudaStream_t st) {
  planck_full_kernel<<<64, 256, 0, st>>>(t, wl, out);
  return cudaGetLastError();
}

cudaError_t launch_planck64(const KTables &t, const float *wl, double *out, cudaStream_t st) {
  planck64_kernel<<<64, 256, 0, st>>>(t, wl, out);
  return cudaGetLastError();
}

cudaError_t launch_forward(const KTables &t, int mode, const float *state, const uint16_t *wv,
                           int64_t n, float noise_rel, float noise_abs, uint64_t seed,
                           uint64_t stream_id, int64_t pix0, float *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int warps = 8;
  long long blocks = (n + warps - 1) / warps;
  if (blocks > 148 * 64) blocks = 148 * 64;
  forward_kernel<<<(int)blocks, warps * 32, warps * 2 * kMaxTgrid * sizeof(float), st>>>(
      t, mode, state, wv, n, noise_rel, noise_abs, seed, stream_id, pix0, out);
  return cudaGetLastError();
}

cudaError_t launch_block_mean(const float *src, int w, int h, int nb, int blk, float *dst,
                              cudaStream_t st) {
  long long total = (long long)(w / blk) * (h / blk) * nb;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 148 * 32) blocks = 148 * 32;
  block_mean_kernel<<<(int)blocks, 256, 0, st>>>(src, w, h, nb, blk, dst);
  return cudaGetLastError();
}

}  // namespace firert
