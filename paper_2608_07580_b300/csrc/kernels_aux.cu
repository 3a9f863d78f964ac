// kernels_aux.cu — table construction, the forward model (with optional
// counter-based noise) and the block-mean coarsening kernel.
#include "internal.cuh"

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

__device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
  // SplitMix64 output function (Steele, Lea & Flood 2014)
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float counter_uniform(unsigned long long kpix, unsigned long long idx) {
  unsigned long long u = sm_mix(kpix ^ idx);
  return (float)(((double)(u >> 11) + 1.0) * 1.1102230246251565e-16);  // (0, 1]
}

// Forward model, one warp per state: lanes build the grid weights of the two
// mixture components (mode 2), then sweep the bands.
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
  const float *img = t.image;
  for (long long i = gw; i < n; i += nw) {
    const float *s = state + i * ns;
    if (wv[i] >= t.nwv) {   // invalid water-vapour bin: NaN radiance, no table read
      for (int b = lane; b < t.nb; b += 32) out[i * t.nb + b] = __int_as_float(0x7fc00000);
      continue;
    }
    const float4 *row = t.wvtab + (size_t)wv[i] * t.nb;
    float a = mode == 1 ? s[K] : s[K + 5];
    if (mode == 2 && a != 0.f) {
      float mh = s[K], sh_ = s[K + 1], ms = s[K + 2], ss = s[K + 3], eta = s[K + 4];
      float uh[4], us[4], Uh = 0.f, Us = 0.f;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        int j = lane + 32 * q;
        uh[q] = us[q] = 0.f;
        if (j < t.nt) {
          float T = t.tglo + j * t.tgstep;
          float dh = T - mh, ds = T - ms;
          uh[q] = __expf(-dh * dh / (2.f * sh_ * sh_));
          us[q] = __expf(-ds * ds / (2.f * ss * ss));
        }
        Uh += uh[q];
        Us += us[q];
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        Uh += __shfl_xor_sync(0xffffffffu, Uh, o);
        Us += __shfl_xor_sync(0xffffffffu, Us, o);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 4; q++) {
        int j = lane + 32 * q;
        if (j < t.nt) wsc[j] = eta * uh[q] / Uh + (1.f - eta) * us[q] / Us;
      }
      __syncwarp();
    }
    unsigned long long kpix = 0;
    if (nrel > 0.f || nabs > 0.f)
      kpix = sm_mix(sm_mix(sm_mix(seed) ^ sid) ^ (unsigned long long)(pix0 + i));
    for (int b = lane; b < t.nb; b += 32) {
      float4 q = row[b];
      float rho = 0.f;
      for (int k = 0; k < K; k++) rho += s[k] * img[t.lay.off_endm + k * t.nb + b];
      float Lv = q.y + q.x * rho / (1.f - q.z * rho);
      if (a != 0.f) {
        if (mode == 1) {
          float x = img[t.lay.off_c2l + b] / s[K + 1];
          float e = expf(-x);
          Lv += a * q.w * img[t.lay.off_c1l5 + b] * e / (1.f - e);
        } else {
          // thermal term on the grid: sum_j p_j B(lambda_b, T_j)
          float x0 = img[t.lay.off_c2l + b], c1 = img[t.lay.off_c1l5 + b], acc = 0.f;
          for (int j = 0; j < t.nt; j++) {
            float e = expf(-x0 / (t.tglo + j * t.tgstep));
            acc += wsc[j] * c1 * e / (1.f - e);
          }
          Lv += a * q.w * acc;
        }
      }
      if (kpix) {
        float u1 = counter_uniform(kpix, 2ull * b), u2 = counter_uniform(kpix, 2ull * b + 1);
        float z = sqrtf(-2.f * logf(u1)) * cosf(6.283185307179586f * u2);
        Lv += sqrtf(nrel * nrel * Lv * Lv + nabs * nabs) * z;
      }
      out[i * t.nb + b] = Lv;
    }
    __syncwarp();
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
