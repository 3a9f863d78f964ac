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

// Eq. (inject): out = L_bg + alpha tau_up B(lambda, T) for each band of each
// pixel, the Planck term in FP64 (an input generator: exact to the fp32
// store), tau_up of the pixel's water-vapour bin; an invalid bin gives NaN
__global__ void inject_kernel(KTables t, const float *wl, const float *bg, const uint16_t *wv,
                              const float *alpha, const float *T, long long n, float *out) {
  const long long total = n * t.nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / t.nb;
    const int b = (int)(e % t.nb);
    const int w = wv[i];
    if (w >= t.nwv) {
      out[e] = __int_as_float(0x7fc00000);
      continue;
    }
    const double lam = (double)wl[b] * 1e-9;
    const double x = kH * kC / (kKB * lam * (double)T[i]);
    const double B = 2.0 * kH * kC * kC / (lam * lam * lam * lam * lam) * 1e-9 / expm1(x);
    out[e] = (float)((double)bg[e] + (double)alpha[i] * (double)t.wvtab[(size_t)w * t.nb + b].w * B);
  }
}

// HFDI (Sec. 2.1): (L_hi - L_lo) / (L_hi + L_lo) at the two gate bands, one
// thread per pixel; NaN where either band is not finite
__global__ void hfdi_kernel(const float *rad, int nb, long long n, int bhi, int blo, float *out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float h = __ldg(rad + i * nb + bhi), l = __ldg(rad + i * nb + blo);
    out[i] = (isfinite(h) && isfinite(l)) ? (h - l) / (h + l) : __int_as_float(0x7fc00000);
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

// ---- water-vapour presolve (Sec. 2.5): one warp per super-pixel. Each lane
// forms the 940 nm band depth of up to kWvPerLane of the block's pixels,
// D = 1 - L_c / fma(L_hi - L_lo, cf, L_lo), in single precision; the warp
// then selects the lower median (rank (n - 1) / 2 of the n finite depths)
// by a most-significant-bit-first radix select on order-preserving integer
// keys (32 ballot-count rounds), interpolates its fractional bin index
// between the bracketing depths of the table and rounds it to the nearest
// bin, and writes that bin for every pixel of the block. Three floats of
// each 1136-byte radiance row are read: DRAM moves one 32-byte sector per
// band per pixel.
constexpr int kWvPerLane = 8;     // 32 x 8 = 256 pixels: blocks up to 16 x 16

__device__ __forceinline__ unsigned order_key(float v) {
  const unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void __launch_bounds__(256) wv_presolve_kernel(const float *rad, int nb, long long W,
                                                          long long H, int B, int blo, int bc, int bhi,
                                                          float cf, const float *sat, WvLut lut,
                                                          uint16_t *bins, float *depth) {
  const int lane = threadIdx.x & 31;
  const long long nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
  const long long blk = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (blk >= nbx * nby) return;                 // warp-uniform
  const long long by = blk / nbx, bx = blk % nbx;
  const long long x0 = bx * B, y0 = by * B;
  const int bw = (int)min((long long)B, W - x0), bh = (int)min((long long)B, H - y0);
  const int np = bw * bh;
  unsigned key[kWvPerLane];
  bool ok[kWvPerLane];
  int nv = 0;
#pragma unroll
  for (int q = 0; q < kWvPerLane; q++) {
    const int i = lane + 32 * q;
    ok[q] = false;
    key[q] = 0u;
    if (i < np) {
      const long long p = (y0 + i / bw) * W + x0 + i % bw;
      const float *row = rad + p * nb;
      const float lo = __ldg(row + blo), c = __ldg(row + bc), hi = __ldg(row + bhi);
      bool v = isfinite(lo) && isfinite(c) && isfinite(hi);
      if (sat) v = v && lo < __ldg(sat + blo) && c < __ldg(sat + bc) && hi < __ldg(sat + bhi);
      const float cont = fmaf(hi - lo, cf, lo);
      v = v && cont > 0.f;
      const float D = v ? 1.f - c / cont : __int_as_float(0x7fc00000);
      if (depth) depth[p] = D;
      ok[q] = v;
      key[q] = order_key(D);
      nv += v;
    }
  }
  const int n = __reduce_add_sync(0xffffffffu, nv);
  uint16_t bin = 0xFFFF;
  if (n > 0) {
    // the k-th smallest key, k = (n - 1) / 2, bit by bit from the top
    unsigned want = 0u;
    int k = (n - 1) / 2;
    for (int bit = 31; bit >= 0; bit--) {
      const unsigned hi_mask = bit == 31 ? 0u : (0xffffffffu << (bit + 1));
      int cnt = 0;
#pragma unroll
      for (int q = 0; q < kWvPerLane; q++)
        cnt += ok[q] && (key[q] & hi_mask) == want && !((key[q] >> bit) & 1u);
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (k >= cnt) {
        want |= 1u << bit;
        k -= cnt;
      }
    }
    const float med = key_value(want);
    const int J = lut.n;
    float fi;
    if (!(med > lut.D[0])) fi = 0.f;
    else if (!(med < lut.D[J - 1])) fi = (float)(J - 1);
    else {
      int j = 0;
      while (!(med < lut.D[j + 1])) j++;        // D[j] <= med < D[j + 1]
      fi = (float)j + (med - lut.D[j]) / (lut.D[j + 1] - lut.D[j]);
    }
    const int b = (int)floorf(fi + 0.5f);
    bin = (uint16_t)(b < 0 ? 0 : (b > J - 1 ? J - 1 : b));
  }
#pragma unroll
  for (int q = 0; q < kWvPerLane; q++) {
    const int i = lane + 32 * q;
    if (i < np) bins[(y0 + i / bw) * W + x0 + i % bw] = bin;
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

cudaError_t launch_wv_presolve(const float *rad, int nb, long long W, long long H, int B, int blo,
                               int bc, int bhi, float cf, const float *sat, const WvLut &lut,
                               uint16_t *bins, float *depth, cudaStream_t st) {
  const long long nblk = ((W + B - 1) / B) * ((H + B - 1) / B);
  if (nblk <= 0) return cudaSuccess;
  const long long grid = (nblk + 7) / 8;         // 8 warps (super-pixels) per CTA
  wv_presolve_kernel<<<(unsigned)grid, 256, 0, st>>>(rad, nb, W, H, B, blo, bc, bhi, cf, sat, lut, bins,
                                                     depth);
  return cudaGetLastError();
}

cudaError_t launch_inject(const KTables &t, const float *wl, const float *bg, const uint16_t *wv,
                          const float *alpha, const float *T, long long n, float *out, cudaStream_t st) {
  const long long total = n * t.nb;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  inject_kernel<<<(int)blocks, 256, 0, st>>>(t, wl, bg, wv, alpha, T, n, out);
  return cudaGetLastError();
}

cudaError_t launch_hfdi(const float *rad, int nb, long long n, int bhi, int blo, float *out,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  hfdi_kernel<<<(int)blocks, 256, 0, st>>>(rad, nb, n, bhi, blo, out);
  return cudaGetLastError();
}

}  // namespace firert
