// model.cuh — device pieces shared by the forward kernel and the training-
// spectrum synthesiser: the counter-based generator and the forward model
// Eq. (fm) = Eq. (solar) + Eq. (thermal) for one state, one warp.
#pragma once
#include "internal.cuh"

namespace firert {

// SplitMix64 output function (Steele, Lea & Flood 2014)
__device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// key of one pixel's stream: nested mixing of (seed, stream id, pixel)
__device__ __forceinline__ unsigned long long sm_key(unsigned long long seed, unsigned long long sid,
                                                     unsigned long long pix) {
  return sm_mix(sm_mix(sm_mix(seed) ^ sid) ^ pix);
}

// uniform in (0, 1] from draw idx of a pixel's stream (top 53 bits + 1 ulp)
__device__ __forceinline__ float counter_uniform(unsigned long long kpix, unsigned long long idx) {
  unsigned long long u = sm_mix(kpix ^ idx);
  return (float)(((double)(u >> 11) + 1.0) * 1.1102230246251565e-16);
}

// standard normal by Box-Muller on draws (2i, 2i+1)
__device__ __forceinline__ float counter_normal(unsigned long long kpix, unsigned long long i) {
  float u1 = counter_uniform(kpix, 2ull * i), u2 = counter_uniform(kpix, 2ull * i + 1);
  return sqrtf(-2.f * logf(u1)) * cosf(6.283185307179586f * u2);
}

// Forward model of one state by one warp. mode 1: s = [x_surf(K), a1, T1];
// mode 2: s = [x_surf(K), mu_h, s_h, mu_s, s_s, eta, a]. wsc: this warp's
// scratch of >= n_tgrid floats. Calls emit(b, L_b) on the owning lane.
template <class Emit>
__device__ __forceinline__ void warp_forward(const KTables &t, const float *img, int lane, int mode,
                                             const float *s, int wvb, float *wsc, Emit &&emit) {
  const int K = t.K;
  const float4 *row = t.wvtab + (size_t)wvb * t.nb;
  const float a = mode == 1 ? s[K] : s[K + 5];
  if (mode == 2 && a != 0.f) {
    const float mh = s[K], sh = s[K + 1], ms = s[K + 2], ss = s[K + 3], eta = s[K + 4];
    float uh[4], us[4], Uh = 0.f, Us = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j = lane + 32 * q;
      uh[q] = us[q] = 0.f;
      if (j < t.nt) {
        float T = t.tglo + j * t.tgstep;
        float dh = T - mh, ds = T - ms;
        uh[q] = __expf(-dh * dh / (2.f * sh * sh));
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
    emit(b, Lv);
  }
  __syncwarp();
}

}  // namespace firert
