// kernels_gemm.cu — BF16 tensor-core GEMM on sm_103a (tcgen05 + TMEM).
//
// C[M x N] = A[M x K] * B[N x K]^T with A, B bf16, K-major (row-major with K
// contiguous), FP32 accumulation in tensor memory, and a fused epilogue:
//   EPI_F32        C_f32 = acc (+ bias)
//   EPI_BIAS_RELU  h = max(acc + bias, 0) -> bf16 (and optionally h^T)
//   EPI_BIAS_TANH  z = tanh(acc + bias) -> f32
//   EPI_RELU_MASK  d = acc * (mask > 0) -> bf16 (and optionally d^T)
// One CTA (4 warps) computes a 128 x BN tile; K is consumed in 64-wide
// chunks in 128-byte-swizzled shared memory (the canonical K-major SW128
// layout the UMMA descriptors read). The default kernel is warp-specialised:
// one thread of warp 0 moves the A and B chunks with TMA
// (cp.async.bulk.tensor, 2D tensor maps with the 128-byte swizzle; the
// tails in M, N and K are zero-filled by the copy) into a ring of four
// stages, each with a full and an empty mbarrier; one thread of warp 1
// issues tcgen05.mma (cta_group::1, kind::f16, M = 128, N = BN, K = 16 per
// instruction) as each stage fills and commits it back to the stage's empty
// barrier; all four warps then read the accumulator with tcgen05.ld
// (32x32b, warp w the TMEM lanes 32w..32w+31) for the epilogue, one row per
// thread. Bases and row pitches must be 16-byte aligned. Where a tensor map
// cannot be encoded (no driver entry point), a second kernel stages the
// operands with 16-byte cp.async copies, double buffered. Every wait is
// bounded and sets an error flag on timeout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace firert {
namespace {

constexpr int kBM = 128, kBK = 64;
constexpr long long kSpin = 1ll << 24;

using tc::idesc_bf16;
using tc::sdesc;
using tc::su32;
using tc::swz;

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  return tc::mbar_wait(bar, parity, kSpin);
}

__device__ __forceinline__ void cp16(unsigned dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0) : "memory");
}

// the epilogue of both kernels: warp w reads TMEM lanes 32w..32w+31 (rows
// m0 + 32w + lane), columns in groups of 16
template <int BN>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs &g, uint32_t tmem, int m0, int n0, int warp,
                                              int lane) {
  const int row = m0 + warp * 32 + lane;
  const bool rv = row < g.M;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    uint32_t v[16];
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!rv) continue;
    if (g.Cb && !g.Cf && !g.CbT && g.epi != EPI_RELU_MASK && !(g.ldcb & 7) && n0 + c0 + 16 <= g.N) {
      // bf16 rows: bias, activation, and 16-byte stores of 8 values
#pragma unroll
      for (int h = 0; h < 16; h += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          const int col = n0 + c0 + h + j;
          float a0 = __uint_as_float(v[h + j]), a1 = __uint_as_float(v[h + j + 1]);
          if (g.bias) { a0 += g.bias[col]; a1 += g.bias[col + 1]; }
          if (g.epi == EPI_BIAS_RELU) { a0 = fmaxf(a0, 0.f); a1 = fmaxf(a1, 0.f); }
          else if (g.epi == EPI_BIAS_TANH) { a0 = tanhf(a0); a1 = tanhf(a1); }
          const __nv_bfloat162 p2 = __floats2bfloat162_rn(a0, a1);
          pk[j / 2] = *reinterpret_cast<const uint32_t *>(&p2);
        }
        *reinterpret_cast<uint4 *>(g.Cb + (size_t)row * g.ldcb + n0 + c0 + h) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const int col = n0 + c0 + j;
      if (col >= g.N) continue;
      float a = __uint_as_float(v[j]);
      if (g.bias) a += g.bias[col];
      switch (g.epi) {
        case EPI_BIAS_RELU: a = fmaxf(a, 0.f); break;
        case EPI_BIAS_TANH: a = tanhf(a); break;
        case EPI_RELU_MASK:
          a = __bfloat162float(g.mask[(size_t)row * g.ldm + col]) > 0.f ? a : 0.f;
          break;
        default: break;
      }
      if (g.Cf) g.Cf[(size_t)row * g.ldc + col] = g.accumulate ? g.Cf[(size_t)row * g.ldc + col] + a : a;
      if (g.Cb) g.Cb[(size_t)row * g.ldcb + col] = __float2bfloat16_rn(a);
      if (g.CbT) g.CbT[(size_t)col * g.ldcbT + row] = __float2bfloat16_rn(a);
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(128) gemm_tn_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_slot;
  constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  constexpr int kCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  // stage buffers, 1024-byte aligned
  unsigned char *base = gsm + ((1024 - (su32(gsm) & 1023)) & 1023);
  unsigned char *As[2] = {base, base + kABytes};
  unsigned char *Bs[2] = {base + 2 * kABytes, base + 2 * kABytes + kBBytes};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nk = (g.K + kBK - 1) / kBK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(su32(&tmem_slot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  auto load_chunk = [&](int kc, int s) {
    const int k0 = kc * kBK;
    for (int e = tid; e < kBM * 8; e += 128) {
      int r = e >> 3, c = e & 7;
      int gr = m0 + r, gk = k0 + c * 8;
      bool ok = gr < g.M && gk < g.K;
      const void *src = ok ? (const void *)(g.A + (size_t)gr * g.lda + gk) : (const void *)g.A;
      cp16(su32(As[s]) + swz(r, c), src, ok);
    }
    for (int e = tid; e < BN * 8; e += 128) {
      int r = e >> 3, c = e & 7;
      int gr = n0 + r, gk = k0 + c * 8;
      bool ok = gr < g.N && gk < g.K;
      const void *src = ok ? (const void *)(g.B + (size_t)gr * g.ldb + gk) : (const void *)g.B;
      cp16(su32(Bs[s]) + swz(r, c), src, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  bool ok = true;
  unsigned uses[2] = {0u, 0u};
  load_chunk(0, 0);
  if (nk > 1) load_chunk(1, 1);
  constexpr uint32_t idesc = idesc_bf16(kBM, BN);
  for (int kc = 0; kc < nk; kc++) {
    const int s = kc & 1;
    if (kc + 1 < nk) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kBK / 16; kk++) {
        uint64_t ad = sdesc(su32(As[s]) + kk * 32), bd = sdesc(su32(Bs[s]) + kk * 32);
        uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
            ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(su32(&bar[s])) : "memory");
    }
    uses[s]++;
    if (kc + 2 < nk) {
      // the stage is reused: wait until the MMAs that read it completed (the
      // decision is made uniform across the CTA)
      const bool w = mbar_wait(su32(&bar[s]), (uses[s] - 1) & 1);
      if (!__syncthreads_and(w)) { ok = false; break; }
      load_chunk(kc + 2, s);
    }
  }
  // wait for the last commit of each stage that was used
  if (ok) {
    bool w = true;
    for (int s = 0; s < 2; s++)
      if (uses[s]) w = mbar_wait(su32(&bar[s]), (uses[s] - 1) & 1) && w;
    ok = __syncthreads_and(w);
  }
  if (!ok) {
    if (tid == 0 && g.err) atomicExch(g.err, 1);
    // drain: bounded waits on whatever is still in flight, then free TMEM
    for (int s = 0; s < 2; s++)
      if (uses[s]) mbar_wait(su32(&bar[s]), (uses[s] - 1) & 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok) gemm_epilogue<BN>(g, tmem, m0, n0, warp, lane);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

constexpr int kStages = 4;   // TMA ring depth

// 2D tile load of a K-major operand chunk: box {64 K elements (128 bytes),
// rows} at coordinates {k0, r0} (k0 a multiple of 64: 128-byte aligned),
// completing on the stage's full barrier
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int k0, int r0,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(k0), "r"(r0), "r"(bar) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(128) gemm_tma_kernel(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB,
                                                       GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  constexpr int kCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  unsigned char *base = gsm + ((1024 - (su32(gsm) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nk = (g.K + kBK - 1) / kBK;
  auto As = [&](int s) { return su32(base + s * (kABytes + kBBytes)); };
  auto Bs = [&](int s) { return su32(base + s * (kABytes + kBBytes) + kABytes); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(su32(&tmem_slot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  int issued = 0;       // producer: chunks whose copies were issued
  int mma_done = 0;     // MMA thread: chunks whose products were issued

  if (warp == 0 && lane == 0) {
    // producer: a stage is refilled once the MMAs that read it have
    // completed (its empty barrier's phase for the previous use)
    for (int kc = 0; kc < nk; kc++) {
      const int s = kc % kStages;
      if (kc >= kStages && !mbar_wait(su32(&empty[s]), ((kc / kStages) - 1) & 1)) {
        atomicExch(&fail, 1);
        break;
      }
      if (*((volatile int *)&fail)) break;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   ::"r"(su32(&full[s])), "r"(kABytes + kBBytes) : "memory");
      tma_load_2d(As(s), &mapA, kc * kBK, m0, su32(&full[s]));
      tma_load_2d(Bs(s), &mapB, kc * kBK, n0, su32(&full[s]));
      issued = kc + 1;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    for (int kc = 0; kc < nk; kc++) {
      const int s = kc % kStages;
      if (*((volatile int *)&fail)) break;
      if (!mbar_wait(su32(&full[s]), (kc / kStages) & 1)) {
        atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kBK / 16; kk++) {
        const uint64_t ad = sdesc(As(s) + kk * 32), bd = sdesc(Bs(s) + kk * 32);
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
            ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(su32(&empty[s])) : "memory");
      mma_done = kc + 1;
    }
    // every product issued so far completes before the accumulator is read
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(su32(&done)) : "memory");
  }
  __syncwarp();
  // every thread: the accumulator is complete (or the fit gave up)
  bool ok = mbar_wait(su32(&done), 0);
  ok = __syncthreads_and(ok && !*((volatile int *)&fail));
  if (!ok) {
    if (tid == 0 && g.err) atomicExch(g.err, 1);
    // drain with bounded waits: the copies the producer issued land on the
    // full barriers; the products the MMA thread issued on the empty ones
    if (warp == 0 && lane == 0)
      for (int kc = (issued > kStages ? issued - kStages : 0); kc < issued; kc++)
        mbar_wait(su32(&full[kc % kStages]), (kc / kStages) & 1);
    if (warp == 1 && lane == 0)
      for (int kc = (mma_done > kStages ? mma_done - kStages : 0); kc < mma_done; kc++)
        mbar_wait(su32(&empty[kc % kStages]), (kc / kStages) & 1);
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) gemm_epilogue<BN>(g, tmem, m0, n0, warp, lane);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// K-major bf16 operand [rows][ld] -> tensor map with box {64, box_rows}
bool make_map(CUtensorMap *m, const __nv_bfloat16 *p, int rows, int K, long long ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_tma_bn(const GemmArgs &g, cudaStream_t st, bool *used) {
  *used = false;
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.M, g.K, g.lda, kBM) || !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
    return cudaSuccess;
  const size_t smem = (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
  cudaError_t e = cudaFuncSetAttribute(gemm_tma_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + kBM - 1) / kBM, (g.N + BN - 1) / BN);
  gemm_tma_kernel<BN><<<grid, 128, smem, st>>>(ma, mb, g);
  *used = true;
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_bn(const GemmArgs &g, cudaStream_t st) {
  const size_t smem = 2 * (size_t)(kBM * kBK * 2) + 2 * (size_t)(BN * kBK * 2) + 1024;
  cudaError_t e = cudaFuncSetAttribute(gemm_tn_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + kBM - 1) / kBM, (g.N + BN - 1) / BN);
  gemm_tn_kernel<BN><<<grid, 128, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace

template <int BN>
cudaError_t launch_any(const GemmArgs &g, cudaStream_t st) {
  bool used = false;
  cudaError_t e = launch_tma_bn<BN>(g, st, &used);
  if (e != cudaSuccess || used) return e;
  return launch_bn<BN>(g, st);      // operands TMA cannot address
}

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if ((g.K & 7) || (g.lda & 7) || (g.ldb & 7)) return cudaErrorInvalidValue;  // 16-byte rows
  if (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15)) return cudaErrorInvalidValue;  // 16-byte bases
  if (g.N <= 16) return launch_any<16>(g, st);
  if (g.N <= 32) return launch_any<32>(g, st);
  if (g.N <= 64) return launch_any<64>(g, st);
  if (g.N <= 128) return launch_any<128>(g, st);
  return launch_any<256>(g, st);
}

}  // namespace firert
