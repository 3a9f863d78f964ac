// tc.cuh — tcgen05 building blocks shared by the tensor-core kernels:
// shared-memory addresses, the UMMA shared-memory and instruction
// descriptors for bf16 K-major operands in the 128-byte-swizzled layout, the
// byte offset of a 16-byte chunk inside such a tile, and a bounded mbarrier
// wait.
#pragma once
#include <stdint.h>

namespace firert {
namespace tc {

__device__ __forceinline__ unsigned su32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor, K-major, 128-byte swizzle: start address,
// leading-byte offset (unused for this layout), stride-byte offset = 1024 B
// between 8-row core-matrix groups, descriptor version 1, layout type 2.
__device__ __forceinline__ uint64_t sdesc(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(1u) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// byte offset of the 16-byte chunk c (K elements 8c..8c+7) of row r inside a
// K-major SW128 tile whose base is 1024-byte aligned
__host__ __device__ __forceinline__ unsigned swz(int r, int c) {
  return (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// wait for the given phase parity of an mbarrier, at most `spins` polls;
// false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long spins) {
  unsigned done = 0;
  for (long long s = 0; s < spins && !done; s++)
    asm volatile(
        "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2; selp.u32 %0, 1, 0, P; }"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}

}  // namespace tc
}  // namespace firert
