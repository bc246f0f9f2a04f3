// Shared device helpers of the tcgen05 kernels: shared-memory matrix
// descriptors for the SWIZZLE_NONE K-major core-matrix layout, time-bounded
// mbarrier waits, powers of two.
//
// Operand tiles are stored as 8-row x 16-byte core matrices: element (r, k)
// of a tile with BK = 16 contracted indices sits at byte
//   (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2,
// LBO = 128 B (next core matrix along K), SBO = 256 B (next 8-row group).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace tctl {
namespace tc {

constexpr int BK = 16;
constexpr uint32_t LBO = 128, SBO = (BK / 8) * 128;  // bytes

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of element (r, k), k < 16, in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)((r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2);
}

// Bounded wait on an mbarrier phase: false once limit_ns nanoseconds (global
// timer) have passed without the phase completing, or after 2^24 polls
// whatever the timer says; the caller records an error and unwinds instead of
// hanging. kWaitNs = 1 s, far above any wait of a working pipeline
// (microseconds).
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ float pow2f(int e) {
  // 2^e for -126 <= e <= 127, 0 below (exact)
  return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}

}  // namespace tc
}  // namespace tctl
