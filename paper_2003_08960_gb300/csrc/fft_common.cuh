// Device helpers shared by the kernels: FFT splits, complex arithmetic,
// compile-time loops, memory-order primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fft_codelets.cuh"
#include "ssoct_internal.h"

namespace ssoct {

template <int N>
struct Split {
  static constexpr int N1 = split_n1(N);
  static constexpr int N2 = N1 ? N / N1 : 0;
  static_assert(N1 > 0 && N2 % N1 == 0, "FFT length not built");
};

// f(integral_constant<int, I>) for I = B .. E-1, unrolled at compile time.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Add to a device counter with release semantics at GPU scope: every write this
// thread has made or observed (e.g. its CTA's writes before a __syncthreads) is
// visible GPU-wide before the new count is.
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// uint16 halves of a 32-bit word to float, exactly: 0x4B000000 | u is 2^23 + u.
__device__ __forceinline__ float u16lo_to_f(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5410)) - 8388608.0f;
}
__device__ __forceinline__ float u16hi_to_f(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5432)) - 8388608.0f;
}

}  // namespace ssoct
