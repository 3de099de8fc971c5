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
  static_assert(N1 > 0 && N1 * N2 == N, "FFT length not built");
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

// L2 eviction-priority policies (createpolicy) and accesses that carry them.
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// L2-only (L1 bypassed) complex store with an L2 policy.
__device__ __forceinline__ void st_cg_hint(float2* a, float2 v, unsigned long long pol) {
  asm volatile("st.global.cg.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}

// Eq. 5 at one pixel of a uint16 frame [.][nx] from its separable taps (weights
// are 0 where a tap falls outside the frame; bases are clamped inside it).
__device__ __forceinline__ float rescale_tap_value(const uint16_t* fr, int nx, const Tap& tx, const Tap& ty) {
  const uint16_t* r0 = fr + (size_t)ty.base * nx + tx.base;
  const uint16_t* r1 = r0 + nx;
  const float v0 = fmaf(tx.w0, (float)__ldg(r0), tx.w1 * (float)__ldg(r0 + 1));
  const float v1 = fmaf(tx.w0, (float)__ldg(r1), tx.w1 * (float)__ldg(r1 + 1));
  return fmaf(ty.w0, v0, ty.w1 * v1);
}

}  // namespace ssoct
