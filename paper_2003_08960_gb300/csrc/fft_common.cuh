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
// L2-only (L1 bypassed) complex load / store with an L2 policy.
__device__ __forceinline__ float2 ld_cg_hint(const float2* a, unsigned long long pol) {
  float2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void st_cg_hint(float2* a, float2 v, unsigned long long pol) {
  asm volatile("st.global.cg.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}
// Read-only 16-byte load, not kept in L1, with an L2 policy.
__device__ __forceinline__ uint4 ld_nc_hint(const uint4* a, unsigned long long pol) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(pol));
  return v;
}
// Asynchronous prefetch of a contiguous block into L2 (16-byte aligned, size a
// multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* a, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
}

// uint16 halves of a 32-bit word to float, exactly: 0x4B000000 | u is 2^23 + u.
__device__ __forceinline__ float u16lo_to_f(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5410)) - 8388608.0f;
}
__device__ __forceinline__ float u16hi_to_f(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5432)) - 8388608.0f;
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
