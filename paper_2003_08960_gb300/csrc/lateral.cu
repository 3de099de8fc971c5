// Lateral stage: chromatic rescale (Eq. 5) + Fresnel transform (Eq. 6) of every
// frame of a sweep, as one persistent kernel.
//
// Work items, taken from a device ticket counter in the order LateralSchedule
// defines:
//  * row item (frame f, band of rows): stage the input rows the band needs in
//    shared memory as float, resample them with the frame's separable linear-
//    interpolation taps, multiply by the input chirp (centring phase folded in),
//    run the Nx-point row DFT in registers (N2-point DFT per thread, twiddle,
//    exchange through shared memory, N1-point DFTs), multiply by the row's y
//    chirp and store the window columns into an L2-resident scratch slot;
//  * column item (frame f, band of columns): after every row item of f has
//    signalled, load the band from the scratch slot, run the Ny-point column DFT
//    the same way, keep the window rows and write them into the sweep-axis
//    intermediate [wy][tile][t][32] that the axial kernel streams.
// The scratch ring holds `slots` frames, so the row-transformed frames never
// leave L2: only the uint16 input is read from HBM and only the windowed
// complex hologram is written to it.
#include <cstdio>

#include "fft_common.cuh"

namespace ssoct {
namespace {

constexpr unsigned kSpinLimit = 1u << 24;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

// One thread waits until *ctr >= target.  Bounded: on timeout it records
// kErrTimeout, raises the abort flag and returns false; it also returns false
// as soon as another CTA raised the abort flag.
__device__ bool wait_counter(const unsigned* ctr, unsigned target, Counters* c) {
  if (ld_acquire_gpu(ctr) >= target) return true;
  const unsigned long long t0 = global_timer_ns();
  for (unsigned it = 0;; ++it) {
    if (ld_acquire_gpu(ctr) >= target) return true;
    if (*(volatile unsigned*)&c->abort) return false;
    if (it > kSpinLimit || global_timer_ns() - t0 > kWaitNs) {
      atomicCAS(&c->err, 0u, kErrTimeout);
      atomicExch(&c->abort, 1u);
      return false;
    }
    __nanosleep(128);
  }
}

// Row item: rows [item*RPI, item*RPI + RPI) of frame f.
template <int NX, int NY, bool FW>
__device__ __forceinline__ bool row_item(const LateralParams& p, int f, int item, unsigned char* smem,
                                         int* s_flag) {
  constexpr int N1 = Split<NX>::N1, N2 = Split<NX>::N2;
  constexpr int RPI = kThreads / N1;
  constexpr int LD = N1 + 1;  // padded exchange row: conflict-free transposed reads
  const int tid = threadIdx.x;
  const int r = tid / N1;
  const int j1 = tid % N1;
  const int row0 = item * RPI;
  const int y = row0 + r;
  const Tap* yt = p.ytab + (size_t)f * NY;
  const int jlo = yt[row0].base;
  const int jhi = yt[row0 + RPI - 1].base + 1;
  const int nrows = jhi - jlo + 1;
  const int fr = (p.ring_start + f) % p.nl;
  const unsigned long long pol_first = policy_evict_first();
  const unsigned long long pol_last = policy_evict_last();
  // 1. stage input rows jlo..jhi as float, each row padded with zeros on both
  //    sides so that taps outside the frame read 0 (8 pixels per 16-byte load)
  constexpr int SP = NX + 2 * kStagePad;
  float* stage = reinterpret_cast<float*>(smem);
  {
    const uint4* s4 = reinterpret_cast<const uint4*>(p.frames + ((size_t)fr * NY + jlo) * NX);
    const int nvec = nrows * (NX / 8);
    for (int i = tid; i < nvec; i += kThreads) {
      const uint4 v = ld_nc_hint(s4 + i, pol_first);
      float4* d4 = reinterpret_cast<float4*>(stage + (i / (NX / 8)) * SP + kStagePad + (i % (NX / 8)) * 8);
      d4[0] = make_float4(u16lo_to_f(v.x), u16hi_to_f(v.x), u16lo_to_f(v.y), u16hi_to_f(v.y));
      d4[1] = make_float4(u16lo_to_f(v.z), u16hi_to_f(v.z), u16lo_to_f(v.w), u16hi_to_f(v.w));
    }
    for (int i = tid; i < nrows; i += kThreads) {
      stage[i * SP + kStagePad - 1] = 0.f;
      stage[i * SP + kStagePad + NX] = 0.f;
    }
  }
  __syncthreads();
  // 2. Eq. 5 resample x input chirp, elements n = j1 + N1 * j2 of row y
  float2 a[N2];
  {
    const Tap ty = yt[y];
    const float* r0 = stage + (ty.base - jlo) * SP + kStagePad;
    const float* r1 = r0 + SP;
    const float4* xt = reinterpret_cast<const float4*>(p.xtab + (size_t)f * NX);
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) {
      const int n = j1 + N1 * j2;
      const float4 t = __ldg(xt + n);
      const int bx = __float_as_int(t.x);
      const float a0 = r0[bx], a1 = r0[bx + 1], b0 = r1[bx], b1 = r1[bx + 1];
      const float v0 = fmaf(t.y, a1 - a0, a0);
      const float v1 = fmaf(t.y, b1 - b0, b0);
      const float v = fmaf(ty.w0, v0, ty.w1 * v1);
      a[j2] = make_float2(v * t.z, v * t.w);
    }
  }
  // 3. row DFT (+ sign of Eq. 6), first factor in registers
  Dft<N2, 1>::template run<1, 0>(a);
  {
    const float2 cyv = ldg2(p.cy + y);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], cmul(ldg2(p.twx + k2 * N1 + j1), cyv));
  }
  // the scratch slot of frame f must be free (the columns of frame f - slots
  // done); thread 0 checks before the barrier that retires the staging rows
  if (tid == 0) {
    *s_flag = 0;
    if (f >= p.sch.slots)
      *s_flag = wait_counter(p.cols_done + (f - p.sch.slots), (unsigned)p.sch.n_col, p.ctr) ? 0 : 1;
  }
  __syncthreads();  // staging rows are dead: the exchange buffer reuses them
  if (*s_flag) return false;
  float2* exr = reinterpret_cast<float2*>(smem) + r * (N2 * LD);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) exr[k2 * LD + j1] = a[k2];
  __syncwarp();  // a row's N1 threads lie in one warp
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = exr[k2 * LD + jj];
    Dft<N1, 1>::template run<1, i * N1>(a);
  });
  float2* dst = p.scratch + ((size_t)(f % p.sch.slots) * NY + y) * p.wxp;
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      if constexpr (FW) {
        st_cg_hint(dst + k2 + N2 * k1, a[i * N1 + k1], pol_last);
      } else {
        const int kw = k2 + N2 * k1 - p.x0;
        if (kw >= 0 && kw < p.wx) st_cg_hint(dst + kw, a[i * N1 + k1], pol_last);
      }
    }
  });
  __syncthreads();
  if (tid == 0) red_release_gpu(p.rows_done + f, 1u);
  return true;
}

// Column item: window columns [item*BC, item*BC + BC) of frame f.
template <int NY, bool FW>
__device__ __forceinline__ bool col_item(const LateralParams& p, int f, int item, unsigned char* smem,
                                         int* s_flag) {
  constexpr int N1 = Split<NY>::N1, N2 = Split<NY>::N2;
  constexpr int BC = kThreads / N1;
  // padded k2 block: the 16 lanes of a half-warp read 16/BC k2 blocks at once,
  // shifted by 2*BC banks each, so they never share a bank
  constexpr int KP = N1 * BC + (BC < 16 ? BC : 0);
  const int tid = threadIdx.x;
  const int b = tid % BC;
  const int j1 = tid / BC;
  if (tid == 0) *s_flag = wait_counter(p.rows_done + f, (unsigned)p.sch.n_row, p.ctr) ? 0 : 1;
  __syncthreads();
  if (*s_flag) return false;
  const unsigned long long pol_first = policy_evict_first();
  const unsigned long long pol_last = policy_evict_last();
  const int c0 = item * BC;
  const float2* src = p.scratch + (size_t)(f % p.sch.slots) * NY * p.wxp + c0 + b;
  float2 a[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = ld_cg_hint(src + (size_t)(j1 + N1 * j2) * p.wxp, pol_last);
  Dft<N2, 1>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], ldg2(p.twy + k2 * N1 + j1));
  float2* ex = reinterpret_cast<float2*>(smem);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[k2 * KP + j1 * BC + b] = a[k2];
  __syncthreads();
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[k2 * KP + jj * BC + b];
    Dft<N1, 1>::template run<1, i * N1>(a);
  });
  const int kxw = c0 + b;
  if (kxw < p.wx) {
    float2* dst = p.inter + (size_t)(kxw / kTile) * p.nl * kTile + (size_t)f * kTile + (kxw % kTile);
    const size_t row_pitch = (size_t)p.ntx * p.nl * kTile;
    static_for<0, N2 / N1>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const int k2 = j1 + N1 * i;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        if constexpr (FW) {
          st_cg_hint(dst + (size_t)(k2 + N2 * k1) * row_pitch, a[i * N1 + k1], pol_first);
        } else {
          const int kyw = k2 + N2 * k1 - p.y0;
          if (kyw >= 0 && kyw < p.wy) st_cg_hint(dst + (size_t)kyw * row_pitch, a[i * N1 + k1], pol_first);
        }
      }
    });
  }
  __syncthreads();
  if (tid == 0) red_release_gpu(p.cols_done + f, 1u);
  return true;
}

// L2 prefetch of the input rows a row item will stage (nothing for a column item).
template <int NX, int NY>
__device__ __forceinline__ void prefetch_row_input(const LateralParams& p, unsigned t) {
  int kind, f, item;
  p.sch.decode(t, kind, f, item);
  if (kind != 0) return;
  constexpr int RPI = kThreads / Split<NX>::N1;
  const Tap* yt = p.ytab + (size_t)f * NY;
  const int jlo = yt[item * RPI].base;
  const int jhi = yt[item * RPI + RPI - 1].base + 1;
  const int fr = (p.ring_start + f) % p.nl;
  prefetch_l2_bulk(p.frames + ((size_t)fr * NY + jlo) * NX, (unsigned)((jhi - jlo + 1) * NX * sizeof(uint16_t)));
}

template <int NX, int NY, bool FW>
__global__ void __launch_bounds__(kThreads, 2) lateral_kernel(const __grid_constant__ LateralParams p) {
  static_assert(kThreads / Split<NX>::N1 <= NY, "a row item must not exceed the frame");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_ticket;
  __shared__ int s_flag;
  const long long total = p.sch.total();
  // Thread 0 keeps the ticket after the current one (t1) in hand and takes the
  // one after that while the current item runs, so the atomic round trip hides
  // behind the item; t1's input rows are prefetched into L2 meanwhile.  A CTA
  // holds at most two unstarted tickets, and the lowest unfinished ticket is
  // always the one its CTA is working on, so the queue still drains.
  unsigned t1 = 0xffffffffu;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(&p.ctr->ticket, 1u);
    t1 = atomicAdd(&p.ctr->ticket, 1u);
  }
  for (;;) {
    __syncthreads();
    const long long k = s_ticket;
    if (k >= total) break;
    int kind, f, item;
    p.sch.decode(k, kind, f, item);
    unsigned t2 = 0xffffffffu;
    if (threadIdx.x == 0) {
      t2 = (*(volatile unsigned*)&p.ctr->abort) ? 0xffffffffu : atomicAdd(&p.ctr->ticket, 1u);
      if (t1 < total) prefetch_row_input<NX, NY>(p, t1);
    }
    const bool ok = kind == 0 ? row_item<NX, NY, FW>(p, f, item, smem, &s_flag)
                              : col_item<NY, FW>(p, f, item, smem, &s_flag);
    if (!ok) break;
    if (threadIdx.x == 0) {  // every thread read s_ticket before the item's barriers
      s_ticket = t1;
      t1 = t2;
    }
  }
}

template <int NX, int NY>
size_t smem_for(const Plan& p) {
  constexpr int N1x = Split<NX>::N1, N2x = Split<NX>::N2;
  constexpr int N1y = Split<NY>::N1;
  constexpr int N2y = Split<NY>::N2;
  const size_t stage = (size_t)p.stage_rows * (NX + 2 * kStagePad) * sizeof(float);
  const size_t rows = (size_t)(kThreads / N1x) * N2x * (N1x + 1) * sizeof(float2);
  constexpr int BCy = kThreads / N1y;
  const size_t cols = (size_t)N2y * (N1y * BCy + (BCy < 16 ? BCy : 0)) * sizeof(float2);
  size_t m = stage > rows ? stage : rows;
  return m > cols ? m : cols;
}

template <int NX, int NY, bool FW>
cudaError_t launch_fw(const Plan& p, const LateralParams& lp, cudaStream_t s) {
  const size_t smem = smem_for<NX, NY>(p);
  cudaError_t e = cudaFuncSetAttribute(lateral_kernel<NX, NY, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  long long total = lp.sch.total();
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lateral_kernel<NX, NY, FW>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = (p.num_sms > 0 ? p.num_sms : 1) * per_sm;
  if (grid > total) grid = (int)total;
  lateral_kernel<NX, NY, FW><<<grid, kThreads, smem, s>>>(lp);
  return cudaGetLastError();
}

template <int NX, int NY>
cudaError_t launch(const Plan& p, const LateralParams& lp, cudaStream_t s) {
  const bool full = p.x0 == 0 && p.y0 == 0 && p.wx == NX && p.wy == NY;
  return full ? launch_fw<NX, NY, true>(p, lp, s) : launch_fw<NX, NY, false>(p, lp, s);
}

#define SSOCT_LATERAL_SIZES(X) \
  X(64, 64) X(128, 128) X(256, 256) X(512, 512) X(1024, 1024) X(128, 64) X(64, 128)

}  // namespace

bool lateral_supported(int nx, int ny) {
#define X(a, b) if (nx == a && ny == b) return true;
  SSOCT_LATERAL_SIZES(X)
#undef X
  return false;
}

size_t lateral_smem_bytes(const Plan& p) {
#define X(a, b) if (p.nx == a && p.ny == b) return smem_for<a, b>(p);
  SSOCT_LATERAL_SIZES(X)
#undef X
  return 0;
}

cudaError_t launch_lateral(const Plan& p, const LateralParams& lp, cudaStream_t s) {
#define X(a, b) if (p.nx == a && p.ny == b) return launch<a, b>(p, lp, s);
  SSOCT_LATERAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ssoct
