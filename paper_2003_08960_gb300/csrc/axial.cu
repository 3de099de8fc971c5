// Axial stage: transform over the sweep (Eq. 7, rectangular gate of N_lambda
// frames, kernel exp(-2 pi i q t / N_lambda), unnormalised) at every window
// pixel, then the envelope |V|^2 (or |V|) written as the float32 volume
// [q][y][x].  Optionally also V itself with the Eq. 6 prefactor and output
// chirp applied (unit-modulus factors apart from |K|, so |V|^2 needs only |K|^2).
//
// The unit of work is a 32-pixel tile of one window row: its N_lambda x 32
// complex values (contiguous in the intermediate) go through the
// N_lambda-point DFT as N2-point DFTs in registers, a twiddle, an exchange
// through shared memory and N1-point DFTs, and leave as 128-byte runs of the
// volume per depth bin.  Sweeps of 64 to 256 frames take the persistent
// streaming form (axial_stream_kernel: TMA-fed ring of stage buffers, two
// consumer groups per SM); the others one CTA per tile (axial_kernel).
#include <cuda.h>

#include "fft_common.cuh"
#include "mbarrier.cuh"

namespace ssoct {
namespace {

template <int NL>
__global__ void __launch_bounds__(kTile * Split<NL>::N1) axial_kernel(const __grid_constant__ AxialParams p) {
  constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  static_assert(N2 % N1 == 0, "the second stage needs N1 | N2");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ex = reinterpret_cast<float2*>(smem);
  const int tile = blockIdx.x;
  const int kyw = blockIdx.y;
  const int pix = threadIdx.x % kTile;
  const int j1 = threadIdx.x / kTile;
  const float2* src = p.inter + ((size_t)kyw * p.ntx + tile) * NL * kTile + pix;
  float2 a[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = __ldcs(src + (j1 + N1 * j2) * kTile);
  Dft<N2, -1>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], ldg2(p.twl + k2 * N1 + j1));
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * kTile + pix] = a[k2];
  __syncthreads();
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[(k2 * N1 + jj) * kTile + pix];
    Dft<N1, -1>::template run<1, i * N1>(a);
  });
  const int kxw = tile * kTile + pix;
  if (kxw >= p.wx) return;
  const size_t plane = (size_t)p.wy * p.wx;
  float* vol = p.vol + (size_t)kyw * p.wx + kxw;
  float2 of = make_float2(0.f, 0.f);
  if (p.cplx) of = cmul(ldg2(p.ox + kxw), ldg2(p.oy + kyw));
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int q = k2 + N2 * k1;
      const float2 v = a[i * N1 + k1];
      float pw = fmaf(v.x, v.x, v.y * v.y) * p.power_scale;
      if (p.magnitude) pw = sqrtf(pw);
      __stcs(vol + (size_t)q * plane, pw);
      if (p.cplx) __stcs(p.cplx + (size_t)q * plane + (size_t)kyw * p.wx + kxw, cmul(v, of));
    }
  });
}

// Streaming form for sweeps of up to 256 frames: one persistent CTA per SM,
// two consumer groups and a ring of shared-memory stage buffers.  Whole tiles
// (N_lambda x 32 complex values, contiguous in the intermediate) arrive by 1D
// TMA bulk copies, a ring's worth ahead; group g computes the CTA's tiles
// g, g + 2, ... with the same two-stage DFT as axial_kernel, doing the exchange
// in place in the stage buffer, and once all its threads are done with a
// buffer one of them issues the copy of the tile kStages further on into it.
// The loads never wait for the arithmetic, so HBM keeps streaming.
constexpr int kAxGroups = 2;
constexpr size_t kAxRingBytes = 192 * 1024;
constexpr unsigned long long kAxWaitNs = 4000000000ull;  // 4 s

template <int NL>
struct AxStream {
  static constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  static constexpr int kGroupThreads = kTile * N1;
  static constexpr int kThreadsAll = kAxGroups * kGroupThreads;
  static constexpr size_t kTileBytes = (size_t)NL * kTile * sizeof(float2);
  static constexpr int kStages = kAxRingBytes / kTileBytes > 8 ? 8 : (int)(kAxRingBytes / kTileBytes);
  // one full barrier per tile index mod lcm(kStages, kAxGroups): each is waited
  // on by one group only, which has consumed its previous fill, and its fills
  // follow one another through the buffer chain t -> t + kStages
  static constexpr int kFull = kStages % kAxGroups == 0 ? kStages : kStages * kAxGroups;
};

__device__ bool mbar_wait_bounded(uint64_t* b, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try(b, parity))
    if (global_timer_ns() - t0 > limit_ns) return false;
  return true;
}

// Barrier of one consumer group (named barrier id, T threads); returns the OR of v.
template <int T>
__device__ __forceinline__ bool group_sync_or(int id, bool v) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
               : "=r"(r)
               : "r"((unsigned)v), "r"(id), "n"(T)
               : "memory");
  return r != 0;
}
template <int T>
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(T) : "memory");
}

// Copy of the CTA's tile t (global tile blockIdx.x + t * gridDim.x) into stage
// buffer t mod kStages; fills[] counts the copies issued on each full barrier.
template <int NL>
__device__ __forceinline__ void axial_fill(const AxialParams& p, unsigned char* ring, uint64_t* full_bar,
                                           unsigned* fills, int t) {
  using S = AxStream<NL>;
  const int f = t % S::kFull;
  atomicAdd(&fills[f], 1u);
  mbar_arrive_tx(&full_bar[f], (unsigned)S::kTileBytes);
  const size_t gt = blockIdx.x + (size_t)t * gridDim.x;
  tma_load_1d(ring + (size_t)(t % S::kStages) * S::kTileBytes, p.inter + gt * NL * kTile, (unsigned)S::kTileBytes,
              &full_bar[f]);
}

// End of a streaming tile: the depth bins q = k2 + N2 k1 this thread holds (a[])
// for window pixel (kxw, kyw): |V|^2 |K|^2 (|V| |K| if MAG) into the volume and,
// if CPLX, V with the output chirp and K into the complex volume.
template <int NL, bool MAG, bool CPLX>
__device__ __forceinline__ void axial_epilogue(const AxialParams& p, const float2* a, int j1, int kyw, int kxw) {
  constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  const size_t plane = (size_t)p.wy * p.wx;
  float* vol = p.vol + (size_t)kyw * p.wx + kxw;
  float2 of = make_float2(0.f, 0.f);
  if constexpr (CPLX) of = cmul(ldg2(p.ox + kxw), ldg2(p.oy + kyw));
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int ii = decltype(I)::value;
    const int k2 = j1 + N1 * ii;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int q = k2 + N2 * k1;
      const float2 v = a[ii * N1 + k1];
      float pw = fmaf(v.x, v.x, v.y * v.y) * p.power_scale;
      if constexpr (MAG) pw = sqrtf(pw);
      __stcs(vol + (size_t)q * plane, pw);
      if constexpr (CPLX) __stcs(p.cplx + (size_t)q * plane + (size_t)kyw * p.wx + kxw, cmul(v, of));
    }
  });
}

template <int NL>
__global__ void __launch_bounds__(AxStream<NL>::kThreadsAll, 1)
    axial_stream_kernel(const __grid_constant__ AxialParams p) {
  using S = AxStream<NL>;
  constexpr int N1 = S::N1, N2 = S::N2, T = S::kGroupThreads;
  static_assert(N2 % N1 == 0, "the second stage needs N1 | N2");
  extern __shared__ __align__(16) unsigned char smem[];  // 16 B: the bulk copies need no more
  __shared__ __align__(8) uint64_t full_bar[S::kFull];
  __shared__ unsigned fills[S::kFull];
  const int tid = threadIdx.x;
  const int ntiles = p.ntx * p.wy;
  const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < S::kFull; ++b) {
      mbar_init(&full_bar[b], 1);
      fills[b] = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int t = 0; t < S::kStages && t < mine; ++t) axial_fill<NL>(p, smem, full_bar, fills, t);
  }
  __syncthreads();
  const int g = tid / T;
  const int lt = tid % T;
  const int pix = lt % kTile;
  const int j1 = lt / kTile;
  for (int i = g, prev = -1;; prev = i, i += kAxGroups) {
    group_sync<T>(1 + g);  // every thread of the group is done with tile prev's buffer
    if (lt == 0 && prev >= 0 && prev + S::kStages < mine) axial_fill<NL>(p, smem, full_bar, fills, prev + S::kStages);
    if (i >= mine) break;
    // one thread waits for the tile; the others sleep at the group barrier
    bool ok = true;
    if (lt == 0) {
      ok = mbar_wait_bounded(&full_bar[i % S::kFull], (unsigned)(i / S::kFull) & 1u, kAxWaitNs);
      if (!ok) atomicOr(p.err, kErrAxial);
    }
    if (group_sync_or<T>(1 + g, !ok)) break;
    float2* ex = reinterpret_cast<float2*>(smem + (size_t)(i % S::kStages) * S::kTileBytes);
    float2 a[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) a[j2] = ex[(j1 + N1 * j2) * kTile + pix];
    Dft<N2, -1>::template run<1, 0>(a);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], ldg2(p.twl + k2 * N1 + j1));
    // t = k2 N1 + j1 runs over the same frames j1 + N1 j2 this thread read
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * kTile + pix] = a[k2];
    // these writes come before the buffer's next TMA fill (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    group_sync<T>(1 + g);
    static_for<0, N2 / N1>([&](auto I) {
      constexpr int ii = decltype(I)::value;
      const int k2 = j1 + N1 * ii;
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[ii * N1 + jj] = ex[(k2 * N1 + jj) * kTile + pix];
      Dft<N1, -1>::template run<1, ii * N1>(a);
    });
    const int gt = (int)blockIdx.x + i * (int)gridDim.x;
    const int kyw = gt / p.ntx;
    const int kxw = (gt - kyw * p.ntx) * kTile + pix;
    if (kxw >= p.wx) continue;
    // the options are tested once per tile: inside the unrolled loop they were
    // predicated on every value
    if (p.cplx) {
      if (p.magnitude) axial_epilogue<NL, true, true>(p, a, j1, kyw, kxw);
      else axial_epilogue<NL, false, true>(p, a, j1, kyw, kxw);
    } else {
      if (p.magnitude) axial_epilogue<NL, true, false>(p, a, j1, kyw, kxw);
      else axial_epilogue<NL, false, false>(p, a, j1, kyw, kxw);
    }
  }
  // copies still in flight (after a time-out) write this CTA's shared memory:
  // they land before it exits.  The last fill of each barrier is its latest
  // phase, so the parity is exact.
  __syncthreads();
  if (tid == 0)
    for (int f = 0; f < S::kFull; ++f)
      if (fills[f] && !mbar_wait_bounded(&full_bar[f], (fills[f] - 1u) & 1u, kAxWaitNs)) atomicOr(p.err, kErrAxial);
}

struct RescaleAxialParams {
  const uint16_t* frames;  // gate frame t at frames[(ring_start + t) mod nl]
  int ring_start;
  const Tap* xtab;         // [nl][nx]
  const Tap* ytab;         // [nl][ny]
  const float2* twl;       // [N2l][N1l], sign -
  float2* planes;          // [nl/2 + 1][ny][nx]
  const float2* cx;        // [nx] input chirp of Eq. 6 (with the centring phase)
  const float2* cy;        // [ny]
  float k_abs;             // |K| of Eq. 6
  int nx, ny, nl;
};

// Axial-first order, first pass: at every sensor pixel of a 32-pixel tile, the
// Eq. 5 resample of each frame of the gate (a real series over t), its Eq. 7
// transform over t, and bins q = 0 .. nl/2 as complex planes.  The rest of the
// spectrum is the conjugate mirror (real input) and is formed by the lateral
// pass.  Eq. 6 is linear and the same for every frame, so transforming over t
// before it gives the same V as the paper's order.  The planes are stored times
// the input chirp of Eq. 6 and |K| (X c |K|): bins up to nl/2 then enter the
// lateral pass's DFTs as they are, and the mirrored bins take c^2 there.
template <int NL>
__global__ void __launch_bounds__(kTile * Split<NL>::N1) rescale_axial_kernel(const __grid_constant__ RescaleAxialParams p) {
  constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  static_assert(N2 % N1 == 0, "the second stage needs N1 | N2");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ex = reinterpret_cast<float2*>(smem);
  const int pix = threadIdx.x % kTile, j1 = threadIdx.x / kTile;
  const int x = blockIdx.x * kTile + pix, y = blockIdx.y;
  float2 a[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int t = j1 + N1 * j2;
    const uint16_t* fr = p.frames + (size_t)((p.ring_start + t) % p.nl) * p.ny * p.nx;
    const float u = rescale_tap_value(fr, p.nx, p.xtab[(size_t)t * p.nx + x], p.ytab[(size_t)t * p.ny + y]);
    a[j2] = make_float2(u, 0.f);
  }
  Dft<N2, -1>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], ldg2(p.twl + k2 * N1 + j1));
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * kTile + pix] = a[k2];
  __syncthreads();
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[(k2 * N1 + jj) * kTile + pix];
    Dft<N1, -1>::template run<1, i * N1>(a);
  });
  const size_t plane = (size_t)p.ny * p.nx;
  float2* dst = p.planes + (size_t)y * p.nx + x;
  float2 c = cmul(ldg2(p.cx + x), ldg2(p.cy + y));
  c = make_float2(c.x * p.k_abs, c.y * p.k_abs);
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int q = k2 + N2 * k1;
      if (q <= NL / 2) dst[(size_t)q * plane] = cmul(a[i * N1 + k1], c);
    }
  });
}

// ---------------------------------------------------------------- axial-first pass, tiled form
//
// Same output as rescale_axial_kernel for sweeps of 64, 96, 128, 160, 200 and
// 256 frames, with the frames read once and the real input used twice over:
//  * a tile is 64 consecutive pixels of one sensor row (a 64-pixel strip x one
//    row), tiles numbered row by row, so that the CTAs running together cover
//    neighbouring strips of neighbouring rows and share in L2 the source lines
//    their staged boxes overlap on (numbered strip by strip, the frames were
//    read 2.2 times from DRAM); pixels p and p + 32 are paired into one complex series
//    z_t = u_t(p) + i u_t(p + 32), so 32 complex N_lambda-point DFTs give the
//    64 real ones: X(p) = (Z_q + conj Z_{N-q}) / 2 and
//    X(p + 32) = (Z_q - conj Z_{N-q}) / (2i);
//  * every frame's two source rows of the tile (the rows of its y taps) are
//    staged in shared memory by one 2D tensor copy per frame (TMA), which
//    reads zeros outside the frame; the next tile's copies are issued as soon
//    as the current tile's samples have been read, and land while it finishes
//    its transform and writes its planes.  (16-byte cp.async copies of the
//    same rows, ten per row, took 0.39 of 0.88 ms at 1024 x 1024 x 256);
//  * the x taps of Eq. 5 follow u(x0 + k) = u(x0) + k s_t along the strip, so
//    one record per (frame, strip), built in float64 (first staged column,
//    integer and fractional part of u(x0) relative to it, s_t - 1), gives every
//    pixel's taps: g = frac(u(x0)) + k (s_t - 1) in float32, column
//    off + k + floor(g), weight g - floor(g); out-of-frame taps read the zero
//    fill, as Eq. 5 is read here (taps outside the frame are 0).
// The DFT over t is a two-stage split N1 x N2 (ra_split_n1: the axial
// kernel's where that gives 8 to 16 warps per tile, 16 x 6, 16 x 10 and
// 20 x 10 for 96, 160 and 200 frames): N2-point DFTs in registers, twiddle,
// exchange through shared memory, N1-point DFTs (idle in some threads where N1
// does not divide N2), the second stage in place, so that the pair separation
// reads Z_{N-q} from the same buffer after a barrier.
struct RescaleAxialTileParams {
  int ring_start;            // gate frame t is frame (ring_start + t) mod nl of the tensor map
  const StripTap* xstrip;    // [nl][nx / 64]
  const Tap* ytab;           // [nl][ny]
  const float2* twl;         // [N2][N1] of this pass's split (ra_split_n1), sign -
  float2* planes;            // [nl/2 + 1][ny][nx]
  const float2* cx;          // [nx] input chirp of Eq. 6 (with the centring phase)
  const float2* cy;          // [ny]
  float k_abs;               // |K| of Eq. 6
  int nx, ny, w;             // w: staged columns per source row (multiple of 8)
  unsigned* err;             // kErrAxial is ORed in if a staging wait runs out
};

constexpr int kRaStrip = 64;  // pixels per tile (two per complex series)

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Eq. 5 at strip pixel k of a frame whose two staged source rows are r0, r1.
__device__ __forceinline__ float ra_sample(int k, const StripTap& xs, const Tap& yt, const uint16_t* r0,
                                           const uint16_t* r1) {
  const float g = fmaf((float)k, xs.e, xs.f);
  const float fl = floorf(g);
  const float fr = g - fl;
  const int col = xs.off + k + (int)fl;
  const float a0 = __uint2float_rn(r0[col]), a1 = __uint2float_rn(r0[col + 1]);
  const float b0 = __uint2float_rn(r1[col]), b1 = __uint2float_rn(r1[col + 1]);
  const float h0 = fmaf(fr, a1 - a0, a0), h1 = fmaf(fr, b1 - b0, b0);
  return fmaf(yt.w0, h0, yt.w1 * h1);
}

template <int NL>
struct RaTile {
  static constexpr int N1 = ra_split_n1(NL), N2 = NL / N1;
  using S2 = Stage2<NL, N1>;  // stage 2: NI N1-point DFTs per thread, idle where N1 does not divide N2
  static constexpr int kThreads = 32 * N1;
  // shared memory: exchange [NL][32] complex, strip records [NL], y taps [NL],
  // twiddles [NL], then frame t's two staged rows (2 x w uint16) at t * stride,
  // then the staging mbarrier.  A tensor copy's shared-memory destination must
  // be 128-byte aligned: the staged rows start on a 128-byte boundary and each
  // frame's block is padded to a multiple of 128 bytes.
  static constexpr size_t kStageOffset = ((size_t)NL * 32 * sizeof(float2) +
                                          (size_t)NL * (sizeof(StripTap) + sizeof(Tap) + sizeof(float2)) + 127) /
                                         128 * 128;
  static_assert(kStageOffset % 128 == 0, "staged rows on a 128-byte boundary");
  __host__ __device__ static size_t frame_stride(int w) { return ((size_t)2 * w * sizeof(uint16_t) + 127) / 128 * 128; }
  static size_t smem_bytes(int w) { return kStageOffset + (size_t)NL * frame_stride(w) + sizeof(uint64_t); }
};

template <int NL>
__global__ void __launch_bounds__(RaTile<NL>::kThreads, 1)
    rescale_axial_tile_kernel(const __grid_constant__ RescaleAxialTileParams p,
                              const __grid_constant__ CUtensorMap fmap) {
  using R = RaTile<NL>;
  constexpr int N1 = R::N1, N2 = R::N2, T = R::kThreads;
  using S2 = typename R::S2;
  static_assert(T >= NL, "one loader thread per frame");
  // its own name: the other kernels of this file declare the dynamic shared
  // memory with 16-byte alignment, and a tensor copy needs 128 here
  extern __shared__ __align__(1024) unsigned char smem_ra[];
  unsigned char* smem = smem_ra;
  float2* ex = reinterpret_cast<float2*>(smem);
  StripTap* xsm = reinterpret_cast<StripTap*>(ex + NL * 32);
  Tap* ysm = reinterpret_cast<Tap*>(xsm + NL);
  float2* tw = reinterpret_cast<float2*>(ysm + NL);
  unsigned char* st = smem + R::kStageOffset;  // frame t's rows at st + t * fstride
  const size_t fstride = R::frame_stride(p.w);
  uint64_t& full = *reinterpret_cast<uint64_t*>(st + NL * fstride);
  const int tid = threadIdx.x;
  const int pp = tid % 32, j1 = tid / 32;
  const int w = p.w;
  const int strips = p.nx / kRaStrip;
  const int ntiles = strips * p.ny;
  const size_t plane = (size_t)p.ny * p.nx;
  for (int i = tid; i < NL; i += T) tw[i] = p.twl[i];
  if (tid == 0) {
    mbar_init(&full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // loader role: thread t < NL stages frame t's two source rows of a tile
  const bool loader = tid < NL;
  const int frow = loader ? ((p.ring_start + tid) % NL) * p.ny : 0;  // first row of frame t in the map
  const unsigned tile_bytes = (unsigned)(NL * 2 * w * sizeof(uint16_t));
  auto stage = [&](const StripTap& xr, const Tap& yr) {
    if (tid == 0) mbar_arrive_tx(&full, tile_bytes);
    if (loader) {
      xsm[tid] = xr;
      ysm[tid] = yr;
      // earlier generic reads of the buffer come before this async-proxy write
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      unsigned char* dst = st + (size_t)tid * fstride;
      // a tensor copy needs a 128-byte aligned destination and an x start whose
      // byte offset is a multiple of 16; a copy that would break either is not
      // issued (the wait for it then runs out and reports kErrAxial)
      if ((smem_u32(dst) & 127u) == 0u && (xr.xs & 7) == 0)
        tma_load_2d(dst, &fmap, xr.xs, frow + yr.base, &full);
      else
        atomicOr(p.err, kErrAxial);
    }
  };
  auto records = [&](int tile, StripTap& xr, Tap& yr) {
    if (loader && tile < ntiles) {
      const int y = tile / strips, strip = tile - y * strips;
      xr = p.xstrip[(size_t)tid * strips + strip];
      yr = p.ytab[(size_t)tid * p.ny + y];
    }
  };
  StripTap xr{};
  Tap yr{};
  int tile = blockIdx.x;
  unsigned phase = 0;     // tiles staged and consumed so far
  bool pending = false;   // a staging copy is in flight on `full`
  records(tile, xr, yr);
  if (tile < ntiles) {
    stage(xr, yr);
    pending = true;
  }
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    records(next, xr, yr);  // in flight while this tile is transformed
    // one thread waits for the copies; the others sleep at the barrier
    bool ok = true;
    if (tid == 0) {
      ok = mbar_wait_bounded(&full, phase & 1u, kAxWaitNs);
      if (!ok) atomicOr(p.err, kErrAxial);
    }
    // this tile's rows and records are in; every thread is done with the last tile
    if (__syncthreads_or(!ok)) break;
    pending = false;
    ++phase;
    const int y = tile / strips, strip = tile - y * strips;
    // 1. Eq. 5 samples of frames t = j1 + N1 j2 at pixels pp and pp + 32 (one
    //    complex series), N2-point DFT over j2, twiddle, exchange
    float2 a[S2::A];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) {
      const int t = j1 + N1 * j2;
      const StripTap xs = xsm[t];
      const Tap yt = ysm[t];
      const uint16_t* r0 = reinterpret_cast<const uint16_t*>(st + (size_t)t * fstride);
      a[j2] = make_float2(ra_sample(pp, xs, yt, r0, r0 + w), ra_sample(pp + 32, xs, yt, r0, r0 + w));
    }
    Dft<N2, -1>::template run<1, 0>(a);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * 32 + pp] = cmul(a[k2], tw[k2 * N1 + j1]);
    __syncthreads();  // the staged rows are read: the next tile's copies may overwrite them
    if (next < ntiles) {
      stage(xr, yr);
      pending = true;
    }
    // 2. N1-point DFTs, results back into the slots just read: Z_q, q = k2 + N2 k1,
    //    at row k2 N1 + k1
    static_for<0, S2::NI>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const int k2 = j1 + N1 * i;
      if (!S2::live(i, j1)) return;
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[(k2 * N1 + jj) * 32 + pp];
      Dft<N1, -1>::template run<1, i * N1>(a);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) ex[(k2 * N1 + k1) * 32 + pp] = a[i * N1 + k1];
    });
    __syncthreads();
    // 3. the two real series' spectra, bins q = 0 .. NL/2, as plane rows, times
    //    the input chirp and |K| of Eq. 6 at their pixels (the factor 1/2 of the
    //    separation folded in)
    const int xa = strip * kRaStrip + pp;
    float2* dst = p.planes + (size_t)y * p.nx + xa;
    const float2 cyv = ldg2(p.cy + y);
    const float h = 0.5f * p.k_abs;
    float2 ca = cmul(ldg2(p.cx + xa), cyv), cb = cmul(ldg2(p.cx + xa + 32), cyv);
    ca = make_float2(ca.x * h, ca.y * h);
    cb = make_float2(cb.x * h, cb.y * h);
    static_for<0, S2::NI>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const int k2 = j1 + N1 * i;
      if (!S2::live(i, j1)) return;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int q = k2 + N2 * k1;
        if (q <= NL / 2) {
          const int qm = (NL - q) % NL;
          const float2 zq = a[i * N1 + k1];
          const float2 zm = ex[((qm % N2) * N1 + qm / N2) * 32 + pp];
          __stcs(dst + (size_t)q * plane, cmul(make_float2(zq.x + zm.x, zq.y - zm.y), ca));
          __stcs(dst + (size_t)q * plane + 32, cmul(make_float2(zq.y + zm.y, zm.x - zq.x), cb));
        }
      }
    });
  }
  // after a time-out, the copy still in flight lands before the CTA exits
  if (pending && tid == 0 && !mbar_wait_bounded(&full, phase & 1u, kAxWaitNs)) atomicOr(p.err, kErrAxial);
}

struct GateCutsParams {
  const float2* inter;   // [wy][ntx][nl][32]
  const float2* wq;      // [nl] exp(-2 pi i k / nl)
  const float2* twl;     // [N2l][N1l], sign - (the axial kernel's table)
  float* xy;             // [wy][wx] or NULL
  float* xz;             // [nl][wx] or NULL
  float* yz;             // [nl][wy] or NULL
  float2* xy_state;      // [wy][ntx * 32] X(z0) of the xy cut, or NULL
  int nl, wx, wy, ntx, x0, y0, z0;
  float power_scale;
  int magnitude;
};

__device__ __forceinline__ float envelope(float2 v, float scale, int magnitude) {
  const float pw = fmaf(v.x, v.x, v.y * v.y) * scale;
  return magnitude ? sqrtf(pw) : pw;
}

// xy cut at depth bin z0 straight from the intermediate: at every window pixel
// the single bin V_z0 = sum_t H_t exp(-2 pi i z0 t / N) of Eq. 7.
__global__ void __launch_bounds__(256) gate_xy_kernel(const __grid_constant__ GateCutsParams c) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* w = reinterpret_cast<float2*>(smem);
  for (int k = threadIdx.x; k < c.nl; k += blockDim.x) w[k] = ldg2(c.wq + k);
  __syncthreads();
  const size_t row = (size_t)c.ntx * kTile;
  const size_t n = (size_t)c.wy * row;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kyw = (int)(i / row), tile = (int)(i % row) / kTile, pix = (int)(i % kTile);
    const int kxw = tile * kTile + pix;
    const float2* h = c.inter + ((size_t)kyw * c.ntx + tile) * c.nl * kTile + pix;
    float2 acc = make_float2(0.f, 0.f);
    int k = 0;
#pragma unroll 8
    for (int t = 0; t < c.nl; ++t) {
      const float2 v = __ldcs(h + (size_t)t * kTile);
      const float2 e = w[k];
      acc.x = fmaf(v.x, e.x, fmaf(-v.y, e.y, acc.x));
      acc.y = fmaf(v.x, e.y, fmaf(v.y, e.x, acc.y));
      k += c.z0;
      if (k >= c.nl) k -= c.nl;
    }
    if (c.xy_state) c.xy_state[i] = acc;
    if (kxw < c.wx) c.xy[(size_t)kyw * c.wx + kxw] = envelope(acc, c.power_scale, c.magnitude);
  }
}

struct XySlideParams {
  const float2* inter;   // [wy][ntx][nl][32]
  const float2* wq;      // [nl] exp(-2 pi i k / nl)
  float2* state;         // [wy][ntx * 32] running X(z0)
  float* xy;             // [wy][wx] or NULL
  int nl, wx, wy, ntx, z0, slot0, k;
  float sign;
  float power_scale;
  int magnitude;
};

// Running xy cut of a sliding gate.  X(z0) = sum_t h_t exp(-2 pi i z0 t / nl)
// over the gate's slots t is linear in the holograms, so a frame that replaces
// slot t changes it by (h_new - h_old) exp(-2 pi i z0 t / nl): one pass with
// sign -1 over the slots about to be overwritten (before the lateral pass) and
// one with sign +1 after it read k slots per pixel instead of nl.
__global__ void __launch_bounds__(256) xy_slide_kernel(const __grid_constant__ XySlideParams c) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* w = reinterpret_cast<float2*>(smem);
  for (int k = threadIdx.x; k < c.nl; k += blockDim.x) w[k] = ldg2(c.wq + k);
  __syncthreads();
  const size_t row = (size_t)c.ntx * kTile;
  const size_t n = (size_t)c.wy * row;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kyw = (int)(i / row), tile = (int)(i % row) / kTile, pix = (int)(i % kTile);
    const int kxw = tile * kTile + pix;
    const float2* h = c.inter + ((size_t)kyw * c.ntx + tile) * c.nl * kTile + pix;
    float2 d = make_float2(0.f, 0.f);
    int t = c.slot0;
    for (int j = 0; j < c.k; ++j) {
      const float2 v = __ldcs(h + (size_t)t * kTile);
      const float2 e = w[(c.z0 * t) % c.nl];
      d.x = fmaf(v.x, e.x, fmaf(-v.y, e.y, d.x));
      d.y = fmaf(v.x, e.y, fmaf(v.y, e.x, d.y));
      if (++t == c.nl) t = 0;
    }
    float2 acc = c.state[i];
    acc.x = fmaf(c.sign, d.x, acc.x);
    acc.y = fmaf(c.sign, d.y, acc.y);
    c.state[i] = acc;
    if (c.xy && kxw < c.wx) c.xy[(size_t)kyw * c.wx + kxw] = envelope(acc, c.power_scale, c.magnitude);
  }
}

// xz and yz cuts: the axial kernel's transform on the tiles of row y0 (blocks
// 0 .. ntx-1) and on the tile holding column x0 of every row (the next wy
// blocks), keeping only the cut's pixels.
template <int NL>
__global__ void __launch_bounds__(kTile * Split<NL>::N1) gate_lines_kernel(const __grid_constant__ GateCutsParams c) {
  constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ex = reinterpret_cast<float2*>(smem);
  const bool xz_block = (int)blockIdx.x < c.ntx;
  const int kyw = xz_block ? c.y0 : (int)blockIdx.x - c.ntx;
  const int tile = xz_block ? (int)blockIdx.x : c.x0 / kTile;
  const int pix = threadIdx.x % kTile, j1 = threadIdx.x / kTile;
  const float2* src = c.inter + ((size_t)kyw * c.ntx + tile) * NL * kTile + pix;
  float2 a[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = __ldcs(src + (j1 + N1 * j2) * kTile);
  Dft<N2, -1>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], ldg2(c.twl + k2 * N1 + j1));
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * kTile + pix] = a[k2];
  __syncthreads();
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[(k2 * N1 + jj) * kTile + pix];
    Dft<N1, -1>::template run<1, i * N1>(a);
  });
  const int kxw = tile * kTile + pix;
  if (kxw >= c.wx) return;
  if (xz_block ? !c.xz : (!c.yz || kxw != c.x0)) return;
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int q = k2 + N2 * k1;
      const float pw = envelope(a[i * N1 + k1], c.power_scale, c.magnitude);
      if (xz_block) c.xz[(size_t)q * c.wx + kxw] = pw;
      else c.yz[(size_t)q * c.wy + kyw] = pw;
    }
  });
}

template <int NL>
cudaError_t launch_lines(const GateCutsParams& c, cudaStream_t s) {
  const size_t smem = (size_t)NL * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(gate_lines_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gate_lines_kernel<NL><<<c.ntx + c.wy, kTile * Split<NL>::N1, smem, s>>>(c);
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch_ra(const RescaleAxialParams& rp, cudaStream_t s) {
  const size_t smem = (size_t)NL * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(rescale_axial_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rescale_axial_kernel<NL><<<dim3(rp.nx / kTile, rp.ny), kTile * Split<NL>::N1, smem, s>>>(rp);
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch_ra_tiles(const RescaleAxialTileParams& rp, const CUtensorMap& fmap, int num_sms, cudaStream_t s) {
  using R = RaTile<NL>;
  const size_t smem = R::smem_bytes(rp.w);
  cudaError_t e = cudaFuncSetAttribute(rescale_axial_tile_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)(rp.nx / kRaStrip) * rp.ny;
  long long grid = num_sms > 0 ? num_sms : 1;
  if (grid > ntiles) grid = ntiles;
  rescale_axial_tile_kernel<NL><<<(unsigned)grid, R::kThreads, smem, s>>>(rp, fmap);
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch_stream(const AxialParams& ap, int num_sms, cudaStream_t s) {
  using S = AxStream<NL>;
  const size_t smem = (size_t)S::kStages * S::kTileBytes;
  cudaError_t e = cudaFuncSetAttribute(axial_stream_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, axial_stream_kernel<NL>, S::kThreadsAll, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long ntiles = (long long)ap.ntx * ap.wy;
  long long grid = (long long)(num_sms > 0 ? num_sms : 1) * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  axial_stream_kernel<NL><<<(unsigned)grid, S::kThreadsAll, smem, s>>>(ap);
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch(const AxialParams& ap, int num_sms, cudaStream_t s) {
  // the streaming form where a tile fits a third of the ring and a group has
  // eight warps or more; otherwise one CTA per tile
  constexpr bool kStream = (size_t)NL * kTile * sizeof(float2) <= 64 * 1024 && kTile * split_n1(NL) >= 256;
  if constexpr (kStream) return launch_stream<NL>(ap, num_sms, s);
  const size_t smem = (size_t)NL * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(axial_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ap.ntx, ap.wy);
  axial_kernel<NL><<<grid, kTile * Split<NL>::N1, smem, s>>>(ap);
  return cudaGetLastError();
}

#define SSOCT_AXIAL_SIZES(X) X(16) X(32) X(64) X(96) X(128) X(160) X(200) X(256) X(512)

}  // namespace

cudaError_t launch_xy_slide(const Plan& p, int slot0, int k, int z0, float sign, float* xy, cudaStream_t s) {
  XySlideParams c;
  c.inter = (const float2*)(p.ws + p.off_inter);
  c.wq = (const float2*)(p.ws + p.off_wq);
  c.state = (float2*)(p.ws + p.off_xys);
  c.xy = xy;
  c.nl = p.nl; c.wx = p.wx; c.wy = p.wy; c.ntx = p.ntx;
  c.z0 = z0; c.slot0 = slot0; c.k = k;
  c.sign = sign;
  c.power_scale = (float)(p.alpha * p.alpha);
  c.magnitude = (p.flags & SSOCT_FLAG_MAGNITUDE) ? 1 : 0;
  xy_slide_kernel<<<4 * p.num_sms, 256, (size_t)p.nl * sizeof(float2), s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_gate_cuts(const Plan& p, int x0, int y0, int z0, float* xy, float* xz, float* yz,
                             float2* xy_state, cudaStream_t s) {
  GateCutsParams c;
  c.inter = (const float2*)(p.ws + p.off_inter);
  c.wq = (const float2*)(p.ws + p.off_wq);
  c.twl = (const float2*)(p.ws + p.off_twl);
  c.xy = xy;
  c.xz = xz;
  c.yz = yz;
  c.xy_state = xy_state;
  c.nl = p.nl; c.wx = p.wx; c.wy = p.wy; c.ntx = p.ntx;
  c.x0 = x0; c.y0 = y0; c.z0 = z0;
  c.power_scale = (float)(p.alpha * p.alpha);
  c.magnitude = (p.flags & SSOCT_FLAG_MAGNITUDE) ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (xy) {
    gate_xy_kernel<<<4 * p.num_sms, 256, (size_t)p.nl * sizeof(float2), s>>>(c);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || (!xz && !yz)) return e;
#define X(a) if (p.nl == a) return launch_lines<a>(c, s);
  SSOCT_AXIAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
}

bool rescale_axial_tiled(int nx, int nl) {
  return nx % kRaStrip == 0 && (nl == 64 || nl == 96 || nl == 128 || nl == 160 || nl == 200 || nl == 256);
}

size_t rescale_axial_tile_smem(int nl, int w) {
  if (nl == 64) return RaTile<64>::smem_bytes(w);
  if (nl == 96) return RaTile<96>::smem_bytes(w);
  if (nl == 128) return RaTile<128>::smem_bytes(w);
  if (nl == 160) return RaTile<160>::smem_bytes(w);
  if (nl == 200) return RaTile<200>::smem_bytes(w);
  if (nl == 256) return RaTile<256>::smem_bytes(w);
  return 0;
}

cudaError_t launch_rescale_axial(const Plan& p, const uint16_t* frames, int ring_start, float2* planes,
                                 cudaStream_t s) {
  if (p.ra_w > 0) {
    alignas(64) CUtensorMap fmap;
    if (!encode_frames_map(p, frames, p.ra_w, &fmap)) return cudaErrorInvalidValue;
    RescaleAxialTileParams tp;
    tp.ring_start = ring_start;
    tp.xstrip = (const StripTap*)(p.ws + p.off_xstrip);
    tp.ytab = (const Tap*)(p.ws + p.off_ytab);
    tp.twl = (const float2*)(p.ws + p.off_twra);
    tp.planes = planes;
    tp.cx = (const float2*)(p.ws + p.off_cx);
    tp.cy = (const float2*)(p.ws + p.off_cy);
    tp.k_abs = (float)p.alpha;
    tp.nx = p.nx;
    tp.ny = p.ny;
    tp.w = p.ra_w;
    tp.err = &((Counters*)(p.ws + p.off_ctr))->err;
    if (p.nl == 64) return launch_ra_tiles<64>(tp, fmap, p.num_sms, s);
    if (p.nl == 96) return launch_ra_tiles<96>(tp, fmap, p.num_sms, s);
    if (p.nl == 128) return launch_ra_tiles<128>(tp, fmap, p.num_sms, s);
    if (p.nl == 160) return launch_ra_tiles<160>(tp, fmap, p.num_sms, s);
    if (p.nl == 200) return launch_ra_tiles<200>(tp, fmap, p.num_sms, s);
    if (p.nl == 256) return launch_ra_tiles<256>(tp, fmap, p.num_sms, s);
    return cudaErrorInvalidValue;
  }
  RescaleAxialParams rp;
  rp.frames = frames;
  rp.ring_start = ring_start;
  rp.xtab = (const Tap*)(p.ws + p.off_xtab);
  rp.ytab = (const Tap*)(p.ws + p.off_ytab);
  rp.twl = (const float2*)(p.ws + p.off_twl);
  rp.planes = planes;
  rp.cx = (const float2*)(p.ws + p.off_cx);
  rp.cy = (const float2*)(p.ws + p.off_cy);
  rp.k_abs = (float)p.alpha;
  rp.nx = p.nx;
  rp.ny = p.ny;
  rp.nl = p.nl;
#define X(a) if (p.nl == a) return launch_ra<a>(rp, s);
  SSOCT_AXIAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
}

bool axial_supported(int nl) {
#define X(a) if (nl == a) return true;
  SSOCT_AXIAL_SIZES(X)
#undef X
  return false;
}

cudaError_t launch_axial_with(const Plan& p, const AxialParams& ap, int num_sms, cudaStream_t s) {
#define X(a) if (p.nl == a) return launch<a>(ap, num_sms, s);
  SSOCT_AXIAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_axial(const Plan& p, const AxialParams& ap, cudaStream_t s) {
  return launch_axial_with(p, ap, p.num_sms, s);
}

// The three orthogonal cuts: plain gathers from the volume [q][y][x].
__global__ void cuts_kernel(const __grid_constant__ CutsParams c) {
  const size_t nxy = c.xy ? (size_t)c.wy * c.wx : 0;
  const size_t nxz = c.xz ? (size_t)c.nl * c.wx : 0;
  const size_t nyz = c.yz ? (size_t)c.nl * c.wy : 0;
  const size_t plane = (size_t)c.wy * c.wx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nxy + nxz + nyz;
       i += (size_t)gridDim.x * blockDim.x) {
    if (i < nxy) {
      c.xy[i] = c.vol[(size_t)c.z0 * plane + i];
    } else if (i < nxy + nxz) {
      const size_t k = i - nxy;
      const size_t q = k / c.wx, x = k % c.wx;
      c.xz[k] = c.vol[q * plane + (size_t)c.y0 * c.wx + x];
    } else {
      const size_t k = i - nxy - nxz;
      const size_t q = k / c.wy, y = k % c.wy;
      c.yz[k] = c.vol[q * plane + y * c.wx + c.x0];
    }
  }
}

cudaError_t launch_cuts(const CutsParams& cp, cudaStream_t s) {
  const size_t n = (cp.xy ? (size_t)cp.wy * cp.wx : 0) + (cp.xz ? (size_t)cp.nl * cp.wx : 0) +
                   (cp.yz ? (size_t)cp.nl * cp.wy : 0);
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  cuts_kernel<<<blocks, 256, 0, s>>>(cp);
  return cudaGetLastError();
}

}  // namespace ssoct
