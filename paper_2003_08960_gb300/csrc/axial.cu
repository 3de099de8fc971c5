// Axial stage: transform over the sweep (Eq. 7, rectangular gate of N_lambda
// frames, kernel exp(-2 pi i q t / N_lambda), unnormalised) at every window
// pixel, then the envelope |V|^2 (or |V|) written as the float32 volume
// [q][y][x].  Optionally also V itself with the Eq. 6 prefactor and output
// chirp applied (unit-modulus factors apart from |K|, so |V|^2 needs only |K|^2).
//
// One CTA per 32-pixel tile of one window row: it streams the tile's
// N_lambda x 32 complex values (contiguous in the intermediate), runs the
// N_lambda-point DFT as N2-point DFTs in registers, a twiddle, an exchange
// through shared memory and N1-point DFTs, and stores 128-byte runs of the
// volume per depth bin.
#include "fft_common.cuh"

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

struct RescaleAxialParams {
  const uint16_t* frames;  // gate frame t at frames[(ring_start + t) mod nl]
  int ring_start;
  const Tap* xtab;         // [nl][nx]
  const Tap* ytab;         // [nl][ny]
  const float2* twl;       // [N2l][N1l], sign -
  float2* planes;          // [nl/2 + 1][ny][nx]
  int nx, ny, nl;
};

// Axial-first order, first pass: at every sensor pixel of a 32-pixel tile, the
// Eq. 5 resample of each frame of the gate (a real series over t), its Eq. 7
// transform over t, and bins q = 0 .. nl/2 as complex planes.  The rest of the
// spectrum is the conjugate mirror (real input) and is formed by the lateral
// pass.  Eq. 6 is linear and the same for every frame, so transforming over t
// before it gives the same V as the paper's order.
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
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int q = k2 + N2 * k1;
      if (q <= NL / 2) dst[(size_t)q * plane] = a[i * N1 + k1];
    }
  });
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
cudaError_t launch(const AxialParams& ap, cudaStream_t s) {
  const size_t smem = (size_t)NL * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(axial_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ap.ntx, ap.wy);
  axial_kernel<NL><<<grid, kTile * Split<NL>::N1, smem, s>>>(ap);
  return cudaGetLastError();
}

#define SSOCT_AXIAL_SIZES(X) X(16) X(32) X(64) X(96) X(128) X(160) X(200) X(256) X(512)

}  // namespace

cudaError_t launch_rescale_axial(const Plan& p, const uint16_t* frames, int ring_start, float2* planes,
                                 cudaStream_t s) {
  RescaleAxialParams rp;
  rp.frames = frames;
  rp.ring_start = ring_start;
  rp.xtab = (const Tap*)(p.ws + p.off_xtab);
  rp.ytab = (const Tap*)(p.ws + p.off_ytab);
  rp.twl = (const float2*)(p.ws + p.off_twl);
  rp.planes = planes;
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

cudaError_t launch_axial(const Plan& p, const AxialParams& ap, cudaStream_t s) {
#define X(a) if (p.nl == a) return launch<a>(ap, s);
  SSOCT_AXIAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
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
