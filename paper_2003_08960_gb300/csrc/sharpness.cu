// Aberration correction: the reconstruction with a Zernike phase screen in the
// sensor plane, the sharpness of its intensity volume and the gradient of that
// sharpness with respect to the reconstruction distance z and the coefficients
// c_1..c_15, by one hand-written adjoint pass.
//
// Forward (the chain of Eq. 5 - Eq. 7 with the screen P = exp(i sum_j c_j Z_j)
// multiplied into the input chirp c of Eq. 6):
//   rows    u_t = Eq. 5 resample of frame t;  row DFT (+) of c P u_t      -> F[t][y][x]
//   columns column DFT (+), window crop                                  -> sweep-axis intermediate
//   axial   Eq. 7 over t, P_v = |K|^2 |V~_v|^2                            -> volume
//   sums    S1 = sum P_v, S2 = sum P_v^2 (FP64); L = -S2 / S1^2
// Adjoint (W = 2 |K|^2 dL/dP V~, dL/dP = -2 P / S1^2 + 2 S2 / S1^3):
//   axial   V~ recomputed, W formed, sum_q W_q exp(+2 pi i q t / N)      -> intermediate (in place)
//   columns zero outside the window, column DFT (-)                      -> F[t][y][x]
//   rows    row DFT (-) = Y_t; Q = sum_t conj(Y_t) u_t with u_t recomputed from the uint16 frames
//   grad    M = -Im(c P Q); dL/dc_j = sum Z_j M; dL/dz = (pi |K| / z) sum r_pix^2 M
// The DFTs here are the uncentred ones of the lateral kernel, with the centring
// phase (-1)^n folded into c; the unit-modulus factors this moves onto V~ cancel
// in W's round trip, so M is the same as with the centred transform.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fft_common.cuh"

namespace ssoct {
namespace {

constexpr int kRowThreads = 256;
constexpr int kGradThreads = 256;

// Split N = N1 x N2 of one axis for these kernels: stage 1 is N2-point DFTs in
// the N1 threads of a transform, stage 2 the N2 N1-point DFTs spread over those
// threads, NI per thread (the last ones idle when N1 does not divide N2, e.g.
// 640 = 32 x 20).  AS is the register array length, TW the width of a column
// tile (16 when 32 N1 threads would exceed 512).
template <int N>
struct Lat {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int NI = (N2 + N1 - 1) / N1;
  static constexpr int AS = NI * N1 > N2 ? NI * N1 : N2;
};
// Column-tile width for axis length N (a variable template, instantiated only
// for the column kernels that use it).
template <int N>
constexpr int kLatTW = kTile * Split<N>::N1 <= 512 ? kTile : kTile / 2;

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }


// Row DFT of sign S over the registers of thread (r, j1) of an N1 x N2 split:
// on entry a[j2] = x[j1 + N1 j2]; on exit a[i N1 + k1] = X[k2 + N2 k1] with
// k2 = j1 + N1 i for the i with k2 < N2.  ex is this row's padded exchange
// block; a row's N1 threads lie in one warp.
template <int N, int S>
__device__ __forceinline__ void row_dft(float2 (&a)[Lat<N>::AS], const float2* tw, float2* ex, int j1) {
  constexpr int N1 = Lat<N>::N1, N2 = Lat<N>::N2, NI = Lat<N>::NI;
  Dft<N2, S>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const float2 w = ldg2(tw + k2 * N1 + j1);
    a[k2] = cmul(a[k2], S > 0 ? w : conjf2(w));
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[k2 * (N1 + 1) + j1] = a[k2];
  __syncwarp();
  static_for<0, NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[k2 * (N1 + 1) + jj];
      Dft<N1, S>::template run<1, i * N1>(a);
    }
  });
}

// Column DFT of sign S over 32-wide tiles: thread (pix, j1), a[j2] = x[j1 + N1 j2]
// on entry, a[i N1 + k1] = X[k2 + N2 k1] (k2 = j1 + N1 i) on exit.  tw holds the
// twiddles of sign TS (conjugated when S differs).
template <int N, int S, int TS, int TW>
__device__ __forceinline__ void col_dft(float2 (&a)[Lat<N>::AS], const float2* tw, float2* ex, int j1, int pix) {
  constexpr int N1 = Lat<N>::N1, N2 = Lat<N>::N2, NI = Lat<N>::NI;
  Dft<N2, S>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const float2 w = ldg2(tw + k2 * N1 + j1);
    a[k2] = cmul(a[k2], S == TS ? w : conjf2(w));
  }
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[(k2 * N1 + j1) * TW + pix] = a[k2];
  __syncthreads();
  static_for<0, NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[(k2 * N1 + jj) * TW + pix];
      Dft<N1, S>::template run<1, i * N1>(a);
    }
  });
}

struct ShParams {
  const uint16_t* frames;  // [nl][ny][nx]
  const Tap* xtab;         // [nl][nx]
  const Tap* ytab;         // [nl][ny]
  const float2* cp;        // [ny][nx] input chirp (with centring) x pupil screen
  const float2* twx;       // [N2x][N1x], sign +
  const float2* twy;       // [N2y][N1y], sign +
  const float2* twl;       // [N2l][N1l], sign -
  float2* F;               // [nl][ny][nx] lateral work frames
  float2* inter;           // [wy][ntx][nl][32] sweep-axis intermediate
  float2* qpart;           // [chunks][ny][nx] partial Q
  const float* vol;        // [nl][wy][wx] P_v
  double* red;             // [0] S1, [1] S2, [2..18] loss, dL/dz, dL/dc_1..15
  int nx, ny, nl, x0, y0, wx, wy, ntx, tpc;
  int ring_start;          // frame t of the gate is frames[(ring_start + t) mod nl]
  float alpha2;            // |K|^2
  double scale_z;          // pi |K| / z
};

// ----------------------------------------------------------------- forward

template <int NX>
__global__ void __launch_bounds__(kRowThreads) rows_fwd_kernel(const __grid_constant__ ShParams p) {
  constexpr int N1 = Lat<NX>::N1, N2 = Lat<NX>::N2, RPI = kRowThreads / N1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x / N1, j1 = threadIdx.x % N1;
  const int y = blockIdx.x * RPI + r, t = blockIdx.y;
  float2* ex = reinterpret_cast<float2*>(smem) + r * N2 * (N1 + 1);
  const uint16_t* fr = p.frames + (size_t)((p.ring_start + t) % p.nl) * p.ny * NX;
  const Tap ty = p.ytab[(size_t)t * p.ny + y];
  const float2* cp = p.cp + (size_t)y * NX;
  float2 a[Lat<NX>::AS];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int n = j1 + N1 * j2;
    const float u = rescale_tap_value(fr, NX, p.xtab[(size_t)t * NX + n], ty);
    const float2 c = ldg2(cp + n);
    a[j2] = make_float2(u * c.x, u * c.y);
  }
  row_dft<NX, 1>(a, p.twx, ex, j1);
  float2* dst = p.F + ((size_t)t * p.ny + y) * NX;
  static_for<0, Lat<NX>::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) dst[k2 + N2 * k1] = a[i * N1 + k1];
    }
  });
}

template <int NY>
__global__ void __launch_bounds__(kLatTW<NY> * Lat<NY>::N1) cols_fwd_kernel(const __grid_constant__ ShParams p) {
  constexpr int N1 = Lat<NY>::N1, N2 = Lat<NY>::N2, TW = kLatTW<NY>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int pix = threadIdx.x % TW, j1 = threadIdx.x / TW;
  const int x = blockIdx.x * TW + pix, t = blockIdx.y;
  const float2* src = p.F + (size_t)t * NY * p.nx + x;
  float2 a[Lat<NY>::AS];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = src[(size_t)(j1 + N1 * j2) * p.nx];
  col_dft<NY, 1, 1, TW>(a, p.twy, reinterpret_cast<float2*>(smem), j1, pix);
  const int kxw = x - p.x0;
  if (kxw < 0 || kxw >= p.wx) return;
  float2* dst = p.inter + ((size_t)(kxw / kTile) * p.nl + t) * kTile + kxw % kTile;
  const size_t row_pitch = (size_t)p.ntx * p.nl * kTile;
  static_for<0, Lat<NY>::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int kyw = k2 + N2 * k1 - p.y0;
        if (kyw >= 0 && kyw < p.wy) dst[(size_t)kyw * row_pitch] = a[i * N1 + k1];
      }
    }
  });
}

// S1 = sum P, S2 = sum P^2 over the volume, FP64.
__global__ void __launch_bounds__(kGradThreads) sums_kernel(const __grid_constant__ ShParams p, size_t n) {
  double s1 = 0.0, s2 = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = p.vol[i];
    s1 += v;
    s2 += v * v;
  }
  __shared__ double sh[2][kGradThreads / 32];
  for (int o = 16; o; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (threadIdx.x % 32 == 0) {
    sh[0][threadIdx.x / 32] = s1;
    sh[1][threadIdx.x / 32] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kGradThreads / 32; ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    atomicAdd(p.red + 0, a);
    atomicAdd(p.red + 1, b);
  }
}

// ----------------------------------------------------------------- adjoint

template <int NL>
__global__ void __launch_bounds__(kTile * Split<NL>::N1) axial_adj_kernel(const __grid_constant__ ShParams p) {
  constexpr int N1 = Split<NL>::N1, N2 = Split<NL>::N2;
  static_assert(N2 % N1 == 0, "sweep lengths split with N1 | N2");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ex = reinterpret_cast<float2*>(smem);
  const int pix = threadIdx.x % kTile, j1 = threadIdx.x / kTile;
  float2* g = p.inter + ((size_t)blockIdx.y * p.ntx + blockIdx.x) * NL * kTile + pix;
  const double s1 = p.red[0], s2 = p.red[1];
  const float a1 = (float)(-2.0 / (s1 * s1)), a0 = (float)(2.0 * s2 / (s1 * s1 * s1));
  float2 a[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = g[(j1 + N1 * j2) * kTile];
  col_dft<NL, -1, -1, kTile>(a, p.twl, ex, j1, pix);  // V~[q = k2 + N2 k1]
  __syncthreads();
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 v = a[i * N1 + k1];
      const float pw = p.alpha2 * fmaf(v.x, v.x, v.y * v.y);
      const float s = 2.f * p.alpha2 * fmaf(a1, pw, a0);
      ex[(k2 + N2 * k1) * kTile + pix] = make_float2(s * v.x, s * v.y);  // W in natural order
    }
  });
  __syncthreads();
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = ex[(j1 + N1 * j2) * kTile + pix];
  // sum_q W_q exp(+2 pi i q t / NL): the same split with the conjugate twiddles
  col_dft<NL, 1, -1, kTile>(a, p.twl, ex, j1, pix);
  static_for<0, N2 / N1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) g[(k2 + N2 * k1) * kTile] = a[i * N1 + k1];
  });
}

template <int NY>
__global__ void __launch_bounds__(kLatTW<NY> * Lat<NY>::N1) cols_adj_kernel(const __grid_constant__ ShParams p) {
  constexpr int N1 = Lat<NY>::N1, N2 = Lat<NY>::N2, TW = kLatTW<NY>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int pix = threadIdx.x % TW, j1 = threadIdx.x / TW;
  const int x = blockIdx.x * TW + pix, t = blockIdx.y;
  const int kxw = x - p.x0;
  const bool inx = kxw >= 0 && kxw < p.wx;
  const float2* src = p.inter + ((size_t)(inx ? kxw / kTile : 0) * p.nl + t) * kTile + (inx ? kxw % kTile : 0);
  const size_t row_pitch = (size_t)p.ntx * p.nl * kTile;
  float2 a[Lat<NY>::AS];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int kyw = j1 + N1 * j2 - p.y0;
    a[j2] = (inx && kyw >= 0 && kyw < p.wy) ? src[(size_t)kyw * row_pitch] : make_float2(0.f, 0.f);
  }
  // the adjoint of the forward column DFT (+) is the column DFT (-), with the forward table conjugated
  col_dft<NY, -1, 1, TW>(a, p.twy, reinterpret_cast<float2*>(smem), j1, pix);
  float2* dst = p.F + (size_t)t * NY * p.nx + x;
  static_for<0, Lat<NY>::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) dst[(size_t)(k2 + N2 * k1) * p.nx] = a[i * N1 + k1];
    }
  });
}

template <int NX>
__global__ void __launch_bounds__(kRowThreads) rows_adj_kernel(const __grid_constant__ ShParams p) {
  constexpr int N1 = Lat<NX>::N1, N2 = Lat<NX>::N2, RPI = kRowThreads / N1, AS = Lat<NX>::AS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x / N1, j1 = threadIdx.x % N1;
  const int y = blockIdx.x * RPI + r, chunk = blockIdx.y;
  float2* ex = reinterpret_cast<float2*>(smem) + r * N2 * (N1 + 1);
  const int t0 = chunk * p.tpc, t1 = min(p.nl, t0 + p.tpc);
  float2 acc[AS];
#pragma unroll
  for (int i = 0; i < AS; ++i) acc[i] = make_float2(0.f, 0.f);
  for (int t = t0; t < t1; ++t) {
    const float2* src = p.F + ((size_t)t * p.ny + y) * NX;
    float2 a[AS];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) a[j2] = src[j1 + N1 * j2];
    row_dft<NX, -1>(a, p.twx, ex, j1);
    const uint16_t* fr = p.frames + (size_t)((p.ring_start + t) % p.nl) * p.ny * NX;
    const Tap ty = p.ytab[(size_t)t * p.ny + y];
    const Tap* xt = p.xtab + (size_t)t * NX;
    static_for<0, Lat<NX>::NI>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const int k2 = j1 + N1 * i;
      if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          const float u = rescale_tap_value(fr, NX, xt[k2 + N2 * k1], ty);
          const float2 v = a[i * N1 + k1];
          acc[i * N1 + k1].x = fmaf(v.x, u, acc[i * N1 + k1].x);   // conj(Y) u
          acc[i * N1 + k1].y = fmaf(-v.y, u, acc[i * N1 + k1].y);
        }
      }
    });
  }
  float2* dst = p.qpart + ((size_t)chunk * p.ny + y) * NX;
  static_for<0, Lat<NX>::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (N2 % N1 == 0 || k2 < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) dst[k2 + N2 * k1] = acc[i * N1 + k1];
    }
  });
}

}  // namespace

// Z_1..Z_15 (Noll order, RMS-normalised on the unit disk; Noll 1976) at radius
// rho and angle (cos th, sin th).
__host__ __device__ __forceinline__ void zernike15(double rho, double c1, double s1, double (&z)[15]) {
  const double r2 = rho * rho, r3 = r2 * rho, r4 = r2 * r2;
  const double c2 = c1 * c1 - s1 * s1, s2 = 2.0 * s1 * c1;
  const double c3 = c2 * c1 - s2 * s1, s3 = s2 * c1 + c2 * s1;
  const double c4 = c2 * c2 - s2 * s2, s4 = 2.0 * s2 * c2;
  const double q3 = 1.7320508075688772935, q5 = 2.2360679774997896964, q6 = 2.4494897427831780982,
               q8 = 2.8284271247461900976, q10 = 3.1622776601683793320;
  z[0] = 1.0;
  z[1] = 2.0 * rho * c1;
  z[2] = 2.0 * rho * s1;
  z[3] = q3 * (2.0 * r2 - 1.0);
  z[4] = q6 * r2 * s2;
  z[5] = q6 * r2 * c2;
  z[6] = q8 * (3.0 * r3 - 2.0 * rho) * s1;
  z[7] = q8 * (3.0 * r3 - 2.0 * rho) * c1;
  z[8] = q8 * r3 * s3;
  z[9] = q8 * r3 * c3;
  z[10] = q5 * (6.0 * r4 - 6.0 * r2 + 1.0);
  z[11] = q10 * (4.0 * r4 - 3.0 * r2) * c2;
  z[12] = q10 * (4.0 * r4 - 3.0 * r2) * s2;
  z[13] = q10 * r4 * c4;
  z[14] = q10 * r4 * s4;
}

namespace {

__global__ void __launch_bounds__(kGradThreads) grad_kernel(const __grid_constant__ ShParams p, int chunks) {
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  const size_t npix = (size_t)p.nx * p.ny;
  const double cxp = p.nx / 2.0, cyp = p.ny / 2.0;
  const double inv_radius = 2.0 / (double)min(p.nx, p.ny);  // rho = r_pix / (min(nx, ny) / 2)
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
    double qx = 0.0, qy = 0.0;
    for (int c = 0; c < chunks; ++c) {
      const float2 q = p.qpart[(size_t)c * npix + i];
      qx += q.x;
      qy += q.y;
    }
    const float2 cp = p.cp[i];
    const double m = -((double)cp.x * qy + (double)cp.y * qx);  // -Im(c P Q)
    const double dx = (double)(i % p.nx) - cxp, dy = (double)(i / p.nx) - cyp;
    const double r2 = dx * dx + dy * dy;
    const double rp = sqrt(r2);
    const double c1 = rp > 0.0 ? dx / rp : 1.0, s1 = rp > 0.0 ? dy / rp : 0.0;
    double z[15];
    zernike15(rp * inv_radius, c1, s1, z);
    acc[0] += r2 * m;
#pragma unroll
    for (int j = 0; j < 15; ++j) acc[1 + j] += z[j] * m;
  }
  __shared__ double sh[16][kGradThreads / 32];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    double v = acc[j];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x % 32 == 0) sh[j][threadIdx.x / 32] = v;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    double v = 0.0;
    for (int w = 0; w < kGradThreads / 32; ++w) v += sh[threadIdx.x][w];
    atomicAdd(p.red + 3 + threadIdx.x, threadIdx.x == 0 ? v * p.scale_z : v);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.red[2] = -p.red[1] / (p.red[0] * p.red[0]);
}

// ----------------------------------------------------------------- launchers

template <class K>
cudaError_t launch_k(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t s, const ShParams& p) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NX>
size_t row_smem() {
  return (size_t)(kRowThreads / Lat<NX>::N1) * Lat<NX>::N2 * (Lat<NX>::N1 + 1) * sizeof(float2);
}

template <int NX>
cudaError_t rows(bool adjoint, const ShParams& p, int chunks, cudaStream_t s) {
  constexpr int RPI = kRowThreads / Lat<NX>::N1;
  if (adjoint) return launch_k(rows_adj_kernel<NX>, dim3(p.ny / RPI, chunks), kRowThreads, row_smem<NX>(), s, p);
  return launch_k(rows_fwd_kernel<NX>, dim3(p.ny / RPI, p.nl), kRowThreads, row_smem<NX>(), s, p);
}

template <int NY>
cudaError_t cols(bool adjoint, const ShParams& p, cudaStream_t s) {
  constexpr int TW = kLatTW<NY>;
  const size_t smem = (size_t)Lat<NY>::N2 * Lat<NY>::N1 * TW * sizeof(float2);
  const dim3 grid(p.nx / TW, p.nl);
  if (adjoint) return launch_k(cols_adj_kernel<NY>, grid, TW * Lat<NY>::N1, smem, s, p);
  return launch_k(cols_fwd_kernel<NY>, grid, TW * Lat<NY>::N1, smem, s, p);
}

template <int NL>
cudaError_t axial_adj(const ShParams& p, cudaStream_t s) {
  return launch_k(axial_adj_kernel<NL>, dim3(p.ntx, p.wy), kTile * Split<NL>::N1, (size_t)NL * kTile * sizeof(float2),
                  s, p);
}

cudaError_t rows_any(bool adj, const ShParams& p, int chunks, cudaStream_t s) {
  switch (p.nx) {
    case 64: return rows<64>(adj, p, chunks, s);
    case 128: return rows<128>(adj, p, chunks, s);
    case 256: return rows<256>(adj, p, chunks, s);
    case 384: return rows<384>(adj, p, chunks, s);
    case 512: return rows<512>(adj, p, chunks, s);
    case 640: return rows<640>(adj, p, chunks, s);
    case 768: return rows<768>(adj, p, chunks, s);
    case 1024: return rows<1024>(adj, p, chunks, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t cols_any(bool adj, const ShParams& p, cudaStream_t s) {
  switch (p.ny) {
    case 64: return cols<64>(adj, p, s);
    case 128: return cols<128>(adj, p, s);
    case 256: return cols<256>(adj, p, s);
    case 384: return cols<384>(adj, p, s);
    case 512: return cols<512>(adj, p, s);
    case 640: return cols<640>(adj, p, s);
    case 768: return cols<768>(adj, p, s);
    case 1024: return cols<1024>(adj, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t axial_adj_any(const ShParams& p, cudaStream_t s) {
  switch (p.nl) {
    case 16: return axial_adj<16>(p, s);
    case 32: return axial_adj<32>(p, s);
    case 64: return axial_adj<64>(p, s);
    case 96: return axial_adj<96>(p, s);
    case 128: return axial_adj<128>(p, s);
    case 160: return axial_adj<160>(p, s);
    case 200: return axial_adj<200>(p, s);
    case 256: return axial_adj<256>(p, s);
    case 512: return axial_adj<512>(p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// c P on the sensor grid: the input chirp of Eq. 6 with its centring phase,
// exp(-i pi [alpha (n - N/2)^2 + n]) per axis, times exp(i sum_j c_j Z_j).  Phases
// are reduced in units of pi in float64 before the float32 rounding.
void build_pupil_table(int nx, int ny, double alpha, const double* coeffs, int ncoeffs, std::vector<float2>& out) {
  out.resize((size_t)nx * ny);
  const double pi = 3.14159265358979323846264338327950288;
  const double inv_radius = 2.0 / (double)(nx < ny ? nx : ny);
  for (int l = 0; l < ny; ++l)
    for (int n = 0; n < nx; ++n) {
      const double dx = n - nx / 2.0, dy = l - ny / 2.0;
      double turns = -(std::fmod(alpha * dx * dx, 2.0) + (double)(n & 1)) - (std::fmod(alpha * dy * dy, 2.0) + (double)(l & 1));
      const double rp = std::sqrt(dx * dx + dy * dy);
      double z[15];
      zernike15(rp * inv_radius, rp > 0.0 ? dx / rp : 1.0, rp > 0.0 ? dy / rp : 0.0, z);
      double phi = 0.0;
      for (int j = 0; j < ncoeffs; ++j) phi += coeffs[j] * z[j];
      turns += std::fmod(phi / pi, 2.0);
      out[(size_t)l * nx + n] = make_float2((float)std::cos(pi * turns), (float)std::sin(pi * turns));
    }
}

namespace {

struct PupilParams {
  float2* cp;
  int nx, ny, ncoeffs;
  double alpha;
  double c[15];
};

// c P per sensor pixel, the device twin of build_pupil_table: phases reduced in
// units of pi in float64, one rounding to float32 at the end.
__global__ void __launch_bounds__(256) pupil_table_kernel(const __grid_constant__ PupilParams p) {
  const size_t npix = (size_t)p.nx * p.ny;
  const double inv_radius = 2.0 / (double)min(p.nx, p.ny);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(i % p.nx), l = (int)(i / p.nx);
    const double dx = n - p.nx / 2.0, dy = l - p.ny / 2.0;
    double turns = -(fmod(p.alpha * dx * dx, 2.0) + (double)(n & 1)) - (fmod(p.alpha * dy * dy, 2.0) + (double)(l & 1));
    const double rp = sqrt(dx * dx + dy * dy);
    double z[15];
    zernike15(rp * inv_radius, rp > 0.0 ? dx / rp : 1.0, rp > 0.0 ? dy / rp : 0.0, z);
    double phi = 0.0;
    for (int j = 0; j < p.ncoeffs; ++j) phi += p.c[j] * z[j];
    turns += fmod(phi / 3.14159265358979323846, 2.0);
    double sn, cs;
    sincospi(turns, &sn, &cs);
    p.cp[i] = make_float2((float)cs, (float)sn);
  }
}

}  // namespace

cudaError_t launch_pupil_table(const Plan& pl, cudaStream_t s) {
  PupilParams p;
  p.cp = (float2*)(pl.ws + pl.off_cp);
  p.nx = pl.nx;
  p.ny = pl.ny;
  p.ncoeffs = pl.sh_ncoeffs;
  p.alpha = pl.sh_alpha;
  for (int j = 0; j < 15; ++j) p.c[j] = j < pl.sh_ncoeffs ? pl.sh_coeffs[j] : 0.0;
  pupil_table_kernel<<<2 * pl.num_sms, 256, 0, s>>>(p);
  return cudaGetLastError();
}

bool generic_lateral_supported(int nx, int ny) {
  auto ok = [](int n) {
    return n == 64 || n == 128 || n == 256 || n == 384 || n == 512 || n == 640 || n == 768 || n == 1024;
  };
  return ok(nx) && ok(ny);
}

bool sharpness_supported(int nx, int ny, int nl) { return generic_lateral_supported(nx, ny) && axial_supported(nl); }

cudaError_t launch_lateral_generic(const Plan& pl, const uint16_t* frames, int ring_start, cudaStream_t s) {
  char* ws = pl.ws;
  ShParams p = {};
  p.frames = frames;
  p.xtab = (const Tap*)(ws + pl.off_xtab);
  p.ytab = (const Tap*)(ws + pl.off_ytab);
  p.cp = (const float2*)(ws + pl.off_cg);
  p.twx = (const float2*)(ws + pl.off_twx);
  p.twy = (const float2*)(ws + pl.off_twy);
  p.twl = (const float2*)(ws + pl.off_twl);
  p.F = (float2*)(ws + pl.off_F);
  p.inter = (float2*)(ws + pl.off_inter);
  p.nx = pl.nx; p.ny = pl.ny; p.nl = pl.nl;
  p.x0 = pl.x0; p.y0 = pl.y0; p.wx = pl.wx; p.wy = pl.wy; p.ntx = pl.ntx;
  p.ring_start = ring_start;
  cudaError_t e = rows_any(false, p, 1, s);
  if (e == cudaSuccess) e = cols_any(false, p, s);
  return e;
}

cudaError_t launch_sharpness(const Plan& pl, const uint16_t* frames, float* vol, cudaStream_t s) {
  char* ws = pl.ws;
  ShParams p = {};
  p.frames = frames;
  p.xtab = (const Tap*)(ws + pl.off_xtab);
  p.ytab = (const Tap*)(ws + pl.off_ytab);
  p.cp = (const float2*)(ws + pl.off_cp);
  p.twx = (const float2*)(ws + pl.off_twx);
  p.twy = (const float2*)(ws + pl.off_twy);
  p.twl = (const float2*)(ws + pl.off_twl);
  p.F = (float2*)(ws + pl.off_F);
  p.inter = (float2*)(ws + pl.off_inter);
  p.qpart = (float2*)(ws + pl.off_Q);
  p.vol = vol;
  p.red = (double*)(ws + pl.off_red);
  p.nx = pl.nx; p.ny = pl.ny; p.nl = pl.nl;
  p.x0 = pl.x0; p.y0 = pl.y0; p.wx = pl.wx; p.wy = pl.wy; p.ntx = pl.ntx;
  p.tpc = pl.sh_tpc;
  p.alpha2 = (float)(pl.sh_alpha * pl.sh_alpha);
  p.scale_z = 3.14159265358979323846 * pl.sh_alpha / pl.sh_z;
  const int chunks = (pl.nl + pl.sh_tpc - 1) / pl.sh_tpc;

  cudaError_t e = cudaMemsetAsync(p.red, 0, kShRedDoubles * sizeof(double), s);
  if (e == cudaSuccess) e = rows_any(false, p, chunks, s);
  if (e == cudaSuccess) e = cols_any(false, p, s);
  if (e == cudaSuccess) {
    AxialParams ap;
    ap.inter = p.inter;
    ap.vol = vol;
    ap.cplx = nullptr;
    ap.twl = p.twl;
    ap.ox = (const float2*)(ws + pl.off_ox);
    ap.oy = (const float2*)(ws + pl.off_oy);
    ap.nl = pl.nl; ap.wx = pl.wx; ap.wy = pl.wy; ap.ntx = pl.ntx;
    ap.power_scale = p.alpha2;
    ap.magnitude = 0;
    ap.err = &((Counters*)(ws + pl.off_ctr))->err;
    e = launch_axial(pl, ap, s);
  }
  const size_t nvox = (size_t)pl.nl * pl.wy * pl.wx;
  if (e == cudaSuccess) {
    sums_kernel<<<2 * pl.num_sms, kGradThreads, 0, s>>>(p, nvox);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = axial_adj_any(p, s);
  if (e == cudaSuccess) e = cols_any(true, p, s);
  if (e == cudaSuccess) e = rows_any(true, p, chunks, s);
  if (e == cudaSuccess) {
    grad_kernel<<<2 * pl.num_sms, kGradThreads, 0, s>>>(p, chunks);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace ssoct
