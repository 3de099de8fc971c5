// Axial stage on the tensor cores: the transform over the sweep (Eq. 7) as two
// dense 16-point DFT stages (256 = 16 x 16) issued as tcgen05 MMAs, with FP32
// accumulation in tensor memory and split-precision BF16 operands.
//
// Stage 1, for every pixel p and j1 in [0, 16):
//   Y[k2] = sum_j2 H[j1 + 16 j2] w16^(j2 k2),   w16 = exp(-2 pi i / 16)
// then Y is multiplied by the twiddle w256^(j1 k2) (FP32, CUDA cores), and
// stage 2, for every pixel and k2:
//   V[k2 + 16 k1] = sum_j1 Y'[j1][k2] w16^(j1 k1).
// Each stage is a real GEMM D[M=128][N=32] = A[128][K=32] B[32][32]^T per block
// of 8 pixels: rows are (pixel, j1) (stage 1) or (pixel, k2) (stage 2), the K
// index runs over (real parts, imaginary parts) of the 16 inputs, and B is the
// real 32 x 32 form of the complex 16-point DFT matrix.  Operands are split as
// x = hi + lo with hi, lo in BF16 (BF16 keeps FP32's exponent range, so no
// scaling is needed), and D = Ahi Bhi + Ahi Blo + Alo Bhi; the dropped Alo Blo
// term and the rounding of lo put the relative error near 2^-16 per stage.
//
// One 256-thread CTA per 32-pixel tile of one window row (the sweep-axis
// intermediate stores such a tile as 256 x 32 contiguous complex values): 4
// blocks of 8 pixels, 24 MMAs per stage issued by one thread into 128 TMEM
// columns, results read back with tcgen05.ld, |V|^2 staged in shared memory and
// written as 128-byte rows of the volume.  70 KB of shared memory, 128 TMEM
// columns and at most 80 registers per thread let three CTAs share an SM, so
// that one CTA's loads overlap the others' conversions and MMAs; one thread
// waits for the MMAs while the rest wait at the CTA barrier.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fft_common.cuh"

namespace ssoct {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcN = 256;          // sweep length this kernel is built for
constexpr int kTcR = 16;           // radix of both stages
constexpr int kTcBlocks = 4;       // 8-pixel M blocks per 32-pixel tile
constexpr int kTcK = 2 * kTcR;     // 32: real + imaginary parts
constexpr unsigned kTcCols = kTcBlocks * kTcK;  // TMEM columns (fp32 accumulators)
constexpr unsigned long long kTcWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// K-major operand layout without swizzle: 8 x 8 core matrices of BF16 (8 rows
// of 16 bytes, contiguous), ordered [row group][k group]; offset in elements.
__host__ __device__ __forceinline__ int tc_core_off(int r, int k) {
  return ((r >> 3) * (kTcK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
constexpr unsigned kTcLbo = 128;                   // bytes between core matrices along K
constexpr unsigned kTcSbo = (kTcK / 8) * 128;      // bytes between 8-row groups

// Shared-memory matrix descriptor (no swizzle).
__device__ __forceinline__ uint64_t tc_desc(const void* base) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr(base) >> 4) & 0x3FFF);
  d |= (uint64_t)((kTcLbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kTcSbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__device__ __forceinline__ unsigned tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned d_tmem, uint64_t a, uint64_t b, unsigned idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"((unsigned)accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 lanes x 32 columns of fp32 from tensor memory (this warp's lane quadrant).
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32]) {
  unsigned u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}
// Bounded wait for an mbarrier phase (true on completion).
__device__ bool tc_wait(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_timer_ns() - t0 > kTcWaitNs) return false;
  }
}

// x = hi + lo, both BF16 (round to nearest even).
__device__ __forceinline__ void split_bf16(float x, unsigned short& hi, unsigned short& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

struct TcParams {
  const float2* inter;          // [wy][ntx][256][32]
  float* vol;                   // [256][wy][wx]
  float2* cplx;                 // optional
  const unsigned short* bmat;   // [2][32 x 32] BF16 hi, lo of the 16-point DFT matrix (core layout)
  const float2* twl;            // [16][16] w256^(j1 k2) at [k2 * 16 + j1]
  const float2* ox;
  const float2* oy;
  int wx, wy, ntx;
  float power_scale;
  int magnitude;
  unsigned* err;                // set to 1 if a wait ran out
};

__device__ __forceinline__ void split2_bf16(float a, float b, unsigned& hi, unsigned& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const unsigned*>(&h);
  lo = *reinterpret_cast<const unsigned*>(&l);
}

// Row of the M = 128 operand block for (8-pixel block entry pl, radix index i):
// i * 8 + pl keeps a warp's 32 pixels on distinct 16-byte slots of a core matrix.
__device__ __forceinline__ int tc_row(int i, int pl) { return i * 8 + pl; }

__global__ void __launch_bounds__(kTcThreads, 3) axial_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // A operands: [hi / lo][block][128 x 32] BF16; the |V|^2 tile reuses them
  unsigned short* A = reinterpret_cast<unsigned short*>(smem);
  constexpr int kABlock = 128 * kTcK;                        // elements per block
  unsigned short* Bs = A + 2 * kTcBlocks * kABlock;          // [hi / lo][32 x 32]
  float2* tw = reinterpret_cast<float2*>(Bs + 2 * kTcK * kTcK);
  constexpr int kOutStride = 40;                             // floats; conflict-free both ways
  float* out = reinterpret_cast<float*>(smem);               // [256][kOutStride] after stage 2
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tmem_base;
  __shared__ int ok_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tile = blockIdx.x, kyw = blockIdx.y;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "n"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  reinterpret_cast<uint4*>(Bs)[tid] = __ldg(reinterpret_cast<const uint4*>(p.bmat) + tid);  // 4 KB
  tw[tid] = ldg2(p.twl + tid);                                                             // 256 twiddles

  // 1. t = j1 + 16 j2 -> stage-1 row (pixel, j1), K = j2 (real) / 16 + j2 (imaginary).
  //    Work unit c = (j1, half of j2): 8 coalesced loads, 4 16-byte stores.
  {
    const float2* src = p.inter + ((size_t)kyw * p.ntx + tile) * kTcN * kTile + lane;
    const int blk = lane >> 3, pl = lane & 7;
    unsigned short* Ahi = A + blk * kABlock;
    unsigned short* Alo = A + (kTcBlocks + blk) * kABlock;
#pragma unroll 2
    for (int c = warp; c < 2 * kTcR; c += kTcThreads / 32) {
      const int j1 = c & 15, h = c >> 4;
      float2 x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = __ldcs(src + (j1 + 16 * (8 * h + i)) * kTile);
      uint4 hr, lr, hm, lm;
      split2_bf16(x[0].x, x[1].x, hr.x, lr.x);
      split2_bf16(x[2].x, x[3].x, hr.y, lr.y);
      split2_bf16(x[4].x, x[5].x, hr.z, lr.z);
      split2_bf16(x[6].x, x[7].x, hr.w, lr.w);
      split2_bf16(x[0].y, x[1].y, hm.x, lm.x);
      split2_bf16(x[2].y, x[3].y, hm.y, lm.y);
      split2_bf16(x[4].y, x[5].y, hm.z, lm.z);
      split2_bf16(x[6].y, x[7].y, hm.w, lm.w);
      const int r = tc_row(j1, pl);
      *reinterpret_cast<uint4*>(Ahi + tc_core_off(r, 8 * h)) = hr;
      *reinterpret_cast<uint4*>(Alo + tc_core_off(r, 8 * h)) = lr;
      *reinterpret_cast<uint4*>(Ahi + tc_core_off(r, 16 + 8 * h)) = hm;
      *reinterpret_cast<uint4*>(Alo + tc_core_off(r, 16 + 8 * h)) = lm;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_base;
  const unsigned idesc = tc_idesc(128, kTcK);
  // D = Ahi Bhi + Ahi Blo + Alo Bhi for each block, K = 32 as two K = 16 steps
  auto issue_stage = [&]() {
#pragma unroll 1
    for (int blk = 0; blk < kTcBlocks; ++blk) {
      const unsigned short* a_terms[3] = {A + blk * kABlock, A + blk * kABlock, A + (kTcBlocks + blk) * kABlock};
      const unsigned short* b_terms[3] = {Bs, Bs + kTcK * kTcK, Bs};
      bool acc = false;
#pragma unroll
      for (int term = 0; term < 3; ++term)
#pragma unroll
        for (int ks = 0; ks < kTcK / 16; ++ks) {
          tc_mma(tmem + (unsigned)(blk * kTcK), tc_desc(a_terms[term] + ks * 2 * 64), tc_desc(b_terms[term] + ks * 2 * 64),
                 idesc, acc);
          acc = true;
        }
    }
    tc_commit(&bar);
  };
  if (tid == 0) {
    issue_stage();
    ok_flag = tc_wait(&bar, 0) ? 1 : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok1 = ok_flag != 0;

  // 2. twiddle w256^(j1 k2) and re-layout as the stage-2 operand: row (pixel, k2),
  //    K = j1 (real) / 16 + j1 (imaginary).  Warp quadrant quad holds TMEM lanes
  //    32 quad .. 32 quad + 31, i.e. j1 = 4 quad + lane / 8 of each block.
  const int quad = warp & 3;
  if (ok1) {
#pragma unroll 1
    for (int hblk = 0; hblk < 2; ++hblk) {
      const int blk = (warp >> 2) + 2 * hblk;
      float v[32];
      tc_ld32(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(blk * kTcK), v);
      const int r = quad * 32 + lane;
      const int j1 = r >> 3, pl = r & 7;
      unsigned short* Ahi = A + blk * kABlock;
      unsigned short* Alo = A + (kTcBlocks + blk) * kABlock;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const float2 z = cmul(make_float2(v[k2], v[16 + k2]), tw[k2 * 16 + j1]);
        const int r2 = tc_row(k2, pl);
        unsigned short hr, lr, hm, lm;
        split_bf16(z.x, hr, lr);
        split_bf16(z.y, hm, lm);
        Ahi[tc_core_off(r2, j1)] = hr;
        Alo[tc_core_off(r2, j1)] = lr;
        Ahi[tc_core_off(r2, 16 + j1)] = hm;
        Alo[tc_core_off(r2, 16 + j1)] = lm;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    if (ok1) issue_stage();
    ok_flag = (ok1 && tc_wait(&bar, 1)) ? 1 : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok2 = ok_flag != 0;

  // 3. V[k2 + 16 k1] sits in row (pixel, k2), columns k1 (real) / 16 + k1 (imaginary)
  const int kx0 = tile * kTile;
#pragma unroll 1
  for (int hblk = 0; hblk < 2; ++hblk) {
    const int blk = (warp >> 2) + 2 * hblk;
    float v[32];
    if (ok2) tc_ld32(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(blk * kTcK), v);
    else
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
    const int r = quad * 32 + lane;
    const int k2 = r >> 3, px = blk * 8 + (r & 7);
    const bool in = kx0 + px < p.wx;
    float2 of = make_float2(0.f, 0.f);
    if (p.cplx && in) of = cmul(ldg2(p.ox + kx0 + px), ldg2(p.oy + kyw));
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      const int q = k2 + 16 * k1;
      const float2 x = make_float2(v[k1], v[16 + k1]);
      float pw = fmaf(x.x, x.x, x.y * x.y) * p.power_scale;
      if (p.magnitude) pw = sqrtf(pw);
      out[q * kOutStride + px] = pw;
      if (p.cplx && in) __stcs(p.cplx + ((size_t)q * p.wy + kyw) * p.wx + kx0 + px, cmul(x, of));
    }
  }
  __syncthreads();
  // 4. 128-byte rows of the volume
  if (kx0 + lane < p.wx) {
    float* dst = p.vol + (size_t)kyw * p.wx + kx0 + lane;
    const size_t plane = (size_t)p.wy * p.wx;
#pragma unroll 8
    for (int q = warp; q < kTcN; q += kTcThreads / 32) __stcs(dst + (size_t)q * plane, out[q * kOutStride + lane]);
  }
  if (tid == 0 && !ok2) atomicOr(p.err, kErrAxialTc);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcCols) : "memory");
}

}  // namespace

bool axial_tc_supported(int nl) { return nl == kTcN; }

size_t axial_tc_smem_bytes() {
  return (size_t)2 * kTcBlocks * 128 * kTcK * 2 + (size_t)2 * kTcK * kTcK * 2 + kTcN * sizeof(float2);
}

size_t axial_tc_table_elems() { return 2 * kTcK * kTcK; }

// BF16 hi / lo of the real form of the 16-point DFT matrix (sign -), already in
// the K-major core layout the kernel's B operand uses: B[n][k] with n = output
// (k2 real for n < 16, k2 imaginary for n >= 16) and k = input (j2 real for
// k < 16, j2 imaginary for k >= 16).
void axial_tc_table(std::vector<unsigned short>& out) {
  out.assign(axial_tc_table_elems(), 0);
  const double pi = 3.14159265358979323846264338327950288;
  auto bf16_bits = [](float x) {
    unsigned u;
    std::memcpy(&u, &x, 4);
    const unsigned rounding = 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
    return (unsigned short)((u + rounding) >> 16);
  };
  auto bf16_val = [](unsigned short b) {
    const unsigned u = (unsigned)b << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
  };
  for (int n = 0; n < kTcK; ++n)
    for (int k = 0; k < kTcK; ++k) {
      const int k2 = n % kTcR, j2 = k % kTcR;
      const double a = -2.0 * pi * (double)((j2 * k2) % kTcR) / kTcR;
      const double c = std::cos(a), s = std::sin(a);
      double w;
      if (n < kTcR) w = (k < kTcR) ? c : -s;   // Re Y = sum Hr c - Hi s
      else w = (k < kTcR) ? s : c;             // Im Y = sum Hr s + Hi c
      const unsigned short hi = bf16_bits((float)w);
      const unsigned short lo = bf16_bits((float)(w - (double)bf16_val(hi)));
      out[tc_core_off(n, k)] = hi;
      out[kTcK * kTcK + tc_core_off(n, k)] = lo;
    }
}

cudaError_t launch_axial_tc(const Plan& pl, const AxialParams& ap, const unsigned short* bmat, unsigned* err,
                            cudaStream_t s) {
  TcParams p;
  p.inter = ap.inter;
  p.vol = ap.vol;
  p.cplx = ap.cplx;
  p.bmat = bmat;
  p.twl = ap.twl;
  p.ox = ap.ox;
  p.oy = ap.oy;
  p.wx = ap.wx;
  p.wy = ap.wy;
  p.ntx = ap.ntx;
  p.power_scale = ap.power_scale;
  p.magnitude = ap.magnitude;
  p.err = err;
  const size_t smem = axial_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(axial_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ap.ntx, ap.wy);
  axial_tc_kernel<<<grid, kTcThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ssoct
