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
// index runs over the 16 inputs with real and imaginary parts interleaved
// (K = 2 j + 0 / 1), the N index likewise over the 16 outputs, and B is the
// real 32 x 32 form of the complex 16-point DFT matrix in that order.  With
// the parts interleaved, one packed BF16x2 split of a complex value gives the
// two adjacent operand entries (hi and lo), stored with one 4-byte store each.  Operands are split as
// x = hi + lo with hi, lo in BF16 (BF16 keeps FP32's exponent range, so no
// scaling is needed), and D = Ahi Bhi + Ahi Blo + Alo Bhi; the dropped Alo Blo
// term and the rounding of lo put the relative error near 2^-16 per stage.
//
// The kernel is persistent, one CTA per SM.  Its unit of work is half a tile:
// 16 pixels x 256 frames (two 8-pixel M blocks), which a 2D tensor copy (TMA)
// takes out of the 32-pixel tile of the sweep-axis intermediate into a ring of
// six 32 KB shared-memory buffers, a ring's worth ahead.  Four groups of 8
// warps compute the CTA's half-tiles g, g + 4, ...; while one group waits for
// its MMAs or its next half-tile, three others compute.  (Two groups on whole
// 64 KB tiles spent 43 % of their stall samples at barriers and took 0.73 ms.)
// A half-tile never leaves its buffer: the FP32 values are read into registers
// and written back as the BF16 hi / lo stage-1 operands (the same 32 KB), the
// stage-2 operands overwrite those once the stage-1 MMAs are done, and the
// |V|^2 rows overwrite those once the stage-2 MMAs are done.  Each group owns
// 64 TMEM columns (2 blocks x N = 32 fp32 accumulators); one of its threads
// issues its 12 MMAs per stage and waits on its commit barrier.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fft_common.cuh"
#include "mbarrier.cuh"

namespace ssoct {
namespace {

constexpr int kTcN = 256;          // sweep length this kernel is built for
constexpr int kTcR = 16;           // radix of both stages
constexpr int kTcK = 2 * kTcR;     // 32: real + imaginary parts
constexpr int kTcGroups = 4;       // half-tiles computed at once per CTA
constexpr int kTcGroupThreads = 256;
constexpr int kTcThreads = kTcGroups * kTcGroupThreads;
constexpr int kTcHalf = 16;                     // pixels per work item (half a 32-pixel tile)
constexpr int kTcItemBlocks = kTcHalf / 8;      // 8-pixel M blocks per work item
constexpr unsigned kTcCols = kTcItemBlocks * kTcK;  // TMEM columns (fp32 accumulators) per group
constexpr int kTcStages = 6;                    // ring buffers
constexpr int kTcFull = 12;                     // full barriers: item mod lcm(stages, groups)
constexpr size_t kTcItemBytes = (size_t)kTcN * kTcHalf * sizeof(float2);  // 32 KB
constexpr unsigned long long kTcLoadWaitNs = 4000000000ull;
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
__device__ bool tc_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns = kTcWaitNs) {
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
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
  float k_abs;                  // |K|, folded into the stage-2 twiddles (so |V|^2 |K|^2 = |v|^2)
  float inv_k_abs;              // 1 / |K|, taken back out of the complex output (oy holds K)
  int magnitude;
  unsigned* err;                // kErrAxialTc (MMA wait) / kErrAxial (tile wait) ORed in on a time-out
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

// Barrier of one group (named barrier 1 + g, 256 threads); returns the OR of v.
__device__ __forceinline__ bool tc_group_sync_or(int g, bool v) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
               : "=r"(r)
               : "r"((unsigned)v), "r"(1 + g), "n"(kTcGroupThreads)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ void tc_group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kTcGroupThreads) : "memory");
}

__device__ __forceinline__ void tc_tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

constexpr int kABlock = 128 * kTcK;  // elements of one M block of an operand
constexpr int kOutStride = 24;       // floats per |V|^2 row in the buffer: conflict-free writes

// Copy of the CTA's work item t (global item blockIdx.x + t * gridDim.x: half
// item % 2 of tile item / 2) into ring buffer t mod kTcStages.  The tensor map
// sees the intermediate as float [tiles * 256][64]; a box is 32 floats (16
// complex values) x 256 rows.
__device__ __forceinline__ void tc_fill(const CUtensorMap* map, unsigned char* ring, uint64_t* full, unsigned* fills,
                                        int t) {
  const int f = t % kTcFull;
  atomicAdd(&fills[f], 1u);
  mbar_arrive_tx(&full[f], (unsigned)kTcItemBytes);
  const int gi = (int)blockIdx.x + t * (int)gridDim.x;
  tc_tma_2d(ring + (size_t)(t % kTcStages) * kTcItemBytes, map, (gi & 1) * 2 * kTcHalf, (gi >> 1) * kTcN, &full[f]);
}

// 12 MMAs of one stage: D[blk] = Ahi Bhi + Ahi Blo + Alo Bhi, K = 32 as two K = 16 steps.
__device__ __forceinline__ void tc_issue_stage(unsigned tmem, const unsigned short* A, const unsigned short* Bs,
                                               uint64_t* bar) {
  const unsigned idesc = tc_idesc(128, kTcK);
#pragma unroll 1
  for (int blk = 0; blk < kTcItemBlocks; ++blk) {
    const unsigned short* a_terms[3] = {A + blk * kABlock, A + blk * kABlock, A + (kTcItemBlocks + blk) * kABlock};
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
  tc_commit(bar);
}

// |V|^2 |K|^2 (|V| |K| if MAG) of the 16 depth bins q = k2 + 16 k1 this thread
// holds (v carries |K| from the twiddles) into the item's output rows; with
// CPLX also V with the output chirp and K.
template <bool MAG, bool CPLX>
__device__ __forceinline__ void tc_epilogue(const TcParams& p, const float (&v)[32], float* out, int k2, int px,
                                            int kx0, int kyw) {
  const bool in = kx0 + px < p.wx;
  float2 of = make_float2(0.f, 0.f);
  if constexpr (CPLX) {
    if (in) of = cmul(ldg2(p.ox + kx0 + px), ldg2(p.oy + kyw));
    of = make_float2(of.x * p.inv_k_abs, of.y * p.inv_k_abs);
  }
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const int q = k2 + 16 * k1;
    const float2 x = make_float2(v[2 * k1], v[2 * k1 + 1]);
    float pw = fmaf(x.x, x.x, x.y * x.y);
    if constexpr (MAG) pw = sqrtf(pw);
    out[q * kOutStride + px] = pw;
    if constexpr (CPLX) {
      if (in) __stcs(p.cplx + ((size_t)q * p.wy + kyw) * p.wx + kx0 + px, cmul(x, of));
    }
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    axial_tc_kernel(const __grid_constant__ TcParams p, const __grid_constant__ CUtensorMap imap) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* ring = smem;                                                      // [6][32 KB]
  unsigned short* Bs = reinterpret_cast<unsigned short*>(ring + kTcStages * kTcItemBytes);  // [hi / lo][32 x 32]
  float2* tw = reinterpret_cast<float2*>(Bs + 2 * kTcK * kTcK);                    // [256]
  __shared__ __align__(8) uint64_t full[kTcFull];
  __shared__ __align__(8) uint64_t mma_bar[kTcGroups];
  __shared__ unsigned fills[kTcFull];
  __shared__ unsigned tmem_base;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nitems = 2 * p.ntx * p.wy;
  const int mine = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "n"(kTcGroups * kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int f = 0; f < kTcFull; ++f) {
      mbar_init(&full[f], 1);
      fills[f] = 0u;
    }
    for (int g = 0; g < kTcGroups; ++g) mbar_init(&mma_bar[g], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int t = 0; t < kTcStages && t < mine; ++t) tc_fill(&imap, ring, full, fills, t);
  }
  if (tid < 256) reinterpret_cast<uint4*>(Bs)[tid] = __ldg(reinterpret_cast<const uint4*>(p.bmat) + tid);  // 4 KB
  if (tid < kTcN) {
    const float2 t = ldg2(p.twl + tid);
    tw[tid] = make_float2(t.x * p.k_abs, t.y * p.k_abs);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const int g = tid / kTcGroupThreads;
  const int lt = tid % kTcGroupThreads;
  const int gw = lt / 32;                       // warp within the group (0..7)
  const int quad = gw & 3, qblk = gw >> 2;      // TMEM lane quadrant, M block read by this warp
  const unsigned tmem = tmem_base + (unsigned)(g * kTcCols);
  for (int i = g, prev = -1;; prev = i, i += kTcGroups) {
    tc_group_sync(g);  // every thread of the group is done with item prev's buffer
    if (lt == 0 && prev >= 0 && prev + kTcStages < mine) tc_fill(&imap, ring, full, fills, prev + kTcStages);
    if (i >= mine) break;
    // one thread waits for the item; the others sleep at the group barrier
    bool ok0 = true;
    if (lt == 0) {
      ok0 = tc_wait(&full[i % kTcFull], (unsigned)(i / kTcFull) & 1u, kTcLoadWaitNs);
      if (!ok0) atomicOr(p.err, kErrAxial);
    }
    if (tc_group_sync_or(g, !ok0)) break;
    unsigned char* buf = ring + (size_t)(i % kTcStages) * kTcItemBytes;
    unsigned short* A = reinterpret_cast<unsigned short*>(buf);  // [hi / lo][block][128 x 32]
    const int gi = (int)blockIdx.x + i * (int)gridDim.x;
    const int gt = gi >> 1;
    const int kyw = gt / p.ntx;
    const int kx0 = (gt - kyw * p.ntx) * kTile + (gi & 1) * kTcHalf;

    // 1. t = j1 + 16 j2 -> stage-1 row (pixel, j1), K = 2 j2 (real) / 2 j2 + 1 (imaginary).
    //    Work units c = (j1, half of j2): a warp takes four, a thread two
    //    (lanes 0-15 and 16-31 on different units); every value is read before
    //    any operand is written over it.
    {
      const int px = lane & (kTcHalf - 1), usel = lane >> 4;
      const float2* src = reinterpret_cast<const float2*>(buf) + px;
      float2 x[2][8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = gw * 4 + u * 2 + usel, j1 = c & 15, h = c >> 4;
#pragma unroll
        for (int k = 0; k < 8; ++k) x[u][k] = src[(j1 + 16 * (8 * h + k)) * kTcHalf];
      }
      tc_group_sync(g);
      const int blk = px >> 3, pl = px & 7;
      unsigned short* Ahi = A + blk * kABlock;
      unsigned short* Alo = A + (kTcItemBlocks + blk) * kABlock;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = gw * 4 + u * 2 + usel, j1 = c & 15, h = c >> 4;
        // j2 = 8h .. 8h + 3 fill K = 16h .. 16h + 7, j2 = 8h + 4 .. 8h + 7 the next 8
        uint4 h0, l0, h1, l1;
        split2_bf16(x[u][0].x, x[u][0].y, h0.x, l0.x);
        split2_bf16(x[u][1].x, x[u][1].y, h0.y, l0.y);
        split2_bf16(x[u][2].x, x[u][2].y, h0.z, l0.z);
        split2_bf16(x[u][3].x, x[u][3].y, h0.w, l0.w);
        split2_bf16(x[u][4].x, x[u][4].y, h1.x, l1.x);
        split2_bf16(x[u][5].x, x[u][5].y, h1.y, l1.y);
        split2_bf16(x[u][6].x, x[u][6].y, h1.z, l1.z);
        split2_bf16(x[u][7].x, x[u][7].y, h1.w, l1.w);
        const int r = tc_row(j1, pl);
        *reinterpret_cast<uint4*>(Ahi + tc_core_off(r, 16 * h)) = h0;
        *reinterpret_cast<uint4*>(Alo + tc_core_off(r, 16 * h)) = l0;
        *reinterpret_cast<uint4*>(Ahi + tc_core_off(r, 16 * h + 8)) = h1;
        *reinterpret_cast<uint4*>(Alo + tc_core_off(r, 16 * h + 8)) = l1;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    tc_group_sync(g);
    tc_fence_after();
    bool ok = true;
    if (lt == 0) {
      tc_issue_stage(tmem, A, Bs, &mma_bar[g]);
      ok = tc_wait(&mma_bar[g], 0u);
      if (!ok) atomicOr(p.err, kErrAxialTc);
    }
    tc_fence_before();
    const bool bad1 = tc_group_sync_or(g, !ok);
    tc_fence_after();
    if (bad1) break;

    // 2. twiddle w256^(j1 k2) and re-layout as the stage-2 operand: row (pixel, k2),
    //    K = 2 j1 (real) / 2 j1 + 1 (imaginary), over the stage-1 operand (its MMAs are done)
    {
      float v[32];
      tc_ld32(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(qblk * kTcK), v);
      const int r = quad * 32 + lane;
      const int j1 = r >> 3, pl = r & 7;
      unsigned short* Ahi = A + qblk * kABlock;
      unsigned short* Alo = A + (kTcItemBlocks + qblk) * kABlock;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const float2 z = cmul(make_float2(v[2 * k2], v[2 * k2 + 1]), tw[k2 * 16 + j1]);
        const int off = tc_core_off(tc_row(k2, pl), 2 * j1);
        unsigned hi, lo;
        split2_bf16(z.x, z.y, hi, lo);
        *reinterpret_cast<unsigned*>(Ahi + off) = hi;
        *reinterpret_cast<unsigned*>(Alo + off) = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    tc_group_sync(g);
    tc_fence_after();
    if (lt == 0) {
      tc_issue_stage(tmem, A, Bs, &mma_bar[g]);
      ok = tc_wait(&mma_bar[g], 1u);
      if (!ok) atomicOr(p.err, kErrAxialTc);
    }
    tc_fence_before();
    const bool bad2 = tc_group_sync_or(g, !ok);
    tc_fence_after();
    if (bad2) break;

    // 3. V[k2 + 16 k1] sits in row (pixel, k2), columns 2 k1 (real) / 2 k1 + 1
    //    (imaginary); |V|^2 rows over the stage-2 operand (its MMAs are done)
    float* out = reinterpret_cast<float*>(buf);  // [256][kOutStride]
    {
      float v[32];
      tc_ld32(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(qblk * kTcK), v);
      const int r = quad * 32 + lane;
      const int k2 = r >> 3, px = qblk * 8 + (r & 7);
      if (p.cplx) {
        if (p.magnitude) tc_epilogue<true, true>(p, v, out, k2, px, kx0, kyw);
        else tc_epilogue<false, true>(p, v, out, k2, px, kx0, kyw);
      } else {
        if (p.magnitude) tc_epilogue<true, false>(p, v, out, k2, px, kx0, kyw);
        else tc_epilogue<false, false>(p, v, out, k2, px, kx0, kyw);
      }
    }
    tc_group_sync(g);
    // 4. 64-byte rows of the volume: per pass 16 depth bins, a warp's two halves
    //    on bins two apart (distinct banks with the 24-float row stride)
    {
      const int px = lane & (kTcHalf - 1);
      const int qa = (gw & 1) + 4 * (gw >> 1) + 2 * (lane >> 4);
      if (kx0 + px < p.wx) {
        float* dst = p.vol + (size_t)kyw * p.wx + kx0 + px;
        const size_t plane = (size_t)p.wy * p.wx;
#pragma unroll 4
        for (int q = qa; q < kTcN; q += 16) __stcs(dst + (size_t)q * plane, out[q * kOutStride + px]);
      }
    }
    // this thread's accesses to the buffer come before its next TMA fill (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  // copies still in flight (after a time-out) land before the CTA exits; the
  // last fill of each barrier is its latest phase
  tc_fence_before();
  __syncthreads();
  if (tid == 0)
    for (int f = 0; f < kTcFull; ++f)
      if (fills[f] && !tc_wait(&full[f], (fills[f] - 1u) & 1u, kTcLoadWaitNs)) atomicOr(p.err, kErrAxial);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kTcGroups * kTcCols)
                 : "memory");
  }
}

}  // namespace

bool axial_tc_supported(int nl) { return nl == kTcN; }

size_t axial_tc_smem_bytes() {
  return (size_t)kTcStages * kTcItemBytes + (size_t)2 * kTcK * kTcK * 2 + kTcN * sizeof(float2);
}

size_t axial_tc_table_elems() { return 2 * kTcK * kTcK; }

// BF16 hi / lo of the real form of the 16-point DFT matrix (sign -), already in
// the K-major core layout the kernel's B operand uses: B[n][k] with n = output
// (2 k2: real part, 2 k2 + 1: imaginary part of output k2) and k = input
// (2 j2: real part, 2 j2 + 1: imaginary part of input j2).
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
      const int k2 = n / 2, j2 = k / 2;
      const double a = -2.0 * pi * (double)((j2 * k2) % kTcR) / kTcR;
      const double c = std::cos(a), s = std::sin(a);
      double w;
      if (n % 2 == 0) w = (k % 2 == 0) ? c : -s;   // Re Y = sum Hr c - Hi s
      else w = (k % 2 == 0) ? s : c;               // Im Y = sum Hr s + Hi c
      const unsigned short hi = bf16_bits((float)w);
      const unsigned short lo = bf16_bits((float)(w - (double)bf16_val(hi)));
      out[tc_core_off(n, k)] = hi;
      out[kTcK * kTcK + tc_core_off(n, k)] = lo;
    }
}

cudaError_t launch_axial_tc(const Plan& pl, const AxialParams& ap, const unsigned short* bmat, unsigned* err,
                            int num_sms, cudaStream_t s) {
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
  p.k_abs = (float)std::sqrt((double)ap.power_scale);
  p.inv_k_abs = (float)(1.0 / std::sqrt((double)ap.power_scale));
  p.magnitude = ap.magnitude;
  p.err = err;
  const size_t smem = axial_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(axial_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  alignas(64) CUtensorMap imap;
  if (!encode_inter_map(ap.inter, (long long)ap.ntx * ap.wy * kTcN, kTcHalf, &imap)) return cudaErrorInvalidValue;
  const long long nitems = 2ll * ap.ntx * ap.wy;
  long long grid = num_sms > 0 ? num_sms : 1;  // persistent: one CTA per SM
  if (grid > nitems) grid = nitems;
  if (grid < 1) return cudaSuccess;
  axial_tc_kernel<<<(unsigned)grid, kTcThreads, smem, s>>>(p, imap);
  return cudaGetLastError();
}

}  // namespace ssoct
