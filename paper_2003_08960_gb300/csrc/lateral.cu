// Lateral stage: chromatic rescale (Eq. 5) + Fresnel transform (Eq. 6) of every
// frame of a sweep, as one persistent, warp-specialised kernel.
//
// Each CTA has two producer warps, two consumer groups of eight warps and a
// publisher warp.  A producer takes work items from a device ticket counter (in
// the order LateralSchedule defines), waits until an item's inputs are ready,
// and copies them into one of three shared-memory stage buffers with the Tensor
// Memory Accelerator (1D bulk copies of the uint16 input rows and tap tables,
// or 2D tensor copies of an L2 scratch column band), handing the item over
// through an mbarrier; producer g feeds consumer group g, hand-overs alternate
// between them, and two items are computed at once.  Consumers compute in
// place in the stage buffer, store the item's outputs themselves and arrive on
// a second mbarrier; the publisher then frees the buffer for the producers and
// makes the outputs visible to the other CTAs (release increment of the
// frame's counter), off the producer's path.
// Items:
//  * row item (frame f, band of rows): stage the uint16 input rows the band
//    needs in shared memory, resample them with the frame's separable linear-
//    interpolation taps, multiply by the input chirp (centring phase folded in),
//    run the Nx-point row DFT in registers (N2-point DFT per thread, twiddle,
//    exchange through shared memory, N1-point DFTs), multiply by the row's y
//    chirp and store the window columns into an L2-resident scratch slot;
//  * column item (frame f, band of columns): after every row item of f has
//    signalled, load the band from the scratch slot, run the Ny-point column DFT
//    the same way, keep the window rows and write them into the sweep-axis
//    intermediate [wy][tile][t][32] that the axial kernel streams.
// The scratch ring holds `slots` frames, so that most row-transformed frames
// are read back from L2: the uint16 input is read from HBM once and the
// windowed complex hologram written to it (lines of the ring evicted dirty
// after their column items are written back as well).
// Axial-first order (AF): frame f is depth bin af_bin(f); row items read rows
// of the half-spectrum plane of that bin, which the first pass stored times
// the input chirp and |K| (bins above N/2 take the plane conjugated, times the
// squared chirp), and column items write |V|^2 straight into the volume.
#include <cuda.h>

#include "fft_common.cuh"
#include "mbarrier.cuh"

namespace ssoct {
namespace {

constexpr int kGroups = 2;                            // consumer groups, each works on its own item
constexpr int kCtaThreads = kGroups * kThreads + 96;  // 2 x 8 consumer warps, 2 producer warps, a publisher warp
constexpr unsigned long long kProducerWaitNs = 2000000000ull;   // 2 s
constexpr unsigned long long kConsumerWaitNs = 4000000000ull;   // longer: the producer gives up first
enum : int { kRowItem = 0, kColItem = 1, kEndItem = 2 };

struct Desc {
  int kind, f, item, jlo, nrows, slot;  // slot: wavelength / intermediate index of frame f
};

// Axial-first order: frame f of the lateral pass is depth bin af_bin(f), in the
// order 0, 1, N-1, 2, N-2, ..., N/2, so that the two bins sharing a half-spectrum
// plane (q and N - q) follow each other and the second read of the plane hits L2.
__host__ __device__ __forceinline__ int af_bin(int f, int nl) {
  if (f == 0) return 0;
  const int k = (f + 1) / 2;
  return (f & 1) ? k : nl - k;
}

// ---------------------------------------------------------------- waits

// Bounded wait for an mbarrier phase; on timeout records kErrTimeout and aborts.
__device__ bool mbar_wait(uint64_t* b, unsigned parity, Counters* c, unsigned long long limit_ns) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    if (mbar_try(b, parity)) return true;
    if (global_timer_ns() - t0 > limit_ns) {
      atomicCAS(&c->err, 0u, kErrTimeout);
      atomicExch(&c->abort, 1u);
      return false;
    }
  }
}
// Barrier of consumer group g only (named barrier 1 + g); returns the OR of `v`.
__device__ __forceinline__ bool consumers_sync_or(int g, bool v) {
  unsigned r;
  if (g == 0)
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((unsigned)v), "n"(kThreads)
                 : "memory");
  else
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((unsigned)v), "n"(kThreads)
                 : "memory");
  return r != 0;
}
__device__ __forceinline__ void consumers_sync(int g) {
  if (g == 0) asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
  else asm volatile("bar.sync 2, %0;" ::"n"(kThreads) : "memory");
}

// ---------------------------------------------------------------- consumer work

constexpr int kStages = 3;  // stage buffers: one computed, one or two loaded ahead
// Items' outputs leave through the consumers' own stores.  (Producer-issued TMA
// stores of them were measured slower on GB300: the single producer thread
// serialises on writing and waiting for 1024 64-byte column rows per band.)

// A row item's stage buffer: nrows uint16 input rows, then (16-byte aligned) the
// frame's NX x taps, the RPI y taps and the RPI y chirps of its rows.
template <int NX>
__host__ __device__ constexpr size_t row_taps_offset(int nrows) {
  return ((size_t)nrows * NX * sizeof(uint16_t) + 15) / 16 * 16;
}
template <int NX>
__host__ __device__ constexpr size_t row_stage_bytes(int nrows) {
  return row_taps_offset<NX>(nrows) + (size_t)NX * sizeof(Tap) +
         (size_t)(kThreads / split_n1(NX)) * (sizeof(Tap) + sizeof(float2));
}

// Position of element (k2, j1) in a row's N2 x N1 transpose block: the column is
// XOR-swizzled by k2 so that both the writes (fixed k2, all j1) and the
// transposed reads (fixed j1, all k2) hit distinct banks without padding.
template <int N1>
__device__ __forceinline__ int xswz(int k2, int j1) {
  return k2 * N1 + (j1 ^ (k2 & (N1 - 1)));
}

// Exact (every uint16 is a float).  One conversion instruction: the kernel is
// bound by instruction issue, and the two-instruction form (OR into the
// mantissa of 2^23, subtract 2^23) measured 1.5-2 % slower overall.
__device__ __forceinline__ float u16_to_f(unsigned short u) {
  return __uint2float_rn((unsigned)u);
}

// Row item: rows [item*RPI, item*RPI + RPI) of frame d.f.  The stage buffer holds
// input rows jlo .. jlo + nrows - 1 (uint16) and the taps (in axial-first
// order the RPI plane rows); it then serves as the transpose block.
template <int NX, int NY, bool FW, bool AF>
__device__ __forceinline__ void row_item(const LateralParams& p, const Desc& d, unsigned char* buf,
                                         const float2* twx, const float2* cxs, int g) {
  constexpr int N1 = Split<NX>::N1, N2 = Split<NX>::N2;
  constexpr int RPI = kThreads / N1;
  static_assert(32 % N1 == 0, "a row's N1 threads lie in one warp");
  const int tid = threadIdx.x % kThreads;
  const int r = tid / N1;
  const int j1 = tid % N1;
  const int f = d.f;
  const int y = d.item * RPI + r;
  const uint16_t* in = reinterpret_cast<const uint16_t*>(buf);
  const Tap* xtaps = reinterpret_cast<const Tap*>(buf + row_taps_offset<NX>(d.nrows));
  const Tap* ytaps = xtaps + NX;
  const float2* ychirp = reinterpret_cast<const float2*>(ytaps + RPI);
  // 1. Eq. 5 resample (taps outside the frame carry weight 0) x input chirp,
  //    elements n = j1 + N1 * j2 of row y; in axial-first order the row of the
  //    half-spectrum plane of bin q, which already carries the input chirp c
  //    (and |K|), as it is for q <= N/2 and conjugated x c^2 above
  using S2 = Stage2<NX>;
  float2 a[S2::A];
  float2 cyv;
  bool mirrored = false;
  if constexpr (AF) {
    const float2* in2 = reinterpret_cast<const float2*>(buf) + r * NX;
    mirrored = af_bin(f, p.nl) > p.nl / 2;
    if (mirrored) {
      // conj(v) c2 = (v.x c2.x + v.y c2.y, v.x c2.y - v.y c2.x); cxs holds c2 in this order
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) {
        const int n = j1 + N1 * j2;
        const float2 v = in2[n], c = cxs[n];
        a[j2] = make_float2(fmaf(v.x, c.x, v.y * c.y), fmaf(v.x, c.y, -v.y * c.x));
      }
      cyv = ldg2(p.cy2 + y);
    } else {
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) a[j2] = in2[j1 + N1 * j2];
    }
  } else {
    cyv = ychirp[r];
    const Tap ty = ytaps[r];
    const uint16_t* r0 = in + (ty.base - d.jlo) * NX;
    const uint16_t* r1 = r0 + NX;
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) {
      const int n = j1 + N1 * j2;
      const Tap t = xtaps[n];
      const float v0 = fmaf(t.w0, u16_to_f(r0[t.base]), t.w1 * u16_to_f(r0[t.base + 1]));
      const float v1 = fmaf(t.w0, u16_to_f(r1[t.base]), t.w1 * u16_to_f(r1[t.base + 1]));
      const float v = fmaf(ty.w0, v0, ty.w1 * v1);
      const float2 c = cxs[n];
      a[j2] = make_float2(v * c.x, v * c.y);
    }
  }
  // 2. row DFT (+ sign of Eq. 6): N2-point DFT in registers, twiddle with the
  //    row's y chirp folded in (none for the planes' own bins in axial-first
  //    order), transpose in the stage buffer, N1-point DFTs
  Dft<N2, 1>::template run<1, 0>(a);
  if (AF && !mirrored) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], twx[k2 * N1 + j1]);
  } else {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], cmul(twx[k2 * N1 + j1], cyv));
  }
  // every input of the buffer has been read.  In axial-first order row r's
  // input is its own block of the buffer, read by its own warp only, so the
  // warp's barrier suffices; otherwise the staged uint16 rows and taps are
  // shared by the group.
  if constexpr (AF) __syncwarp();
  else consumers_sync(g);
  float2* ex = reinterpret_cast<float2*>(buf) + r * NX;  // this row's block (N2 x N1 = NX values)
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) ex[xswz<N1>(k2, j1)] = a[k2];
  __syncwarp();  // a row's N1 threads lie in one warp
  static_for<0, S2::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (S2::live(i, j1)) {
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = ex[xswz<N1>(k2, jj)];
      Dft<N1, 1>::template run<1, i * N1>(a);
    }
  });
  {
    // 3. window columns straight into the scratch slot of frame f
    const unsigned long long pol_last = policy_evict_last();
    float2* dst = p.scratch + ((size_t)(f % p.sch.slots) * NY + y) * p.wxp;
    static_for<0, S2::NI>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const int k2 = j1 + N1 * i;
      if (!S2::live(i, j1)) return;
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
  }
}

// Row of the band where the first column pass leaves element (j1, k2).  With
// 64-byte band rows (BC = 8), the second pass's reads of rows jj + N1 k2 for a
// warp's four consecutive k2 would all fall in the same 16 banks; swapping the
// row pair (2m, 2m + 1) for odd k2 puts two of them in each half.  The swapped
// partner row belongs to thread j1 ^ 1 of the same warp.
template <int N1, int BC>
__device__ __forceinline__ int col_row(int j1, int k2) {
  if constexpr (BC == 8) return (j1 ^ (k2 & 1)) + N1 * k2;
  else return j1 + N1 * k2;
}

// Axial-first order, end of a column item: V of depth bin q at window column
// kxw for the rows this thread holds (a[], rows k2 + N2 k1 of the column DFT),
// already scaled by |K| through the planes: |V|^2 |K|^2 (|V| |K| if MAG)
// into the volume and, if CPLX, V with the output chirp and K into the complex
// volume.  Full-window plans use the frame's sizes as the volume's strides, so
// that the stores take constant offsets.
template <int NY, bool FW, bool MAG, bool CPLX, int NX>
__device__ __forceinline__ void af_epilogue(const LateralParams& p, const Desc& d, const float2* a, int j1,
                                            int kxw) {
  constexpr int N1 = Split<NY>::N1, N2 = Split<NY>::N2;
  const int q = af_bin(d.f, p.nl);
  const int wx = FW ? NX : p.wx, wy = FW ? NY : p.wy;
  float* vdst = p.vol + (size_t)q * wy * wx + kxw;
  float2 ox = make_float2(0.f, 0.f);
  if constexpr (CPLX) {
    ox = ldg2(p.ox + kxw);
    ox = make_float2(ox.x * p.inv_k_abs, ox.y * p.inv_k_abs);
  }
  static_for<0, Stage2<NY>::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (!Stage2<NY>::live(i, j1)) return;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int kyw = k2 + N2 * k1 - (FW ? 0 : p.y0);
      if (FW || (kyw >= 0 && kyw < wy)) {
        const float2 v = a[i * N1 + k1];
        float pw = fmaf(v.x, v.x, v.y * v.y);
        if constexpr (MAG) pw = sqrtf(pw);
        __stcs(vdst + (size_t)kyw * wx, pw);
        if constexpr (CPLX)
          __stcs(p.cplx + ((size_t)q * wy + kyw) * wx + kxw, cmul(v, cmul(ox, ldg2(p.oy + kyw))));
      }
    }
  });
}

// Column item: window columns [item*BC, item*BC + BC) of frame d.f.  The stage
// buffer holds the band [NY][BC] copied from the scratch slot; the first DFT
// pass writes back in place (up to the row-pair swap of col_row), the second
// stores the item's outputs straight from registers.
template <int NX, int NY, bool FW, bool AF>
__device__ __forceinline__ void col_item(const LateralParams& p, const Desc& d, unsigned char* buf,
                                         const float2* twy, int g) {
  constexpr int N1 = Split<NY>::N1, N2 = Split<NY>::N2;
  constexpr int BC = kThreads / N1;
  static_assert(BC != 8 || N1 % 2 == 0, "the swapped row pairs lie in one warp");
  const int tid = threadIdx.x % kThreads;
  const int b = tid % BC;
  const int j1 = tid / BC;
  float2* tile = reinterpret_cast<float2*>(buf);
  using S2 = Stage2<NY>;
  float2 a[S2::A];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = tile[(j1 + N1 * j2) * BC + b];
  Dft<N2, 1>::template run<1, 0>(a);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmul(a[k2], twy[k2 * N1 + j1]);
  if constexpr (BC == 8) __syncwarp();  // the partner thread has read the rows it will be given
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) tile[col_row<N1, BC>(j1, k2) * BC + b] = a[k2];
  consumers_sync(g);
  static_for<0, S2::NI>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int k2 = j1 + N1 * i;
    if (!S2::live(i, j1)) return;
    if constexpr (BC == 8) {
      // row jj ^ sw: jj + sw for even jj, jj - sw for odd jj (two bases, constant offsets)
      const int sw = k2 & 1;
      const float2* ev = tile + (N1 * k2 + sw) * BC + b;
      const float2* od = tile + (N1 * k2 - sw) * BC + b;
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = (jj & 1) ? od[jj * BC] : ev[jj * BC];
    } else {
#pragma unroll
      for (int jj = 0; jj < N1; ++jj) a[i * N1 + jj] = tile[(jj + N1 * k2) * BC + b];
    }
    Dft<N1, 1>::template run<1, i * N1>(a);
  });
  if constexpr (AF) {
    // axial-first order: the column DFT completes V of bin q; write |V|^2 |K|^2
    // (or |V| |K|) and optionally V with the output chirp and K.  The two
    // options are tested once per item, not per value: tested inside the
    // unrolled loop they were predicated on every value.
    const int kxw = d.item * BC + b;  // column bands already span the window's columns
    if (kxw < p.wx) {
      if (p.cplx) {
        if (p.magnitude) af_epilogue<NY, FW, true, true, NX>(p, d, a, j1, kxw);
        else af_epilogue<NY, FW, false, true, NX>(p, d, a, j1, kxw);
      } else {
        if (p.magnitude) af_epilogue<NY, FW, true, false, NX>(p, d, a, j1, kxw);
        else af_epilogue<NY, FW, false, false, NX>(p, d, a, j1, kxw);
      }
    }
  } else {
    const int kxw = d.item * BC + b;
    if (kxw < p.wx) {
      const unsigned long long pol_first = policy_evict_first();
      float2* dst = p.inter + (size_t)(kxw / kTile) * p.nl * kTile + (size_t)d.slot * kTile + (kxw % kTile);
      const size_t row_pitch = (size_t)p.ntx * p.nl * kTile;
      static_for<0, S2::NI>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const int k2 = j1 + N1 * i;
        if (!S2::live(i, j1)) return;
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
  }
}

// ---------------------------------------------------------------- producer

// Hand-over bookkeeping in shared memory between the producers and the
// publisher.  Hand-over s is prepared by producer s mod kProducers and computed
// by consumer group s mod kGroups (kProducers == kGroups: producer g feeds group
// g).  Producer 0 claims tickets in pairs, so hand-over positions follow ticket
// order.  Producers run at most kStages positions ahead of the publisher, so
// kPubQ > kStages slots of item info suffice.
constexpr int kProducers = kGroups;
constexpr int kPubQ = 4;
constexpr int kTicketQ = 4;
// Full barriers: one per position mod lcm(kStages, kGroups), so that each is
// filled by one producer in position order and waited on by one group, which
// has consumed its previous fill: parity waits cannot pass early even though
// the two producers' hand-overs may complete out of order.
constexpr int kFullBars = kStages * kGroups;
constexpr unsigned kEndStamp = 0x80000000u;
struct Handover {
  int kind[kPubQ];
  int f[kPubQ];
  unsigned stamp[kPubQ];     // s + 1 once hand-over s is in place (| kEndStamp for an end mark)
  unsigned freed;            // hand-overs whose consumers are done with their buffer (publisher)
  unsigned tk[kTicketQ];     // ticket of position 2k + 1, from producer 0 to producer 1
  unsigned tk_stamp[kTicketQ];
};

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* a) { return *(const volatile unsigned*)a; }
__device__ __forceinline__ void st_volatile_u32(unsigned* a, unsigned v) { *(volatile unsigned*)a = v; }

// Producer warp pi (one thread each), hand-over positions s = 2k + pi.  For
// each it takes the position's ticket, waits (bounded) for the item's
// dependency on other CTAs, waits until the consumers of hand-over s - kStages,
// the previous user of stage buffer s mod kStages, are done with it (the
// publisher's freed count), copies the item's inputs into the buffer with TMA
// and hands it over to consumer group pi; its last hand-over is that group's
// end mark.  It publishes nothing: the publisher does, and a buffer is freed
// before its item is published, so the release of one item's outputs (a wait
// for its stores, which leave from registers) never delays preparing the next.  Positions follow ticket order
// and every dependency is on lower tickets, so the queue drains.
template <int NX, int NY, bool FW, bool AF>
__device__ void producer(const LateralParams& p, const CUtensorMap* tmap, uint64_t* full_bar, Desc* desc,
                         unsigned char* stage0, Handover* ho, int pi) {
  constexpr int RPI = kThreads / Split<NX>::N1;
  constexpr int BC = kThreads / Split<NY>::N1;
  constexpr int BOX_ROWS = band_box_rows(NY);
  const unsigned total = (unsigned)p.sch.total();
  auto give_up = [&]() {
    atomicCAS(&p.ctr->err, 0u, kErrTimeout);
    atomicExch(&p.ctr->abort, 1u);
  };
  auto aborted = [&]() { return *(volatile unsigned*)&p.ctr->abort != 0u; };
  const unsigned long long wait_limit = p.wait_ns ? p.wait_ns : kProducerWaitNs;
  // producer 0: tickets of the pair (2k, 2k + 1), the next pair requested early
  unsigned pair_next = (pi == 0 && !aborted()) ? atomicAdd(&p.ctr->ticket, 2u) : 0xffffffffu;
  for (unsigned k = 0;; ++k) {
    const unsigned s = 2u * k + (unsigned)pi;
    const int b = (int)(s % kStages);
    uint64_t* full = &full_bar[s % kFullBars];
    unsigned char* buf = stage0 + (size_t)b * p.stage_bytes;
    unsigned t = 0xffffffffu;
    if (pi == 0) {
      t = pair_next;
      ho->tk[k % kTicketQ] = t == 0xffffffffu ? t : t + 1u;
      __threadfence_block();
      st_volatile_u32(&ho->tk_stamp[k % kTicketQ], k + 1u);
    } else {
      const unsigned long long t0 = global_timer_ns();
      bool ok = true;
      while (ld_volatile_u32(&ho->tk_stamp[k % kTicketQ]) != k + 1u) {
        if (global_timer_ns() - t0 > wait_limit) {
          give_up();
          ok = false;
          break;
        }
        __nanosleep(32);  // leave the issue slots to the consumers meanwhile
      }
      if (ok) {
        __threadfence_block();
        t = ho->tk[k % kTicketQ];
      }
    }
    int kind = kEndItem, f = 0, item = 0;
    if (t < total && !aborted()) p.sch.decode(t, kind, f, item);
    const int slot = (p.tab0 + f) % p.nl;
    // input rows a row item stages (from its rows' y taps): loaded before the
    // dependency wait so that the two round trips overlap
    int ylo = 0, yhi = 0;
    if (kind == kRowItem && !AF) {
      const Tap* yt = p.ytab + (size_t)slot * NY;
      ylo = yt[item * RPI].base;
      yhi = yt[item * RPI + RPI - 1].base;
    }
    // 1. its dependency: a column item needs every row item of its frame; a row
    //    item needs the columns of the frame whose scratch slot it reuses
    if (kind != kEndItem) {
      const unsigned* dep = nullptr;
      unsigned target = 0;
      if (kind == kColItem) {
        dep = p.rows_done + f;
        target = (unsigned)p.sch.n_row;
      } else if (f >= p.sch.slots) {
        dep = p.cols_done + (f - p.sch.slots);
        target = (unsigned)p.sch.n_col;
      }
      if (dep && ld_acquire_gpu(dep) < target) {
        const unsigned long long t0 = global_timer_ns();
        while (ld_acquire_gpu(dep) < target) {
          if (aborted() || global_timer_ns() - t0 > wait_limit) {
            give_up();
            kind = kEndItem;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    fence_proxy_async_global();  // the acquired data is read by TMA (async proxy)
    Desc d{kind, f, item, 0, 0, slot};
    if (kind == kRowItem && !AF) {
      d.jlo = ylo;
      d.nrows = yhi + 1 - ylo + 1;
    }
    // 2. the consumers of the buffer's previous hand-over must be done with it
    if (s >= (unsigned)kStages && ld_volatile_u32(&ho->freed) + kStages <= s) {
      const unsigned long long t0 = global_timer_ns();
      while (ld_volatile_u32(&ho->freed) + kStages <= s) {
        if (global_timer_ns() - t0 > wait_limit) {
          give_up();
          kind = kEndItem;  // the buffer's old item is lost; the group still gets its end mark
          break;
        }
        __nanosleep(32);  // leave the issue slots to the consumers meanwhile
      }
    }
    // 3. hand over
    if (kind == kEndItem) {
      desc[b] = Desc{kEndItem, 0, 0, 0, 0, 0};
      mbar_arrive(full);
      __threadfence_block();
      st_volatile_u32(&ho->stamp[s % kPubQ], (s + 1u) | kEndStamp);
      break;
    }
    ho->kind[s % kPubQ] = kind;
    ho->f[s % kPubQ] = f;
    desc[b] = d;
    if (AF && kind == kRowItem) {
      // RPI contiguous rows of the half-spectrum plane of bin af_bin(f)
      const int q = af_bin(f, p.nl);
      const int plane = q <= p.nl / 2 ? q : p.nl - q;
      const unsigned bytes = (unsigned)(RPI * NX * sizeof(float2));
      mbar_arrive_tx(full, bytes);
      tma_load_1d(buf, p.aplanes + ((size_t)plane * NY + item * RPI) * NX, bytes, full);
    } else if (kind == kRowItem) {
      const unsigned bytes = (unsigned)(d.nrows * NX * sizeof(uint16_t));
      const unsigned tap_off = (unsigned)row_taps_offset<NX>(d.nrows);
      const unsigned tap_bytes = (unsigned)(NX * sizeof(Tap));
      const unsigned yt_bytes = (unsigned)(RPI * sizeof(Tap));
      const unsigned cy_bytes = (unsigned)(RPI * sizeof(float2));
      mbar_arrive_tx(full, bytes + tap_bytes + yt_bytes + cy_bytes);
      const int fr = (p.ring_start + f) % p.nl;
      tma_load_1d(buf, p.frames + ((size_t)fr * NY + d.jlo) * NX, bytes, full);
      tma_load_1d(buf + tap_off, p.xtab + (size_t)slot * NX, tap_bytes, full);
      tma_load_1d(buf + tap_off + tap_bytes, p.ytab + (size_t)slot * NY + item * RPI, yt_bytes, full);
      tma_load_1d(buf + tap_off + tap_bytes + yt_bytes, p.cy + item * RPI, cy_bytes, full);
    } else {
      mbar_arrive_tx(full, (unsigned)(NY * BC * sizeof(float2)));
      const int x = 2 * item * BC;
      const int y0 = (f % p.sch.slots) * NY;
#pragma unroll
      for (int i = 0; i < NY / BOX_ROWS; ++i)
        tma_load_2d(buf + (size_t)i * BOX_ROWS * BC * sizeof(float2), tmap, x, y0 + i * BOX_ROWS, full);
    }
    __threadfence_block();
    st_volatile_u32(&ho->stamp[s % kPubQ], s + 1u);
    if (pi == 0) pair_next = aborted() ? 0xffffffffu : atomicAdd(&p.ctr->ticket, 2u);
  }
}

// Publisher warp, one thread: in hand-over order, waits (bounded) for the
// position to be handed over and for its consumers to arrive on its buffer's
// done barrier, marks the buffer free for the producers, then publishes the
// item to other CTAs with a release increment of its frame's counter, which
// orders the item's outputs (the consumers' stores) before it at GPU scope.
// The first end mark ends it: tickets grow with positions, so no item follows
// an end mark.
__device__ void publisher(const LateralParams& p, uint64_t* done_bar, Handover* ho) {
  auto give_up = [&]() {
    atomicCAS(&p.ctr->err, 0u, kErrTimeout);
    atomicExch(&p.ctr->abort, 1u);
  };
  const unsigned long long wait_limit = 2 * (p.wait_ns ? p.wait_ns : kProducerWaitNs);
  for (unsigned s = 0;; ++s) {
    unsigned st = ld_volatile_u32(&ho->stamp[s % kPubQ]);
    if ((st & ~kEndStamp) != s + 1u) {
      const unsigned long long t0 = global_timer_ns();
      while (((st = ld_volatile_u32(&ho->stamp[s % kPubQ])) & ~kEndStamp) != s + 1u) {
        if (global_timer_ns() - t0 > wait_limit) {
          give_up();
          return;
        }
        __nanosleep(32);
      }
    }
    if (st & kEndStamp) return;
    __threadfence_block();
    const int kind = ho->kind[s % kPubQ];
    const int f = ho->f[s % kPubQ];
    const int b = (int)(s % kStages);
    const unsigned parity = (s / kStages) & 1u;
    // try_wait suspends the thread in hardware between checks: a test_wait spin
    // here would take issue slots from the consumer warps of its scheduler
    if (!mbar_try(&done_bar[b], parity)) {
      const unsigned long long t0 = global_timer_ns();
      while (!mbar_try(&done_bar[b], parity)) {
        if (global_timer_ns() - t0 > wait_limit) {
          give_up();
          return;
        }
      }
    }
    // the buffer can be refilled now: the item's outputs leave from registers
    st_volatile_u32(&ho->freed, s + 1u);
    red_release_gpu((kind == kRowItem ? p.rows_done : p.cols_done) + f, 1u);
  }
}

template <int NX, int NY, bool FW, bool AF>
__global__ void __launch_bounds__(kCtaThreads, 1)
    lateral_kernel(const __grid_constant__ LateralParams p, const __grid_constant__ CUtensorMap tmap) {
  static_assert(kThreads / Split<NX>::N1 <= NY, "a row item must not exceed the frame");
  static_assert(NY % band_box_rows(NY) == 0, "whole tensor copies cover a column band");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kFullBars];
  __shared__ __align__(8) uint64_t done_bar[kStages];
  __shared__ Desc desc[kStages];
  __shared__ Handover ho;
  const int tid = threadIdx.x;
  if (tid == 0) {
    ho.freed = 0u;
    for (int i = 0; i < kPubQ; ++i) ho.stamp[i] = 0u;
    for (int i = 0; i < kTicketQ; ++i) ho.tk_stamp[i] = 0u;
#pragma unroll
    for (int b = 0; b < kFullBars; ++b) mbar_init(&full_bar[b], 1);
#pragma unroll
    for (int b = 0; b < kStages; ++b) mbar_init(&done_bar[b], kThreads);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned char* stage0 = smem;
  float2* twx = reinterpret_cast<float2*>(smem + kStages * (size_t)p.stage_bytes);
  float2* twy = twx + NX;
  float2* cxs = twy + NY;
  if (tid >= kGroups * kThreads) {
    const int w = (tid - kGroups * kThreads) / 32;
    if (tid % 32 == 0) {
      if (w < kProducers) producer<NX, NY, FW, AF>(p, &tmap, full_bar, desc, stage0, &ho, w);
      else publisher(p, done_bar, &ho);
    }
    return;
  }
  for (int i = tid; i < NX; i += kGroups * kThreads) {
    twx[i] = ldg2(p.twx + i);
    cxs[i] = ldg2((AF ? p.cx2 : p.cx) + i);  // axial-first order: the squared chirp, for the mirrored bins
  }
  for (int i = tid; i < NY; i += kGroups * kThreads) twy[i] = ldg2(p.twy + i);
  asm volatile("bar.sync 3, %0;" ::"n"(kGroups * kThreads) : "memory");  // tables seen by both groups
  // Group g takes hand-overs s = g, g + kGroups, ...: buffer s mod kStages, full
  // barrier s mod kFullBars, whose previous fill (s - kFullBars) this group has
  // consumed and whose next fill needs this one freed, so the parity wait is
  // exact.
  const int g = tid / kThreads;
  for (unsigned s = g;; s += kGroups) {
    const int b = (int)(s % kStages);
    // consumers wait longer than the producer, which gives up first and hands
    // each group an end mark.  One thread of the group waits; the others sleep
    // at the group barrier instead of spinning (a spinning group takes issue
    // slots from the group that has work), and see the buffer's contents
    // through that barrier.
    bool ok = true;
    if (threadIdx.x % kThreads == 0)
      ok = mbar_wait(&full_bar[s % kFullBars], (s / kFullBars) & 1u, p.ctr, p.wait_ns ? 2 * p.wait_ns : kConsumerWaitNs);
    // the group agrees, and its previous item is finished in all its threads
    if (consumers_sync_or(g, !ok)) break;
    const Desc d = desc[b];
    if (d.kind == kEndItem) break;
    unsigned char* buf = stage0 + (size_t)b * p.stage_bytes;
    if (d.kind == kRowItem)
      row_item<NX, NY, FW, AF>(p, d, buf, twx, cxs, g);
    else
      col_item<NX, NY, FW, AF>(p, d, buf, twy, g);
    // this thread's writes to the buffer come before its next TMA fill (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(&done_bar[b]);
  }
}

// Shared memory: three stage buffers (a row item's inputs / transpose / output,
// or a column band), then the row and column twiddles and the x input chirp.
template <int NX, int NY>
void smem_layout(const Plan& p, size_t& stage_bytes, size_t& total) {
  constexpr int N1y = Split<NY>::N1;
  constexpr int BCy = kThreads / N1y;
  constexpr int RPI = kThreads / Split<NX>::N1;
  const size_t in_rows = row_stage_bytes<NX>(p.stage_rows);
  const size_t rows = (size_t)RPI * NX * sizeof(float2);     // transpose block / output of a row item
  const size_t cols = (size_t)NY * BCy * sizeof(float2);     // a column band
  size_t sbm = in_rows > rows ? in_rows : rows;
  sbm = sbm > cols ? sbm : cols;
  stage_bytes = (sbm + 1023) / 1024 * 1024;
  total = kStages * stage_bytes + (size_t)(2 * NX + NY) * sizeof(float2);
}

template <int NX, int NY>
size_t smem_for(const Plan& p) {
  size_t sb, total;
  smem_layout<NX, NY>(p, sb, total);
  return total;
}

template <int NX, int NY, bool FW, bool AF>
cudaError_t launch_fw(const Plan& p, const LateralParams& lp_in, const void* tmap, int num_sms, cudaStream_t s) {
  size_t sb, smem;
  smem_layout<NX, NY>(p, sb, smem);
  LateralParams lp = lp_in;
  lp.stage_bytes = (int)sb;
  cudaError_t e = cudaFuncSetAttribute(lateral_kernel<NX, NY, FW, AF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const long long total = lp.sch.total();
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lateral_kernel<NX, NY, FW, AF>, kCtaThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = (num_sms > 0 ? num_sms : 1) * per_sm;
  if (grid > total) grid = (int)total;
  lateral_kernel<NX, NY, FW, AF><<<grid, kCtaThreads, smem, s>>>(lp, *reinterpret_cast<const CUtensorMap*>(tmap));
  return cudaGetLastError();
}

template <int NX, int NY>
cudaError_t launch(const Plan& p, const LateralParams& lp, const void* tmap, int num_sms,
                   cudaStream_t s) {
  if (p.axial_first)
    return lateral_full_window(p) ? launch_fw<NX, NY, true, true>(p, lp, tmap, num_sms, s)
                                  : launch_fw<NX, NY, false, true>(p, lp, tmap, num_sms, s);
  return lateral_full_window(p) ? launch_fw<NX, NY, true, false>(p, lp, tmap, num_sms, s)
                                : launch_fw<NX, NY, false, false>(p, lp, tmap, num_sms, s);
}

#define SSOCT_LATERAL_SIZES(X) \
  X(64, 64) X(128, 128) X(256, 256) X(384, 384) X(512, 512) X(640, 640) X(768, 768) X(1024, 1024) X(128, 64) X(64, 128)

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

int lateral_col_band(int ny) { return kThreads / split_n1(ny); }

cudaError_t launch_lateral_with(const Plan& p, const LateralParams& lp, const void* tmap,
                                int num_sms, cudaStream_t s) {
#define X(a, b) if (p.nx == a && p.ny == b) return launch<a, b>(p, lp, tmap, num_sms, s);
  SSOCT_LATERAL_SIZES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_lateral(const Plan& p, const LateralParams& lp, cudaStream_t s) {
  return launch_lateral_with(p, lp, p.tmap, p.num_sms, s);
}

}  // namespace ssoct
