// Internal types shared by the host plan code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ssoct.h"

namespace ssoct {

constexpr int kThreads = 256;          // threads of a lateral-stage CTA (two CTAs per SM)
constexpr int kTile = 32;              // pixels per sweep-axis tile (one x-run)

// FFT length N = N1 * N2 as the kernels split it: an N2-point DFT per thread,
// a twiddle, an exchange through shared memory, N1-point DFTs (0 = not built).
__host__ __device__ constexpr int split_n1(int n) {
  return n == 16 ? 4 : n == 32 ? 4 : n == 64 ? 8 : n == 96 ? 4 : n == 128 ? 8 : n == 160 ? 4 : n == 200 ? 5
       : n == 256 ? 16 : n == 384 ? 16 : n == 512 ? 16 : n == 640 ? 32 : n == 768 ? 32 : n == 1024 ? 32 : 0;
}

// Stage 2 of a transform of length N = N1 x N2 (N1 = split_n1(N)) in the
// persistent lateral kernel: N2 N1-point DFTs spread over the transform's N1
// threads, NI per thread; where N1 does not divide N2 (384 = 16 x 24,
// 640 = 32 x 20, 768 = 32 x 24) the last one is idle in the threads
// j1 >= N2 - N1 (NI - 1).  A is the register array length.
template <int N, int N1_ = split_n1(N)>
struct Stage2 {
  static constexpr int N1 = N1_, N2 = N / N1_;
  static constexpr int NI = (N2 + N1 - 1) / N1;
  static constexpr int A = NI * N1 > N2 ? NI * N1 : N2;
  // stage-2 DFT i of thread j1 exists (always, for the iterations N1 fills)
  __host__ __device__ static constexpr bool live(int i, int j1) { return (i + 1) * N1 <= N2 || j1 + N1 * i < N2; }
};

// Split of the axial-first first pass's transform over nl frames, N1 x nl/N1
// with a tile of 32 N1 threads: the axial split where it gives 8 to 16 warps,
// and 16 x 6, 16 x 10, 20 x 10 for 96, 160, 200 frames, whose axial splits
// (4 x 24, 4 x 40, 5 x 40) would leave four or five warps per tile.
__host__ __device__ constexpr int ra_split_n1(int nl) {
  return nl == 96 ? 16 : nl == 160 ? 16 : nl == 200 ? 20 : split_n1(nl);
}

// Rows per tensor copy of a lateral column band: the largest divisor of ny up
// to 256 (a box dimension's limit), so that whole boxes cover the column.
__host__ __device__ constexpr int band_box_rows(int ny) {
  int r = ny < 256 ? ny : 256;
  while (r > 1 && ny % r != 0) --r;
  return r;
}

// Separable linear-interpolation tap for one output coordinate of one frame
// (Eq. 5): the value is w0 * in[base] + w1 * in[base + 1]; base is clamped so
// both reads are inside the frame, and a weight is 0 where its tap fell outside.
struct __align__(16) Tap {
  int base;
  float w0;
  float w1;
  float pad;
};

// Eq. 5 along a 64-pixel strip x0 .. x0 + 63 of one frame (axial-first order):
// the position u(x0 + k) = u(x0) + k s_t lies at staged column
// off + k + floor(f + k e) with weight frac(f + k e), where the strip's source
// rows are staged from column xs (a multiple of 8) on.  Built in float64.
struct __align__(16) StripTap {
  int xs;    // first staged source column (multiple of 8; may be negative)
  int off;   // floor(u(x0)) - xs (>= 1)
  float f;   // u(x0) - floor(u(x0))
  float e;   // s_t - 1
};

// Device work-queue counters of the lateral kernel (zeroed before each launch).
struct Counters {
  unsigned ticket;
  unsigned abort;
  unsigned err;
  unsigned pad[29];
  // followed by rows_done[nlambda], cols_done[nlambda]
};

constexpr unsigned kErrTimeout = 1u;      // lateral kernel: a queue wait ran out
constexpr unsigned kErrAxialTc = 2u;      // tensor-core axial kernel: an MMA wait ran out
constexpr unsigned kErrAxial = 4u;        // streaming axial kernel: a stage-buffer wait ran out

// Order in which the lateral kernel takes its items.  Step s holds the row
// items of frame s (if s < nl) and then the column items of frame s - lag (if
// s >= lag).  A column item of frame f waits for every row item of f; a row item
// of frame f (f >= slots) waits for every column item of f - slots, whose L2
// scratch slot it reuses.  Both wait on items of earlier tickets, and a ticket
// is only taken by a running CTA, so the queue always drains (requires
// slots > lag).
struct LateralSchedule {
  int nl;
  int n_row;   // row items per frame
  int n_col;   // column items per frame
  int lag;
  int slots;

  __host__ __device__ long long total() const { return (long long)nl * (n_row + n_col); }

  // 32-bit arithmetic: a sweep has at most 512 x 2 x 1024 tickets, and the
  // producer decodes one per item, so 64-bit division would cost it hundreds
  // of cycles.
  __host__ __device__ void decode(unsigned k, int& kind, int& frame, int& item) const {
    const unsigned nr = (unsigned)n_row, nc = (unsigned)n_col;
    const unsigned head = (unsigned)lag * nr;
    if (k < head) {
      kind = 0;
      frame = (int)(k / nr);
      item = (int)(k - (unsigned)frame * nr);
      return;
    }
    k -= head;
    const unsigned per = nr + nc;
    const unsigned both = (unsigned)(nl - lag) * per;
    if (k < both) {
      const unsigned st = k / per;
      const unsigned r = k - st * per;
      if (r < nr) {
        kind = 0;
        frame = lag + (int)st;
        item = (int)r;
      } else {
        kind = 1;
        frame = (int)st;
        item = (int)(r - nr);
      }
      return;
    }
    k -= both;
    kind = 1;
    const unsigned q = k / nc;
    frame = nl - lag + (int)q;
    item = (int)(k - q * nc);
  }
};

// Everything the lateral kernel (rescale + chirp + row FFT, column FFT) reads.
struct LateralParams {
  const uint16_t* frames;  // batch frame f at frames + ((ring_start + f) % nl) * nx * ny
  int ring_start;
  int tab0;                // batch frame f has wavelength / intermediate index (tab0 + f) % nl
  int nx, ny, nl;
  int x0, y0, wx, wy;      // window
  int wxp;                 // scratch row pitch (complex elements)
  int ntx;                 // sweep-axis tiles per window row
  const Tap* xtab;         // [nl][nx]
  const Tap* ytab;         // [nl][ny]
  const float2* cx;        // [nx] input chirp incl. centring phase
  const float2* cy;        // [ny]
  const float2* cx2;       // [nx] squared input chirp (axial-first order, bins above nl/2)
  const float2* cy2;       // [ny]
  const float2* twx;       // [N2x][N1x] row-FFT twiddles
  const float2* twy;       // [N2y][N1y] column-FFT twiddles
  float2* scratch;         // [slots][ny][wxp]
  float2* inter;           // [wy][ntx][nl][32]
  Counters* ctr;
  unsigned* rows_done;     // [nl]
  unsigned* cols_done;     // [nl]
  LateralSchedule sch;
  int stage_rows;          // input rows staged per row item (max over items)
  int stage_bytes;         // bytes of one shared-memory stage buffer (set at launch)
  unsigned long long wait_ns;  // limit of every device-side wait (0 = default)
  // axial-first order (SSOCT_FLAG_AXIAL_FIRST): frame f is depth bin af_bin(f);
  // row items read half-spectrum planes, column items write the volume
  const float2* aplanes;   // [nl/2 + 1][ny][nx]
  float* vol;              // [nl][wy][wx]
  float2* cplx;            // optional [nl][wy][wx]
  const float2* ox;        // [wx] output chirp (x)
  const float2* oy;        // [wy] output chirp (y) times K
  float inv_k_abs;         // 1 / |K|: the planes carry |K| (so |V|^2 |K|^2 = |v|^2), oy holds K as well
  int magnitude;
};

struct AxialParams {
  const float2* inter;     // [wy][ntx][nl][32]
  float* vol;              // [nl][wy][wx]
  float2* cplx;            // optional [nl][wy][wx]
  const float2* twl;       // [N2l][N1l], sign -
  const float2* ox;        // [wx] output chirp (x), incl. centring phase
  const float2* oy;        // [wy] output chirp (y) times the prefactor K
  int nl, wx, wy, ntx;
  float power_scale;       // |K|^2
  int magnitude;           // 1: write |V| instead of |V|^2
  unsigned* err;           // error word (kErrAxial), the plan's Counters::err
};

struct CutsParams {
  const float* vol;
  float* xy;
  float* xz;
  float* yz;
  int nl, wx, wy, x0, y0, z0;
};

// Host-side plan.
struct Plan {
  int nx, ny, nl;
  int x0, y0, wx, wy;
  unsigned flags;
  double pitch, z, lambda1;
  std::vector<double> lambdas;
  double kre, kim;          // prefactor K
  double alpha;             // d^2 / (lambda_1 z) = |K|
  // host tables
  std::vector<Tap> xtab, ytab;
  std::vector<float2> cx, cy, cx2, cy2, ox, oy, twx, twy, twl, twra;
  std::vector<float2> wq;   // [nl] exp(-2 pi i k / nl), for single-bin transforms
  std::vector<unsigned short> tcb;  // SSOCT_FLAG_TC_AXIAL: BF16 hi / lo 16-point DFT matrix (operand layout)
  // SSOCT_FLAG_PUPIL: input chirp x Zernike screen, its distance z and |K|, frames per Q chunk
  double sh_z = 0.0, sh_alpha = 0.0;
  double sh_coeffs[15] = {};
  int sh_ncoeffs = 0;
  bool sh_dirty = false;     // the device table is built by the next ssoct_sharpness
  int sh_tpc = 8;
  bool sh_ready = false;
  // geometry of the device work
  int n1x, n2x, n1y, n2y, n1l, n2l;
  int rows_per_item, cols_per_item;
  int wxp, ntx;
  int stage_rows;
  LateralSchedule sch;
  int slots_alloc = 0;       // scratch-ring slots the workspace holds (sch.slots <= slots_alloc)
  bool use_tc = false;       // axial pass on the tensor cores (flag, or the autotuner's choice)
  // workspace layout (byte offsets)
  size_t off_ctr, off_xtab, off_ytab, off_cx, off_cy, off_cx2, off_cy2, off_ox, off_oy, off_twx, off_twy, off_twl;
  size_t off_twra = 0;       // twiddles of the tiled first pass's split (ra_split_n1)
  size_t off_tcb, off_wq, off_ring, off_scratch, off_inter, ws_bytes;
  size_t off_cp = 0, off_F = 0, off_Q = 0, off_red = 0;  // SSOCT_FLAG_PUPIL regions
  // Frame sizes the persistent lateral kernel does not compile (384, 640, 768)
  // take the two-pass lateral path of sharpness.cu: chirp table and frame buffer.
  bool generic = false;
  size_t off_cg = 0;
  // SSOCT_FLAG_AXIAL_FIRST: Eq. 5 + Eq. 7 first (half spectrum of the real
  // rescaled frames), then the lateral kernel on the planes
  bool axial_first = false;  // order of whole-volume reconstructions (the flag's, or the autotuner's choice)
  bool af_forced = false;    // created with SSOCT_FLAG_AXIAL_FIRST: every call runs that order
  bool af_option = false;    // the autotuner may pick the axial-first order (its planes fit the intermediate)
  size_t off_aplanes = 0;
  // tiled first pass (rescale_axial_tiled): strip records [nl][nx / 64] and the
  // staged columns per source row (0: the one-tile-per-CTA kernel instead)
  std::vector<StripTap> xstrip;
  size_t off_xstrip = 0;
  int ra_w = 0;
  char* ws = nullptr;
  int device = -1;
  int noalloc_device = -1;   // device of the plan's last no-allocation call (-1: none)
  int num_sms = 0;
  alignas(64) unsigned char tmap[128];        // CUtensorMap of the scratch ring (column bands)
  // frame ring state
  long long pushed = 0;     // frames in the current gate (capped at nl)
  int ring_head = 0;        // next ring slot to write
  long long next_seq = -1;
  long long stream_count = 0;  // frames pushed since the gate (re)started, uncapped
  long long lat_upto = -1;     // sliding gates: stream index up to which the intermediate holds holograms
  // cuts-only sliding gates: running one-bin transform X(z0) of the gate, valid
  // for the intermediate as it stood at lat_upto == xs_lat; xs_updates frames
  // have been swapped in since it was last summed in full
  size_t off_xys = 0;          // [wy][ntx * 32] complex
  bool xs_valid = false;
  int xs_z0 = 0;
  int xs_updates = 0;
  long long xs_lat = -1;
  std::string last_error;
  // failure injection (ssoct_inject_stall)
  unsigned inject_skip = 0;
  unsigned long long wait_ns = 0;
  // stage timing (ssoct_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> events;  // 3 per recorded call: start, after lateral, after axial
  size_t events_used = 0;
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_lateral(const Plan& p, const LateralParams& lp, cudaStream_t s);
cudaError_t launch_axial(const Plan& p, const AxialParams& ap, cudaStream_t s);
cudaError_t launch_cuts(const CutsParams& cp, cudaStream_t s);
// The three cuts of the current gate straight from the sweep-axis intermediate
// (xy: one bin per pixel; xz, yz: the axial transform of the cut's tiles).
// xy_state, if not NULL, receives the xy cut's complex X(z0) ([wy][ntx * 32]).
cudaError_t launch_gate_cuts(const Plan& p, int x0, int y0, int z0, float* xy, float* xz, float* yz,
                             float2* xy_state, cudaStream_t s);
// Running xy cut of the sliding gate (one bin of Eq. 7 is linear in the gate's
// holograms): X(z0) += sign * sum over slots slot0 .. slot0 + k - 1 (mod nl) of
// h_t exp(-2 pi i z0 t / nl), then xy = envelope of X if xy is not NULL.
cudaError_t launch_xy_slide(const Plan& p, int slot0, int k, int z0, float sign, float* xy, cudaStream_t s);
// Axial-first order, first pass: Eq. 5 resample of every frame and Eq. 7 over
// the sweep at every pixel, bins 0..nl/2 written as planes [nl/2 + 1][ny][nx].
cudaError_t launch_rescale_axial(const Plan& p, const uint16_t* frames, int ring_start, float2* planes,
                                 cudaStream_t s);
// The tiled first pass: sizes it is built for, and its dynamic shared memory
// for w staged columns per source row.
bool rescale_axial_tiled(int nx, int nl);
size_t rescale_axial_tile_smem(int nl, int w);
// Tensor map over a gate's frames seen as uint16 [nl * ny][nx], boxes of
// box_cols columns x 2 rows (zero fill outside the frame).
bool encode_frames_map(const Plan& p, const uint16_t* frames, int box_cols, void* map_out);
// Tensor map over the sweep-axis intermediate seen as float [rows][64] (one
// row = 32 complex values of one frame of a tile), boxes of box_complex
// complex values x 256 rows.
bool encode_inter_map(const float2* inter, long long rows, int box_complex, void* map_out);
bool lateral_supported(int nx, int ny);
bool axial_supported(int nl);
// Tensor-core axial kernel (axial_tc.cu): sweep lengths it handles, its DFT
// operand table, dynamic shared memory, and launcher.  err is the plan's error
// word; the kernel ORs kErrAxialTc into it when an MMA wait runs out.
bool axial_tc_supported(int nl);
void axial_tc_table(std::vector<unsigned short>& out);
size_t axial_tc_smem_bytes();
cudaError_t launch_axial_tc(const Plan& pl, const AxialParams& ap, const unsigned short* bmat, unsigned* err,
                            int num_sms, cudaStream_t s);
// Aberration path (sharpness.cu): sizes it compiles, the c P table, and the
// forward + adjoint launches that leave loss and gradient in the FP64 block at
// off_red ([0] S1, [1] S2, [2] loss, [3] dL/dz, [4..18] dL/dc_1..15).
constexpr int kShRedDoubles = 19;
bool sharpness_supported(int nx, int ny, int nl);
bool generic_lateral_supported(int nx, int ny);
// Eq. 5 + Eq. 6 as a row pass and a column pass through the frame buffer at
// off_F, for frames[(ring_start + t) mod nl]; writes the sweep-axis intermediate.
cudaError_t launch_lateral_generic(const Plan& pl, const uint16_t* frames, int ring_start, cudaStream_t s);
void build_pupil_table(int nx, int ny, double alpha, const double* coeffs, int ncoeffs, std::vector<float2>& out);
cudaError_t launch_sharpness(const Plan& pl, const uint16_t* frames, float* vol, cudaStream_t s);
cudaError_t launch_pupil_table(const Plan& pl, cudaStream_t s);
// Dynamic shared memory of the lateral kernel for a plan (bytes).
size_t lateral_smem_bytes(const Plan& p);
// Columns per column item of the lateral kernel for a column length ny.
int lateral_col_band(int ny);

// Used by the no-allocation entry point (noalloc.cu): the plan behind a handle,
// a scratch-ring tensor map for scratch memory at an arbitrary device address,
// and a lateral launch that takes the tensor map and SM count explicitly.
Plan& plan_of(ssoct_plan h);
bool encode_scratch_map_at(const Plan& p, void* scratch_dev, void* map_out);
cudaError_t launch_lateral_with(const Plan& p, const LateralParams& lp, const void* tmap,
                                int num_sms, cudaStream_t s);
// The axial launch with the SM count given explicitly (the persistent streaming
// form sizes its grid by it); launch_axial passes the plan's own.
cudaError_t launch_axial_with(const Plan& p, const AxialParams& ap, int num_sms, cudaStream_t s);
// Error word of the last no-allocation call made with this plan (0 if none, or
// if that call's kernels met no time-out); read after the caller's stream sync.
cudaError_t noalloc_error_word(Plan& p, unsigned* err);
// Runs the paper's order for one call on a plan whose axial-first order was
// only the autotuner's choice (sliding gates and the no-allocation path keep
// the paper's order); restores the plan's order when it goes out of scope.
struct PaperOrderScope {
  Plan& p;
  bool saved;
  explicit PaperOrderScope(Plan& pl) : p(pl), saved(pl.axial_first) {
    if (!p.af_forced) p.axial_first = false;
  }
  ~PaperOrderScope() { p.axial_first = saved; }
};

// Whole-frame window: the lateral kernel then needs no window bounds checks.
inline bool lateral_full_window(const Plan& p) { return p.x0 == 0 && p.y0 == 0 && p.wx == p.nx && p.wy == p.ny; }

}  // namespace ssoct
