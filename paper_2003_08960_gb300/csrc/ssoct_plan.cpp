// Host side of libssoct: plan validation, float64 table construction, workspace
// layout, frame ring, and the C ABI entry points declared in include/ssoct.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "ssoct_internal.h"

using namespace ssoct;

struct ssoct_plan_s {
  Plan p;
};

namespace {

constexpr size_t kAlign = 256;
constexpr double kPi = 3.14159265358979323846264338327950288;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

ssoct_status fail(Plan* p, ssoct_status s, const std::string& msg) {
  if (p) p->last_error = msg;
  return s;
}

ssoct_status cuda_fail(Plan* p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(p, SSOCT_ECUDA, m);
}

// exp(i pi r) for r given already reduced to a few units; float64 then rounded once.
float2 cis_pi(double r) {
  const double a = kPi * r;
  return make_float2((float)std::cos(a), (float)std::sin(a));
}

// Eq. 5 along one axis: output pixel i reads the input at u = c + (i - c) s,
// c = n / 2, by linear interpolation; a tap outside [0, n) reads 0.
Tap make_tap(int i, int n, double s) {
  const double c = n / 2.0;
  const double u = c + (i - c) * s;
  const double fl = std::floor(u);
  const double a = u - fl;
  const long i0 = (long)fl, i1 = i0 + 1;
  const double w0 = (i0 >= 0 && i0 < n) ? 1.0 - a : 0.0;
  const double w1 = (i1 >= 0 && i1 < n) ? a : 0.0;
  long b = i0 < 0 ? 0 : i0;
  if (b > n - 2) b = n - 2;
  double wb = 0.0, wb1 = 0.0;
  if (i0 == b) wb += w0; else if (i0 == b + 1) wb1 += w0;
  if (i1 == b) wb += w1; else if (i1 == b + 1) wb1 += w1;
  Tap t;
  t.base = (int)b;
  t.w0 = (float)wb;
  t.w1 = (float)wb1;
  t.pad = 0.f;
  return t;
}

// Input chirp of Eq. 6 times the centring phase along one axis of length n:
// exp(-i pi [(k - n/2)^2 alpha + k]); alpha = d^2 / (lambda_1 z).  With it the
// centred sum over (k - n/2)(m - n/2) / n becomes a plain DFT over k m / n.
std::vector<float2> input_chirp(int n, double alpha) {
  std::vector<float2> v(n);
  for (int k = 0; k < n; ++k) {
    const double d = k - n / 2.0;
    const double r = std::fmod(d * d * alpha, 2.0) + (double)(k & 1);
    v[k] = cis_pi(-r);
  }
  return v;
}

// Square of the input chirp: exp(-2 i pi (k - n/2)^2 alpha) (the centring
// phase squares to 1).  In axial-first order the planes carry the input chirp
// c, and a bin above nl/2 needs conj(X) c = conj(X c) c^2.
std::vector<float2> input_chirp_squared(int n, double alpha) {
  std::vector<float2> v(n);
  for (int k = 0; k < n; ++k) {
    const double d = k - n / 2.0;
    v[k] = cis_pi(-std::fmod(2.0 * d * d * alpha, 2.0));
  }
  return v;
}

// Output chirp of Eq. 6 on the hologram grid x_m = (m - n/2) d', times the
// remaining centring phase exp(-i pi (m - n/2)):  exp(-i pi [(m - n/2)^2 / (n^2 alpha) + m - n/2]).
std::vector<float2> output_chirp(int n, double alpha, int m0, int count) {
  std::vector<float2> v(count);
  const double inv = 1.0 / ((double)n * (double)n * alpha);
  for (int i = 0; i < count; ++i) {
    const int m = m0 + i;
    const double d = m - n / 2.0;
    const double r = std::fmod(d * d * inv, 2.0) + std::fmod(d, 2.0);
    v[i] = cis_pi(-r);
  }
  return v;
}

// tw[k2][j1] = exp(sign 2 pi i j1 k2 / n) for the n = n1 * n2 split.
std::vector<float2> twiddles(int n, int n1, int n2, int sign) {
  std::vector<float2> v((size_t)n1 * n2);
  for (int k2 = 0; k2 < n2; ++k2)
    for (int j1 = 0; j1 < n1; ++j1) {
      const long e = ((long)j1 * k2) % n;
      v[(size_t)k2 * n1 + j1] = cis_pi(sign * 2.0 * (double)e / n);
    }
  return v;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// Tensor map over the scratch ring seen as float32 [slots * ny][2 * wxp]; one
// box is a column band of the lateral kernel (2 * band floats x band_box_rows(ny) rows).
bool encode_scratch_map(Plan& p) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int band = lateral_col_band(p.ny);
  cuuint64_t dims[2] = {(cuuint64_t)2 * p.wxp, (cuuint64_t)p.slots_alloc * p.ny};
  cuuint64_t strides[1] = {(cuuint64_t)2 * p.wxp * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)(2 * band), (cuuint32_t)band_box_rows(p.ny)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(p.tmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p.ws + p.off_scratch,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

namespace ssoct {

Plan& plan_of(ssoct_plan h) { return h->p; }

bool encode_scratch_map_at(const Plan& p, void* scratch_dev, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int band = lateral_col_band(p.ny);
  cuuint64_t dims[2] = {(cuuint64_t)2 * p.wxp, (cuuint64_t)p.slots_alloc * p.ny};
  cuuint64_t strides[1] = {(cuuint64_t)2 * p.wxp * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)(2 * band), (cuuint32_t)band_box_rows(p.ny)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, scratch_dev, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}


bool encode_inter_map(const float2* inter, long long rows, int box_complex, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)2 * kTile, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kTile * sizeof(float2)};
  cuuint32_t box[2] = {(cuuint32_t)(2 * box_complex), 256};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<float2*>(inter), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_frames_map(const Plan& p, const uint16_t* frames, int box_cols, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.nl * p.ny};
  cuuint64_t strides[1] = {(cuuint64_t)p.nx * sizeof(uint16_t)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, 2};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                   const_cast<uint16_t*>(frames), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace ssoct

extern "C" {

const char* ssoct_status_string(ssoct_status s) {
  switch (s) {
    case SSOCT_OK: return "SSOCT_OK";
    case SSOCT_EINVAL: return "SSOCT_EINVAL";
    case SSOCT_ENOMEM: return "SSOCT_ENOMEM";
    case SSOCT_ECUDA: return "SSOCT_ECUDA";
    case SSOCT_EAGAIN: return "SSOCT_EAGAIN";
    case SSOCT_ENOTREADY: return "SSOCT_ENOTREADY";
    case SSOCT_EDROPPED: return "SSOCT_EDROPPED";
    case SSOCT_ETIMEOUT: return "SSOCT_ETIMEOUT";
    case SSOCT_EUNSUPPORTED: return "SSOCT_EUNSUPPORTED";
  }
  return "SSOCT_?";
}

ssoct_status ssoct_create_plan(int nx, int ny, int nlambda, double pitch_m, double z_m,
                               const double* lambda_m, const ssoct_window* win, unsigned flags,
                               ssoct_plan* out) {
  if (!out) return SSOCT_EINVAL;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nlambda < 1 || !lambda_m) return SSOCT_EINVAL;
  if ((nx & 1) || (ny & 1)) return SSOCT_EINVAL;  // the centred grid needs an even size
  if (!(pitch_m > 0.0) || !std::isfinite(pitch_m) || z_m == 0.0 || !std::isfinite(z_m))
    return SSOCT_EINVAL;
  for (int t = 0; t < nlambda; ++t)
    if (!(lambda_m[t] > 0.0) || !std::isfinite(lambda_m[t])) return SSOCT_EINVAL;
  if (flags & ~(SSOCT_FLAG_MAGNITUDE | SSOCT_FLAG_TC_AXIAL | SSOCT_FLAG_PUPIL | SSOCT_FLAG_AXIAL_FIRST)) return SSOCT_EINVAL;
  ssoct_window w = win ? *win : ssoct_window{0, 0, nx, ny};
  if (w.x0 < 0 || w.y0 < 0 || w.wx < 1 || w.wy < 1 || w.x0 + w.wx > nx || w.y0 + w.wy > ny)
    return SSOCT_EINVAL;
  if (!axial_supported(nlambda)) return SSOCT_EUNSUPPORTED;
  const bool generic = !lateral_supported(nx, ny);  // two-pass lateral path for the other sizes
  if (generic && !generic_lateral_supported(nx, ny)) return SSOCT_EUNSUPPORTED;
  if ((flags & SSOCT_FLAG_AXIAL_FIRST) && (generic || (nlambda & 1) || (flags & SSOCT_FLAG_TC_AXIAL)))
    return SSOCT_EUNSUPPORTED;
  if ((flags & SSOCT_FLAG_TC_AXIAL) && !axial_tc_supported(nlambda)) return SSOCT_EUNSUPPORTED;
  if ((flags & SSOCT_FLAG_PUPIL) && !sharpness_supported(nx, ny, nlambda)) return SSOCT_EUNSUPPORTED;

  ssoct_plan h = new (std::nothrow) ssoct_plan_s();
  if (!h) return SSOCT_ENOMEM;
  Plan& p = h->p;
  p.nx = nx; p.ny = ny; p.nl = nlambda;
  p.x0 = w.x0; p.y0 = w.y0; p.wx = w.wx; p.wy = w.wy;
  p.flags = flags;
  p.generic = generic;
  p.af_forced = (flags & SSOCT_FLAG_AXIAL_FIRST) != 0;
  p.axial_first = p.af_forced;
  p.pitch = pitch_m; p.z = z_m;
  p.lambdas.assign(lambda_m, lambda_m + nlambda);
  p.lambda1 = lambda_m[0];
  p.alpha = pitch_m * pitch_m / (p.lambda1 * z_m);
  {
    // K = (i / (lambda_1 z)) exp(-i k_1 z) d^2; k_1 z = 2 pi z / lambda_1 reduced mod 1 turn.
    const double turns = std::fmod(z_m / p.lambda1, 1.0);
    const double ph = -2.0 * kPi * turns;
    const double mag = pitch_m * pitch_m / (p.lambda1 * z_m);
    // i * exp(i ph) = exp(i (ph + pi/2))
    p.kre = mag * std::cos(ph + 0.5 * kPi);
    p.kim = mag * std::sin(ph + 0.5 * kPi);
  }

  // Eq. 5 taps, per frame and axis (ratio lambda_t / lambda_1).
  p.xtab.resize((size_t)nlambda * nx);
  p.ytab.resize((size_t)nlambda * ny);
  for (int t = 0; t < nlambda; ++t) {
    const double s = lambda_m[t] / p.lambda1;
    for (int i = 0; i < nx; ++i) p.xtab[(size_t)t * nx + i] = make_tap(i, nx, s);
    for (int j = 0; j < ny; ++j) p.ytab[(size_t)t * ny + j] = make_tap(j, ny, s);
  }
  // Axial-first order, tiled first pass: one strip record per (frame, 64-pixel
  // strip), and the staged width that holds every frame's taps of a strip
  // (one column of slack at each end for the float32 position's rounding).
  // Built for every plan whose sizes the tiled pass takes: the autotuner may
  // choose that order for plans created without the flag.
  if (!generic && rescale_axial_tiled(nx, nlambda)) {
    const int strips = nx / 64;
    p.xstrip.resize((size_t)nlambda * strips);
    int wmax = 0;
    const double c = nx / 2.0;
    for (int t = 0; t < nlambda; ++t) {
      const double s = lambda_m[t] / p.lambda1;
      for (int k = 0; k < strips; ++k) {
        const double u0 = c + (64.0 * k - c) * s;
        const double u1 = c + (64.0 * k + 63.0 - c) * s;
        const long n0 = (long)std::floor(u0);
        const long xs = (long)std::floor((double)(n0 - 1) / 8.0) * 8;
        StripTap& r = p.xstrip[(size_t)t * strips + k];
        r.xs = (int)xs;
        r.off = (int)(n0 - xs);
        r.f = (float)(u0 - (double)n0);
        r.e = (float)(s - 1.0);
        const long hi = (long)std::floor(u1) + 1 - xs;  // last staged column the strip reads
        wmax = std::max<int>(wmax, (int)std::max<long>(hi + 2, r.off + 2));
      }
    }
    const int w = (wmax + 7) / 8 * 8;
    // beyond 128 columns (rescale ratios far from 1) the staging buffer would not
    // fit, and the one-tile-per-CTA kernel is used
    const bool ok = w <= 128 && rescale_axial_tile_smem(nlambda, w) <= 227u * 1024u;
    if (ok) p.ra_w = w;
    else p.xstrip.clear();
  }
  // Eq. 6 chirps.  alpha x (k - n/2)^2 is the chirp phase / pi.
  p.cx = input_chirp(nx, p.alpha);
  p.cy = input_chirp(ny, p.alpha);
  p.cx2 = input_chirp_squared(nx, p.alpha);
  p.cy2 = input_chirp_squared(ny, p.alpha);
  p.ox = output_chirp(nx, p.alpha, p.x0, p.wx);
  {
    std::vector<float2> oy = output_chirp(ny, p.alpha, p.y0, p.wy);
    // fold K into the y factor (float64 product, rounded once)
    const double c = ny / 2.0;
    const double inv = 1.0 / ((double)ny * (double)ny * p.alpha);
    for (int i = 0; i < p.wy; ++i) {
      const int m = p.y0 + i;
      const double d = m - c;
      const double r = std::fmod(d * d * inv, 2.0) + std::fmod(d, 2.0);
      const double cr = std::cos(-kPi * r), ci = std::sin(-kPi * r);
      oy[i] = make_float2((float)(p.kre * cr - p.kim * ci), (float)(p.kre * ci + p.kim * cr));
    }
    p.oy = oy;
  }
  p.n1x = split_n1(nx); p.n2x = nx / p.n1x;
  p.n1y = split_n1(ny); p.n2y = ny / p.n1y;
  p.n1l = split_n1(nlambda); p.n2l = nlambda / p.n1l;
  p.twx = twiddles(nx, p.n1x, p.n2x, +1);
  p.twy = twiddles(ny, p.n1y, p.n2y, +1);
  p.twl = twiddles(nlambda, p.n1l, p.n2l, -1);
  p.twra = twiddles(nlambda, ra_split_n1(nlambda), nlambda / ra_split_n1(nlambda), -1);
  p.wq.resize(nlambda);
  for (int k = 0; k < nlambda; ++k) p.wq[k] = cis_pi(-2.0 * (double)k / nlambda);  // exp(-2 pi i k / nlambda)
  if (axial_tc_supported(nlambda)) axial_tc_table(p.tcb);  // kept for every such plan: the autotuner may switch forms
  p.use_tc = (flags & SSOCT_FLAG_TC_AXIAL) != 0;

  // Work decomposition of the lateral kernel.
  p.rows_per_item = kThreads / p.n1x;
  if (p.rows_per_item > ny) p.rows_per_item = ny;
  p.cols_per_item = kThreads / p.n1y;
  p.wxp = (int)align_up((size_t)p.wx, 64);
  p.ntx = (p.wx + kTile - 1) / kTile;
  p.sch.nl = nlambda;
  p.sch.n_row = ny / p.rows_per_item;
  p.sch.n_col = (p.wx + p.cols_per_item - 1) / p.cols_per_item;
  p.sch.lag = nlambda >= 3 ? 2 : nlambda - 1;
  // a row item of frame f reuses the slot of frame f - slots, whose last column
  // items were taken four steps earlier: enough slack that the wait is rare
  p.sch.slots = p.sch.lag + 4;
  // Slots the workspace holds (the autotuner may use them all).  A column item
  // waits for every row item of its frame, so the lag has to span the frames
  // whose items are in flight at once, about 600 on a 152-SM GPU (two groups
  // computing and up to two buffers loaded per SM): 2.4 frames of 1024 x 1024,
  // 9.5 of 512 x 512.  Smaller frames get more slots, as long as the ring
  // stays within 64 MiB of L2.
  {
    const long long items = (long long)p.sch.n_row + p.sch.n_col;
    const long long in_flight = (600 + items - 1) / items;
    const long long slot_bytes = (long long)sizeof(float2) * ny * p.wxp;
    long long n = std::max<long long>(p.sch.slots, in_flight + 4);
    n = std::min<long long>(n, std::max<long long>(p.sch.slots, (64ll << 20) / slot_bytes));
    n = std::min<long long>(n, std::max<long long>(p.sch.slots, nlambda));
    p.slots_alloc = (int)n;
    // default schedule: a lag of about 0.7 of the frames in flight (what the
    // autotuner picked at 512 x 512 and 256 x 256; 3 at 1024 x 1024), four
    // slots of slack
    if (nlambda >= 3) {
      const long long lag = std::min<long long>(std::max<long long>(2, (7 * in_flight + 9) / 10),
                                                std::min<long long>(p.slots_alloc - 4, nlambda - 1));
      if (lag >= 2) {
        p.sch.lag = (int)lag;
        p.sch.slots = (int)lag + 4;
      }
    }
  }
  // input rows a row item stages: from the first row's base to the last row's base + 1
  int st = 0;
  for (int t = 0; t < nlambda; ++t)
    for (int it = 0; it < p.sch.n_row; ++it) {
      const Tap& a = p.ytab[(size_t)t * ny + it * p.rows_per_item];
      const Tap& b = p.ytab[(size_t)t * ny + it * p.rows_per_item + p.rows_per_item - 1];
      const int rows = b.base + 1 - a.base + 1;
      if (rows > st) st = rows;
    }
  p.stage_rows = st;
  if (!generic && lateral_smem_bytes(p) > 227u * 1024u) {
    delete h;
    return SSOCT_EUNSUPPORTED;  // rescale ratio too far from 1 for the staging buffer
  }

  // Workspace layout.
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
  p.off_ctr = take(sizeof(Counters) + 2 * sizeof(unsigned) * (size_t)nlambda);
  p.off_xtab = take(sizeof(Tap) * p.xtab.size());
  p.off_ytab = take(sizeof(Tap) * p.ytab.size());
  p.off_cx = take(sizeof(float2) * nx);
  p.off_cy = take(sizeof(float2) * ny);
  p.off_cx2 = take(sizeof(float2) * nx);
  p.off_cy2 = take(sizeof(float2) * ny);
  p.off_ox = take(sizeof(float2) * p.wx);
  p.off_oy = take(sizeof(float2) * p.wy);
  p.off_twx = take(sizeof(float2) * p.twx.size());
  p.off_twy = take(sizeof(float2) * p.twy.size());
  p.off_twl = take(sizeof(float2) * p.twl.size());
  p.off_twra = take(sizeof(float2) * p.twra.size());
  p.off_tcb = take(sizeof(unsigned short) * p.tcb.size());
  p.off_wq = take(sizeof(float2) * p.wq.size());
  p.off_ring = take(sizeof(uint16_t) * (size_t)nlambda * ny * nx);
  p.off_scratch = take(generic ? 0 : sizeof(float2) * (size_t)p.slots_alloc * ny * p.wxp);
  const size_t inter_bytes = sizeof(float2) * (size_t)p.wy * p.ntx * nlambda * kTile;
  p.off_inter = take(inter_bytes);
  if (generic) p.off_cg = take(sizeof(float2) * (size_t)nx * ny);
  // The axial-first order never uses the sweep-axis intermediate, so its
  // half-spectrum planes share that region when they fit in it.
  const size_t planes_bytes = sizeof(float2) * (size_t)(nlambda / 2 + 1) * ny * nx;
  if (p.af_forced) p.off_aplanes = planes_bytes <= inter_bytes ? p.off_inter : take(planes_bytes);
  else if (!generic && p.ra_w && planes_bytes <= inter_bytes && !(flags & SSOCT_FLAG_PUPIL)) {
    p.off_aplanes = p.off_inter;
    p.af_option = true;
  }
  if (p.ra_w) p.off_xstrip = take(sizeof(StripTap) * p.xstrip.size());
  if (!generic && !p.af_forced) p.off_xys = take(sizeof(float2) * (size_t)p.wy * p.ntx * kTile);
  if (generic || (flags & SSOCT_FLAG_PUPIL)) p.off_F = take(sizeof(float2) * (size_t)nlambda * ny * nx);
  if (flags & SSOCT_FLAG_PUPIL) {
    const size_t chunks = (size_t)(nlambda + p.sh_tpc - 1) / p.sh_tpc;
    p.off_cp = take(sizeof(float2) * (size_t)nx * ny);
    p.off_Q = take(sizeof(float2) * chunks * ny * nx);
    p.off_red = take(sizeof(double) * kShRedDoubles);
  }
  p.ws_bytes = off;
  *out = h;
  return SSOCT_OK;
}

ssoct_status ssoct_plan_info(ssoct_plan h, ssoct_plan_info_t* info) {
  if (!h || !info) return SSOCT_EINVAL;
  const Plan& p = h->p;
  info->nx = p.nx; info->ny = p.ny; info->nlambda = p.nl;
  info->window = ssoct_window{p.x0, p.y0, p.wx, p.wy};
  info->lambda1_m = p.lambda1;
  info->dprime_x_m = p.lambda1 * p.z / (p.nx * p.pitch);
  info->dprime_y_m = p.lambda1 * p.z / (p.ny * p.pitch);
  const int nmax = p.nx > p.ny ? p.nx : p.ny;
  info->z_b_m = nmax * p.pitch * p.pitch / p.lambda1;
  info->aliased_chirp = std::fabs(p.z) < info->z_b_m ? 1 : 0;
  info->prefactor_re = p.kre;
  info->prefactor_im = p.kim;
  info->workspace_bytes = p.ws_bytes;
  info->ring_slots = p.sch.slots;
  return SSOCT_OK;
}

ssoct_status ssoct_workspace_size(ssoct_plan h, size_t* bytes) {
  if (!h || !bytes) return SSOCT_EINVAL;
  *bytes = h->p.ws_bytes;
  return SSOCT_OK;
}

ssoct_status ssoct_workspace_bytes(ssoct_plan h, size_t* bytes) { return ssoct_workspace_size(h, bytes); }

ssoct_status ssoct_set_workspace(ssoct_plan h, void* dev_ptr, size_t bytes) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign)) return fail(&p, SSOCT_EINVAL, "workspace NULL or not 256-byte aligned");
  if (bytes < p.ws_bytes) return fail(&p, SSOCT_ENOMEM, "workspace smaller than ssoct_workspace_size");
  cudaError_t e = cudaGetDevice(&p.device);
  if (e != cudaSuccess) return cuda_fail(&p, e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device);
  if (e != cudaSuccess) return cuda_fail(&p, e, "cudaDeviceGetAttribute");
  char* ws = (char*)dev_ptr;
  struct Up { size_t off; const void* src; size_t n; } ups[] = {
      {p.off_xtab, p.xtab.data(), sizeof(Tap) * p.xtab.size()},
      {p.off_ytab, p.ytab.data(), sizeof(Tap) * p.ytab.size()},
      {p.off_cx, p.cx.data(), sizeof(float2) * p.cx.size()},
      {p.off_cy, p.cy.data(), sizeof(float2) * p.cy.size()},
      {p.off_cx2, p.cx2.data(), sizeof(float2) * p.cx2.size()},
      {p.off_cy2, p.cy2.data(), sizeof(float2) * p.cy2.size()},
      {p.off_ox, p.ox.data(), sizeof(float2) * p.ox.size()},
      {p.off_oy, p.oy.data(), sizeof(float2) * p.oy.size()},
      {p.off_twx, p.twx.data(), sizeof(float2) * p.twx.size()},
      {p.off_twy, p.twy.data(), sizeof(float2) * p.twy.size()},
      {p.off_twl, p.twl.data(), sizeof(float2) * p.twl.size()},
      {p.off_twra, p.twra.data(), sizeof(float2) * p.twra.size()},
      {p.off_tcb, p.tcb.data(), sizeof(unsigned short) * p.tcb.size()},
      {p.off_wq, p.wq.data(), sizeof(float2) * p.wq.size()},
      {p.off_xstrip, p.xstrip.data(), sizeof(StripTap) * p.xstrip.size()},
  };
  for (const Up& u : ups) {
    if (!u.n) continue;
    e = cudaMemcpy(ws + u.off, u.src, u.n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(&p, e, "table upload");
  }
  e = cudaMemset(ws + p.off_ctr, 0, sizeof(Counters) + 2 * sizeof(unsigned) * (size_t)p.nl);
  if (e != cudaSuccess) return cuda_fail(&p, e, "counter reset");
  p.ws = ws;
  p.stream_count = 0;
  p.lat_upto = -1;
  if (p.generic) {
    std::vector<float2> cg;
    build_pupil_table(p.nx, p.ny, p.alpha, nullptr, 0, cg);  // the input chirp alone
    e = cudaMemcpy(ws + p.off_cg, cg.data(), sizeof(float2) * cg.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      p.ws = nullptr;
      return cuda_fail(&p, e, "chirp table upload");
    }
  } else if (!encode_scratch_map(p)) {
    p.ws = nullptr;
    return fail(&p, SSOCT_ECUDA, "cuTensorMapEncodeTiled failed for the scratch ring");
  }
  p.pushed = 0;
  p.ring_head = 0;
  p.next_seq = -1;
  return SSOCT_OK;
}

ssoct_status ssoct_push_frames(ssoct_plan h, const uint16_t* frames, int n, int frames_on_device,
                               int64_t first_seq, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  if (!frames || n < 1) return fail(&p, SSOCT_EINVAL, "frames NULL or n < 1");
  ssoct_status st = SSOCT_OK;
  if (first_seq >= 0) {
    if (p.next_seq >= 0 && first_seq != p.next_seq) {
      // a drop: the current gate can no longer hold consecutive frames
      p.pushed = 0;
      p.ring_head = 0;
      p.stream_count = 0;
      p.lat_upto = -1;
      st = SSOCT_EDROPPED;
    }
    p.next_seq = first_seq + n;
  }
  const size_t fbytes = sizeof(uint16_t) * (size_t)p.nx * p.ny;
  // only the last nl frames of a long push can survive in the ring
  int skip = n > p.nl ? n - p.nl : 0;
  if (skip) {
    p.ring_head = (p.ring_head + skip) % p.nl;
    p.pushed += skip;
  }
  const cudaMemcpyKind kind = frames_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t s = (cudaStream_t)stream;
  int done = skip;
  while (done < n) {
    const int run = std::min(n - done, p.nl - p.ring_head);
    cudaError_t e = cudaMemcpyAsync(p.ws + p.off_ring + fbytes * p.ring_head,
                                    (const char*)frames + fbytes * done, fbytes * run, kind, s);
    if (e != cudaSuccess) return cuda_fail(&p, e, "frame copy");
    done += run;
    p.ring_head = (p.ring_head + run) % p.nl;
    p.pushed += run;
  }
  if (p.pushed > p.nl) p.pushed = p.nl;
  p.stream_count += n;
  if (st != SSOCT_OK) p.last_error = "frame sequence skipped; gate restarted";
  return st;
}

// Lateral-kernel parameters of a plan over its workspace: batch frame f is read
// from ring slot (ring_start + f) % nl and has wavelength / intermediate index
// (tab0 + f) % nl.  The schedule covers all nl frames.
static LateralParams lateral_params(const Plan& p, const uint16_t* frames, int ring_start, int tab0) {
  char* ws = p.ws;
  LateralParams lp;
  lp.frames = frames;
  lp.ring_start = ring_start;
  lp.tab0 = tab0;
  lp.nx = p.nx; lp.ny = p.ny; lp.nl = p.nl;
  lp.x0 = p.x0; lp.y0 = p.y0; lp.wx = p.wx; lp.wy = p.wy;
  lp.wxp = p.wxp; lp.ntx = p.ntx;
  lp.xtab = (const Tap*)(ws + p.off_xtab);
  lp.ytab = (const Tap*)(ws + p.off_ytab);
  lp.cx = (const float2*)(ws + p.off_cx);
  lp.cy = (const float2*)(ws + p.off_cy);
  lp.cx2 = (const float2*)(ws + p.off_cx2);
  lp.cy2 = (const float2*)(ws + p.off_cy2);
  lp.twx = (const float2*)(ws + p.off_twx);
  lp.twy = (const float2*)(ws + p.off_twy);
  lp.scratch = (float2*)(ws + p.off_scratch);
  lp.inter = (float2*)(ws + p.off_inter);
  lp.ctr = (Counters*)(ws + p.off_ctr);
  lp.rows_done = (unsigned*)(ws + p.off_ctr + sizeof(Counters));
  lp.cols_done = lp.rows_done + p.nl;
  lp.sch = p.sch;
  lp.stage_rows = p.stage_rows;
  lp.stage_bytes = 0;
  lp.wait_ns = p.wait_ns;
  return lp;
}

// Reset the work counters and launch the lateral kernel (with the stage events
// of ssoct_profile); *ev receives the event slots of this call, if profiling.
static ssoct_status launch_lateral_pass(Plan& p, const LateralParams& lp, cudaStream_t s, cudaEvent_t** ev) {
  char* ws = p.ws;
  cudaError_t e = cudaMemsetAsync(ws + p.off_ctr, 0, sizeof(Counters) + 2 * sizeof(unsigned) * (size_t)p.nl, s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "counter reset");
  if (p.inject_skip) {
    // start the ticket counter past the first items (ssoct_inject_stall)
    e = cudaMemcpyAsync(ws + p.off_ctr, &p.inject_skip, sizeof(unsigned), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(&p, e, "stall injection");
    e = cudaStreamSynchronize(s);  // the host value must outlive the copy
    if (e != cudaSuccess) return cuda_fail(&p, e, "stall injection");
  }
  *ev = nullptr;
  if (p.profiling) {
    if (p.events_used + 3 > p.events.size()) {
      for (int i = 0; i < 3; ++i) {
        cudaEvent_t x;
        e = cudaEventCreate(&x);
        if (e != cudaSuccess) return cuda_fail(&p, e, "event create");
        p.events.push_back(x);
      }
    }
    *ev = p.events.data() + p.events_used;
    p.events_used += 3;
    cudaEventRecord((*ev)[0], s);
  }
  if (p.axial_first) {
    // Eq. 5 + Eq. 7 first: the interval between events 0 and 1 is this pass
    e = launch_rescale_axial(p, lp.frames, lp.ring_start, (float2*)(ws + p.off_aplanes), s);
    if (e != cudaSuccess) return cuda_fail(&p, e, "rescale-axial kernel launch");
    if (*ev) cudaEventRecord((*ev)[1], s);
  }
  e = p.generic ? launch_lateral_generic(p, lp.frames, lp.ring_start, s) : launch_lateral(p, lp, s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "lateral kernel launch");
  if (p.axial_first) {
    if (*ev) cudaEventRecord((*ev)[2], s);
    return SSOCT_OK;
  }
  if (*ev) cudaEventRecord((*ev)[1], s);
  return SSOCT_OK;
}

static ssoct_status launch_axial_pass(Plan& p, float* vol, void* cplx, cudaStream_t s, cudaEvent_t* ev) {
  char* ws = p.ws;
  AxialParams ap;
  ap.inter = (const float2*)(ws + p.off_inter);
  ap.vol = vol;
  ap.cplx = (float2*)cplx;
  ap.twl = (const float2*)(ws + p.off_twl);
  ap.ox = (const float2*)(ws + p.off_ox);
  ap.oy = (const float2*)(ws + p.off_oy);
  ap.nl = p.nl; ap.wx = p.wx; ap.wy = p.wy; ap.ntx = p.ntx;
  ap.power_scale = (float)(p.alpha * p.alpha);
  ap.magnitude = (p.flags & SSOCT_FLAG_MAGNITUDE) ? 1 : 0;
  ap.err = &((Counters*)(ws + p.off_ctr))->err;
  cudaError_t e = p.use_tc
                      ? launch_axial_tc(p, ap, (const unsigned short*)(ws + p.off_tcb),
                                        &((Counters*)(ws + p.off_ctr))->err, p.num_sms, s)
                      : launch_axial(p, ap, s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "axial kernel launch");
  if (ev) cudaEventRecord(ev[2], s);
  return SSOCT_OK;
}

static ssoct_status run_volume(Plan& p, const uint16_t* frames, int ring_start, float* vol, void* cplx,
                               cudaStream_t s) {
  if (!vol || ((uintptr_t)vol % 16) || ((uintptr_t)cplx % 16))
    return fail(&p, SSOCT_EINVAL, "volume pointer NULL or not 16-byte aligned");
  LateralParams lp = lateral_params(p, frames, ring_start, 0);
  p.lat_upto = -1;  // the intermediate no longer holds the sliding-gate holograms
  if (p.axial_first) {
    // the lateral pass writes the volume itself
    lp.aplanes = (const float2*)(p.ws + p.off_aplanes);
    lp.vol = vol;
    lp.cplx = (float2*)cplx;
    lp.ox = (const float2*)(p.ws + p.off_ox);
    lp.oy = (const float2*)(p.ws + p.off_oy);
    lp.inv_k_abs = (float)(1.0 / p.alpha);
    lp.magnitude = (p.flags & SSOCT_FLAG_MAGNITUDE) ? 1 : 0;
  }
  cudaEvent_t* ev = nullptr;
  ssoct_status st = launch_lateral_pass(p, lp, s, &ev);
  if (st != SSOCT_OK || p.axial_first) return st;
  return launch_axial_pass(p, vol, cplx, s, ev);
}

ssoct_status ssoct_reconstruct_volume(ssoct_plan h, float* vol_dev, void* complex_dev, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  if (p.pushed < p.nl) return fail(&p, SSOCT_ENOTREADY, "fewer than nlambda frames pushed");
  // the ring is full: the oldest frame sits at ring_head
  return run_volume(p, (const uint16_t*)(p.ws + p.off_ring), p.ring_head, vol_dev, complex_dev,
                    (cudaStream_t)stream);
}

ssoct_status ssoct_reconstruct_frames(ssoct_plan h, const uint16_t* frames_dev, float* vol_dev,
                                      void* complex_dev, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  if (!frames_dev || ((uintptr_t)frames_dev % 16)) return fail(&p, SSOCT_EINVAL, "frames NULL or not 16-byte aligned");
  return run_volume(p, frames_dev, 0, vol_dev, complex_dev, (cudaStream_t)stream);
}

// Lateral pass of the sliding gate: frames pushed since the last sliding call
// (at most nl) into their slots of the intermediate; *ev gets the call's events.
static ssoct_status sliding_update(Plan& p, cudaStream_t s, cudaEvent_t** ev_out) {
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  if (p.generic) return fail(&p, SSOCT_EUNSUPPORTED, "sliding gates need a frame size of the persistent lateral kernel");
  if (p.af_forced) return fail(&p, SSOCT_EUNSUPPORTED, "sliding gates need the paper's order (no SSOCT_FLAG_AXIAL_FIRST)");
  if (p.stream_count < p.nl) return fail(&p, SSOCT_ENOTREADY, "fewer than nlambda frames pushed");
  // holograms still missing for the gate of the last nl frames: stream frames
  // [first, stream_count), in ring slots first % nl onwards
  const long long first = std::max(p.lat_upto, p.stream_count - p.nl);
  const int k = (int)(p.stream_count - first);
  cudaEvent_t* ev = nullptr;
  if (k > 0) {
    const int slot0 = (int)(first % p.nl);
    LateralParams lp = lateral_params(p, (const uint16_t*)(p.ws + p.off_ring), slot0, slot0);
    lp.sch.nl = k;
    lp.sch.lag = k >= 3 ? 2 : k - 1;
    lp.sch.slots = lp.sch.lag + 4;  // never more than the plan's ring of scratch slots
    ssoct_status st = launch_lateral_pass(p, lp, s, &ev);
    if (st != SSOCT_OK) return st;
  }
  p.lat_upto = p.stream_count;
  if (k == 0 && p.profiling) {
    // keep the profile's three events per call: an empty lateral interval
    cudaEvent_t* e0 = nullptr;
    if (p.events_used + 3 > p.events.size())
      for (int i = 0; i < 3; ++i) {
        cudaEvent_t x;
        if (cudaEventCreate(&x) != cudaSuccess) return fail(&p, SSOCT_ECUDA, "event create");
        p.events.push_back(x);
      }
    e0 = p.events.data() + p.events_used;
    p.events_used += 3;
    cudaEventRecord(e0[0], s);
    cudaEventRecord(e0[1], s);
    ev = e0;
  }
  *ev_out = ev;
  return SSOCT_OK;
}

ssoct_status ssoct_reconstruct_sliding(ssoct_plan h, float* vol_dev, void* complex_dev, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!vol_dev || ((uintptr_t)vol_dev % 16) || ((uintptr_t)complex_dev % 16))
    return fail(&p, SSOCT_EINVAL, "volume pointer NULL or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  PaperOrderScope paper_order(p);
  cudaEvent_t* ev = nullptr;
  ssoct_status st = sliding_update(p, s, &ev);
  if (st != SSOCT_OK) return st;
  return launch_axial_pass(p, vol_dev, complex_dev, s, ev);
}

ssoct_status ssoct_sliding_cuts(ssoct_plan h, int x0, int y0, int z0, float* xy, float* xz, float* yz, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (x0 < 0 || x0 >= p.wx || y0 < 0 || y0 >= p.wy || z0 < 0 || z0 >= p.nl)
    return fail(&p, SSOCT_EINVAL, "cut position outside the volume");
  cudaStream_t s = (cudaStream_t)stream;
  PaperOrderScope paper_order(p);
  // The xy cut is kept as a running sum X(z0) over the gate's slots while z0
  // stays put: the frames this call swaps in change it by their holograms minus
  // those they replace.  Once nl frames have been swapped in since the last
  // full sum, the next call sums the whole gate again, which bounds the
  // rounding the running sum collects to that of one full sum.
  bool incremental = false;
  int slot0 = 0, k = 0;
  if (xy && p.ws && !p.generic && !p.axial_first && p.stream_count >= p.nl) {
    const long long first = std::max(p.lat_upto, p.stream_count - p.nl);
    k = (int)(p.stream_count - first);
    slot0 = (int)(first % p.nl);
    incremental = p.xs_valid && p.xs_z0 == z0 && p.xs_lat == p.lat_upto && k < p.nl && p.xs_updates + k <= p.nl;
  }
  cudaError_t e = cudaSuccess;
  if (incremental && k > 0) {
    e = launch_xy_slide(p, slot0, k, z0, -1.f, nullptr, s);  // the holograms about to be replaced
    if (e != cudaSuccess) {
      p.xs_valid = false;
      return cuda_fail(&p, e, "running xy cut");
    }
  }
  cudaEvent_t* ev = nullptr;
  ssoct_status st = sliding_update(p, s, &ev);
  if (st != SSOCT_OK) {
    p.xs_valid = false;
    return st;
  }
  if (incremental) e = launch_xy_slide(p, slot0, k, z0, 1.f, xy, s);
  if (e == cudaSuccess)
    e = launch_gate_cuts(p, x0, y0, z0, incremental ? nullptr : xy, xz, yz,
                         incremental || !xy ? nullptr : (float2*)(p.ws + p.off_xys), s);
  if (e != cudaSuccess) {
    p.xs_valid = false;
    return cuda_fail(&p, e, "gate cuts kernels");
  }
  if (xy) {
    p.xs_valid = true;
    p.xs_z0 = z0;
    p.xs_lat = p.lat_upto;
    p.xs_updates = incremental ? p.xs_updates + k : 0;
  }
  if (ev) cudaEventRecord(ev[2], s);
  return SSOCT_OK;
}

ssoct_status ssoct_get_cuts(ssoct_plan h, const float* vol_dev, int x0, int y0, int z0, float* xy,
                            float* xz, float* yz, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!vol_dev) return fail(&p, SSOCT_EINVAL, "volume NULL");
  if (x0 < 0 || x0 >= p.wx || y0 < 0 || y0 >= p.wy || z0 < 0 || z0 >= p.nl)
    return fail(&p, SSOCT_EINVAL, "cut index outside the volume");
  if (!xy && !xz && !yz) return SSOCT_OK;
  CutsParams cp{vol_dev, xy, xz, yz, p.nl, p.wx, p.wy, x0, y0, z0};
  cudaError_t e = launch_cuts(cp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&p, e, "cuts kernel launch");
  return SSOCT_OK;
}

ssoct_status ssoct_sync(ssoct_plan h, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&p, e, "stream synchronize");
  // the last no-allocation call's kernels leave their error word in that
  // path's device array, not in the workspace
  unsigned noalloc_err = 0u;
  e = noalloc_error_word(p, &noalloc_err);
  if (e != cudaSuccess) return cuda_fail(&p, e, "error word read (no-allocation path)");
  if (noalloc_err & kErrTimeout) return fail(&p, SSOCT_ETIMEOUT, "lateral kernel gave up waiting on its work queue (no-allocation call)");
  if (noalloc_err & kErrAxial) return fail(&p, SSOCT_ETIMEOUT, "axial kernel gave up waiting on its stage buffers (no-allocation call)");
  if (noalloc_err) return fail(&p, SSOCT_ETIMEOUT, "tensor-core axial kernel gave up waiting on its MMAs (no-allocation call)");
  if (!p.ws) return SSOCT_OK;
  Counters c;
  e = cudaMemcpy(&c, p.ws + p.off_ctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(&p, e, "error word read");
  if (c.err) {
    cudaMemset(p.ws + p.off_ctr, 0, sizeof(Counters));
    // a kernel gave up part way: the intermediate and the running xy cut no
    // longer describe the gate, so the next sliding call starts over
    p.lat_upto = -1;
    p.xs_valid = false;
    if (c.err & kErrTimeout) return fail(&p, SSOCT_ETIMEOUT, "lateral kernel gave up waiting on its work queue");
    if (c.err & kErrAxial) return fail(&p, SSOCT_ETIMEOUT, "axial kernel gave up waiting on its stage buffers");
    return fail(&p, SSOCT_ETIMEOUT, "tensor-core axial kernel gave up waiting on its MMAs");
  }
  return SSOCT_OK;
}

ssoct_status ssoct_set_pupil(ssoct_plan h, const double* coeffs, int ncoeffs, double z_m) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!(p.flags & SSOCT_FLAG_PUPIL)) return fail(&p, SSOCT_EINVAL, "plan created without SSOCT_FLAG_PUPIL");
  if (ncoeffs < 0 || ncoeffs > 15 || (ncoeffs > 0 && !coeffs)) return fail(&p, SSOCT_EINVAL, "need 0..15 coefficients");
  if (z_m == 0.0 || !std::isfinite(z_m)) return fail(&p, SSOCT_EINVAL, "z must be finite and non-zero");
  for (int j = 0; j < ncoeffs; ++j)
    if (!std::isfinite(coeffs[j])) return fail(&p, SSOCT_EINVAL, "coefficients must be finite");
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  p.sh_z = z_m;
  p.sh_alpha = p.pitch * p.pitch / (p.lambda1 * z_m);
  p.sh_ncoeffs = ncoeffs;
  for (int j = 0; j < 15; ++j) p.sh_coeffs[j] = j < ncoeffs ? coeffs[j] : 0.0;
  p.sh_ready = true;
  p.sh_dirty = true;
  return SSOCT_OK;
}

ssoct_status ssoct_sharpness(ssoct_plan h, const uint16_t* frames_dev, float* vol_dev, double* out_host, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  if (!(p.flags & SSOCT_FLAG_PUPIL)) return fail(&p, SSOCT_EINVAL, "plan created without SSOCT_FLAG_PUPIL");
  if (!p.ws) return fail(&p, SSOCT_ENOMEM, "no workspace");
  if (!p.sh_ready) return fail(&p, SSOCT_ENOTREADY, "ssoct_set_pupil has not been called");
  if (!frames_dev || !vol_dev || !out_host || ((uintptr_t)vol_dev % 16))
    return fail(&p, SSOCT_EINVAL, "frames, volume (16-byte aligned) and output must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  p.lat_upto = -1;  // the intermediate no longer holds sliding-gate holograms
  cudaError_t e = cudaSuccess;
  if (p.sh_dirty) {
    e = launch_pupil_table(p, s);
    if (e != cudaSuccess) return cuda_fail(&p, e, "pupil table kernel");
    p.sh_dirty = false;
  }
  e = launch_sharpness(p, frames_dev, vol_dev, s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "sharpness kernels");
  e = cudaMemcpyAsync(out_host, p.ws + p.off_red + 2 * sizeof(double), 17 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "loss and gradient read-back");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(&p, e, "stream synchronize");
  return SSOCT_OK;
}

ssoct_status ssoct_inject_stall(ssoct_plan h, unsigned skip, unsigned long long wait_limit_ns) {
  if (!h) return SSOCT_EINVAL;
  h->p.inject_skip = skip;
  h->p.wait_ns = wait_limit_ns;
  return SSOCT_OK;
}

ssoct_status ssoct_profile(ssoct_plan h, int enable) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  p.profiling = enable != 0;
  if (enable) p.events_used = 0;
  return SSOCT_OK;
}

ssoct_status ssoct_profile_read(ssoct_plan h, double* lateral_ms, double* axial_ms, int* calls) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = h->p;
  double lat = 0.0, ax = 0.0;
  for (size_t i = 0; i + 2 < p.events_used; i += 3) {
    float a = 0.f, b = 0.f;
    cudaError_t e = cudaEventSynchronize(p.events[i + 2]);
    if (e != cudaSuccess) return cuda_fail(&p, e, "event synchronize");
    e = cudaEventElapsedTime(&a, p.events[i], p.events[i + 1]);
    if (e != cudaSuccess) return cuda_fail(&p, e, "event elapsed");
    e = cudaEventElapsedTime(&b, p.events[i + 1], p.events[i + 2]);
    if (e != cudaSuccess) return cuda_fail(&p, e, "event elapsed");
    // axial-first plans record the rescale-axial pass first
    lat += p.axial_first ? b : a;
    ax += p.axial_first ? a : b;
  }
  if (lateral_ms) *lateral_ms = lat;
  if (axial_ms) *axial_ms = ax;
  if (calls) *calls = (int)(p.events_used / 3);
  return SSOCT_OK;
}

const char* ssoct_last_error(ssoct_plan h) { return h ? h->p.last_error.c_str() : ""; }

void ssoct_destroy_plan(ssoct_plan h) {
  if (!h) return;
  for (cudaEvent_t e : h->p.events) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
