// Reconstruction without any device allocation, for callers that cannot
// allocate device memory themselves.
//
// Who needs this: acquisition software that reserves all its memory up front and
// must not allocate while frames stream in (a device allocation can synchronise
// the device and stall the frame loop, which is exactly the frame drop the
// acquisition buffering exists to prevent), and plug-ins running inside a host
// application whose own memory manager owns the device heap and forbids
// cudaMalloc from third-party code.  Such a caller can still create a plan (host
// memory only) and pass its own frames and output volume; everything else this
// path needs lives in one file-scope device array.
//
// The array holds the plan's tables, the L2 scratch ring and work counters of
// the lateral kernel, and the sweep-axis intermediate, laid out exactly like a
// plan workspace.  It has a fixed size (kNoAllocBytes), and every GPU that loads
// the library keeps it until the process exits.  All calls share it and it keeps
// the last call's contents: each call rewrites the tables and zeroes the
// counters before its kernels run, and calls that overlap on the GPU (different
// streams, or different host threads) race on it.
//
// A kernel that gives up a bounded wait leaves its error word in the array;
// ssoct_sync on the same plan reads it (noalloc_error_word) and reports
// SSOCT_ETIMEOUT, as it does for the workspace path.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "ssoct_internal.h"

namespace ssoct {
namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch and SM count, per device, set once by the
// first call on that device.  Host threads may make their first calls at the
// same time: the set-up runs under a mutex and publishes the address last
// (release), so a thread that sees the address also sees the SM count.
std::atomic<char*> g_scratch_addr[kMaxDevices] = {};
std::atomic<int> g_num_sms[kMaxDevices] = {};
std::mutex g_setup_mutex;

// The array's device address on device dev (the current one), looked up once.
cudaError_t scratch_on_device(int dev, char** addr, int* sms) {
  char* a = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    a = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!a) {
      // In host code the name g_noalloc_scratch is only a host-side stand-in,
      // so the kernels get this address instead.
      cudaError_t e = cudaGetSymbolAddress((void**)&a, g_noalloc_scratch);
      if (e != cudaSuccess) return e;
      int n = 0;
      e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      g_num_sms[dev].store(n, std::memory_order_relaxed);
      g_scratch_addr[dev].store(a, std::memory_order_release);
    }
  }
  *addr = a;
  *sms = g_num_sms[dev].load(std::memory_order_relaxed);
  return cudaSuccess;
}

ssoct_status fail(Plan& p, ssoct_status s, const std::string& msg) {
  p.last_error = msg;
  return s;
}

}  // namespace
}  // namespace ssoct

using namespace ssoct;

extern "C" ssoct_status ssoct_reconstruct_frames_noalloc(ssoct_plan h, const uint16_t* frames_dev, float* vol_dev,
                                                         void* complex_dev, void* stream) {
  if (!h) return SSOCT_EINVAL;
  Plan& p = plan_of(h);
  if (p.af_forced) return fail(p, SSOCT_EUNSUPPORTED, "the no-allocation entry point runs the paper's order");
  PaperOrderScope paper_order(p);  // an autotuned axial-first choice does not apply here
  if (p.generic) return fail(p, SSOCT_EUNSUPPORTED, "the no-allocation entry point needs a frame size of the persistent lateral kernel");
  if (p.ws_bytes > kNoAllocBytes) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "this plan needs %zu bytes of device scratch; the no-allocation entry point holds at most %zu (64 MiB)",
             p.ws_bytes, kNoAllocBytes);
    return fail(p, SSOCT_EUNSUPPORTED, msg);
  }
  if (!frames_dev || ((uintptr_t)frames_dev % 16)) return fail(p, SSOCT_EINVAL, "frames NULL or not 16-byte aligned");
  if (!vol_dev || ((uintptr_t)vol_dev % 16) || ((uintptr_t)complex_dev % 16))
    return fail(p, SSOCT_EINVAL, "volume pointer NULL or not 16-byte aligned");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(p, SSOCT_EUNSUPPORTED, "device index beyond the no-allocation table");
  // One-time set-up on this device (the current one): the array's device address.
  char* ws = nullptr;
  int num_sms = 0;
  e = scratch_on_device(dev, &ws, &num_sms);
  if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("no-allocation set-up: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;

  // Tables of this plan (the previous call may have left another plan's), then
  // zeroed work counters.
  struct Up {
    size_t off;
    const void* src;
    size_t n;
  } ups[] = {
      {p.off_xtab, p.xtab.data(), sizeof(Tap) * p.xtab.size()},
      {p.off_ytab, p.ytab.data(), sizeof(Tap) * p.ytab.size()},
      {p.off_cx, p.cx.data(), sizeof(float2) * p.cx.size()},
      {p.off_cy, p.cy.data(), sizeof(float2) * p.cy.size()},
      {p.off_ox, p.ox.data(), sizeof(float2) * p.ox.size()},
      {p.off_oy, p.oy.data(), sizeof(float2) * p.oy.size()},
      {p.off_twx, p.twx.data(), sizeof(float2) * p.twx.size()},
      {p.off_twy, p.twy.data(), sizeof(float2) * p.twy.size()},
      {p.off_twl, p.twl.data(), sizeof(float2) * p.twl.size()},
      {p.off_tcb, p.tcb.data(), sizeof(unsigned short) * p.tcb.size()},
  };
  for (const Up& u : ups) {
    if (!u.n) continue;
    e = cudaMemcpyAsync(ws + u.off, u.src, u.n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(ws + p.off_ctr, 0, sizeof(Counters) + 2 * sizeof(unsigned) * (size_t)p.nl, s);
  if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("counter reset: ") + cudaGetErrorString(e));
  if (p.inject_skip) {
    // start the ticket counter past the first items (ssoct_inject_stall); the
    // copy reads the plan's own field, and the sync keeps it a test-only cost
    e = cudaMemcpyAsync(ws + p.off_ctr, &p.inject_skip, sizeof(unsigned), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("stall injection: ") + cudaGetErrorString(e));
  }
  p.noalloc_device = dev;

  alignas(64) unsigned char tmap[128];
  if (!encode_scratch_map_at(p, ws + p.off_scratch, tmap))
    return fail(p, SSOCT_ECUDA, "cuTensorMapEncodeTiled failed for the no-allocation scratch ring");

  LateralParams lp;
  lp.frames = frames_dev;
  lp.ring_start = 0;
  lp.tab0 = 0;
  lp.nx = p.nx; lp.ny = p.ny; lp.nl = p.nl;
  lp.x0 = p.x0; lp.y0 = p.y0; lp.wx = p.wx; lp.wy = p.wy;
  lp.wxp = p.wxp; lp.ntx = p.ntx;
  lp.xtab = (const Tap*)(ws + p.off_xtab);
  lp.ytab = (const Tap*)(ws + p.off_ytab);
  lp.cx = (const float2*)(ws + p.off_cx);
  lp.cy = (const float2*)(ws + p.off_cy);
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
  e = launch_lateral_with(p, lp, tmap, num_sms, s);
  if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("lateral kernel launch: ") + cudaGetErrorString(e));

  AxialParams ap;
  ap.inter = lp.inter;
  ap.vol = vol_dev;
  ap.cplx = (float2*)complex_dev;
  ap.twl = (const float2*)(ws + p.off_twl);
  ap.ox = (const float2*)(ws + p.off_ox);
  ap.oy = (const float2*)(ws + p.off_oy);
  ap.nl = p.nl; ap.wx = p.wx; ap.wy = p.wy; ap.ntx = p.ntx;
  ap.power_scale = (float)(p.alpha * p.alpha);
  ap.magnitude = (p.flags & SSOCT_FLAG_MAGNITUDE) ? 1 : 0;
  ap.err = &lp.ctr->err;
  e = p.use_tc ? launch_axial_tc(p, ap, (const unsigned short*)(ws + p.off_tcb), &lp.ctr->err, num_sms, s)
                                      : launch_axial_with(p, ap, num_sms, s);
  if (e != cudaSuccess) return fail(p, SSOCT_ECUDA, std::string("axial kernel launch: ") + cudaGetErrorString(e));
  return SSOCT_OK;
}

namespace ssoct {

cudaError_t noalloc_error_word(Plan& p, unsigned* err) {
  *err = 0u;
  const int dev = p.noalloc_device;
  if (dev < 0) return cudaSuccess;
  char* ws = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!ws) return cudaSuccess;
  Counters c;
  cudaError_t e = cudaMemcpy(&c, ws + p.off_ctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  *err = c.err;
  p.noalloc_device = -1;
  return cudaSuccess;
}

}  // namespace ssoct
