// Batched reconstruction of several volumes of different sizes (one plan each)
// as one CUDA graph.  The first run on a set of frame / volume pointers captures
// every plan's kernels (lateral pass, axial pass), volume i on lane (stream)
// i mod lanes; later runs on the same pointers relaunch the instantiated graph
// with one call.  One lane runs the volumes back to back; more lanes let a
// volume's kernels overlap another's, which pays off only where kernels leave
// SMs idle (the persistent lateral kernel takes every SM).
#include <string>
#include <vector>

#include "ssoct_internal.h"

struct ssoct_batch_s {
  std::vector<ssoct_plan> plans;
  cudaStream_t origin = nullptr;        // capture stream (the caller's may be the legacy stream)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const uint16_t*> frames;  // pointers the graph was captured with
  std::vector<float*> vols;
  int captures = 0;
  std::string last_error;
};

namespace {

ssoct_status batch_fail(ssoct_batch b, ssoct_status s, const std::string& msg) {
  b->last_error = msg;
  return s;
}

void drop_graph(ssoct_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

}  // namespace

using namespace ssoct;

extern "C" ssoct_status ssoct_batch_create(const ssoct_plan* plans, int n, int lanes, ssoct_batch* out) {
  if (!out) return SSOCT_EINVAL;
  *out = nullptr;
  if (!plans || n < 1 || lanes < 0) return SSOCT_EINVAL;
  if (lanes == 0 || lanes > n) lanes = n;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return SSOCT_EINVAL;
    const Plan& p = plan_of(plans[i]);
    if (!p.ws) return SSOCT_ENOMEM;
    if (p.inject_skip || p.profiling) return SSOCT_EINVAL;  // host-side steps that cannot be captured
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return SSOCT_EINVAL;  // one workspace cannot serve two volumes at once
  }
  ssoct_batch b = new (std::nothrow) ssoct_batch_s();
  if (!b) return SSOCT_ENOMEM;
  b->plans.assign(plans, plans + n);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int i = 0; i < lanes && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->done.push_back(ev);
  }
  if (e != cudaSuccess) {
    ssoct_batch_destroy(b);
    return SSOCT_ECUDA;
  }
  *out = b;
  return SSOCT_OK;
}

extern "C" ssoct_status ssoct_batch_run(ssoct_batch b, const uint16_t* const* frames_dev, float* const* vol_dev,
                                        void* stream) {
  if (!b || !frames_dev || !vol_dev) return SSOCT_EINVAL;
  const int n = (int)b->plans.size();
  for (int i = 0; i < n; ++i) {
    if (!frames_dev[i] || ((uintptr_t)frames_dev[i] % 16) || !vol_dev[i] || ((uintptr_t)vol_dev[i] % 16))
      return batch_fail(b, SSOCT_EINVAL, "frames and volumes must be non-NULL and 16-byte aligned");
    const Plan& p = plan_of(b->plans[i]);
    if (p.inject_skip || p.profiling) return batch_fail(b, SSOCT_EINVAL, "a plan has profiling or a stall injection on");
  }
  cudaStream_t s = (cudaStream_t)stream;
  bool same = b->exec != nullptr;
  for (int i = 0; same && i < n; ++i) same = b->frames[i] == frames_dev[i] && b->vols[i] == vol_dev[i];
  if (!same) {
    drop_graph(b);
    cudaStream_t o = b->origin;
    cudaError_t e = cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, SSOCT_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    ssoct_status st = SSOCT_OK;
    e = cudaEventRecord(b->fork, o);
    const int lanes = (int)b->streams.size();
    for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->streams[l], b->fork, 0);
    // volume i runs on lane i mod lanes, after the lane's previous volume
    for (int i = 0; i < n && e == cudaSuccess && st == SSOCT_OK; ++i)
      st = ssoct_reconstruct_frames(b->plans[i], frames_dev[i], vol_dev[i], nullptr, b->streams[i % lanes]);
    for (int l = 0; l < lanes && e == cudaSuccess && st == SSOCT_OK; ++l) {
      e = cudaEventRecord(b->done[l], b->streams[l]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(o, b->done[l], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(o, &g);
    if (st != SSOCT_OK || e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (st != SSOCT_OK) return batch_fail(b, st, "a plan's reconstruct failed while capturing");
      return batch_fail(b, SSOCT_ECUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      drop_graph(b);
      return batch_fail(b, SSOCT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->frames.assign(frames_dev, frames_dev + n);
    b->vols.assign(vol_dev, vol_dev + n);
    ++b->captures;
  }
  const cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return batch_fail(b, SSOCT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return SSOCT_OK;
}

extern "C" ssoct_status ssoct_batch_sync(ssoct_batch b, void* stream) {
  if (!b) return SSOCT_EINVAL;
  ssoct_status worst = SSOCT_OK;
  for (ssoct_plan h : b->plans) {
    const ssoct_status st = ssoct_sync(h, stream);
    if (st != SSOCT_OK && worst == SSOCT_OK) {
      worst = st;
      b->last_error = ssoct_last_error(h);
    }
  }
  return worst;
}

extern "C" int ssoct_batch_captures(ssoct_batch b) { return b ? b->captures : -1; }

extern "C" const char* ssoct_batch_last_error(ssoct_batch b) { return b ? b->last_error.c_str() : "null batch"; }

extern "C" void ssoct_batch_destroy(ssoct_batch b) {
  if (!b) return;
  drop_graph(b);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}
