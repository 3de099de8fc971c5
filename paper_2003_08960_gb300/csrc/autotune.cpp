// Autotuner: picks, per plan and GPU, the order of the steps (the paper's, or
// the axial-first order where the plan offers it), the schedule of the
// persistent lateral kernel (lag between a frame's row and column items,
// number of L2 scratch-ring slots) and the form of the axial pass (FP32 or
// tensor cores, 256-frame sweeps, paper order), by timing whole
// reconstructions on the caller's frames.  Choices are
// cached in a small JSON file, one entry per line, keyed by GPU name, SM count,
// frame size, sweep length and window.
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ssoct_internal.h"

using namespace ssoct;

namespace {

struct Choice {
  int lag, slots, tc, af;
};

std::string tune_key(const Plan& p) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, p.device) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == '"' || c == '\\') c = '_';
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%d|%dx%dx%d|%d,%d,%d,%d%s", name.c_str(), p.num_sms, p.nx, p.ny, p.nl, p.x0, p.y0,
           p.wx, p.wy, p.af_forced ? "|axial-first" : "");
  return buf;
}

// Lines of the cache file other than the header and footer.
std::vector<std::string> read_entries(const char* path) {
  std::vector<std::string> out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line))
    if (line.find("\"key\"") != std::string::npos) {
      while (!line.empty() && (line.back() == ',' || line.back() == ' ')) line.pop_back();
      out.push_back(line);
    }
  return out;
}

bool find_entry(const std::vector<std::string>& entries, const std::string& key, Choice& c, double& ms) {
  const std::string tag = "\"key\": \"" + key + "\"";
  for (const std::string& e : entries) {
    const size_t at = e.find(tag);
    if (at == std::string::npos) continue;
    if (sscanf(e.c_str() + at + tag.size(), ", \"lag\": %d, \"slots\": %d, \"tc_axial\": %d, \"axial_first\": %d, \"ms\": %lf",
               &c.lag, &c.slots, &c.tc, &c.af, &ms) == 5)
      return true;
  }
  return false;
}

bool write_entries(const char* path, std::vector<std::string> entries, const std::string& key, const Choice& c,
                   double ms) {
  const std::string tag = "\"key\": \"" + key + "\"";
  char buf[512];
  snprintf(buf, sizeof buf, "{%s, \"lag\": %d, \"slots\": %d, \"tc_axial\": %d, \"axial_first\": %d, \"ms\": %.6f}",
           tag.c_str(), c.lag, c.slots, c.tc, c.af, ms);
  bool replaced = false;
  for (std::string& e : entries)
    if (e.find(tag) != std::string::npos) {
      e = buf;
      replaced = true;
    }
  if (!replaced) entries.push_back(buf);
  std::ofstream f(path, std::ios::trunc);
  if (!f) return false;
  f << "{\"version\": 1, \"entries\": [\n";
  for (size_t i = 0; i < entries.size(); ++i) f << entries[i] << (i + 1 < entries.size() ? ",\n" : "\n");
  f << "]}\n";
  return (bool)f;
}

bool valid(const Plan& p, const Choice& c) {
  if (c.lag < 1 || c.lag > p.nl - 1) return false;
  if (c.slots < c.lag + 2 || c.slots > p.slots_alloc) return false;
  if (c.tc && !axial_tc_supported(p.nl)) return false;
  if (c.af ? !(p.af_forced || p.af_option) : p.af_forced) return false;
  if (c.af && c.tc) return false;  // the tensor-core form is the paper order's axial pass
  return true;
}

void apply(Plan& p, const Choice& c) {
  p.sch.lag = c.lag;
  p.sch.slots = c.slots;
  p.use_tc = c.tc != 0;
  p.axial_first = c.af != 0;
  p.lat_upto = -1;  // slot numbering of the sliding-gate state changes with the ring
}

}  // namespace

extern "C" ssoct_status ssoct_autotune(ssoct_plan h, const uint16_t* frames_dev, float* vol_dev, const char* cache_path,
                                       void* stream, ssoct_tune_t* result) {
  if (!h || !result) return SSOCT_EINVAL;
  Plan& p = plan_of(h);
  if (!p.ws) return SSOCT_ENOMEM;
  if (!frames_dev || !vol_dev || ((uintptr_t)frames_dev % 16) || ((uintptr_t)vol_dev % 16)) return SSOCT_EINVAL;
  if (p.profiling || p.inject_skip) return SSOCT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = tune_key(p);
  const Choice initial{p.sch.lag, p.sch.slots, p.use_tc ? 1 : 0, p.axial_first ? 1 : 0};
  *result = ssoct_tune_t{initial.lag, initial.slots, initial.tc, 0.0, 0, 0, initial.af};

  std::vector<std::string> entries;
  if (cache_path) {
    entries = read_entries(cache_path);
    Choice c;
    double ms = 0.0;
    if (find_entry(entries, key, c, ms) && valid(p, c)) {
      apply(p, c);
      *result = ssoct_tune_t{c.lag, c.slots, c.tc, ms, 1, 0, c.af};
      return SSOCT_OK;
    }
  }

  // Candidates: the orders the plan offers, times the persistent kernel's
  // schedule (generic-path plans have none), times the axial forms this sweep
  // length has (paper order).  Schedules: lags from 1 up to what the ring
  // allows, each with the fewest slots it needs (lag + 2), two more, and the
  // whole ring.
  std::vector<Choice> cand;
  const int lags[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  for (int af = 0; af <= 1; ++af)
    for (int tc = 0; tc <= 1; ++tc) {
      if (p.generic) {
        const Choice c{initial.lag, initial.slots, tc, af};
        if (valid(p, c)) cand.push_back(c);
        continue;
      }
      for (int lag : lags) {
        const int slot_choices[3] = {lag + 2, lag + 4, p.slots_alloc};
        for (int i = 0; i < 3; ++i) {
          const int slots = slot_choices[i];
          if (i == 1 && slots >= p.slots_alloc) continue;  // the whole ring follows
          if (i == 2 && slots == lag + 2) continue;
          const Choice c{lag, slots, tc, af};
          if (valid(p, c)) cand.push_back(c);
        }
      }
    }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SSOCT_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SSOCT_ECUDA;
  }
  constexpr int kRuns = 3;
  Choice best = initial;
  double best_ms = 1e30;
  ssoct_status st = SSOCT_OK;
  for (const Choice& c : cand) {
    apply(p, c);
    st = ssoct_reconstruct_frames(h, frames_dev, vol_dev, nullptr, s);  // warm-up
    if (st == SSOCT_OK && cudaEventRecord(e0, s) != cudaSuccess) st = SSOCT_ECUDA;
    for (int r = 0; r < kRuns && st == SSOCT_OK; ++r) st = ssoct_reconstruct_frames(h, frames_dev, vol_dev, nullptr, s);
    if (st == SSOCT_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SSOCT_ECUDA;
    if (st == SSOCT_OK) st = ssoct_sync(h, s);
    if (st != SSOCT_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / kRuns < best_ms) {
      best_ms = ms / kRuns;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SSOCT_OK) {
    apply(p, initial);
    return st;
  }
  apply(p, best);
  *result = ssoct_tune_t{best.lag, best.slots, best.tc, best_ms, 0, (int)cand.size(), best.af};
  if (cache_path && !write_entries(cache_path, entries, key, best, best_ms)) {
    p.last_error = std::string("could not write the tuning cache ") + cache_path;
    return SSOCT_EINVAL;
  }
  return SSOCT_OK;
}
