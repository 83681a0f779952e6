// Per-launch CUDA-event timing: events come from a pool, records are folded
// into per-name totals when read.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "prof.cuh"

namespace frac {
namespace prof {

namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
};
struct Totals {
  int64_t launches = 0;
  double ms = 0.0;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_pending;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pool;
std::map<std::string, Totals> g_tot;
}  // namespace

bool enabled() { return g_on.load(std::memory_order_relaxed); }

Scope::Scope(const char* name, cudaStream_t st) : st_(st) {
  if (!enabled()) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // no timing events inside a graph capture
  }
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t a, b;
  if (!g_pool.empty()) {
    a = g_pool.back().first;
    b = g_pool.back().second;
    g_pool.pop_back();
  } else {
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  }
  cudaEventRecord(a, st);
  g_pending.push_back(Rec{name, a, b});
  slot_ = (int)g_pending.size() - 1;
}

Scope::~Scope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot_ < (int)g_pending.size()) cudaEventRecord(g_pending[slot_].b, st_);
}

}  // namespace prof
}  // namespace frac

using namespace frac::prof;

extern "C" int frac_profile_enable(int on) {
  g_on.store(on != 0);
  return FRAC_OK;
}

extern "C" int frac_profile_read(frac_kernel_stat* out, int cap, int* count, int reset) {
  if (!count || cap < 0 || (cap > 0 && !out)) return FRAC_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  int status = FRAC_OK;
  for (Rec& r : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      status = FRAC_ECUDA;
    }
    Totals& t = g_tot[r.name];
    t.launches += 1;
    t.ms += ms;
    g_pool.emplace_back(r.a, r.b);
  }
  g_pending.clear();
  int i = 0;
  for (auto& kv : g_tot) {
    if (i < cap) {
      std::memset(out[i].name, 0, sizeof(out[i].name));
      std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.launches;
      out[i].total_ms = kv.second.ms;
    }
    ++i;
  }
  *count = i;
  if (reset) g_tot.clear();
  return status;
}
