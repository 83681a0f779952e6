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

// ---------------------------------------------------------------------------
// Arithmetic peak: NCH independent FMA chains per thread, x <- x a + b with a
// just below 1 and b small, so the values stay bounded and no chain can be
// folded away (every chain's value is stored).
// ---------------------------------------------------------------------------
constexpr int NCH = 8;

__global__ void __launch_bounds__(256) k_peak_f32(float* out, int iters, float a, float b) {
  float x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f64(double* out, int iters, double a, double b) {
  double x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32x2(float* out, int iters, float a, float b) {
  unsigned long long x[NCH];
  const float2 a2{a, a}, b2{b, b};
  const unsigned long long ra = *reinterpret_cast<const unsigned long long*>(&a2);
  const unsigned long long rb = *reinterpret_cast<const unsigned long long*>(&b2);
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const float2 v{(float)(threadIdx.x + c), (float)(threadIdx.x + 2 * c)};
    x[c] = *reinterpret_cast<const unsigned long long*>(&v);
  }
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(ra), "l"(rb));
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const float2 v = *reinterpret_cast<const float2*>(&x[c]);
    s += v.x + v.y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace prof
}  // namespace frac

using namespace frac;
using namespace frac::prof;

extern "C" int frac_profile_alu_peak(int kind, double* tflops, void* stream) {
  if (!tflops || kind < 0 || kind > 2) return FRAC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  FRAC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = 8 * sms;
  // about 10 ms per launch at the expected rates (FP64 runs far slower on this part)
  const int iters = kind == 1 ? 4096 : (kind == 0 ? 131072 : 65536);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FRAC_ENOMEM;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  int s = FRAC_OK;
  float best = 0.0f;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) s = FRAC_ECUDA;
  for (int rep = 0; rep < 4 && s == FRAC_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(a, st);
    if (kind == 0)
      k_peak_f32<<<blocks, threads, 0, st>>>((float*)buf, iters, 0.9999999f, 1e-7f);
    else if (kind == 1)
      k_peak_f64<<<blocks, threads, 0, st>>>((double*)buf, iters, 0.9999999, 1e-7);
    else
      k_peak_f32x2<<<blocks, threads, 0, st>>>((float*)buf, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(b, st);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      s = FRAC_ECUDA;
      break;
    }
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  if (s != FRAC_OK) return s;
  const double fmas = (double)blocks * threads * iters * NCH * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return FRAC_OK;
}

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
