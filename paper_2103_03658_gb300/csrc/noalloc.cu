// frac_apply_static: the FFT Toeplitz apply without any device allocation.
//
// frac_apply obtains its spectral scratch with cudaMallocAsync on every call.
// Some callers cannot allocate device memory at the point where they apply
// the operator: code that runs under a fixed, pre-reserved memory budget,
// code whose surrounding framework forbids device allocations after start-up,
// or latency-critical loops that cannot risk an allocation stalling or
// failing in the middle of a step.  This entry point serves them: its
// scratch is one file-scope device array of fixed size, reserved when the
// library's device code is loaded on a GPU and held by that GPU until the
// process exits.  Inputs, outputs and the op are still the caller's.
#include <cstdio>
#include <mutex>
#include <vector>

#include "apply.cuh"

namespace frac {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;  // device address of g_static_scratch, per device ordinal

// Looked up once per device, with that device current (the first call on a
// device does this, so that call should come before any stream capture).
int static_scratch(void** out) {
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    FRAC_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FRAC_OK;
}

// device (or managed) memory that the current device's kernels may use
bool on_device(const void* p) { return ptr_kind(p) == PTR_DEVICE; }

}  // namespace
}  // namespace frac

using namespace frac;

extern "C" int frac_apply_static(const frac_op* op, const void* u, void* y, int dtype, int64_t batch,
                                 void* stream) {
  if (!op || batch < 0 || (dtype != FRAC_F32 && dtype != FRAC_F64)) return FRAC_EINVAL;
  if (batch == 0) return FRAC_OK;
  if (!u || !y || u == y) return FRAC_EINVAL;
  const size_t es = dtype == FRAC_F64 ? sizeof(double) : sizeof(float);
  // host buffers would need staging allocations: device memory of the current device only,
  // and the operator's tables must live there too
  if (!op_on_current_device(op)) {
    record_detail("frac_apply_static: the operator was built on device %d, which is not the current device",
                  op->device);
    return FRAC_EINVAL;
  }
  if (!on_device(u) || !on_device(y)) {
    record_detail("frac_apply_static: u and y must be device buffers of the current device");
    return FRAC_EINVAL;
  }
  if (((uintptr_t)u % es) || ((uintptr_t)y % es)) return FRAC_EINVAL;
  const size_t need = apply_workspace_bytes(op, dtype, batch);
  if (need > kStaticScratchBytes) {
    record_detail("frac_apply_static: this call needs %zu bytes of scratch, more than the static %zu bytes; "
                  "split the batch or use frac_apply",
                  need, kStaticScratchBytes);
    return FRAC_EINVAL;
  }
  void* ws = nullptr;
  if (need) FRAC_TRY(static_scratch(&ws));
  cudaStream_t st = (cudaStream_t)stream;
  // every spectral entry the apply reads is written earlier in the same call,
  // so the previous call's leftovers in the array need no clearing
  return dtype == FRAC_F64 ? apply_t<double>(op, (const double*)u, (double*)y, batch, ws, st)
                           : apply_t<float>(op, (const float*)u, (float*)y, batch, ws, st);
}
