// Shared definitions for the sm_103a fractional-Laplacian library.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/frac.h"

namespace frac {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }

// Records the text of a failed CUDA call for frac_error_detail() and consumes the
// thread's last CUDA error (see settle()); returns the status.
int record_cuda_error(cudaError_t e, const char* file, int line, const char* expr);
// Records a failed device-side bounds check (file:line, index); returns FRAC_ECUDA.
int record_check_failure(const char* file, int line, long long index);
// Sets the text returned by frac_error_detail() (printf format).
void record_detail(const char* fmt, ...);

// Status propagation for host code.
#define FRAC_CUDA_TRY(expr)                                                   \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return record_cuda_error(e_, __FILE__, __LINE__, #expr); \
  } while (0)

// A failed runtime call (an allocation above all) leaves its error behind as the
// thread's last CUDA error, where the cudaGetLastError() that follows the next
// launch of this library would report it again, in a later call that did not
// fail. An entry point that fails with a CUDA status consumes it before it
// returns. (A sticky error, one that ends the context, stays reported.)
inline int settle(int s) {
  if (s == FRAC_ENOMEM || s == FRAC_ECUDA) (void)cudaGetLastError();
  return s;
}

#define FRAC_TRY(expr)            \
  do {                            \
    int s_ = (expr);              \
    if (s_ != FRAC_OK) return s_; \
  } while (0)

// Where a caller's pointer lives: host memory (pageable, pinned or unknown to
// CUDA), device memory of the current device (or managed memory), or device
// memory of another device, which the library's kernels on the current device
// must not be given.
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
inline PtrKind ptr_kind(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (at.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (at.type != cudaMemoryTypeDevice) return PTR_HOST;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PTR_OTHER_DEVICE;
  }
  return at.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
}

inline int ilog2(int64_t m) {
  int l = 0;
  while ((int64_t(1) << l) < m) ++l;
  return l;
}

// Twiddle tables exp(-2 pi i t / M), t in [0, M), FP64 and FP32, per M (device-resident,
// built once per M and device, never freed): by log2 M for powers of two, by M for
// the mixed lengths below (prepare_twiddles_len builds them).
const double2* twiddles64(int logm);
const float2* twiddles32(int logm);
const double2* twiddles64_len(int64_t M);
const float2* twiddles32_len(int64_t M);
int prepare_twiddles_len(int64_t M);

// Pass plan of a mixed-radix FFT length M = 2^a 3^b 5^c 7^d, a >= 4 (fft_mixed.cuh):
// the power-of-two factor in ceil(a / 4) passes of radix up to 16 (bits split as
// evenly as in fft.cuh, larger first) and one pass per odd factor, executed as: the
// first power-of-two pass (`first`, from registers), the odd passes (3s, 5s, 7s),
// the other power-of-two passes but the smallest, and that smallest one (`last`, to
// registers; 0 when a <= 4 leaves a single power-of-two pass).  count[] holds the
// middle passes per radix in the order 3, 5, 7, 16, 8, 4, 2; radix[] lists all np
// passes in execution order.  m = 0: the axis has a power-of-two length (fft.cuh).
constexpr int kMxMaxPasses = 12;
struct MxPlan {
  int m = 0;
  int np = 0;
  int8_t radix[kMxMaxPasses] = {};
  int8_t count[7] = {};
  int8_t first = 0, last = 0;
};

// The plan of M; false unless M = 2^a 3^b 5^c 7^d with a >= 4.
inline bool mx_plan(int64_t M, MxPlan* p) {
  if (M < 16 || M > (int64_t(1) << 24)) return false;
  int64_t m = M;
  int a = 0;
  while (m % 2 == 0) {
    m /= 2;
    ++a;
  }
  int odd[kMxMaxPasses], no = 0;
  for (int q : {3, 5, 7})
    while (m % q == 0 && no < kMxMaxPasses) {
      m /= q;
      odd[no++] = q;
    }
  const int np2 = (a + 3) / 4;
  if (m != 1 || a < 4 || np2 + no > kMxMaxPasses) return false;
  int p2[4];
  for (int i = 0; i < np2; ++i) p2[i] = 1 << (a / np2 + (i < a % np2 ? 1 : 0));
  p->m = (int)M;
  p->np = 0;
  for (int c = 0; c < 7; ++c) p->count[c] = 0;
  p->first = (int8_t)p2[0];
  p->last = (int8_t)(np2 > 1 ? p2[np2 - 1] : 0);
  p->radix[p->np++] = p->first;
  for (int i = 0; i < no; ++i) {  // odd[] is sorted: 3s, then 5s, then 7s
    p->radix[p->np++] = (int8_t)odd[i];
    p->count[odd[i] == 3 ? 0 : (odd[i] == 5 ? 1 : 2)] += 1;
  }
  for (int i = 1; i + 1 < np2; ++i) {
    p->radix[p->np++] = (int8_t)p2[i];
    p->count[p2[i] == 16 ? 3 : (p2[i] == 8 ? 4 : (p2[i] == 4 ? 5 : 6))] += 1;
  }
  if (np2 > 1) p->radix[p->np++] = p->last;
  return true;
}

// The smallest M >= lo of that form.
inline int64_t mx_length_at_least(int64_t lo) {
  for (int64_t M = lo < 16 ? 16 : (lo + 15) / 16 * 16;; M += 16) {
    MxPlan p;
    if (mx_plan(M, &p)) return M;
  }
}

}  // namespace frac

// Opaque operator object of the C ABI.
struct frac_op {
  frac_problem prob;
  int64_t N;         // intervals per axis of the generator cube [0, L]^d, L = N h = the largest extent
  int64_t n;         // interior points, FFT length, log2 and M/2 + 1 of axis 0 (x^(1), fastest);
  int64_t M;         //   the same on every axis of a square grid
  int logm;
  int64_t K;
  int64_t na[3];     // per axis i < d: interior points n_i (1 for i >= d)
  int64_t Ma[3];     // FFT length M_i: nextpow2(2 n_i - 1), >= 2, or (FRAC_FFT_SMOOTH) the smallest
                     // 2^a 3^b 5^c 7^d >= 2 n_i + 2 with a >= 4 (1 for i >= d)
  int64_t Ka[3];     // M_i / 2 + 1 (1 for i >= d)
  int logma[3];      // log2 M_i (0 for i >= d; -1 where M_i is not a power of two)
  frac::MxPlan plan[3];  // the pass plan of a 7-smooth M_i that is not a power of two (m = 0 otherwise)
  int square;        // n_i equal on every axis
  int64_t nd;        // prod n_i grid values
  int64_t ngen;      // (N + 1)^d generator entries
  int64_t nsym;      // prod K_i symbol entries (d >= 2: stored in column tiles, below)
  int64_t nsym_alloc;  // entries allocated per symbol array: nsym (d = 1), or the column tiles
                       // ceil(K_1 / 4) 4 prod_{i>0} K_i: d = 2 entry (k2, k1) at (k1 / B) K_2 B + k2 B +
                       // k1 % B, d = 3 entry (k3, k2, k1) at ((k2 KB + k1 / B) K_3 + k3) B + k1 % B
                       // (B = 4 for the FP32 arrays and 2 for the FP64 ones, KB = ceil(K_1 / B);
                       // the padding columns hold zeros)
  double c;          // c_{d,alpha}
  double a0;
  double far_field;
  double norm_bound;
  double kappa_est;  // max / min of the symbol: an estimate of the condition number of A
  double* a;         // device, (N+1)^d FP64 generator
  double* lam64;     // device, prod K_i FP64 scaled symbol
  float* lam32;      // device, prod K_i FP32 scaled symbol
  double* pinv64;    // device, prod K_i FP64 symbol of the tau preconditioner (0 where some k_i is 0 or M_i/2)
  float* pinv32;     // device, prod K_i FP32 copy
  int precond_ok;    // n_i <= M_i/2 - 1 on every axis and the symbol is positive: the tau preconditioner applies
  int xy_fused;      // d = 3: the FP32 apply may run its xy passes fused on thread-block clusters (xy_cluster.cuh)
  size_t device_bytes;
  int device;
};

// The operator's tables live on the device that was current when it was built:
// every call that launches work with it must run with that device current.
inline bool op_on_current_device(const frac_op* op) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == op->device;
}

// Inner tolerance of the mixed-precision refinement when the caller leaves it at 0:
// a well-conditioned operator (kappa_est < 50, so FP32 CG resolves a 1e-6 reduction)
// gets max(1e-6, sqrt(rtol) / 10), two refinement steps for rtol = 1e-10; otherwise
// 1e-4, since FP32 limits each step to about kappa eps_32 anyway.
inline double auto_inner_tol(const frac_op* op, double rtol) {
  if (op->kappa_est < 50.0) {
    const double t = 0.1 * std::sqrt(rtol);
    return t > 1e-6 ? t : 1e-6;
  }
  return 1e-4;
}

