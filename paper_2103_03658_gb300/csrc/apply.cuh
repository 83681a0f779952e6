// Internal interfaces between the translation units of the library.
#pragma once

#include <cmath>

#include <vector>

#include "common.cuh"

namespace frac {

template <typename T> inline const cplx_t<T>* tw_table(int logm);
template <> inline const float2* tw_table<float>(int logm) { return twiddles32(logm); }
template <> inline const double2* tw_table<double>(int logm) { return twiddles64(logm); }

template <typename T> inline const T* sym_table(const frac_op* op);
template <> inline const float* sym_table<float>(const frac_op* op) { return op->lam32; }
template <> inline const double* sym_table<double>(const frac_op* op) { return op->lam64; }

// Device-resident conjugate-gradient state (solve.cu, fused apply kernels).
// Plain CG keeps rz = rr; preconditioned CG (pcg = 1) sets rz = r.z and beta
// in the preconditioner pass (z = P r) that follows each update.
struct CGState {
  double rr;      // r.r
  double pq;      // p.Ap
  double alpha, beta;
  double tol2;    // stop when rr <= tol2
  double rz;      // r.z (= rr without preconditioner); alpha = rz / pq
  int it, maxit, done, status, pcg;
  unsigned int count_pq, count_rr, count_rz;  // arrival counters of the last-block reductions
  int trips;      // loop-body executions in the current launch of a CG graph (reset by the host)
};

// coeffs.cu
int prepare_twiddles(int logm);
int build_coefficients(frac_op* op, cudaStream_t st);
int generator_symbol_axes(const frac_op* op, const int* logm, double* out, double* tmp, cudaStream_t st);
int take_coeff_fault();

// boundary.cu: b = -c (near + far) on device buffers (frac_boundary), and r = f - g.
int boundary_device(const frac_op* op, const double* g_ext, const double* far, double* b, cudaStream_t st);
int subtract_device(const double* f, const double* g, double* r, int64_t count, cudaStream_t st);

// apply_xy.cu: decides op->xy_fused for a 3D operator when it is built (equal
// power-of-two x and y FFT lengths 32..512, a cluster launch that fits the device) and
// sets the fused kernels' attributes; outside any stream capture.
int xy_prepare(frac_op* op);

// apply.cu: y = A u for `batch` vectors on device buffers; ws holds
// apply_workspace_bytes(op, dtype, batch) bytes (unused for d = 1).
size_t apply_workspace_bytes(const frac_op* op, int dtype, int64_t batch);
template <typename T>
int apply_t(const frac_op* op, const T* u, T* y, int64_t batch, void* ws, cudaStream_t st);

// One CG apply for d >= 2 with the vector work fused into the FFT passes:
// p = r + beta p (beta from st) on the way into the forward row pass, q = A p
// stored by the inverse row pass together with per-block partials of p.q;
// the last block of that pass sums the partials in index order and sets
// st->pq and st->alpha (or flags a breakdown).  Every kernel returns at once
// when st->done is set.  `partials` holds apply_cg_partials(op) doubles.
size_t apply_cg_partials(const frac_op* op);
template <typename T>
int apply_cg_t(const frac_op* op, T* p, const T* r, T* q, void* ws, CGState* st, double* partials, cudaStream_t s);

// z = P r with the tau preconditioner (op->precond_ok required) for `batch`
// vectors on device buffers; ws as for apply_t.
template <typename T>
int precond_t(const frac_op* op, const T* r, T* z, int64_t batch, void* ws, cudaStream_t st);
// The preconditioner pass of preconditioned CG (d >= 2): z = P r together with
// per-block partials of r.z; the last block sets st->beta = r.z / st->rz
// (0 when st->rz is 0, the first pass) and st->rz = r.z.  Returns at once when
// st->done.  partials as for apply_cg_t.
template <typename T>
int precond_cg_t(const frac_op* op, const T* r, T* z, void* ws, CGState* st, double* partials, cudaStream_t s);

// solve.cu
int solve_device(const frac_op* op, const double* f, double* u, const frac_solve_opts* opts,
                 frac_solve_info* info, cudaStream_t st);
// Makes every stream of engine e wait for the work already queued on `caller`.
int engine_wait_for(frac_engine* e, cudaStream_t caller);

// Batched work launched on a stream whose per-problem results are still on the
// device: collect() waits for the stream, copies the results to
// info[order[t]] and frees the device buffers (stream ordered); the
// destructor frees them if collect() was never called.
struct BatchPending {
  cudaStream_t st = nullptr;
  std::vector<void*> bufs;
  frac_solve_info* dinfo = nullptr;
  std::vector<int64_t> order;
  template <typename P>
  int alloc(P** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) return record_cuda_error(e, __FILE__, __LINE__, "cudaMallocAsync");
    bufs.push_back(p);
    *out = static_cast<P*>(p);
    return FRAC_OK;
  }
  void* pinned = nullptr;  // host staging of the launch records, freed once st is done
  int collect(frac_solve_info* info);
  ~BatchPending();
};

// Launches the 1D problems listed in idx[0..count) of (ops, f, u) (device
// pointers), grouped by FFT length, one launch per group, on st; the results
// arrive through pend->collect().
int solve_batch_1d(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                   const frac_solve_opts* opts, const int64_t* idx, cudaStream_t st, BatchPending* pend);

}  // namespace frac
