// The tau preconditioner of the CG solves: z = P r = R tau(T_m)^{-1} R^T r,
// m = M/2 - 1, applied as the FFT pipeline of the operator on the odd
// extension of r with the reciprocal symbol (the sine transform of size m is
// that FFT restricted to odd sequences).  Kernels in apply_kernels.cuh.
#include "apply_kernels.cuh"

namespace frac {

template <typename T> static const T* pinv_table(const frac_op* op);
template <> const float* pinv_table<float>(const frac_op* op) { return op->pinv32; }
template <> const double* pinv_table<double>(const frac_op* op) { return op->pinv64; }

template <typename T>
int precond_t(const frac_op* op, const T* r, T* z, int64_t batch, void* ws, cudaStream_t st) {
  if (!op->precond_ok) return FRAC_ENOTSUP;
  if (batch <= 0) return FRAC_OK;
  if (op->prob.d == 1) return conv1d_op<T, true>(op, r, z, batch, pinv_table<T>(op), st);
  return pipeline<T, RF_ODD, RI_ODD, true>(op, pinv_table<T>(op), r, z, batch, ws, CgArgs{}, CgArgs{}, nullptr, st);
}

template int precond_t<float>(const frac_op*, const float*, float*, int64_t, void*, cudaStream_t);
template int precond_t<double>(const frac_op*, const double*, double*, int64_t, void*, cudaStream_t);

template <typename T>
int precond_cg_t(const frac_op* op, const T* r, T* z, void* ws, CGState* cgst, double* partials, cudaStream_t st) {
  if (op->prob.d < 2 || !op->precond_ok) return FRAC_ENOTSUP;
  CgArgs inv;
  inv.p = r;
  inv.st = cgst;
  inv.partials = partials;
  return pipeline<T, RF_ODD, RI_ODD_CG, true>(op, pinv_table<T>(op), r, z, 1, ws, CgArgs{}, inv, cgst, st);
}

template int precond_cg_t<float>(const frac_op*, const float*, float*, void*, CGState*, double*, cudaStream_t);
template int precond_cg_t<double>(const frac_op*, const double*, double*, void*, CGState*, double*, cudaStream_t);

}  // namespace frac
