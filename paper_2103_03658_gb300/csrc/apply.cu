// y = A u by circulant embedding and FFT (Sec. 2.1): the operator apply and
// the fused CG apply; kernels and launch helpers in apply_kernels.cuh.
#include "apply_kernels.cuh"

namespace frac {

size_t apply_workspace_bytes(const frac_op* op, int dtype, int64_t batch) {
  int64_t KB, w1, w2;
  if (dtype == FRAC_F64) {
    layout<double>(op, batch, KB, w1, w2);
    return (size_t)(w1 + w2) * sizeof(double2);
  }
  layout<float>(op, batch, KB, w1, w2);
  return (size_t)(w1 + w2) * sizeof(float2);
}

template <typename T>
int apply_t(const frac_op* op, const T* u, T* y, int64_t batch, void* ws, cudaStream_t st) {
  if (batch <= 0) return FRAC_OK;
  if (op->prob.d == 1) return conv1d_op<T, false>(op, u, y, batch, sym_table<T>(op), st);
  return pipeline<T, RF_PLAIN, RI_PLAIN, false>(op, sym_table<T>(op), u, y, batch, ws, CgArgs{}, CgArgs{}, nullptr,
                                                st);
}

template int apply_t<float>(const frac_op*, const float*, float*, int64_t, void*, cudaStream_t);
template int apply_t<double>(const frac_op*, const double*, double*, int64_t, void*, cudaStream_t);

size_t apply_cg_partials(const frac_op* op) {
  int64_t nrows = 1;  // rows of one field: the extents of the axes after the row axis
  for (int i = 1; i < op->prob.d; ++i) nrows *= op->na[i];
  const int64_t a = rows_grid_op<float>(op, nrows), b = rows_grid_op<double>(op, nrows);
  const int64_t c = xy_grid_blocks(op, 1);  // the fused 3D inverse pass (0 when it does not apply)
  return (size_t)std::max(a, std::max(b, c));
}

template <typename T>
int apply_cg_t(const frac_op* op, T* p, const T* r, T* q, void* ws, CGState* cgst, double* partials, cudaStream_t st) {
  if (op->prob.d < 2) return FRAC_ENOTSUP;
  CgArgs fwd, inv;
  fwd.r = r;
  fwd.st = cgst;
  inv.p = p;
  inv.st = cgst;
  inv.partials = partials;
  return pipeline<T, RF_CG, RI_CG, false>(op, sym_table<T>(op), p, q, 1, ws, fwd, inv, cgst, st);
}

template int apply_cg_t<float>(const frac_op*, float*, const float*, float*, void*, CGState*, double*, cudaStream_t);
template int apply_cg_t<double>(const frac_op*, double*, const double*, double*, void*, CGState*, double*, cudaStream_t);

}  // namespace frac
