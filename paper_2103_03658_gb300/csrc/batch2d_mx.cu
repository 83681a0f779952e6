// The persistent batched 2D kernel instance that also takes mixed (7-smooth) FFT
// lengths (batch2d_kernel.cuh), in a translation unit of its own.
#include "batch2d_kernel.cuh"

namespace frac {
namespace b2 {

int mx_kernel_attrs(size_t smem) { return kernel_attrs<true>(smem); }
int mx_kernel_active_clusters(int C, size_t smem) { return kernel_active_clusters<true>(C, smem); }
int mx_kernel_launch(const B2Args& a, int C, int grid, size_t smem, cudaStream_t st) {
  return kernel_launch<true>(a, C, grid, smem, st);
}

}  // namespace b2
}  // namespace frac
