// Whole 1D solves inside one thread block for the mixed FFT lengths (7-smooth,
// not a power of two; the solver is in solve1d_body.cuh): one kernel per
// precision, M / 16 threads per block, launched once per length.
#include "solve1d_body.cuh"

namespace frac {

template <bool MIXED>
__global__ void __launch_bounds__(512, 1)
k_solve1d_mx(MxLine ln, const Solve1dTask* __restrict__ tasks, int ntasks, const float2* __restrict__ tw32,
             const double2* __restrict__ tw64) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  solve1d_block<MxLine, MIXED>(ln, tasks, ntasks, tw32, tw64, smem_raw, red);
}

template <bool MIXED>
static int launch_solve1d_mx(const MxLine& ln, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  const size_t smem = (size_t)ln.stride() * sizeof(double2);
  auto kern = k_solve1d_mx<MIXED>;
  if (smem > 48 * 1024)
    FRAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  char nb[48];
  std::snprintf(nb, sizeof(nb), "solve1d_%s_M%d", MIXED ? "mixed" : "f64", ln.m());
  prof::Scope ps(nb, st);
  kern<<<ntasks, ln.tpl(), smem, st>>>(ln, d_tasks, ntasks, twiddles32_len(ln.m()), twiddles64_len(ln.m()));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

int solve1d_launch_mx(int64_t M, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  MxPlan plan;
  if (!mx_plan(M, &plan) || M > 8192) return FRAC_ENOTSUP;
  FRAC_TRY(prepare_twiddles_len(M));
  const MxLine ln(plan);
  return mixed ? launch_solve1d_mx<true>(ln, d_tasks, ntasks, st) : launch_solve1d_mx<false>(ln, d_tasks, ntasks, st);
}

}  // namespace frac
