// Whole 1D solves inside one thread block, the power-of-two FFT lengths (the
// solver itself is in solve1d_body.cuh; solve1d_mx.cu has the mixed lengths).
#include "solve1d_body.cuh"

namespace frac {

template <int LOGM, bool MIXED>
__global__ void __launch_bounds__(tpl(LOGM))
k_solve1d(const Solve1dTask* __restrict__ tasks, int ntasks, const float2* __restrict__ tw32,
          const double2* __restrict__ tw64) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  solve1d_block<P2Line<LOGM>, MIXED>(P2Line<LOGM>{}, tasks, ntasks, tw32, tw64, smem_raw, red);
}

template <int LOGM, bool MIXED>
static int launch_solve1d(const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  constexpr int LS = line_stride(LOGM);
  const size_t smem = (size_t)LS * sizeof(double2);
  auto kern = k_solve1d<LOGM, MIXED>;
  if (smem > 48 * 1024)
    FRAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  char nb[48];
  std::snprintf(nb, sizeof(nb), "solve1d_%s_M%d", MIXED ? "mixed" : "f64", 1 << LOGM);
  prof::Scope ps(nb, st);
  kern<<<ntasks, tpl(LOGM), smem, st>>>(d_tasks, ntasks, twiddles32(LOGM), twiddles64(LOGM));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <int LOGM>
static int launch_any(bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  return mixed ? launch_solve1d<LOGM, true>(d_tasks, ntasks, st) : launch_solve1d<LOGM, false>(d_tasks, ntasks, st);
}

int solve1d_launch(int64_t M, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return FRAC_OK;
  FRAC_TRY(prepare_twiddles_len(M));
  if ((M & (M - 1)) != 0) return solve1d_launch_mx(M, mixed, d_tasks, ntasks, st);
  switch (ilog2(M)) {
    case 1: return launch_any<1>(mixed, d_tasks, ntasks, st);
    case 2: return launch_any<2>(mixed, d_tasks, ntasks, st);
    case 3: return launch_any<3>(mixed, d_tasks, ntasks, st);
    case 4: return launch_any<4>(mixed, d_tasks, ntasks, st);
    case 5: return launch_any<5>(mixed, d_tasks, ntasks, st);
    case 6: return launch_any<6>(mixed, d_tasks, ntasks, st);
    case 7: return launch_any<7>(mixed, d_tasks, ntasks, st);
    case 8: return launch_any<8>(mixed, d_tasks, ntasks, st);
    case 9: return launch_any<9>(mixed, d_tasks, ntasks, st);
    case 10: return launch_any<10>(mixed, d_tasks, ntasks, st);
    case 11: return launch_any<11>(mixed, d_tasks, ntasks, st);
    case 12: return launch_any<12>(mixed, d_tasks, ntasks, st);
    case 13: return launch_any<13>(mixed, d_tasks, ntasks, st);
    default: return FRAC_ENOTSUP;
  }
}

}  // namespace frac
