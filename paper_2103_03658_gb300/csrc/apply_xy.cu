// The fused xy passes of the 3D FP32 apply (xy_cluster.cuh): dispatch on the FFT
// length, the per-operator decision taken when it is built, the switch of
// frac_apply_3d_passes, and the instantiations the pipelines of apply.cu and
// precond.cu call.
#include <atomic>
#include <mutex>
#include <vector>

#include "xy_cluster.cuh"

namespace frac {

namespace {

// off by default: measured slower than the five passes on GB300 (the x-spectrum slab of
// a 255^3 field, 135 MB, largely stays in the 129 MB L2 between the five passes, while
// the fused kernels run one 512-thread CTA per SM and cross the cluster through DSMEM)
std::atomic<int> g_xy_on{0};

#define FRAC_XY_DISPATCH(logm, CALL)                                   \
  switch (logm) {                                                      \
    case 5: { constexpr int LG = 5; return CALL; }                     \
    case 6: { constexpr int LG = 6; return CALL; }                     \
    case 7: { constexpr int LG = 7; return CALL; }                     \
    case 8: { constexpr int LG = 8; return CALL; }                     \
    case 9: { constexpr int LG = 9; return CALL; }                     \
    default: return FRAC_ENOTSUP;                                      \
  }

template <typename K>
int allow_smem(K kern, int bytes) {
  FRAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return FRAC_OK;
}

// Kernel attributes of every kind at one length (once per device), and whether a
// cluster of kXyC CTAs with `smem` bytes each can be resident.
template <int LOGM>
int prepare_length(size_t smem, bool* fits) {
  int dev = 0, optin = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  FRAC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  static std::mutex mu;
  static std::vector<int> done;  // per device, bit per length
  {
    std::lock_guard<std::mutex> lk(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (!(done[dev] & (1 << LOGM))) {
      const int lim = optin - 1024;  // room for the kernels' static shared memory
      FRAC_TRY(allow_smem(k_xy_fwd<LOGM, RF_PLAIN, false>, lim));
      FRAC_TRY(allow_smem(k_xy_fwd<LOGM, RF_CG, false>, lim));
      FRAC_TRY(allow_smem(k_xy_fwd<LOGM, RF_ODD, true>, lim));
      FRAC_TRY(allow_smem(k_xy_inv<LOGM, RI_PLAIN, false>, lim));
      FRAC_TRY(allow_smem(k_xy_inv<LOGM, RI_CG, false>, lim));
      FRAC_TRY(allow_smem(k_xy_inv<LOGM, RI_ODD, true>, lim));
      FRAC_TRY(allow_smem(k_xy_inv<LOGM, RI_ODD_CG, true>, lim));
      done[dev] |= 1 << LOGM;
    }
    if (smem + 1024 > (size_t)optin) {
      *fits = false;
      return FRAC_OK;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kXyC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(kXyC);
  cfg.blockDim = dim3(kXyThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int num = 0;
  for (const void* k : {(const void*)k_xy_fwd<LOGM, RF_CG, false>, (const void*)k_xy_inv<LOGM, RI_ODD_CG, true>}) {
    if (cudaOccupancyMaxActiveClusters(&num, k, &cfg) != cudaSuccess) {
      cudaGetLastError();
      num = 0;
    }
    if (num < 1) break;
  }
  *fits = num >= 1;
  return FRAC_OK;
}

}  // namespace

int xy_prepare(frac_op* op) {
  op->xy_fused = 0;
  if (op->prob.d != 3 || op->plan[0].m || op->plan[1].m || op->logma[0] != op->logma[1]) return FRAC_OK;
  const int logm = op->logma[0];
  if (logm < 5 || logm > 9) return FRAC_OK;
  bool fits = false;
  const XyArgs X = xy_args(op, 1);
  switch (logm) {
    case 5: FRAC_TRY(prepare_length<5>(xy_smem_bytes<5>(X), &fits)); break;
    case 6: FRAC_TRY(prepare_length<6>(xy_smem_bytes<6>(X), &fits)); break;
    case 7: FRAC_TRY(prepare_length<7>(xy_smem_bytes<7>(X), &fits)); break;
    case 8: FRAC_TRY(prepare_length<8>(xy_smem_bytes<8>(X), &fits)); break;
    default: FRAC_TRY(prepare_length<9>(xy_smem_bytes<9>(X), &fits)); break;
  }
  op->xy_fused = fits ? 1 : 0;
  return FRAC_OK;
}

bool xy_enabled(const frac_op* op) { return op->xy_fused && g_xy_on.load(std::memory_order_relaxed); }

int64_t xy_grid_blocks(const frac_op* op, int64_t batch) {
  return op->xy_fused ? batch * op->na[2] * kXyC : 0;
}

template <int FK, bool ODD>
int xy_fwd(const frac_op* op, const void* in, void* W2, int64_t batch, const float* lam, const CgArgs& cg,
           const CGState* cgst, cudaStream_t st) {
  FRAC_XY_DISPATCH(op->logma[0], (launch_xy_fwd<LG, FK, ODD>(op, in, W2, batch, lam, cg, cgst, st)));
}

template <int IK, bool ODD>
int xy_inv(const frac_op* op, const void* W2, void* out, int64_t batch, const CgArgs& cg, cudaStream_t st) {
  FRAC_XY_DISPATCH(op->logma[0], (launch_xy_inv<LG, IK, ODD>(op, W2, out, batch, cg, st)));
}

template int xy_fwd<RF_PLAIN, false>(const frac_op*, const void*, void*, int64_t, const float*, const CgArgs&,
                                     const CGState*, cudaStream_t);
template int xy_fwd<RF_CG, false>(const frac_op*, const void*, void*, int64_t, const float*, const CgArgs&,
                                  const CGState*, cudaStream_t);
template int xy_fwd<RF_ODD, true>(const frac_op*, const void*, void*, int64_t, const float*, const CgArgs&,
                                  const CGState*, cudaStream_t);
template int xy_inv<RI_PLAIN, false>(const frac_op*, const void*, void*, int64_t, const CgArgs&, cudaStream_t);
template int xy_inv<RI_CG, false>(const frac_op*, const void*, void*, int64_t, const CgArgs&, cudaStream_t);
template int xy_inv<RI_ODD, true>(const frac_op*, const void*, void*, int64_t, const CgArgs&, cudaStream_t);
template int xy_inv<RI_ODD_CG, true>(const frac_op*, const void*, void*, int64_t, const CgArgs&, cudaStream_t);

}  // namespace frac

extern "C" int frac_apply_3d_passes(int fused) {
  frac::g_xy_on.store(fused ? 1 : 0, std::memory_order_relaxed);
  return FRAC_OK;
}
