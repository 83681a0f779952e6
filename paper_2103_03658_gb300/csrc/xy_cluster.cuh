// Fused xy passes of the 3D FP32 apply on thread-block clusters (Sec. 2.1's FFT
// product; the 3D scheme's trilevel Toeplitz matrix): one cluster of kXyC CTAs per
// z-plane (field b, index j3).  Forward: the row pairs of the plane (two real rows
// per complex FFT along x, as k_rows_fwd) hand their half spectra to the CTA that
// owns each column block (block kb of B = 4 columns lives in CTA kb mod kXyC, as
// local block kb / kXyC), through distributed shared memory; after a cluster
// barrier every CTA runs the y FFTs of its own column blocks (as k_cols YFWD) and
// writes the plane's W2 columns to global memory.  Inverse: the y inverse FFTs of the
// CTA's column blocks (as k_cols YINV) leave the plane's first n_2 rows in its slice;
// after a cluster barrier the row pairs read their half spectra from the owners and
// run the inverse row FFTs (as k_rows_inv).  The x-spectrum slab W1 of the five-pass
// schedule never reaches global memory: per FP32 apply the passes move u, W2 (three
// times), the symbol and y instead of also W1 four times.  The arithmetic is that of
// the five-pass kernels (the same device functions); the compiler may fuse multiplies
// and adds differently in these kernels, so the two agree to FP32 rounding.  Measured
// slower than the five passes on GB300 (W1 largely stays in L2 between those passes,
// and these kernels hold one CTA per SM), so frac_apply_3d_passes selects them.
//
// Waits: two cluster barriers per kernel (forward: at the start, so that every CTA
// has started before remote writes, and after the row phase; inverse: after the
// column phase and before exit, so that no CTA leaves while others read its slice),
// reached by every thread of every CTA; no flag or spin.
#pragma once

#include "apply_kernels.cuh"

namespace frac {

constexpr int kXyC = 8;          // CTAs per cluster (portable size)
constexpr int kXyThreads = 512;  // threads per CTA

struct XyArgs {
  int n1, n2, n3;   // interior points along x, y, z
  int64_t nb;       // fields
  int K1, KB;       // x half-spectrum extent M_1/2 + 1 and its column blocks ceil(K1 / 4)
  int M2, K2;       // y FFT length and M_2/2 + 1
  int lkb;          // column blocks per CTA at most, ceil(KB / kXyC)
  int64_t slice;    // complex entries of a CTA's slice: lkb n2 4
};

__device__ __forceinline__ void xy_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared memory of one CTA: its slice of the plane's x spectra, then the line
// buffers of the row pairs or the column tiles (whichever is larger)
template <int LOGM>
constexpr size_t xy_work_entries() {
  constexpr int TPL = fft::tpl(LOGM), LINES = kXyThreads / TPL, TPR = kXyThreads / (4 * TPL);
  constexpr size_t rows = (size_t)LINES * fft::line_stride(LOGM);
  constexpr size_t cols = (size_t)TPR * 4 * fft::line_stride_tile(LOGM);
  return rows > cols ? rows : cols;
}

// Forward: u (or, RF_CG, p = r + beta p written back to u) -> W2 of the plane.
template <int LOGM, int FK, bool ODD>
__global__ void __launch_bounds__(kXyThreads, 1)
k_xy_fwd(const float* u, float2* __restrict__ W2, XyArgs X, const float* __restrict__ lam,
         const float2* __restrict__ tw, const float* __restrict__ r, const CGState* st) {
  using C = float2;
  using LN = fft::P2Line<LOGM>;
  using LNT = fft::P2Line<LOGM, fft::tile_shift(LOGM)>;
  constexpr int TPL = fft::tpl(LOGM), LINES = kXyThreads / TPL, TPR = kXyThreads / (4 * TPL), B = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;  // set before this launch: the same in every CTA
  C* S = reinterpret_cast<C*>(smem_raw);
  C* work = S + X.slice;
  const int rank = (int)__clusterRelativeBlockRank();
  const int64_t plane = blockIdx.x / kXyC;  // b n3 + j3
  const int tid = threadIdx.x, line = tid / TPL, tl = tid % TPL;
  const int n1 = X.n1, n2 = X.n2;
  const int64_t base = plane * n2 * (int64_t)n1;  // the plane's first row
  xy_cluster_sync();  // every CTA of the cluster has started before any writes into its shared memory
  // ---- x transforms of the plane's row pairs, spectra to their column blocks' owners
  const int npairs = (n2 + 1) / 2, rounds = (npairs + kXyC * LINES - 1) / (kXyC * LINES);
  for (int i = 0; i < rounds; ++i) {
    const int64_t pair = ((int64_t)i * kXyC + rank) * LINES + line;
    const int64_t r0 = 2 * pair;
    auto sink = [&]() {
      return [&](int k, C z0, C z1, bool h0, bool h1) {
        const int kb = k / B, owner = kb % kXyC, lk = kb / kXyC;
        C* dst = static_cast<C*>(__cluster_map_shared_rank((void*)S, owner)) + ((int64_t)lk * n2 + r0) * B + (k % B);
        if (h0) dst[0] = z0;
        if (h1) dst[B] = z1;
      };
    };
    if constexpr (FK == RF_CG) {
      const float be = (float)st->beta;
      float* p = const_cast<float*>(u);
      row_fwd_pair_s<float, LN>(
          LN{},
          [&](int64_t row, int x) {
            const int64_t k = base + row * n1 + x;
            const float v = r[k] + be * p[k];
            p[k] = v;
            return v;
          },
          sink, n1, n2, tw, pair, work + line * LN::stride(), tl);
    } else {
      row_fwd_pair_s<float, LN, FK == RF_ODD>(
          LN{}, [&](int64_t row, int x) { return u[base + row * n1 + x]; }, sink, n1, n2, tw, pair,
          work + line * LN::stride(), tl);
    }
  }
  xy_cluster_sync();  // every slice complete
  // ---- y transforms of this CTA's column blocks -> W2
  const ColArgs Ay{n2, X.K1, X.KB, X.KB, X.nb, X.n3, X.M2, X.K2};
  const int ts = tid / (B * TPL), w = tid % (B * TPL);
  const int mine = (X.KB - rank + kXyC - 1) / kXyC;  // blocks kb = rank + kXyC lk
  const int crounds = (mine + TPR - 1) / TPR;
  for (int i = 0; i < crounds; ++i) {
    const int lk = i * TPR + ts;
    const int64_t tile = lk < mine ? (int64_t)lk * kXyC + rank : X.KB;  // past the spectrum: empty
    col_tile_l<float, LNT, YFWD, ODD>(LNT{}, nullptr, W2, Ay, lam, tw, plane, tile, work + ts * B * LNT::stride_tile(),
                                      w % B, w / B, S + (int64_t)lk * n2 * B);
  }
}

// Inverse: W2 of the plane -> y (IK: RI_CG adds the partials of p.y and its last
// block sets the CG state as k_rows_inv does; RI_ODD / RI_ODD_CG the preconditioner's).
template <int LOGM, int IK, bool ODD>
__global__ void __launch_bounds__(kXyThreads, 1)
k_xy_inv(const float2* __restrict__ W2, float* __restrict__ y, XyArgs X, const float2* __restrict__ tw,
         const float* __restrict__ p, CGState* st, double* partials) {
  using C = float2;
  using LN = fft::P2Line<LOGM>;
  using LNT = fft::P2Line<LOGM, fft::tile_shift(LOGM)>;
  constexpr int TPL = fft::tpl(LOGM), LINES = kXyThreads / TPL, TPR = kXyThreads / (4 * TPL), B = 4;
  constexpr bool CG = IK == RI_CG || IK == RI_ODD_CG;
  constexpr bool RODD = IK == RI_ODD || IK == RI_ODD_CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (CG && st->done) return;  // set before this launch: the same in every CTA
  C* S = reinterpret_cast<C*>(smem_raw);
  C* work = S + X.slice;
  const int rank = (int)__clusterRelativeBlockRank();
  const int64_t plane = blockIdx.x / kXyC;
  const int tid = threadIdx.x, line = tid / TPL, tl = tid % TPL;
  const int n1 = X.n1, n2 = X.n2;
  const int64_t base = plane * n2 * (int64_t)n1;
  // ---- y inverse transforms of this CTA's column blocks -> its slice (rows j2 < n2)
  const ColArgs Ay{n2, X.K1, X.KB, X.KB, X.nb, X.n3, X.M2, X.K2};
  const int ts = tid / (B * TPL), w = tid % (B * TPL);
  const int mine = (X.KB - rank + kXyC - 1) / kXyC;
  const int crounds = (mine + TPR - 1) / TPR;
  for (int i = 0; i < crounds; ++i) {
    const int lk = i * TPR + ts;
    const int64_t tile = lk < mine ? (int64_t)lk * kXyC + rank : X.KB;
    col_tile_l<float, LNT, YINV, ODD>(LNT{}, W2, nullptr, Ay, nullptr, tw, plane, tile,
                                      work + ts * B * LNT::stride_tile(), w % B, w / B, nullptr,
                                      S + (int64_t)lk * n2 * B);
  }
  xy_cluster_sync();  // every slice complete
  // ---- x inverse transforms of the plane's row pairs, half spectra from the owners
  float dot = 0.0f;
  const int npairs = (n2 + 1) / 2, rounds = (npairs + kXyC * LINES - 1) / (kXyC * LINES);
  for (int i = 0; i < rounds; ++i) {
    const int64_t pair = ((int64_t)i * kXyC + rank) * LINES + line;
    const int64_t r0 = 2 * pair;
    auto src = [&](int x, C& v0, C& v1, bool h0, bool h1) {
      const int kb = x / B, owner = kb % kXyC, lk = kb / kXyC;
      const C* from =
          static_cast<const C*>(__cluster_map_shared_rank((void*)S, owner)) + ((int64_t)lk * n2 + r0) * B + (x % B);
      v0 = h0 ? from[0] : C{0.0f, 0.0f};
      v1 = h1 ? from[B] : C{0.0f, 0.0f};
    };
    row_inv_pair_s<float, LN, RODD>(LN{}, src, n1, n2, tw, pair, work + line * LN::stride(), tl,
                                    [&](int64_t row, int x, float v) {
                                      const int64_t k = base + row * n1 + x;
                                      y[k] = v;
                                      if (CG) dot += v * p[k];
                                    });
  }
  xy_cluster_sync();  // every remote read done before any CTA of the cluster exits
  rows_inv_finish<IK>(dot, st, partials, reinterpret_cast<double*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Launchers (one per direction and kind; LOGM from the operator)
// ---------------------------------------------------------------------------

inline XyArgs xy_args(const frac_op* op, int64_t batch) {
  XyArgs X;
  X.n1 = (int)op->na[0];
  X.n2 = (int)op->na[1];
  X.n3 = (int)op->na[2];
  X.nb = batch;
  X.K1 = (int)op->Ka[0];
  X.KB = (X.K1 + 3) / 4;
  X.M2 = (int)op->Ma[1];
  X.K2 = (int)op->Ka[1];
  X.lkb = (X.KB + kXyC - 1) / kXyC;
  X.slice = (int64_t)X.lkb * X.n2 * 4;
  return X;
}

template <int LOGM>
size_t xy_smem_bytes(const XyArgs& X) {
  return ((size_t)X.slice + xy_work_entries<LOGM>()) * sizeof(float2);
}

template <typename K>
int xy_launch(K kern, int64_t planes, size_t smem, cudaStream_t st, const char* name, int logm,
              void** args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kXyC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(planes * kXyC));
  cfg.blockDim = dim3(kXyThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  char nb[48];
  std::snprintf(nb, sizeof(nb), "%s_f32_M%d", name, 1 << logm);
  prof::Scope ps(nb, st);
  FRAC_CUDA_TRY(cudaLaunchKernelExC(&cfg, (const void*)kern, args));
  return FRAC_OK;
}

template <int LOGM, int FK, bool ODD>
int launch_xy_fwd(const frac_op* op, const void* in, void* W2, int64_t batch, const float* lam, const CgArgs& cg,
                  const CGState* cgst, cudaStream_t st) {
  XyArgs X = xy_args(op, batch);
  const float* u = (const float*)in;
  float2* w2 = (float2*)W2;
  const float2* tw = twiddles32(LOGM);
  const float* r = (const float*)cg.r;
  const CGState* s = FK == RF_CG ? cg.st : cgst;
  void* args[] = {(void*)&u, (void*)&w2, (void*)&X, (void*)&lam, (void*)&tw, (void*)&r, (void*)&s};
  return xy_launch(k_xy_fwd<LOGM, FK, ODD>, batch * X.n3, xy_smem_bytes<LOGM>(X), st,
                   FK == RF_CG ? "xy_fwd_cg" : (ODD ? "xy_fwd_tau" : "xy_fwd"), LOGM, args);
}

template <int LOGM, int IK, bool ODD>
int launch_xy_inv(const frac_op* op, const void* W2, void* out, int64_t batch, const CgArgs& cg, cudaStream_t st) {
  XyArgs X = xy_args(op, batch);
  const float2* w2 = (const float2*)W2;
  float* y = (float*)out;
  const float2* tw = twiddles32(LOGM);
  const float* p = (const float*)cg.p;
  CGState* s = cg.st;
  double* partials = cg.partials;
  void* args[] = {(void*)&w2, (void*)&y, (void*)&X, (void*)&tw, (void*)&p, (void*)&s, (void*)&partials};
  static const char* names[4] = {"xy_inv", "xy_inv_cg", "xy_inv_tau", "xy_inv_tau_cg"};
  return xy_launch(k_xy_inv<LOGM, IK, ODD>, batch * X.n3, xy_smem_bytes<LOGM>(X), st, names[IK], LOGM, args);
}

}  // namespace frac
