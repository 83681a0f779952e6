// Device side of the persistent batched 2D solver (batch2d.cu): the problem
// records, the group reductions, the solver over a line policy and the kernel,
// shared by batch2d.cu (the instance for power-of-two lengths) and batch2d_mx.cu
// (the instance that also takes mixed lengths).
#pragma once

#include <type_traits>

#include "apply.cuh"
#include "batch2d.cuh"
#include "passes.cuh"

namespace frac {
namespace b2 {

using namespace fft;

constexpr int kThreads = 512;

struct B2Prob {
  const double* f;
  double* u;
  const float* lam32;
  const double* lam64;
  const float* pinv32;  // tau preconditioner symbol (pcg)
  const float2* tw32;   // twiddles of the problem's FFT length
  const double2* tw64;
  MxPlan plan;          // mixed FFT length (plan.m > 0), else 2^logm
  int n, logm, max_iter, use_x0, pcg;
  double rtol, inner_tol;
};

// Scratch of one worker (a cluster or a CTA), sized for its largest problem.
struct B2Slot {
  void* W;  // spectrum, FP64 layout n ceil(K/2) 2 complex doubles; the FP32 passes use its front
  float *x, *r, *p, *q;
  double* r64;
  size_t w_bytes;  // capacity of W
  int64_t nn;      // capacity of each vector (entries)
};

struct B2Args {
  const B2Prob* probs;
  frac_solve_info* info;  // per problem
  int n_cluster, n_local; // probs[0, n_cluster) cluster-wide, then n_local CTA-local
  unsigned int* next;     // queue heads: [0] cluster, [1] local
  const B2Slot* cslots;   // per cluster
  const B2Slot* lslots;   // per CTA
  size_t smem;            // dynamic shared memory of each CTA (bytes)
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct Group {
  int G, rank;  // CTAs on the problem, this CTA's rank among them
  __device__ __forceinline__ void sync() const {
    if (G > 1)
      cluster_sync_all();
    else
      __syncthreads();
  }
};

// Sum over the group, identical in every thread of every CTA of the group:
// block sum, then (cluster) each CTA's total from the shared memory of ranks
// 0..G-1 in order.  Two slots alternate, so a slot is rewritten only after
// the next reduction's barrier, when every reader is done with it.
__device__ inline double group_sum(double v, const Group& g, double* red, double* slots, int& parity) {
  const double s = block_sum_all(v, red);
  if (g.G == 1) return s;
  double* slot = slots + parity;
  parity ^= 1;
  if (threadIdx.x == 0) *slot = s;
  cluster_sync_all();
  double t = 0.0;
  for (int r = 0; r < g.G; ++r) t += *static_cast<volatile double*>(__cluster_map_shared_rank((void*)slot, r));
  return t;
}

// One problem on one group (cluster or CTA).  The three steps of the
// refinement are separate (non-inlined) functions, so the FP32 CG loop gets
// its own register allocation instead of sharing one with the FP64 passes.
// (Inlined, they once computed a wrong inverse row pass at M = 32: the FFT's
// shared line buffer was a __restrict__ parameter, which let the compiler move
// its accesses across the block barriers; the buffer is no longer restrict and
// the inlined build is exact.)
struct Ctx {
  const B2Prob* P;
  const B2Slot* S;
  Group g;
  const float2* tw32;
  const double2* tw64;
  unsigned char* smem;
  size_t smem_bytes;
  double* red;
  double* slots;
  int parity;
};

// The line policies of a problem: rows (LN) and column tiles (the power-of-two
// tiles pad every 2^tile_shift entries; a mixed line pads the same way in both).
template <typename LN> struct TileLine { using type = LN; };
template <int L> struct TileLine<P2Line<L>> { using type = P2Line<L, tile_shift(L)>; };

// Geometry of one problem's passes on a 512-thread CTA: LINES row lines of TPL
// threads and TPR32 / TPR64 column tiles of 4 / 2 lanes a round.  For a mixed
// length TPL need not divide 512: the threads past the last whole line (tile)
// take an empty unit (no rows, a tile past the spectrum) and a spare buffer.
template <typename LN>
struct Solver {
  using LNT = typename TileLine<LN>::type;
  static __device__ __forceinline__ LN ln(const Ctx& c) {
    if constexpr (std::is_same<LN, MxLine>::value)
      return MxLine(c.P->plan);
    else
      return LN{};
  }
  static __device__ __forceinline__ LNT lnt(const Ctx& c) {
    if constexpr (std::is_same<LN, MxLine>::value)
      return MxLine(c.P->plan);
    else
      return LNT{};
  }
  static __device__ __forceinline__ int tpl(const Ctx& c) { return ln(c).tpl(); }
  static __device__ __forceinline__ int lines(const Ctx& c) { return kThreads / tpl(c); }
  static __device__ __forceinline__ int kk(const Ctx& c) { return ln(c).m() / 2 + 1; }
  static __device__ __forceinline__ int kb32(const Ctx& c) { return (kk(c) + 3) / 4; }
  static __device__ __forceinline__ int kb64(const Ctx& c) { return (kk(c) + 1) / 2; }
  static __device__ __forceinline__ int tpr32(const Ctx& c) { return kThreads / (4 * tpl(c)); }
  static __device__ __forceinline__ int tpr64(const Ctx& c) { return kThreads / (2 * tpl(c)); }
  // this thread's row line (lines(c) for the spare one) and its line buffer
  static __device__ __forceinline__ int my_line(const Ctx& c) { return min((int)threadIdx.x / tpl(c), lines(c)); }
  template <typename C>
  static __device__ __forceinline__ C* row_buf(const Ctx& c) {
    return reinterpret_cast<C*>(c.smem) + my_line(c) * ln(c).stride();
  }

  static __device__ __forceinline__ int rrounds(const Ctx& c) {
    const int npairs = (c.P->n + 1) / 2;
    return (npairs + c.g.G * lines(c) - 1) / (c.g.G * lines(c));
  }
  // the row pair of this thread's line in round i (far past the grid for a spare thread)
  static __device__ __forceinline__ int64_t pair_of(const Ctx& c, int i) {
    const int li = (int)threadIdx.x / tpl(c);
    if (li >= lines(c)) return int64_t(1) << 40;
    return ((int64_t)i * c.g.G + c.g.rank) * lines(c) + li;
  }
  // column tile of round i for the tile group ts of TPR tiles a round (past the
  // spectrum, KB, for a spare group)
  static __device__ __forceinline__ int64_t tile_of(const Ctx& c, int i, int ts, int tpr, int kb) {
    if (ts >= tpr) return kb;
    return ((int64_t)i * c.g.G + c.g.rank) * tpr + ts;
  }
  // the points of this thread: those its row passes read and write
  template <typename Fn>
  static __device__ __forceinline__ void for_own(const Ctx& c, Fn fn) {
    const int n = c.P->n, tl = threadIdx.x % tpl(c), rr = rrounds(c), TPL = tpl(c);
    if ((int)threadIdx.x / TPL >= lines(c)) return;
    for (int i = 0; i < rr; ++i) {
      const int64_t r0 = 2 * pair_of(c, i);
#pragma unroll
      for (int e = 0; e < LN::E / 2; ++e) {
        const int x = tl + e * TPL;
        if (x < n) {
          if (r0 < n) fn(r0 * n + x);
          if (r0 + 1 < n) fn((r0 + 1) * n + x);
        }
      }
    }
  }
  static __device__ __forceinline__ double gsum(Ctx& c, double v) {
    return group_sum(v, c.g, c.red, c.slots, c.parity);
  }

  // ||f||^2, and u = 0 unless it is the initial guess; with u = 0 the first residual is f
  // itself (R64 = F), which spares an FP64 apply
  static __device__ __noinline__ double start(Ctx& c) {
    const double* F = c.P->f;
    double* U = c.P->u;
    double* R64 = c.S->r64;
    const bool zero = !c.P->use_x0;
    double ff = 0.0;
    for_own(c, [&](int64_t k) {
      const double fv = F[k];
      ff += fv * fv;
      if (zero) {
        U[k] = 0.0;
        R64[k] = fv;
      }
    });
    return gsum(c, ff);
  }

  // R64 = F - A64 U (FP64 passes); returns ||R64||^2
  static __device__ __noinline__ double residual(Ctx& c) {
    const int n = c.P->n, tid = threadIdx.x, TPL = tpl(c), tl = tid % TPL, rr = rrounds(c);
    const int K = kk(c), KB64 = kb64(c), TPR64 = tpr64(c), LST = lnt(c).stride_tile();
    const double* F = c.P->f;
    const double* U = c.P->u;
    double* R64 = c.S->r64;
    double2* W = static_cast<double2*>(c.S->W);
    double2* rb = row_buf<double2>(c);
    for (int i = 0; i < rr; ++i)
      row_fwd_pair_l<double, LN>(ln(c), [&](int64_t row, int x) { return U[row * n + x]; }, W, n, n, KB64, c.tw64,
                                 pair_of(c, i), rb, tl);
    c.g.sync();
    {
      const ColArgs A{n, K, KB64, KB64, 1, 0, 0, K};
      const int ts = tid / (2 * TPL), w = tid % (2 * TPL);
      const int cr = (KB64 + c.g.G * TPR64 - 1) / (c.g.G * TPR64);
      for (int i = 0; i < cr; ++i)
        col_tile_l<double, LNT, SYM2>(lnt(c), W, W, A, c.P->lam64, c.tw64, 0, tile_of(c, i, ts, TPR64, KB64),
                                      reinterpret_cast<double2*>(c.smem) + min(ts, TPR64) * 2 * LST, w % 2, w / 2);
    }
    c.g.sync();
    double part = 0.0;
    for (int i = 0; i < rr; ++i)
      row_inv_pair_l<double, LN>(ln(c), W, n, n, KB64, c.tw64, pair_of(c, i), rb, tl, [&](int64_t row, int x, double v) {
        const double rv = F[row * n + x] - v;
        R64[row * n + x] = rv;
        part += rv * rv;
      });
    return gsum(c, part);
  }

  // Z = P R (tau preconditioner, FP32 passes on the odd extension; Z in the
  // storage of Q, which is dead once R is updated); returns the group sum of
  // R.Z.  The odd passes read entries that other threads of the CTA own; the
  // block barriers of the group sums before and after order those accesses.
  static __device__ __forceinline__ double precond(Ctx& c) {
    const int n = c.P->n, tid = threadIdx.x, TPL = tpl(c), tl = tid % TPL, rr = rrounds(c);
    const int K = kk(c), KB32 = kb32(c), TPR32 = tpr32(c), LST = lnt(c).stride_tile();
    const float* R = c.S->r;
    float* Z = c.S->q;
    float2* W = static_cast<float2*>(c.S->W);
    float2* rb = row_buf<float2>(c);
    for (int i = 0; i < rr; ++i)
      row_fwd_pair_l<float, LN, true>(ln(c), [&](int64_t row, int x) { return R[row * n + x]; }, W, n, n, KB32,
                                      c.tw32, pair_of(c, i), rb, tl);
    c.g.sync();
    {
      // two real columns per transform (col_pair_tau_l): QT groups of 4 column pairs
      const ColArgs A{n, K, KB32, KB32, 1, 0, 0, K};
      const int ts = tid / (4 * TPL), w = tid % (4 * TPL);
      const int QT = ((K + 1) / 2 + 3) / 4;
      const int cr = (QT + c.g.G * TPR32 - 1) / (c.g.G * TPR32);
      for (int i = 0; i < cr; ++i)
        col_pair_tau_l<float, LNT, SYM2>(lnt(c), W, W, A, c.P->pinv32, c.tw32, 0, tile_of(c, i, ts, TPR32, QT) * 4 + w % 4,
                                   reinterpret_cast<float2*>(c.smem) + min(ts, TPR32) * 4 * LST, w % 4, w / 4);
    }
    c.g.sync();
    float s = 0.0f;
    for (int i = 0; i < rr; ++i)
      row_inv_pair_l<float, LN, true>(ln(c), W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl, [&](int64_t row, int x, float v) {
        Z[row * n + x] = v;
        s += v * R[row * n + x];
      });
    return gsum(c, s);
  }

  // FP32 CG (preconditioned when pcg) on A d = R64 / ||R64|| (||R64||^2 = rn2)
  // to a relative reduction inner_tol, then U += ||R64|| d.  Returns the
  // iteration count after it.
  static __device__ __noinline__ int inner(Ctx& c, double rn2, int iters) {
    const int n = c.P->n, tid = threadIdx.x, TPL = tpl(c), tl = tid % TPL, rr = rrounds(c), max_iter = c.P->max_iter;
    const int K = kk(c), KB32 = kb32(c), TPR32 = tpr32(c), LST = lnt(c).stride_tile();
    const double* R64 = c.S->r64;
    double* U = c.P->u;
    float* X = c.S->x;
    float* R = c.S->r;
    float* Pv = c.S->p;
    float* Q = c.S->q;
    float2* W = static_cast<float2*>(c.S->W);
    float2* rb = row_buf<float2>(c);
    const ColArgs A{n, K, KB32, KB32, 1, 0, 0, K};
    const int ts = tid / (4 * TPL), w = tid % (4 * TPL);
    const int cr = (KB32 + c.g.G * TPR32 - 1) / (c.g.G * TPR32);
    const double sc = 1.0 / sqrt(rn2);
    float rf = 0.0f;
    for_own(c, [&](int64_t k) {
      const float rv = (float)(R64[k] * sc);
      R[k] = rv;
      X[k] = 0.0f;
      rf += rv * rv;
    });
    double rrv = gsum(c, rf);
    const double stop = c.P->inner_tol * c.P->inner_tol * rrv;
    const bool pcg = c.P->pcg;
    const float* Zs = pcg ? Q : R;  // the vector the direction is built from
    double rz = (pcg && rrv > stop) ? precond(c) : rrv;
    bool first = true;
    float be = 0.0f;
    while (rrv > stop && iters < max_iter) {
      for (int i = 0; i < rr; ++i)
        row_fwd_pair_l<float, LN>(
            ln(c),
            [&](int64_t row, int x) {
              const int64_t k = row * n + x;
              const float v = first ? Zs[k] : Zs[k] + be * Pv[k];
              Pv[k] = v;
              return v;
            },
            W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl);
      c.g.sync();
      for (int i = 0; i < cr; ++i)
        col_tile_l<float, LNT, SYM2>(lnt(c), W, W, A, c.P->lam32, c.tw32, 0, tile_of(c, i, ts, TPR32, KB32),
                                     reinterpret_cast<float2*>(c.smem) + min(ts, TPR32) * 4 * LST, w % 4, w / 4);
      c.g.sync();
      float pqf = 0.0f;
      for (int i = 0; i < rr; ++i)
        row_inv_pair_l<float, LN>(ln(c), W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl, [&](int64_t row, int x, float v) {
          const int64_t k = row * n + x;
          Q[k] = v;
          pqf += v * Pv[k];
        });
      const double pq = gsum(c, pqf);
      if (!(pq > 0.0) || !isfinite(pq)) break;  // inner breakdown: refine from here
      const float al = (float)(rz / pq);
      float rf1 = 0.0f;
      for_own(c, [&](int64_t k) {
        X[k] += al * Pv[k];
        const float rv = R[k] - al * Q[k];
        R[k] = rv;
        rf1 += rv * rv;
      });
      rrv = gsum(c, rf1);
      first = false;
      ++iters;
      if (!(rrv > stop)) break;
      const double rz1 = pcg ? precond(c) : rrv;
      be = (float)(rz1 / rz);
      rz = rz1;
    }
    const double s = sqrt(rn2);
    for_own(c, [&](int64_t k) { U[k] += s * (double)X[k]; });
    return iters;
  }

  // mixed-precision refinement to ||f - A u|| <= rtol ||f||
  // Geometry guard: the problem's spectrum and vectors fit its worker's slot, and its row
  // lines and column tiles (spare ones included) fit the CTA's shared memory.  The
  // same in every thread of the group; a problem that fails it is not touched and
  // reports FRAC_ECUDA.
  static __device__ bool fits(const Ctx& c) {
    const int n = c.P->n, TPL = tpl(c);
    const size_t w = (size_t)n * kb64(c) * 2 * sizeof(double2);
    const int sr = lines(c) * TPL < kThreads, s64 = tpr64(c) * 2 * TPL < kThreads, s32 = tpr32(c) * 4 * TPL < kThreads;
    const size_t rows = (size_t)(lines(c) + sr) * ln(c).stride() * sizeof(double2);
    const size_t t64 = (size_t)(tpr64(c) + s64) * 2 * lnt(c).stride_tile() * sizeof(double2);
    const size_t t32 = (size_t)(tpr32(c) + s32) * 4 * lnt(c).stride_tile() * sizeof(float2);
    return w <= c.S->w_bytes && (int64_t)n * n <= c.S->nn && rows <= c.smem_bytes && t64 <= c.smem_bytes &&
           t32 <= c.smem_bytes;
  }

  static __device__ __noinline__ void solve(Ctx& c, frac_solve_info* info) {
    if (!fits(c)) {
      if (c.g.rank == 0 && threadIdx.x == 0) *info = frac_solve_info{FRAC_ECUDA, 0, 0, c.P->pcg, INFINITY};
      return;
    }
    const double fn2 = start(c);
    const double tol2 = c.P->rtol * c.P->rtol * fn2;
    int iters = 0, outer = 0, status = FRAC_OK;
    double rn2 = 0.0;
    if (fn2 != 0.0) {
      rn2 = c.P->use_x0 ? residual(c) : fn2;  // u = 0: R64 = f, set by start()
      double prev = INFINITY;
      while (rn2 > tol2 && iters < c.P->max_iter && outer < 100) {
        iters = inner(c, rn2, iters);
        rn2 = residual(c);
        ++outer;
        if (!(rn2 < prev) && outer > 3) break;  // refinement stagnated
        prev = rn2;
      }
    }
    if (c.g.rank == 0 && threadIdx.x == 0) {
      frac_solve_info out;
      out.iters = iters;
      out.outer = outer;
      out.precond = c.P->pcg;
      out.rel_resid = fn2 > 0.0 ? sqrt(rn2 / fn2) : (fn2 == 0.0 ? 0.0 : NAN);  // NaN: non-finite f
      if (status == FRAC_OK && !(out.rel_resid <= c.P->rtol)) status = FRAC_ENOCONV;
      if (!isfinite(out.rel_resid)) status = FRAC_EINVAL;
      out.status = status;
      *info = out;
    }
  }
};

// MX: the launch holds mixed lengths.  Only then is the mixed solver part of the
// kernel: its out-of-line FFT passes in the same call graph cost the power-of-two
// solvers registers (2D batch of power-of-two lengths 51.8 -> 57.7 ms when it was
// always there), so batches without mixed lengths launch the kernel without it.
template <bool MX>
__device__ inline void solve_any(const B2Args& A, int item, const B2Slot& S, const Group g, unsigned char* smem,
                          double* red, double* slots) {
  const B2Prob& P = A.probs[item];
  frac_solve_info* info = A.info + item;
  Ctx c{&P, &S, g, P.tw32, P.tw64, smem, A.smem, red, slots, 0};
  if constexpr (MX) {
    if (P.plan.m) {  // a mixed length (uniform over the group)
      Solver<MxLine>::solve(c, info);
      return;
    }
  }
  switch (P.logm) {  // uniform over the group
#define FRAC_B2_CASE(L)                 \
  case L:                               \
    Solver<P2Line<L>>::solve(c, info);  \
    break;
    FRAC_B2_CASE(5)
    FRAC_B2_CASE(6)
    FRAC_B2_CASE(7)
    FRAC_B2_CASE(8)
    FRAC_B2_CASE(9)
    FRAC_B2_CASE(10)
#undef FRAC_B2_CASE
    default: break;
  }
}

template <bool MX>
__global__ void __launch_bounds__(kThreads, 1) k_batch2d(B2Args A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double slots[2];
  __shared__ unsigned int s_item;
  const int C = (int)__clusterSizeInBlocks(), rank = (int)__clusterRelativeBlockRank();
  const int cid = (int)(blockIdx.x / C);
  // cluster-wide problems: rank 0 takes the next one, every CTA reads it from rank 0
  while (true) {
    if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(A.next, 1u);
    cluster_sync_all();
    const unsigned int item = *static_cast<volatile unsigned int*>(__cluster_map_shared_rank((void*)&s_item, 0));
    cluster_sync_all();  // every read of rank 0's slot is done before it changes or its CTA moves on
    if (item >= (unsigned int)A.n_cluster) break;
    solve_any<MX>(A, (int)item, A.cslots[cid], Group{C, rank}, smem, red, slots);
  }
  // then one problem per CTA
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.next + 1, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    __syncthreads();
    if (item >= (unsigned int)A.n_local) break;
    solve_any<MX>(A, A.n_cluster + (int)item, A.lslots[blockIdx.x], Group{1, 0}, smem, red, slots);
  }
}


// Host helpers of the two kernel instances: MX = false is compiled in batch2d.cu,
// MX = true (with the mixed-length solver) in batch2d_mx.cu, so that no translation
// unit holds both call graphs.
template <bool MX>
int kernel_attrs(size_t smem) {
  FRAC_CUDA_TRY(cudaFuncSetAttribute(k_batch2d<MX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FRAC_CUDA_TRY(cudaFuncSetAttribute(k_batch2d<MX>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  return FRAC_OK;
}

// Clusters of size C that can be resident at once (0: C not launchable).
template <bool MX>
int kernel_active_clusters(int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, k_batch2d<MX>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

template <bool MX>
int kernel_launch(const B2Args& args, int C, int grid, size_t smem, cudaStream_t st) {
  B2Args a = args;
  a.smem = smem;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  FRAC_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch2d<MX>, a));
  return FRAC_OK;
}

// The MX = true instance (batch2d_mx.cu).
int mx_kernel_attrs(size_t smem);
int mx_kernel_active_clusters(int C, size_t smem);
int mx_kernel_launch(const B2Args& a, int C, int grid, size_t smem, cudaStream_t st);

}  // namespace b2
}  // namespace frac
