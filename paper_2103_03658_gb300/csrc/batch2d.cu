// Batched 2D fractional Poisson solves in one persistent launch.
//
// A batch of problems of different sizes, alpha, basis degree and lambda
// (each its own operator of Eq. (2D-scheme), A = -c T(a) SPD) is solved by
// one kernel launch: a grid of thread-block clusters, one 512-thread CTA per
// SM, takes problems from two queues ordered largest first.  A problem of the
// cluster queue is solved by a whole cluster: its CTAs split the row pairs
// and column tiles of every FFT pass (passes.cuh), the spectrum lives in
// global memory (L2 for these sizes), the passes are separated by cluster
// barriers, and the CG scalars are reduced through distributed shared memory
// in rank order, so every CTA of the cluster holds the same values and takes
// the same branches.  When that queue is empty every CTA takes problems of
// the local queue and solves each alone.  The cluster size and which FFT
// lengths go cluster-wide are chosen by an autotuner that times each size
// class on one of its problems (timings cached per device and FFT length)
// and simulates the queue on those timings.
//
// Each problem runs mixed-precision iterative refinement inside the kernel:
// r = f - A u with the FP64 apply, FP32 CG on A d = r / ||r|| to a relative
// reduction inner_tol, u += ||r|| d, until ||f - A u|| <= rtol ||f||.  Every
// vector entry is read and written by the same thread in every phase (the
// row-pair mapping of the row passes), so only the spectrum crosses threads.
// No thread ever waits on a flag: the only cross-CTA waits are the hardware
// cluster barriers, reached the same number of times by every CTA.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "apply.cuh"
#include "batch2d.cuh"
#include "passes.cuh"
#include "prof.cuh"

namespace frac {
namespace {

using namespace fft;

constexpr int kThreads = 512;

struct B2Prob {
  const double* f;
  double* u;
  const float* lam32;
  const double* lam64;
  const float* pinv32;  // tau preconditioner symbol (pcg)
  int n, logm, max_iter, use_x0, pcg;
  double rtol, inner_tol;
};

// Scratch of one worker (a cluster or a CTA), sized for its largest problem.
struct B2Slot {
  void* W;  // spectrum, FP64 layout n ceil(K/2) 2 complex doubles; the FP32 passes use its front
  float *x, *r, *p, *q;
  double* r64;
};

struct B2Args {
  const B2Prob* probs;
  frac_solve_info* info;  // per problem
  int n_cluster, n_local; // probs[0, n_cluster) cluster-wide, then n_local CTA-local
  unsigned int* next;     // queue heads: [0] cluster, [1] local
  const B2Slot* cslots;   // per cluster
  const B2Slot* lslots;   // per CTA
  const float2* tw32[kBatch2dMaxLog + 1];
  const double2* tw64[kBatch2dMaxLog + 1];
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
__device__ double group_sum(double v, const Group& g, double* red, double* slots, int& parity) {
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
  double* red;
  double* slots;
  int parity;
};

template <int LOGM>
struct Solver {
  static constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LINES = kThreads / TPL;
  static constexpr int LS = line_stride(LOGM), LST = line_stride_tile(LOGM);
  static constexpr int K = M / 2 + 1, KB32 = (K + 3) / 4, KB64 = (K + 1) / 2;
  static constexpr int TPR32 = kThreads / (4 * TPL), TPR64 = kThreads / (2 * TPL);  // column tiles per CTA round

  static __device__ __forceinline__ int rrounds(const Ctx& c) {
    const int npairs = (c.P->n + 1) / 2;
    return (npairs + c.g.G * LINES - 1) / (c.g.G * LINES);
  }
  static __device__ __forceinline__ int64_t pair_of(const Ctx& c, int i) {
    return ((int64_t)i * c.g.G + c.g.rank) * LINES + threadIdx.x / TPL;
  }
  // the points of this thread: those its row passes read and write
  template <typename Fn>
  static __device__ __forceinline__ void for_own(const Ctx& c, Fn fn) {
    const int n = c.P->n, tl = threadIdx.x % TPL, rr = rrounds(c);
    for (int i = 0; i < rr; ++i) {
      const int64_t r0 = 2 * pair_of(c, i);
#pragma unroll
      for (int e = 0; e < E / 2; ++e) {
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
    const int n = c.P->n, tid = threadIdx.x, tl = tid % TPL, rr = rrounds(c);
    const double* F = c.P->f;
    const double* U = c.P->u;
    double* R64 = c.S->r64;
    double2* W = static_cast<double2*>(c.S->W);
    double2* rb = reinterpret_cast<double2*>(c.smem) + (tid / TPL) * LS;
    for (int i = 0; i < rr; ++i)
      row_fwd_pair<double, LOGM>([&](int64_t row, int x) { return U[row * n + x]; }, W, n, n, KB64, c.tw64,
                                 pair_of(c, i), rb, tl);
    c.g.sync();
    {
      const ColArgs A{n, K, KB64, KB64, 1, 0, 0, K};
      const int ts = tid / (2 * TPL), w = tid % (2 * TPL);
      const int cr = (KB64 + c.g.G * TPR64 - 1) / (c.g.G * TPR64);
      for (int i = 0; i < cr; ++i)
        col_tile<double, LOGM, SYM2>(W, W, A, c.P->lam64, c.tw64, 0, ((int64_t)i * c.g.G + c.g.rank) * TPR64 + ts,
                                     reinterpret_cast<double2*>(c.smem) + ts * 2 * LST, w % 2, w / 2);
    }
    c.g.sync();
    double part = 0.0;
    for (int i = 0; i < rr; ++i)
      row_inv_pair<double, LOGM>(W, n, n, KB64, c.tw64, pair_of(c, i), rb, tl, [&](int64_t row, int x, double v) {
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
    const int n = c.P->n, tid = threadIdx.x, tl = tid % TPL, rr = rrounds(c);
    const float* R = c.S->r;
    float* Z = c.S->q;
    float2* W = static_cast<float2*>(c.S->W);
    float2* rb = reinterpret_cast<float2*>(c.smem) + (tid / TPL) * LS;
    for (int i = 0; i < rr; ++i)
      row_fwd_pair<float, LOGM, true>([&](int64_t row, int x) { return R[row * n + x]; }, W, n, n, KB32, c.tw32,
                                      pair_of(c, i), rb, tl);
    c.g.sync();
    {
      const ColArgs A{n, K, KB32, KB32, 1, 0, 0, K};
      const int ts = tid / (4 * TPL), w = tid % (4 * TPL);
      const int cr = (KB32 + c.g.G * TPR32 - 1) / (c.g.G * TPR32);
      for (int i = 0; i < cr; ++i)
        col_tile<float, LOGM, SYM2, true>(W, W, A, c.P->pinv32, c.tw32, 0,
                                          ((int64_t)i * c.g.G + c.g.rank) * TPR32 + ts,
                                          reinterpret_cast<float2*>(c.smem) + ts * 4 * LST, w % 4, w / 4);
    }
    c.g.sync();
    float s = 0.0f;
    for (int i = 0; i < rr; ++i)
      row_inv_pair<float, LOGM, true>(W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl, [&](int64_t row, int x, float v) {
        Z[row * n + x] = v;
        s += v * R[row * n + x];
      });
    return gsum(c, s);
  }

  // FP32 CG (preconditioned when pcg) on A d = R64 / ||R64|| (||R64||^2 = rn2)
  // to a relative reduction inner_tol, then U += ||R64|| d.  Returns the
  // iteration count after it.
  static __device__ __noinline__ int inner(Ctx& c, double rn2, int iters) {
    const int n = c.P->n, tid = threadIdx.x, tl = tid % TPL, rr = rrounds(c), max_iter = c.P->max_iter;
    const double* R64 = c.S->r64;
    double* U = c.P->u;
    float* X = c.S->x;
    float* R = c.S->r;
    float* Pv = c.S->p;
    float* Q = c.S->q;
    float2* W = static_cast<float2*>(c.S->W);
    float2* rb = reinterpret_cast<float2*>(c.smem) + (tid / TPL) * LS;
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
        row_fwd_pair<float, LOGM>(
            [&](int64_t row, int x) {
              const int64_t k = row * n + x;
              const float v = first ? Zs[k] : Zs[k] + be * Pv[k];
              Pv[k] = v;
              return v;
            },
            W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl);
      c.g.sync();
      for (int i = 0; i < cr; ++i)
        col_tile<float, LOGM, SYM2>(W, W, A, c.P->lam32, c.tw32, 0, ((int64_t)i * c.g.G + c.g.rank) * TPR32 + ts,
                                    reinterpret_cast<float2*>(c.smem) + ts * 4 * LST, w % 4, w / 4);
      c.g.sync();
      float pqf = 0.0f;
      for (int i = 0; i < rr; ++i)
        row_inv_pair<float, LOGM>(W, n, n, KB32, c.tw32, pair_of(c, i), rb, tl, [&](int64_t row, int x, float v) {
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
  static __device__ __noinline__ void solve(Ctx& c, frac_solve_info* info) {
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

__device__ void solve_any(const B2Args& A, int item, const B2Slot& S, const Group g, unsigned char* smem,
                          double* red, double* slots) {
  const B2Prob& P = A.probs[item];
  frac_solve_info* info = A.info + item;
  Ctx c{&P, &S, g, nullptr, nullptr, smem, red, slots, 0};
  switch (P.logm) {  // uniform over the group
#define FRAC_B2_CASE(L)       \
  case L:                     \
    c.tw32 = A.tw32[L];       \
    c.tw64 = A.tw64[L];       \
    Solver<L>::solve(c, info); \
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
    solve_any(A, (int)item, A.cslots[cid], Group{C, rank}, smem, red, slots);
  }
  // then one problem per CTA
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.next + 1, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    __syncthreads();
    if (item >= (unsigned int)A.n_local) break;
    solve_any(A, A.n_cluster + (int)item, A.lslots[blockIdx.x], Group{1, 0}, smem, red, slots);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

constexpr int kProbeIters = 24;
constexpr int kClusterSizes[] = {1, 2, 4, 8, 16};
constexpr int kNumSizes = 5;

size_t smem_bytes(int logm) {
  const int tplv = tpl(logm), lines = kThreads / tplv;
  const size_t rows = (size_t)lines * line_stride(logm) * sizeof(double2);
  const size_t cols = (size_t)(kThreads / tplv) * line_stride_tile(logm) * sizeof(double2);
  return std::max(rows, cols);
}

size_t slot_bytes(int n, int logm) {
  const int64_t K = (int64_t(1) << logm) / 2 + 1, KB64 = (K + 1) / 2, nn = (int64_t)n * n;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al((size_t)n * KB64 * 2 * sizeof(double2)) + 4 * al(nn * sizeof(float)) + al(nn * sizeof(double));
}

B2Slot carve(unsigned char* base, int n, int logm) {
  const int64_t K = (int64_t(1) << logm) / 2 + 1, KB64 = (K + 1) / 2, nn = (int64_t)n * n;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  B2Slot s;
  s.W = base;
  base += al((size_t)n * KB64 * 2 * sizeof(double2));
  s.x = reinterpret_cast<float*>(base);
  base += al(nn * sizeof(float));
  s.r = reinterpret_cast<float*>(base);
  base += al(nn * sizeof(float));
  s.p = reinterpret_cast<float*>(base);
  base += al(nn * sizeof(float));
  s.q = reinterpret_cast<float*>(base);
  base += al(nn * sizeof(float));
  s.r64 = reinterpret_cast<double*>(base);
  return s;
}

struct DevBuf {
  cudaStream_t st;
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <typename P>
  int get(P** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) return record_cuda_error(e, __FILE__, __LINE__, "cudaMallocAsync");
    ptrs.push_back(p);
    *out = static_cast<P*>(p);
    return FRAC_OK;
  }
};

int configure_kernel() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, 0);
  if (!done[dev]) {
    size_t mx = 0;
    for (int l = kBatch2dMinLog; l <= kBatch2dMaxLog; ++l) mx = std::max(mx, smem_bytes(l));
    FRAC_CUDA_TRY(cudaFuncSetAttribute(k_batch2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    FRAC_CUDA_TRY(cudaFuncSetAttribute(k_batch2d, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    done[dev] = 1;
  }
  return FRAC_OK;
}

// Clusters of size C that can be resident at once (0: C not launchable).
int active_clusters(int C, size_t smem) {
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
  if (cudaOccupancyMaxActiveClusters(&num, k_batch2d, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

int launch(const B2Args& a, int C, int grid, size_t smem, cudaStream_t st) {
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
  FRAC_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch2d, a));
  return FRAC_OK;
}

void fill_twiddles(B2Args& a) {
  for (int l = 0; l <= kBatch2dMaxLog; ++l) {
    a.tw32[l] = l >= kBatch2dMinLog ? twiddles32(l) : nullptr;
    a.tw64[l] = l >= kBatch2dMinLog ? twiddles64(l) : nullptr;
  }
}

// Autotuner timings: microseconds per CG iteration of a class's probe problem
// (size n_probe) with one CTA, and with one cluster of each size.
struct ClassTiming {
  int n_probe = 0;
  double t[kNumSizes] = {-1, -1, -1, -1, -1};
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, ClassTiming> g_tune;  // (device, logm)

B2Prob make_prob(const frac_op* op, const double* f, double* u, const frac_solve_opts* o) {
  B2Prob p;
  p.f = f;
  p.u = u;
  p.lam32 = op->lam32;
  p.lam64 = op->lam64;
  p.pinv32 = op->pinv32;
  p.pcg = (o->precond == FRAC_PRECOND_TAU && op->precond_ok) ? 1 : 0;
  p.n = (int)op->n;
  p.logm = op->logm;
  p.max_iter = o->max_iter;
  p.use_x0 = o->use_x0 ? 1 : 0;
  p.rtol = o->rtol;
  p.inner_tol = o->inner_tol > 0.0 ? o->inner_tol : auto_inner_tol(op, o->rtol);
  return p;
}

// Times kProbeIters CG iterations of (op, f) alone, on one CTA and on one
// cluster of each launchable size; the solution goes to scratch.
int probe_class(const frac_op* op, const double* f, cudaStream_t st, ClassTiming* out) {
  const int logm = op->logm, n = (int)op->n;
  const size_t smem = smem_bytes(logm);
  DevBuf b{st, {}};
  double* u;
  B2Prob* dp;
  B2Slot* ds;
  frac_solve_info* di;
  unsigned int* next;
  unsigned char* scratch;
  FRAC_TRY(b.get(&u, (size_t)n * n * sizeof(double)));
  FRAC_TRY(b.get(&dp, sizeof(B2Prob)));
  FRAC_TRY(b.get(&ds, sizeof(B2Slot)));
  FRAC_TRY(b.get(&di, sizeof(frac_solve_info)));
  FRAC_TRY(b.get(&next, 2 * sizeof(unsigned int)));
  FRAC_TRY(b.get(&scratch, slot_bytes(n, logm)));
  frac_solve_opts o{0.0, kProbeIters, FRAC_MIXED_IR, 0, FRAC_PRECOND_TAU, 1e-30};  // exactly kProbeIters iterations
  B2Prob hp = make_prob(op, f, u, &o);
  B2Slot hs = carve(scratch, n, logm);
  FRAC_CUDA_TRY(cudaMemcpyAsync(dp, &hp, sizeof(hp), cudaMemcpyHostToDevice, st));
  FRAC_CUDA_TRY(cudaMemcpyAsync(ds, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  cudaEvent_t e0, e1;
  FRAC_CUDA_TRY(cudaEventCreate(&e0));
  FRAC_CUDA_TRY(cudaEventCreate(&e1));
  int rc = FRAC_OK;
  out->n_probe = n;
  for (int i = 0; i < kNumSizes && rc == FRAC_OK; ++i) {
    const int C = kClusterSizes[i];
    if (active_clusters(C, smem) < 1) continue;
    B2Args a = {};
    a.probs = dp;
    a.info = di;
    a.n_cluster = C > 1 ? 1 : 0;
    a.n_local = C > 1 ? 0 : 1;
    a.next = next;
    a.cslots = ds;
    a.lslots = ds;
    fill_twiddles(a);
    float best = 1e30f;
    for (int rep = 0; rep < 2 && rc == FRAC_OK; ++rep) {  // the first run also loads the code
      if (cudaMemsetAsync(next, 0, 2 * sizeof(unsigned int), st) != cudaSuccess ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        rc = FRAC_ECUDA;
        break;
      }
      rc = launch(a, C, C, smem, st);
      if (rc != FRAC_OK) break;
      float ms = 0.0f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = FRAC_ECUDA;
        break;
      }
      best = std::min(best, ms);
    }
    if (rc == FRAC_OK) out->t[i] = 1e3 * best / kProbeIters;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return settle(rc);
}

// Relative cost model of one problem: plain CG iterations ~ n^(alpha/2)
// (condition number ~ n^alpha); with the tau preconditioner they hardly grow
// (about 5-15 to 1e-10 in 2D); per-iteration time of its class measured at
// n_probe, half of it proportional to the number of rows.
double est_iters(int n, double alpha, bool pcg) {
  return pcg ? 10.0 + std::log2((double)n) : 20.0 + 6.0 * std::pow((double)n, 0.5 * alpha);
}

struct Item {
  int64_t idx;  // problem index in the caller's arrays
  int logm, n;
  double alpha;
  bool pcg;
};

// Makespan of the two queues on `ncl` clusters of C CTAs, classes with logm >= cut cluster-wide.
double simulate(const std::vector<Item>& items, const std::map<int, ClassTiming>& tm, int si, int ncl, int cut,
                std::vector<const Item*>* cl_out, std::vector<const Item*>* lo_out) {
  const int C = kClusterSizes[si];
  std::vector<std::pair<double, const Item*>> cl, lo;
  for (const Item& it : items) {
    const ClassTiming& t = tm.at(it.logm);
    const double scale = 0.5 + 0.5 * (double)it.n / t.n_probe;
    const bool wide = C > 1 && it.logm >= cut && t.t[si] > 0;
    const double per = wide ? t.t[si] : t.t[0];
    (wide ? cl : lo).emplace_back(est_iters(it.n, it.alpha, it.pcg) * per * scale, &it);
  }
  auto desc = [](const std::pair<double, const Item*>& a, const std::pair<double, const Item*>& b) {
    return a.first > b.first;
  };
  std::sort(cl.begin(), cl.end(), desc);
  std::sort(lo.begin(), lo.end(), desc);
  std::vector<double> free_cl(ncl, 0.0);
  for (auto& c : cl) {
    auto m = std::min_element(free_cl.begin(), free_cl.end());
    *m += c.first;
  }
  std::vector<double> free_cta;
  for (double t0 : free_cl)
    for (int r = 0; r < C; ++r) free_cta.push_back(t0);
  for (auto& c : lo) {
    auto m = std::min_element(free_cta.begin(), free_cta.end());
    *m += c.first;
  }
  double span = 0.0;
  for (double t0 : free_cta) span = std::max(span, t0);
  if (cl_out) {
    cl_out->clear();
    lo_out->clear();
    for (auto& c : cl) cl_out->push_back(c.second);
    for (auto& c : lo) lo_out->push_back(c.second);
  }
  return span;
}

}  // namespace

int batch2d_prepare(int64_t count, const frac_op* const* ops, const double* const* f, const int64_t* idx,
                    cudaStream_t st) {
  if (count <= 0) return FRAC_OK;
  FRAC_TRY(configure_kernel());
  for (int l = kBatch2dMinLog; l <= kBatch2dMaxLog; ++l) FRAC_TRY(prepare_twiddles(l));
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::map<int, int64_t> rep;  // logm -> largest problem of that class
  for (int64_t t = 0; t < count; ++t) {
    const frac_op* op = ops[idx[t]];
    auto it = rep.find(op->logm);
    if (it == rep.end() || ops[it->second]->n < op->n) rep[op->logm] = idx[t];
  }
  for (auto& kv : rep) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      if (g_tune.count({dev, kv.first})) continue;
    }
    ClassTiming t;
    prof::Scope ps("batch2d_autotune", st);
    FRAC_TRY(probe_class(ops[kv.second], f[kv.second], st, &t));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{dev, kv.first}] = t;
  }
  return FRAC_OK;
}

bool batch2d_eligible(const frac_op* op, const frac_solve_opts* opts) {
  return op->prob.d == 2 && op->square && opts->precision == FRAC_MIXED_IR && op->logm >= kBatch2dMinLog &&
         op->logm <= kBatch2dMaxLog;
}

int solve_batch_2d(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                   const frac_solve_opts* opts, const int64_t* idx, cudaStream_t st, frac_batch_plan* plan_out,
                   int pin_size, int pin_cut, BatchPending* pend) {
  if (count <= 0) return FRAC_OK;
  FRAC_TRY(configure_kernel());
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<Item> items;
  std::map<int, int64_t> rep;  // logm -> largest problem of that class
  for (int64_t t = 0; t < count; ++t) {
    const frac_op* op = ops[idx[t]];
    items.push_back(Item{idx[t], op->logm, (int)op->n, op->prob.alpha,
                         opts->precond == FRAC_PRECOND_TAU && op->precond_ok != 0});
    auto it = rep.find(op->logm);
    if (it == rep.end() || ops[it->second]->n < op->n) rep[op->logm] = idx[t];
  }
  for (int l = kBatch2dMinLog; l <= kBatch2dMaxLog; ++l) FRAC_TRY(prepare_twiddles(l));
  // timings of every class present (measured once per device and FFT length)
  std::map<int, ClassTiming> tm;
  for (auto& kv : rep) {
    ClassTiming t;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find({dev, kv.first});
      if (it != g_tune.end()) {
        t = it->second;
        have = true;
      }
    }
    if (!have) {
      prof::Scope ps("batch2d_autotune", st);
      FRAC_TRY(probe_class(ops[kv.second], f[kv.second], st, &t));
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[{dev, kv.first}] = t;
    }
    if (!(t.t[0] > 0)) return FRAC_ECUDA;
    tm[kv.first] = t;
  }
  // plan: cluster size and the first cluster-wide FFT length, by simulated makespan
  size_t smem = 0;
  for (auto& kv : rep) smem = std::max(smem, smem_bytes(kv.first));
  int best_si = 0, best_cut = kBatch2dMaxLog + 1, best_ncl = 0;
  double best = INFINITY;
  for (int si = 0; si < kNumSizes; ++si) {
    const int C = kClusterSizes[si];
    if (pin_size > 0 && C != pin_size) continue;
    const int ncl = active_clusters(C, smem);
    if (ncl < 1) continue;
    for (int cut = kBatch2dMinLog; cut <= kBatch2dMaxLog + 1; ++cut) {
      if (C == 1 && cut <= kBatch2dMaxLog) continue;
      if (pin_size > 0 && C > 1 && cut != pin_cut) continue;
      const double span = simulate(items, tm, si, ncl, cut, nullptr, nullptr);
      if (span < best) {
        best = span;
        best_si = si;
        best_cut = cut;
        best_ncl = ncl;
      }
    }
  }
  if (best_ncl < 1) return pin_size > 0 ? FRAC_ENOTSUP : FRAC_ECUDA;
  const int C = kClusterSizes[best_si];
  std::vector<const Item*> cl, lo;
  simulate(items, tm, best_si, best_ncl, best_cut, &cl, &lo);
  if (plan_out) {
    plan_out->cluster_size = C;
    plan_out->clusters = best_ncl;
    plan_out->first_cluster_logm = best_cut;
    plan_out->cluster_problems = (int)cl.size();
    plan_out->local_problems = (int)lo.size();
    plan_out->predicted_ms = best * 1e-3;
  }

  // device records: problems in queue order, scratch per cluster and per CTA
  const int grid = best_ncl * C;
  int ncl_max = 0, nlo_max = 0, lcl = kBatch2dMinLog, llo = kBatch2dMinLog;
  for (const Item* it : cl)
    if (it->n > ncl_max) ncl_max = it->n, lcl = it->logm;
  for (const Item* it : lo)
    if (it->n > nlo_max) nlo_max = it->n, llo = it->logm;
  const size_t cslot = cl.empty() ? 0 : slot_bytes(ncl_max, lcl), lslot = lo.empty() ? 0 : slot_bytes(nlo_max, llo);
  const int n_cslots = cl.empty() ? 0 : best_ncl, n_lslots = lo.empty() ? 0 : grid;
  pend->st = st;
  B2Prob* dp;
  B2Slot* ds;
  unsigned int* next;
  unsigned char* scratch;
  FRAC_TRY(pend->alloc(&dp, count * sizeof(B2Prob)));
  FRAC_TRY(pend->alloc(&ds, (size_t)(n_cslots + n_lslots + 1) * sizeof(B2Slot)));
  FRAC_TRY(pend->alloc(&pend->dinfo, count * sizeof(frac_solve_info)));
  FRAC_TRY(pend->alloc(&next, 2 * sizeof(unsigned int)));
  FRAC_TRY(pend->alloc(&scratch, (size_t)n_cslots * cslot + (size_t)n_lslots * lslot));
  std::vector<B2Prob> hp;
  for (const Item* it : cl) {
    hp.push_back(make_prob(ops[it->idx], f[it->idx], u[it->idx], opts));
    pend->order.push_back(it->idx);
  }
  for (const Item* it : lo) {
    hp.push_back(make_prob(ops[it->idx], f[it->idx], u[it->idx], opts));
    pend->order.push_back(it->idx);
  }
  std::vector<B2Slot> hs;
  for (int i = 0; i < n_cslots; ++i) hs.push_back(carve(scratch + (size_t)i * cslot, ncl_max, lcl));
  for (int i = 0; i < n_lslots; ++i)
    hs.push_back(carve(scratch + (size_t)n_cslots * cslot + (size_t)i * lslot, nlo_max, llo));
  if (hs.empty()) hs.push_back(B2Slot{});
  // pinned staging kept until collect(), so the uploads do not wait for the stream
  const size_t hb = hp.size() * sizeof(B2Prob), sb = hs.size() * sizeof(B2Slot);
  unsigned char* stage = nullptr;
  FRAC_CUDA_TRY(cudaMallocHost(&stage, hb + sb));
  pend->pinned = stage;
  std::memcpy(stage, hp.data(), hb);
  std::memcpy(stage + hb, hs.data(), sb);
  FRAC_CUDA_TRY(cudaMemcpyAsync(dp, stage, hb, cudaMemcpyHostToDevice, st));
  FRAC_CUDA_TRY(cudaMemcpyAsync(ds, stage + hb, sb, cudaMemcpyHostToDevice, st));
  FRAC_CUDA_TRY(cudaMemsetAsync(next, 0, 2 * sizeof(unsigned int), st));
  B2Args a = {};
  a.probs = dp;
  a.info = pend->dinfo;
  a.n_cluster = (int)cl.size();
  a.n_local = (int)lo.size();
  a.next = next;
  a.cslots = ds;
  a.lslots = ds + n_cslots;
  fill_twiddles(a);
  prof::Scope ps("batch2d", st);
  return launch(a, C, grid, smem, st);
}

}  // namespace frac
