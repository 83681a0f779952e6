// Conjugate-gradient solves of A u = f (A symmetric positive definite; the
// paper asks for an FFT-based fast solver for the Toeplitz system without
// naming one, Example 3.2.3).
//
//   FRAC_PLAIN_F64: CG with the FP64 FFT apply.
//   FRAC_MIXED_IR : iterative refinement: r64 = f - A64 u (FP64 apply), the
//                   correction from CG with the FP32 FFT apply on r64 / ||r64||
//                   to a relative reduction inner_tol, u += ||r64|| d, until the
//                   true FP64 residual meets rtol.
//
// Every CG scalar lives on the device (struct CGState); the host launches
// iterations in chunks and reads the state back between chunks; once a
// kernel marks the state done, the remaining launches of the chunk are no-ops
// for x and r.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <thread>
#include <map>
#include <vector>

#include "apply.cuh"
#include "solve1d.cuh"

namespace frac {


constexpr int kRedBlocks = 1024;  // partial-sum slots of the two-stage reductions
constexpr int kTB = 256;

// ---- reductions -----------------------------------------------------------

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// partial[b] = sum over this block's grid-stride share of a[i] * b[i]
// (each thread accumulates in T, the block in FP64)
template <typename T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* __restrict__ partial,
                      const CGState* st) {
  __shared__ double sh[32];
  if (st && st->done) return;
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__device__ double sum_partials(const double* __restrict__ partial, int np, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += partial[i];
  return block_sum(v, sh);
}

// start: rr = sum partials (of r.r), tol2 = tol^2 * rr_ref (rr_ref < 0: use rr);
// pcg: preconditioned (rz and beta come from the preconditioner pass that
// follows), else rz = rr
__global__ void k_cg_start(const double* __restrict__ partial, int np, CGState* st, double tol, double rr_ref,
                           int maxit, int pcg) {
  __shared__ double sh[32];
  double rr = sum_partials(partial, np, sh);
  if (threadIdx.x == 0) {
    st->rr = rr;
    st->rz = pcg ? 0.0 : rr;
    st->pcg = pcg;
    st->tol2 = tol * tol * (rr_ref < 0.0 ? rr : rr_ref);
    st->it = 0;
    st->maxit = maxit;
    st->status = FRAC_OK;
    st->done = (rr <= st->tol2 || rr == 0.0) ? 1 : 0;
    st->alpha = st->beta = st->pq = 0.0;
    st->count_pq = st->count_rr = st->count_rz = 0;
  }
}

// Fused update (d >= 2): x += alpha p, r -= alpha q, per-block r.r partials;
// the last block sums them in index order and sets rr, the iteration count,
// the stop flag and (plain CG) beta and rz = rr.
template <typename T>
__global__ void k_cg_update_fused(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                  const T* __restrict__ q, int64_t n, double* __restrict__ partial, CGState* st) {
  __shared__ double red[32];
  __shared__ bool last;
  if (st->done) return;
  const T al = (T)st->alpha;
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    T ri = r[i] - al * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = tot;
    __threadfence();
    last = atomicAdd(&st->count_rr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sacc = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) sacc += __ldcg(partial + i);
  __syncthreads();
  const double rr = block_sum(sacc, red);
  if (threadIdx.x == 0) {
    st->count_rr = 0;
    if (!st->pcg) {
      st->beta = rr / st->rr;
      st->rz = rr;
    }
    st->rr = rr;
    st->it += 1;
    if (!isfinite(rr)) {
      st->status = FRAC_EBREAKDOWN;
      st->done = 1;
    } else if (rr <= st->tol2) {
      st->done = 1;
    } else if (st->it >= st->maxit) {
      st->status = FRAC_ENOCONV;
      st->done = 1;
    }
  }
}

// ---- elementwise helpers --------------------------------------------------

// r = f - Ay; partial r.r (all FP64)
__global__ void k_residual(const double* __restrict__ f, const double* __restrict__ Ay, double* __restrict__ r,
                           int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = f[i] - Ay[i];
    r[i] = v;
    acc += v * v;
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_to(const double* __restrict__ partial, int np, double* out) {
  __shared__ double sh[32];
  double s = sum_partials(partial, np, sh);
  if (threadIdx.x == 0) *out = s;
}

// r32 = r64 * s (s = 1 / ||r64||, read from device), x32 = 0, p32 = r32
__global__ void k_ir_scale_down(const double* __restrict__ r64, const double* __restrict__ nrm2, float* __restrict__ r32,
                                float* __restrict__ p32, float* __restrict__ x32, int64_t n) {
  const double s = 1.0 / sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = (float)(r64[i] * s);
    r32[i] = v;
    p32[i] = v;
    x32[i] = 0.0f;
  }
}

// u += ||r64|| * d32
__global__ void k_ir_correct(double* __restrict__ u, const float* __restrict__ d32, const double* __restrict__ nrm2,
                             int64_t n) {
  const double s = sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] += s * (double)d32[i];
}

template <typename T>
__global__ void k_copy2(const T* __restrict__ a, T* __restrict__ b, T* __restrict__ c, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    b[i] = a[i];
    c[i] = a[i];
  }
}

// ---- host drivers ---------------------------------------------------------

static int red_blocks(int64_t n) {
  int64_t b = (n + kTB * 4 - 1) / (kTB * 4);
  if (b < 1) b = 1;
  if (b > kRedBlocks) b = kRedBlocks;
  return (int)b;
}

struct Ws {
  cudaStream_t st;
  std::vector<void*> ptrs;
  ~Ws() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <typename P>
  int get(P** out, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) return record_cuda_error(e, __FILE__, __LINE__, "cudaMallocAsync");
    ptrs.push_back(p);
    *out = (P*)p;
    return FRAC_OK;
  }
};

// Library stream used for graph replay (the caller's stream may be the legacy
// default stream, which cannot be captured); fenced to the caller's stream with events.
static cudaStream_t graph_stream() {
  static std::mutex mu;
  static std::vector<cudaStream_t> per_dev;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1, nullptr);
  if (!per_dev[dev]) cudaStreamCreateWithFlags(&per_dev[dev], cudaStreamNonBlocking);
  return per_dev[dev];
}

// CG iterations on A_T x = b for d >= 2, fused kernels, run as a CUDA graph whose
// body (one iteration) sits in a device-side WHILE node: the loop guard kernel at
// the end of the body keeps it going while the state is not done, for at most
// kLoopTrips iterations per graph launch (so every launch ends by construction;
// the host relaunches while the state is not done).  Captured on first use, kept
// in *exec for later calls with the same buffers.  On entry r = b - A x, p holds
// any finite values and the state was set by k_cg_start (beta = 0) and,
// preconditioned (z != nullptr), by cg_precond_start.
constexpr int kLoopTrips = 256;

__global__ void k_loop_guard(CGState* st, cudaGraphConditionalHandle h) {
  const int t = ++st->trips;
  cudaGraphSetConditional(h, (!st->done && t < kLoopTrips) ? 1u : 0u);
}

// One (P)CG iteration: q = A p with p = (z or r) + beta p fused in, the x/r
// update, and (z != nullptr) the preconditioner pass z = P r that sets beta.
template <typename T>
static int cg_iteration(const frac_op* op, T* x, T* r, T* p, T* q, T* z, void* apply_ws, CGState* dst,
                        double* part_inv, double* part_upd, cudaStream_t s) {
  const int64_t nd = op->nd;
  FRAC_TRY(apply_cg_t<T>(op, p, z ? z : r, q, apply_ws, dst, part_inv, s));
  k_cg_update_fused<T><<<red_blocks(nd), kTB, 0, s>>>(x, r, p, q, nd, part_upd, dst);
  FRAC_CUDA_TRY(cudaGetLastError());
  if (z) FRAC_TRY(precond_cg_t<T>(op, r, z, apply_ws, dst, part_inv, s));
  return FRAC_OK;
}

// After k_cg_start(pcg = 1): p = 0 and the first z = P r (rz, beta = 0).
template <typename T>
static int cg_precond_start(const frac_op* op, T* r, T* p, T* z, void* apply_ws, CGState* dst, double* part_inv,
                            cudaStream_t s) {
  FRAC_CUDA_TRY(cudaMemsetAsync(p, 0, op->nd * sizeof(T), s));
  return precond_cg_t<T>(op, r, z, apply_ws, dst, part_inv, s);
}

// Build the looping CG graph: [WHILE (condition set by k_loop_guard) { one iteration; k_loop_guard }].
template <typename T>
static int capture_cg_loop(const frac_op* op, T* x, T* r, T* p, T* q, T* z, void* apply_ws, CGState* dst,
                           double* part_inv, double* part_upd, cudaStream_t s, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  FRAC_CUDA_TRY(cudaGraphCreate(&g, 0));
  struct GFree {
    cudaGraph_t g;
    ~GFree() { cudaGraphDestroy(g); }
  } gf{g};
  cudaGraphConditionalHandle h;
  FRAC_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  FRAC_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  FRAC_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int st = cg_iteration<T>(op, x, r, p, q, z, apply_ws, dst, part_inv, part_upd, s);
  if (st == FRAC_OK) {
    k_loop_guard<<<1, 1, 0, s>>>(dst, h);
    if (cudaPeekAtLastError() != cudaSuccess) st = FRAC_ECUDA;
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &captured);
  if (st != FRAC_OK) return st;
  FRAC_CUDA_TRY(e);
  FRAC_CUDA_TRY(cudaGraphInstantiate(exec, g, 0));
  return FRAC_OK;
}

// One launch of the looping CG graph (at most kLoopTrips iterations).
static int launch_cg_loop(cudaGraphExec_t exec, CGState* dst, cudaStream_t s) {
  FRAC_CUDA_TRY(cudaMemsetAsync(&dst->trips, 0, sizeof(int), s));
  FRAC_CUDA_TRY(cudaGraphLaunch(exec, s));
  return FRAC_OK;
}

template <typename T>
static int cg_run_fused(const frac_op* op, T* x, T* r, T* p, T* q, T* z, void* apply_ws, CGState* dst, CGState* hst,
                        double* part_inv, double* part_upd, cudaGraphExec_t* exec, int* iters_total,
                        cudaStream_t caller) {
  cudaStream_t gs = graph_stream();
  if (!gs) return FRAC_ECUDA;
  cudaEvent_t ev;
  FRAC_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  struct EvFree {
    cudaEvent_t e;
    ~EvFree() { cudaEventDestroy(e); }
  } evf{ev};
  FRAC_CUDA_TRY(cudaEventRecord(ev, caller));
  FRAC_CUDA_TRY(cudaStreamWaitEvent(gs, ev, 0));
  if (!*exec) {
    // one plain iteration first: sets kernel attributes outside the capture
    FRAC_TRY(cg_iteration<T>(op, x, r, p, q, z, apply_ws, dst, part_inv, part_upd, gs));
    FRAC_TRY(capture_cg_loop<T>(op, x, r, p, q, z, apply_ws, dst, part_inv, part_upd, gs, exec));
  }
  for (;;) {
    FRAC_CUDA_TRY(cudaMemcpyAsync(hst, dst, sizeof(CGState), cudaMemcpyDeviceToHost, gs));
    FRAC_CUDA_TRY(cudaStreamSynchronize(gs));
    if (hst->done) break;
    FRAC_TRY(launch_cg_loop(*exec, dst, gs));
  }
  FRAC_CUDA_TRY(cudaEventRecord(ev, gs));
  FRAC_CUDA_TRY(cudaStreamWaitEvent(caller, ev, 0));
  *iters_total += hst->it;
  return FRAC_OK;
}

// d = 1: the whole solve runs inside one thread block (solve1d.cu).
static int solve_1d(const frac_op* op, const double* f, double* u, const frac_solve_opts* opts,
                    frac_solve_info* info, cudaStream_t st) {
  Ws ws{st, {}};
  Solve1dTask* dt;
  frac_solve_info* di;
  FRAC_TRY(ws.get(&dt, sizeof(Solve1dTask)));
  FRAC_TRY(ws.get(&di, sizeof(frac_solve_info)));
  Solve1dTask t = make_task1d(op, f, u, di, opts);
  FRAC_CUDA_TRY(cudaMemcpyAsync(dt, &t, sizeof(t), cudaMemcpyHostToDevice, st));
  FRAC_TRY(solve1d_launch(op->M, opts->precision == FRAC_MIXED_IR, dt, 1, st));
  FRAC_CUDA_TRY(cudaMemcpyAsync(info, di, sizeof(frac_solve_info), cudaMemcpyDeviceToHost, st));
  FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  if (info->status == FRAC_EINVAL) {  // non-finite data: report through rel_resid as the other paths do
    info->status = FRAC_OK;
    info->rel_resid = NAN;
  }
  return FRAC_OK;
}

int BatchPending::collect(frac_solve_info* info) {
  std::vector<frac_solve_info> hi(order.size());
  if (!order.empty()) {
    FRAC_CUDA_TRY(cudaMemcpyAsync(hi.data(), dinfo, hi.size() * sizeof(frac_solve_info), cudaMemcpyDeviceToHost, st));
    FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  else if (pinned) {
    FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (size_t t = 0; t < order.size(); ++t) info[order[t]] = hi[t];
  for (void* p : bufs) cudaFreeAsync(p, st);
  bufs.clear();
  order.clear();
  if (pinned) cudaFreeHost(pinned);
  pinned = nullptr;
  return FRAC_OK;
}

BatchPending::~BatchPending() {
  if (pinned) {
    cudaStreamSynchronize(st);
    cudaFreeHost(pinned);
  }
  for (void* p : bufs) cudaFreeAsync(p, st);
}

int solve_batch_1d(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                   const frac_solve_opts* opts, const int64_t* idx, cudaStream_t st, BatchPending* pend) {
  // group the listed problems by FFT length; one launch per group, largest first
  pend->st = st;
  std::map<int64_t, std::vector<int64_t>> groups;  // M -> problems
  for (int64_t t = 0; t < count; ++t) groups[ops[idx[t]]->M].push_back(idx[t]);
  Solve1dTask* dt;
  FRAC_TRY(pend->alloc(&pend->dinfo, count * sizeof(frac_solve_info)));
  FRAC_TRY(pend->alloc(&dt, count * sizeof(Solve1dTask)));
  std::vector<Solve1dTask> tasks;
  std::vector<std::pair<int64_t, int64_t>> launches;  // (M, first task)
  for (auto g = groups.rbegin(); g != groups.rend(); ++g) {
    launches.emplace_back(g->first, (int64_t)tasks.size());
    for (int64_t i : g->second) {
      const frac_op* op = ops[i];
      tasks.push_back(make_task1d(op, f[i], u[i], pend->dinfo + tasks.size(), opts));
      pend->order.push_back(i);
    }
  }
  // pinned staging, kept until collect(), so the upload does not wait for the stream
  Solve1dTask* ht = nullptr;
  FRAC_CUDA_TRY(cudaMallocHost(&ht, tasks.size() * sizeof(Solve1dTask)));
  pend->pinned = ht;
  std::copy(tasks.begin(), tasks.end(), ht);
  FRAC_CUDA_TRY(cudaMemcpyAsync(dt, ht, tasks.size() * sizeof(Solve1dTask), cudaMemcpyHostToDevice, st));
  for (size_t g = 0; g < launches.size(); ++g) {
    const int64_t first = launches[g].second;
    const int64_t last = g + 1 < launches.size() ? launches[g + 1].second : (int64_t)tasks.size();
    FRAC_TRY(solve1d_launch(launches[g].first, opts->precision == FRAC_MIXED_IR, dt + first, (int)(last - first), st));
  }
  return FRAC_OK;
}

int solve_device(const frac_op* op, const double* f, double* u, const frac_solve_opts* opts,
                 frac_solve_info* info, cudaStream_t st) {
  if (op->prob.d == 1) return solve_1d(op, f, u, opts, info, st);
  const int64_t nd = op->nd;
  const int nb = red_blocks(nd);
  const unsigned gb = (unsigned)nb;
  Ws ws{st, {}};
  double *r64, *Au64, *partial, *scal, *part_inv;
  CGState *dst, *hst = nullptr;
  void* ws64;
  cudaGraphExec_t exec = nullptr;
  struct ExecFree {
    cudaGraphExec_t* e;
    ~ExecFree() { if (*e) cudaGraphExecDestroy(*e); }
  } exf{&exec};
  FRAC_TRY(ws.get(&r64, nd * sizeof(double)));
  FRAC_TRY(ws.get(&Au64, nd * sizeof(double)));
  FRAC_TRY(ws.get(&partial, kRedBlocks * sizeof(double)));
  FRAC_TRY(ws.get(&part_inv, apply_cg_partials(op) * sizeof(double)));
  FRAC_TRY(ws.get(&scal, 4 * sizeof(double)));
  FRAC_TRY(ws.get(&dst, sizeof(CGState)));
  FRAC_TRY(ws.get(&ws64, apply_workspace_bytes(op, FRAC_F64, 1)));
  FRAC_CUDA_TRY(cudaMallocHost(&hst, sizeof(CGState) + 4 * sizeof(double)));
  double* hscal = reinterpret_cast<double*>(hst + 1);
  struct HostFree {
    void* p;
    ~HostFree() { if (p) cudaFreeHost(p); }
  } hf{hst};

  // ||f||^2
  k_dot<double><<<gb, kTB, 0, st>>>(f, f, nd, partial, nullptr);
  k_sum_to<<<1, kTB, 0, st>>>(partial, nb, scal + 0);
  // initial residual r64 = f - A u (or f)
  if (opts->use_x0) {
    FRAC_TRY(apply_t<double>(op, u, Au64, 1, ws64, st));
  } else {
    FRAC_CUDA_TRY(cudaMemsetAsync(u, 0, nd * sizeof(double), st));
    FRAC_CUDA_TRY(cudaMemsetAsync(Au64, 0, nd * sizeof(double), st));
  }
  k_residual<<<gb, kTB, 0, st>>>(f, Au64, r64, nd, partial);
  k_sum_to<<<1, kTB, 0, st>>>(partial, nb, scal + 1);
  FRAC_CUDA_TRY(cudaGetLastError());
  FRAC_CUDA_TRY(cudaMemcpyAsync(hscal, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  const double fnorm = std::sqrt(hscal[0]);
  double rnorm = std::sqrt(hscal[1]);
  info->iters = 0;
  info->outer = 0;
  info->status = FRAC_OK;
  if (fnorm == 0.0) {
    FRAC_CUDA_TRY(cudaMemsetAsync(u, 0, nd * sizeof(double), st));
    info->rel_resid = 0.0;
    FRAC_CUDA_TRY(cudaStreamSynchronize(st));
    return FRAC_OK;
  }
  const double rtol = opts->rtol;
  int iters = 0;
  const bool pcg = opts->precond == FRAC_PRECOND_TAU && op->precond_ok;
  info->precond = pcg ? 1 : 0;

  if (opts->precision == FRAC_PLAIN_F64) {
    double *p, *q, *z = nullptr;
    FRAC_TRY(ws.get(&p, nd * sizeof(double)));
    FRAC_TRY(ws.get(&q, nd * sizeof(double)));
    if (pcg) FRAC_TRY(ws.get(&z, nd * sizeof(double)));
    int restarts = 0;
    while (rnorm > rtol * fnorm && iters < opts->max_iter && restarts < 8) {
      // CG on the current residual; the recursive residual is checked against rtol ||f||
      k_copy2<double><<<gb, kTB, 0, st>>>(r64, p, q, nd);  // p = r (q overwritten by the apply)
      k_dot<double><<<gb, kTB, 0, st>>>(r64, r64, nd, partial, nullptr);
      k_cg_start<<<1, kTB, 0, st>>>(partial, nb, dst, rtol * fnorm / std::max(rnorm, 1e-300), -1.0,
                                    opts->max_iter - iters, pcg ? 1 : 0);
      if (pcg) FRAC_TRY(cg_precond_start<double>(op, r64, p, z, ws64, dst, part_inv, st));
      FRAC_TRY(cg_run_fused<double>(op, u, r64, p, q, z, ws64, dst, hst, part_inv, partial, &exec, &iters, st));
      if (hst->status == FRAC_EBREAKDOWN) {
        info->status = FRAC_EBREAKDOWN;
        break;
      }
      // true residual
      FRAC_TRY(apply_t<double>(op, u, Au64, 1, ws64, st));
      k_residual<<<gb, kTB, 0, st>>>(f, Au64, r64, nd, partial);
      k_sum_to<<<1, kTB, 0, st>>>(partial, nb, scal + 1);
      FRAC_CUDA_TRY(cudaMemcpyAsync(hscal + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      FRAC_CUDA_TRY(cudaStreamSynchronize(st));
      rnorm = std::sqrt(hscal[1]);
      ++restarts;
    }
  } else {
    float *x32, *r32, *p32, *q32, *z32 = nullptr;
    void* ws32;
    FRAC_TRY(ws.get(&x32, nd * sizeof(float)));
    FRAC_TRY(ws.get(&r32, nd * sizeof(float)));
    FRAC_TRY(ws.get(&p32, nd * sizeof(float)));
    FRAC_TRY(ws.get(&q32, nd * sizeof(float)));
    if (pcg) FRAC_TRY(ws.get(&z32, nd * sizeof(float)));
    FRAC_TRY(ws.get(&ws32, apply_workspace_bytes(op, FRAC_F32, 1)));
    const double inner = opts->inner_tol > 0.0 ? opts->inner_tol : auto_inner_tol(op, opts->rtol);
    int outer = 0;
    while (rnorm > rtol * fnorm && iters < opts->max_iter && outer < 100) {
      // inner FP32 CG on A d = r / ||r||
      k_ir_scale_down<<<gb, kTB, 0, st>>>(r64, scal + 1, r32, p32, x32, nd);
      k_dot<float><<<gb, kTB, 0, st>>>(r32, r32, nd, partial, nullptr);
      k_cg_start<<<1, kTB, 0, st>>>(partial, nb, dst, inner, -1.0, opts->max_iter - iters, pcg ? 1 : 0);
      if (pcg) FRAC_TRY(cg_precond_start<float>(op, r32, p32, z32, ws32, dst, part_inv, st));
      FRAC_TRY(cg_run_fused<float>(op, x32, r32, p32, q32, z32, ws32, dst, hst, part_inv, partial, &exec, &iters,
                                   st));
      k_ir_correct<<<gb, kTB, 0, st>>>(u, x32, scal + 1, nd);
      // true FP64 residual
      FRAC_TRY(apply_t<double>(op, u, Au64, 1, ws64, st));
      k_residual<<<gb, kTB, 0, st>>>(f, Au64, r64, nd, partial);
      k_sum_to<<<1, kTB, 0, st>>>(partial, nb, scal + 1);
      FRAC_CUDA_TRY(cudaGetLastError());
      FRAC_CUDA_TRY(cudaMemcpyAsync(hscal + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      FRAC_CUDA_TRY(cudaStreamSynchronize(st));
      double prev = rnorm;
      rnorm = std::sqrt(hscal[1]);
      ++outer;
      if (!(rnorm < prev) && outer > 3) break;  // refinement stagnated
    }
    info->outer = outer;
  }
  info->iters = iters;
  info->rel_resid = rnorm / fnorm;
  if (info->status == FRAC_OK && !(info->rel_resid <= rtol)) info->status = FRAC_ENOCONV;
  return FRAC_OK;
}

}  // namespace frac

// ===========================================================================
// Solve engine (frac_engine_*): the computation of solve_device as an
// asynchronous state machine per job, so that many jobs progress at once on
// a pool of streams.  poll() advances every job whose last device step has
// finished (cudaEventQuery) by issuing its next step.
// ===========================================================================

namespace frac {
namespace {

enum Phase { PH_WHOLE1D, PH_NORM, PH_INNER, PH_REFINE, PH_COPYOUT, PH_DONE };

struct Mirror {  // pinned host copies of the small device results
  CGState st;
  double scal[4];
  frac_solve_info info;
  Solve1dTask task;
};

struct Job {
  int64_t id = 0;
  const frac_op* op = nullptr;
  frac_solve_opts opts{};
  double* u_user = nullptr;
  bool host_u = false;
  const double* f = nullptr;  // device
  double* u = nullptr;        // device
  cudaStream_t s = nullptr;
  Mirror* hm = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> bufs;
  size_t bytes = 0;
  // device buffers (d >= 2)
  double *r64 = nullptr, *Au64 = nullptr, *partial = nullptr, *part_inv = nullptr, *scal = nullptr;
  CGState* st = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *z32 = nullptr;
  double *p64 = nullptr, *q64 = nullptr, *z64 = nullptr;
  bool pcg = false;
  void *ws32 = nullptr, *ws64 = nullptr;
  frac_solve_info* dinfo = nullptr;
  Solve1dTask* dtask = nullptr;
  Phase phase = PH_NORM;
  int iters = 0, outer = 0, restarts = 0, status = FRAC_OK;
  double fnorm = 0.0, rnorm = 0.0, prev = INFINITY;
  std::chrono::steady_clock::time_point t0;
  frac_solve_info result{};
};

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace frac

struct frac_engine {
  int device = 0;
  std::vector<cudaStream_t> streams;
  size_t next_stream = 0;
  std::vector<frac::Job*> jobs;  // in flight
  std::vector<frac_job_result> finished;
  int64_t next_id = 1;
  size_t bytes = 0;
  std::vector<frac::Mirror*> free_mirrors;
  std::vector<frac::Mirror*> mirror_blocks;
};

namespace frac {
namespace {

template <typename P>
int jalloc(Job* j, P** out, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, j->s);
  if (e != cudaSuccess) return record_cuda_error(e, __FILE__, __LINE__, "cudaMallocAsync");
  j->bufs.push_back(p);
  j->bytes += bytes;
  *out = (P*)p;
  return FRAC_OK;
}

Mirror* get_mirror(frac_engine* e) {
  if (e->free_mirrors.empty()) {
    Mirror* blk = nullptr;
    if (cudaMallocHost(&blk, 64 * sizeof(Mirror)) != cudaSuccess) return nullptr;
    e->mirror_blocks.push_back(blk);
    for (int i = 0; i < 64; ++i) e->free_mirrors.push_back(blk + i);
  }
  Mirror* m = e->free_mirrors.back();
  e->free_mirrors.pop_back();
  return m;
}

// Launch the next chunk of the current inner/plain CG and the state read-back.
template <typename T>
int launch_chunk(Job* j, T* x, T* r, T* p, T* q, T* z, void* ws) {
  if (!j->exec) {
    FRAC_TRY(cg_iteration<T>(j->op, x, r, p, q, z, ws, j->st, j->part_inv, j->partial, j->s));
    FRAC_TRY(capture_cg_loop<T>(j->op, x, r, p, q, z, ws, j->st, j->part_inv, j->partial, j->s, &j->exec));
  } else {
    FRAC_TRY(launch_cg_loop(j->exec, j->st, j->s));
  }
  FRAC_CUDA_TRY(cudaMemcpyAsync(&j->hm->st, j->st, sizeof(CGState), cudaMemcpyDeviceToHost, j->s));
  FRAC_CUDA_TRY(cudaEventRecord(j->ev, j->s));
  return FRAC_OK;
}

int launch_chunk_resume(Job* j);

// Start an inner (mixed) or plain CG run from the current residual r64.
int start_cg(Job* j) {
  const int64_t nd = j->op->nd;
  const int nb = red_blocks(nd);
  const unsigned gb = (unsigned)nb;
  const int left = j->opts.max_iter - j->iters;
  if (j->opts.precision == FRAC_MIXED_IR) {
    const double inner = j->opts.inner_tol > 0.0 ? j->opts.inner_tol : auto_inner_tol(j->op, j->opts.rtol);
    k_ir_scale_down<<<gb, kTB, 0, j->s>>>(j->r64, j->scal + 1, j->r32, j->p32, j->x32, nd);
    k_dot<float><<<gb, kTB, 0, j->s>>>(j->r32, j->r32, nd, j->partial, nullptr);
    k_cg_start<<<1, kTB, 0, j->s>>>(j->partial, nb, j->st, inner, -1.0, left, j->pcg ? 1 : 0);
    FRAC_CUDA_TRY(cudaGetLastError());
    if (j->pcg) FRAC_TRY(cg_precond_start<float>(j->op, j->r32, j->p32, j->z32, j->ws32, j->st, j->part_inv, j->s));
    j->phase = PH_INNER;
    return launch_chunk<float>(j, j->x32, j->r32, j->p32, j->q32, j->z32, j->ws32);
  }
  k_copy2<double><<<gb, kTB, 0, j->s>>>(j->r64, j->p64, j->q64, nd);
  k_dot<double><<<gb, kTB, 0, j->s>>>(j->r64, j->r64, nd, j->partial, nullptr);
  k_cg_start<<<1, kTB, 0, j->s>>>(j->partial, nb, j->st, j->opts.rtol * j->fnorm / std::max(j->rnorm, 1e-300), -1.0,
                                  left, j->pcg ? 1 : 0);
  FRAC_CUDA_TRY(cudaGetLastError());
  if (j->pcg) FRAC_TRY(cg_precond_start<double>(j->op, j->r64, j->p64, j->z64, j->ws64, j->st, j->part_inv, j->s));
  j->phase = PH_INNER;
  return launch_chunk<double>(j, j->u, j->r64, j->p64, j->q64, j->z64, j->ws64);
}

// r64 = f - A64 u, ||r64||^2 -> scal[1] -> host; phase REFINE
int start_residual(Job* j) {
  const int64_t nd = j->op->nd;
  const int nb = red_blocks(nd);
  FRAC_TRY(apply_t<double>(j->op, j->u, j->Au64, 1, j->ws64, j->s));
  k_residual<<<(unsigned)nb, kTB, 0, j->s>>>(j->f, j->Au64, j->r64, nd, j->partial);
  k_sum_to<<<1, kTB, 0, j->s>>>(j->partial, nb, j->scal + 1);
  FRAC_CUDA_TRY(cudaGetLastError());
  FRAC_CUDA_TRY(cudaMemcpyAsync(j->hm->scal, j->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, j->s));
  FRAC_CUDA_TRY(cudaEventRecord(j->ev, j->s));
  j->phase = PH_REFINE;
  return FRAC_OK;
}

int finish(Job* j) {
  frac_solve_info& r = j->result;
  r.iters = j->iters;
  r.outer = j->outer;
  r.precond = j->pcg ? 1 : 0;
  if (j->op->prob.d == 1) {
    r = j->hm->info;
    if (r.status == FRAC_EINVAL || std::isnan(r.rel_resid)) r.status = FRAC_EINVAL;
  } else {
    r.rel_resid = j->fnorm > 0.0 ? j->rnorm / j->fnorm : (j->fnorm == 0.0 ? 0.0 : NAN);
    if (std::isnan(r.rel_resid)) j->status = FRAC_EINVAL;
    if (j->status == FRAC_OK && !(r.rel_resid <= j->opts.rtol)) j->status = FRAC_ENOCONV;
    r.status = j->status;
  }
  if (j->host_u) {
    FRAC_CUDA_TRY(cudaMemcpyAsync(j->u_user, j->u, j->op->nd * sizeof(double), cudaMemcpyDeviceToHost, j->s));
    FRAC_CUDA_TRY(cudaEventRecord(j->ev, j->s));
    j->phase = PH_COPYOUT;
  } else {
    j->phase = PH_DONE;
  }
  return FRAC_OK;
}

// One step of job j whose last device work has completed.
int advance(Job* j) {
  switch (j->phase) {
    case PH_WHOLE1D:
      return finish(j);
    case PH_NORM:
      j->fnorm = std::sqrt(j->hm->scal[0]);
      j->rnorm = std::sqrt(j->hm->scal[1]);
      if (!(j->fnorm > 0.0) || j->rnorm <= j->opts.rtol * j->fnorm) {
        if (j->fnorm == 0.0) {
          FRAC_CUDA_TRY(cudaMemsetAsync(j->u, 0, j->op->nd * sizeof(double), j->s));
          j->rnorm = 0.0;
        }
        return finish(j);
      }
      return start_cg(j);
    case PH_INNER: {
      const CGState& st = j->hm->st;
      if (!st.done) return launch_chunk_resume(j);
      j->iters += st.it;
      if (j->opts.precision == FRAC_MIXED_IR) {
        k_ir_correct<<<(unsigned)red_blocks(j->op->nd), kTB, 0, j->s>>>(j->u, j->x32, j->scal + 1, j->op->nd);
        FRAC_CUDA_TRY(cudaGetLastError());
      } else if (st.status == FRAC_EBREAKDOWN) {
        j->status = FRAC_EBREAKDOWN;
      }
      return start_residual(j);
    }
    case PH_REFINE: {
      const double rn = std::sqrt(j->hm->scal[1]);
      j->rnorm = rn;
      ++j->outer;
      if (j->opts.precision != FRAC_MIXED_IR) ++j->restarts;
      const bool converged = rn <= j->opts.rtol * j->fnorm;
      const bool stagnated = j->opts.precision == FRAC_MIXED_IR ? (!(rn < j->prev) && j->outer > 3) : j->restarts >= 8;
      j->prev = rn;
      if (converged || stagnated || j->status != FRAC_OK || j->iters >= j->opts.max_iter || j->outer >= 100 ||
          !std::isfinite(rn))
        return finish(j);
      return start_cg(j);
    }
    case PH_COPYOUT:
      j->phase = PH_DONE;
      return FRAC_OK;
    default:
      return FRAC_OK;
  }
}

}  // namespace
}  // namespace frac

namespace frac {
namespace {
int launch_chunk_resume(Job* j) {
  if (j->opts.precision == FRAC_MIXED_IR)
    return launch_chunk<float>(j, j->x32, j->r32, j->p32, j->q32, j->z32, j->ws32);
  return launch_chunk<double>(j, j->u, j->r64, j->p64, j->q64, j->z64, j->ws64);
}
}  // namespace
}  // namespace frac

using namespace frac;

extern "C" int frac_engine_create(int nstreams, frac_engine** out) {
  if (!out || nstreams < 1) return FRAC_EINVAL;
  *out = nullptr;
  frac_engine* e = new (std::nothrow) frac_engine();
  if (!e) return FRAC_ENOMEM;
  cudaGetDevice(&e->device);
  for (int i = 0; i < nstreams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      frac_engine_destroy(e);
      return FRAC_ECUDA;
    }
    e->streams.push_back(s);
  }
  *out = e;
  return FRAC_OK;
}

static void release_job(frac_engine* e, Job* j) {
  for (void* p : j->bufs) cudaFreeAsync(p, j->s);
  if (j->exec) cudaGraphExecDestroy(j->exec);
  if (j->ev) cudaEventDestroy(j->ev);
  if (j->hm) e->free_mirrors.push_back(j->hm);
  e->bytes -= j->bytes;
  delete j;
}

static int submit_impl(frac_engine* e, Job* j, const double* f, double* u) {
  const frac_op* op = j->op;
  const int64_t nd = op->nd;
  FRAC_CUDA_TRY(cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming));
  j->hm = get_mirror(e);
  if (!j->hm) return FRAC_ENOMEM;
  const bool df = dev_ptr(f);
  j->host_u = !dev_ptr(u);
  j->u_user = u;
  if (df) {
    j->f = f;
  } else {
    for (int64_t i = 0; i < nd; ++i)
      if (!std::isfinite(f[i])) return FRAC_EINVAL;
    double* fd;
    FRAC_TRY(jalloc(j, &fd, nd * sizeof(double)));
    FRAC_CUDA_TRY(cudaMemcpyAsync(fd, f, nd * sizeof(double), cudaMemcpyHostToDevice, j->s));
    j->f = fd;
  }
  if (!j->host_u) {
    j->u = u;
  } else {
    FRAC_TRY(jalloc(j, &j->u, nd * sizeof(double)));
    if (j->opts.use_x0) FRAC_CUDA_TRY(cudaMemcpyAsync(j->u, u, nd * sizeof(double), cudaMemcpyHostToDevice, j->s));
  }
  if (op->prob.d == 1) {
    FRAC_TRY(jalloc(j, &j->dinfo, sizeof(frac_solve_info)));
    FRAC_TRY(jalloc(j, &j->dtask, sizeof(Solve1dTask)));
    j->hm->task = make_task1d(op, j->f, j->u, j->dinfo, &j->opts);
    FRAC_CUDA_TRY(cudaMemcpyAsync(j->dtask, &j->hm->task, sizeof(Solve1dTask), cudaMemcpyHostToDevice, j->s));
    FRAC_TRY(solve1d_launch(op->M, j->opts.precision == FRAC_MIXED_IR, j->dtask, 1, j->s));
    FRAC_CUDA_TRY(cudaMemcpyAsync(&j->hm->info, j->dinfo, sizeof(frac_solve_info), cudaMemcpyDeviceToHost, j->s));
    FRAC_CUDA_TRY(cudaEventRecord(j->ev, j->s));
    j->phase = PH_WHOLE1D;
    return FRAC_OK;
  }
  const int nb = red_blocks(nd);
  FRAC_TRY(jalloc(j, &j->r64, nd * sizeof(double)));
  FRAC_TRY(jalloc(j, &j->Au64, nd * sizeof(double)));
  FRAC_TRY(jalloc(j, &j->partial, kRedBlocks * sizeof(double)));
  FRAC_TRY(jalloc(j, &j->part_inv, apply_cg_partials(op) * sizeof(double)));
  FRAC_TRY(jalloc(j, &j->scal, 4 * sizeof(double)));
  FRAC_TRY(jalloc(j, &j->st, sizeof(CGState)));
  FRAC_TRY(jalloc(j, &j->ws64, apply_workspace_bytes(op, FRAC_F64, 1)));
  j->pcg = j->opts.precond == FRAC_PRECOND_TAU && op->precond_ok;
  if (j->opts.precision == FRAC_MIXED_IR) {
    FRAC_TRY(jalloc(j, &j->x32, nd * sizeof(float)));
    FRAC_TRY(jalloc(j, &j->r32, nd * sizeof(float)));
    FRAC_TRY(jalloc(j, &j->p32, nd * sizeof(float)));
    FRAC_TRY(jalloc(j, &j->q32, nd * sizeof(float)));
    if (j->pcg) FRAC_TRY(jalloc(j, &j->z32, nd * sizeof(float)));
    FRAC_TRY(jalloc(j, &j->ws32, apply_workspace_bytes(op, FRAC_F32, 1)));
  } else {
    FRAC_TRY(jalloc(j, &j->p64, nd * sizeof(double)));
    FRAC_TRY(jalloc(j, &j->q64, nd * sizeof(double)));
    if (j->pcg) FRAC_TRY(jalloc(j, &j->z64, nd * sizeof(double)));
  }
  k_dot<double><<<(unsigned)nb, kTB, 0, j->s>>>(j->f, j->f, nd, j->partial, nullptr);
  k_sum_to<<<1, kTB, 0, j->s>>>(j->partial, nb, j->scal + 0);
  if (j->opts.use_x0) {
    FRAC_TRY(apply_t<double>(op, j->u, j->Au64, 1, j->ws64, j->s));
  } else {
    FRAC_CUDA_TRY(cudaMemsetAsync(j->u, 0, nd * sizeof(double), j->s));
    FRAC_CUDA_TRY(cudaMemsetAsync(j->Au64, 0, nd * sizeof(double), j->s));
  }
  k_residual<<<(unsigned)nb, kTB, 0, j->s>>>(j->f, j->Au64, j->r64, nd, j->partial);
  k_sum_to<<<1, kTB, 0, j->s>>>(j->partial, nb, j->scal + 1);
  FRAC_CUDA_TRY(cudaGetLastError());
  FRAC_CUDA_TRY(cudaMemcpyAsync(j->hm->scal, j->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, j->s));
  FRAC_CUDA_TRY(cudaEventRecord(j->ev, j->s));
  j->phase = PH_NORM;
  return FRAC_OK;
}

extern "C" int frac_engine_submit(frac_engine* e, const frac_op* op, const double* f, double* u,
                                  const frac_solve_opts* opts, int64_t* job) {
  if (!e || !op || !f || !u || !opts || !job) return FRAC_EINVAL;
  if (!(opts->rtol > 0.0) || opts->max_iter < 1) return FRAC_EINVAL;
  if (opts->precision != FRAC_PLAIN_F64 && opts->precision != FRAC_MIXED_IR) return FRAC_EINVAL;
  Job* j = new (std::nothrow) Job();
  if (!j) return FRAC_ENOMEM;
  j->id = e->next_id++;
  j->op = op;
  j->opts = *opts;
  j->s = e->streams[e->next_stream++ % e->streams.size()];
  j->t0 = std::chrono::steady_clock::now();
  const int s = submit_impl(e, j, f, u);
  e->bytes += j->bytes;
  if (s != FRAC_OK) {
    cudaStreamSynchronize(j->s);
    release_job(e, j);
    return settle(s);
  }
  e->jobs.push_back(j);
  *job = j->id;
  return FRAC_OK;
}

extern "C" int frac_engine_poll(frac_engine* e, int block, frac_job_result* out, int cap, int* count) {
  if (!e || !count || cap < 0 || (cap > 0 && !out)) return FRAC_EINVAL;
  int first_err = FRAC_OK;
  for (;;) {
    for (size_t i = 0; i < e->jobs.size();) {
      Job* j = e->jobs[i];
      cudaError_t q = cudaEventQuery(j->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      int s = (q == cudaSuccess) ? FRAC_OK : record_cuda_error(q, __FILE__, __LINE__, "cudaEventQuery");
      if (s == FRAC_OK) {
        const size_t before = j->bytes;
        s = advance(j);
        e->bytes += j->bytes - before;
      }
      if (s != FRAC_OK) {
        j->result.status = s;
        j->phase = PH_DONE;
        if (first_err == FRAC_OK) first_err = s;
        cudaStreamSynchronize(j->s);
      }
      if (j->phase == PH_DONE) {
        frac_job_result r;
        r.job = j->id;
        r.info = j->result;
        r.submit_to_done_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - j->t0).count();
        e->finished.push_back(r);
        release_job(e, j);
        e->jobs.erase(e->jobs.begin() + i);
      } else {
        ++i;
      }
    }
    if (!block || !e->finished.empty() || e->jobs.empty()) break;
    std::this_thread::yield();
  }
  const int n = (int)std::min<size_t>((size_t)cap, e->finished.size());
  for (int i = 0; i < n; ++i) out[i] = e->finished[i];
  e->finished.erase(e->finished.begin(), e->finished.begin() + n);
  *count = n;
  return first_err;
}

extern "C" int frac_engine_stats(const frac_engine* e, int64_t* active, size_t* device_bytes) {
  if (!e) return FRAC_EINVAL;
  if (active) *active = (int64_t)e->jobs.size();
  if (device_bytes) *device_bytes = e->bytes;
  return FRAC_OK;
}

extern "C" void frac_engine_destroy(frac_engine* e) {
  if (!e) return;
  for (cudaStream_t s : e->streams) cudaStreamSynchronize(s);
  for (Job* j : e->jobs) release_job(e, j);
  e->jobs.clear();
  for (cudaStream_t s : e->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (Mirror* m : e->mirror_blocks) cudaFreeHost(m);
  delete e;
}

namespace frac {
// Make every engine stream wait for the work already queued on `caller`.
int engine_wait_for(frac_engine* e, cudaStream_t caller) {
  cudaEvent_t ev;
  FRAC_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t r = cudaEventRecord(ev, caller);
  for (cudaStream_t s : e->streams)
    if (r == cudaSuccess) r = cudaStreamWaitEvent(s, ev, 0);
  cudaEventDestroy(ev);
  FRAC_CUDA_TRY(r);
  return FRAC_OK;
}
}  // namespace frac
