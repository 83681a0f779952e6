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
#include <type_traits>
#include <utility>
#include <vector>

#include "batch2d_kernel.cuh"
#include "prof.cuh"

namespace frac {
namespace {

using namespace b2;
using namespace fft;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

constexpr int kProbeIters = 24;
constexpr int kClusterSizes[] = {1, 2, 4, 8, 16};
constexpr int kNumSizes = 5;

// Problem classes are FFT lengths M (a power of two 2^5 .. 2^10 or a mixed length up
// to 2^10); lvl(M) = ceil(log2 M) orders them against the cluster cut-over.
bool is_pow2(int64_t M) { return (M & (M - 1)) == 0; }
int lvl(int64_t M) { return ilog2(M); }

// Dynamic shared memory of one CTA for a class: the row lines or the column tiles of
// its FP64 passes (FP32 ones take half); a mixed length adds the spare line and tile.
size_t smem_bytes(int64_t M) {  // M: a power of two or a length with a plan
  if (is_pow2(M)) {
    const int logm = ilog2(M);
    const int tplv = tpl(logm), lines = kThreads / tplv;
    const size_t rows = (size_t)lines * line_stride(logm) * sizeof(double2);
    const size_t cols = (size_t)(kThreads / tplv) * line_stride_tile(logm) * sizeof(double2);
    return std::max(rows, cols);
  }
  MxPlan plan;
  mx_plan(M, &plan);
  const MxLine ln(plan);
  const int lines = kThreads / ln.tpl(), tpr64 = kThreads / (2 * ln.tpl());
  const size_t rows = (size_t)(lines + 1) * ln.stride() * sizeof(double2);
  const size_t cols = (size_t)(tpr64 + 1) * 2 * ln.stride_tile() * sizeof(double2);
  return std::max(rows, cols);
}

// Scratch of a worker for the problems it may take: the FP64 spectrum layout
// (n ceil(K/2) 2 complex doubles, the largest over the problems: with mixed
// lengths the largest n need not have the largest M) and five vectors of the
// largest n^2.
struct SlotSize {
  size_t w = 0;   // bytes of the spectrum
  int64_t nn = 0; // entries of a vector
  void add(int n, int64_t M) {
    const int64_t K = M / 2 + 1, KB64 = (K + 1) / 2;
    w = std::max(w, (size_t)n * KB64 * 2 * sizeof(double2));
    nn = std::max(nn, (int64_t)n * n);
  }
};
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
size_t slot_bytes(const SlotSize& z) {
  return al256(z.w) + 4 * al256(z.nn * sizeof(float)) + al256(z.nn * sizeof(double));
}

B2Slot carve(unsigned char* base, const SlotSize& z) {
  B2Slot s;
  s.W = base;
  s.w_bytes = z.w;
  s.nn = z.nn;
  base += al256(z.w);
  s.x = reinterpret_cast<float*>(base);
  base += al256(z.nn * sizeof(float));
  s.r = reinterpret_cast<float*>(base);
  base += al256(z.nn * sizeof(float));
  s.p = reinterpret_cast<float*>(base);
  base += al256(z.nn * sizeof(float));
  s.q = reinterpret_cast<float*>(base);
  base += al256(z.nn * sizeof(float));
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
    // the largest over every length the kernel takes (powers of two and mixed lengths)
    size_t mx = 0;
    for (int64_t M = 1 << kBatch2dMinLog; M <= (1 << kBatch2dMaxLog); M += 16) {
      MxPlan plan;
      if (is_pow2(M) || mx_plan(M, &plan)) mx = std::max(mx, smem_bytes(M));
    }
    FRAC_TRY(kernel_attrs<false>(mx));
    FRAC_TRY(mx_kernel_attrs(mx));
    done[dev] = 1;
  }
  return FRAC_OK;
}

// Clusters of size C that can be resident at once, and the launch, of the kernel
// instance without (mx = false) or with the mixed-length solver.
int active_clusters(int C, size_t smem, bool mx) {
  return mx ? mx_kernel_active_clusters(C, smem) : kernel_active_clusters<false>(C, smem);
}

int launch(const B2Args& a, int C, int grid, size_t smem, bool mx, cudaStream_t st) {
  return mx ? mx_kernel_launch(a, C, grid, smem, st) : kernel_launch<false>(a, C, grid, smem, st);
}

// Autotuner timings of a class's probe problem (size n_probe) with one CTA, and with
// one cluster of each size: microseconds per FP32 CG iteration (t) and per
// refinement residual, the FP64 apply with the solve's fixed costs (t64).
struct ClassTiming {
  int n_probe = 0;
  double t[kNumSizes] = {-1, -1, -1, -1, -1};
  double t64[kNumSizes] = {0, 0, 0, 0, 0};
};
std::mutex g_tune_mu;
std::map<std::pair<int, int64_t>, ClassTiming> g_tune;  // (device, FFT length M)

B2Prob make_prob(const frac_op* op, const double* f, double* u, const frac_solve_opts* o) {
  B2Prob p;
  p.f = f;
  p.u = u;
  p.lam32 = op->lam32;
  p.lam64 = op->lam64;
  p.pinv32 = op->pinv32;
  p.pcg = (o->precond == FRAC_PRECOND_TAU && op->precond_ok) ? 1 : 0;
  p.tw32 = twiddles32_len(op->M);
  p.tw64 = twiddles64_len(op->M);
  p.plan = op->plan[0];
  p.n = (int)op->n;
  p.logm = op->logm;
  p.max_iter = o->max_iter;
  p.use_x0 = o->use_x0 ? 1 : 0;
  p.rtol = o->rtol;
  p.inner_tol = o->inner_tol > 0.0 ? o->inner_tol : auto_inner_tol(op, o->rtol);
  return p;
}

// Times (op, f) alone, on one CTA and on one cluster of each launchable size, as
// solves of exactly kProbeIters and 2 kProbeIters FP32 CG iterations (each followed by
// one FP64 residual); their difference gives the time of an iteration, the rest that
// of the residual.  The solution goes to scratch.
int probe_class(const frac_op* op, const double* f, cudaStream_t st, ClassTiming* out) {
  const int64_t M = op->M;
  const int n = (int)op->n;
  const size_t smem = smem_bytes(M);
  const bool mx = !is_pow2(M);
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
  SlotSize z;
  z.add(n, M);
  FRAC_TRY(b.get(&scratch, slot_bytes(z)));
  // rtol 0 and an unreachable inner tolerance: exactly max_iter iterations, then one residual
  frac_solve_opts o1{0.0, kProbeIters, FRAC_MIXED_IR, 0, FRAC_PRECOND_TAU, 1e-30};
  frac_solve_opts o2 = o1;
  o2.max_iter = 2 * kProbeIters;
  const B2Prob hp[2] = {make_prob(op, f, u, &o1), make_prob(op, f, u, &o2)};
  B2Slot hs = carve(scratch, z);
  FRAC_CUDA_TRY(cudaMemcpyAsync(ds, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  cudaEvent_t e0, e1;
  FRAC_CUDA_TRY(cudaEventCreate(&e0));
  FRAC_CUDA_TRY(cudaEventCreate(&e1));
  int rc = FRAC_OK;
  out->n_probe = n;
  for (int i = 0; i < kNumSizes && rc == FRAC_OK; ++i) {
    const int C = kClusterSizes[i];
    if (active_clusters(C, smem, mx) < 1) continue;
    B2Args a = {};
    a.probs = dp;
    a.info = di;
    a.n_cluster = C > 1 ? 1 : 0;
    a.n_local = C > 1 ? 0 : 1;
    a.next = next;
    a.cslots = ds;
    a.lslots = ds;
    float best[2] = {1e30f, 1e30f};
    for (int k = 0; k < 2 && rc == FRAC_OK; ++k) {
      if (cudaMemcpyAsync(dp, &hp[k], sizeof(B2Prob), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = FRAC_ECUDA;
        break;
      }
      for (int rep = 0; rep < 2 - k && rc == FRAC_OK; ++rep) {  // the first run also loads the code
        if (cudaMemsetAsync(next, 0, 2 * sizeof(unsigned int), st) != cudaSuccess ||
            cudaEventRecord(e0, st) != cudaSuccess) {
          rc = FRAC_ECUDA;
          break;
        }
        rc = launch(a, C, C, smem, mx, st);
        if (rc != FRAC_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = FRAC_ECUDA;
          break;
        }
        best[k] = std::min(best[k], ms);
      }
    }
    if (rc == FRAC_OK) {
      // the second solve's extra kProbeIters iterations; at least a tenth of the first
      // solve's mean (timing noise), the residual what is left of the first solve
      const double it = std::max(1e3 * (best[1] - best[0]), 0.1 * 1e3 * best[0]) / kProbeIters;
      out->t[i] = it;
      out->t64[i] = std::max(0.0, 1e3 * best[0] - kProbeIters * it);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return settle(rc);
}

// Cost model of one problem: `outer` refinement steps, each an FP32 CG solve to the
// inner tolerance and an FP64 residual; the CG iterations of a step grow like
// alpha log n with the tau preconditioner (about 2 + alpha log2 n per step in the 2D
// mixes measured) and like n^(alpha/2) without it (condition number ~ n^alpha).
// Per-iteration and per-residual times of its class measured at n_probe, scaled by the
// number of line transforms (the columns' share is the same for every n of a class).
double est_iters(int n, double alpha, bool pcg, int outer) {
  return pcg ? outer * (2.0 + alpha * std::log2((double)n)) : 20.0 + 6.0 * std::pow((double)n, 0.5 * alpha);
}

// Refinement steps to rtol when each gains a factor inner_tol (the last residual
// included), at least one.
int est_outer(double rtol, double inner_tol) {
  if (!(rtol > 0.0 && rtol < 1.0 && inner_tol > 0.0 && inner_tol < 1.0)) return 1;
  return std::max(1, (int)std::ceil(std::log(rtol) / std::log(inner_tol) - 1e-9));
}

struct Item {
  int64_t idx;  // problem index in the caller's arrays
  int64_t M;    // class: the FFT length
  int n;
  double alpha;
  bool pcg;
  int outer;  // estimated refinement steps
};

// Makespan of the two queues on `ncl` clusters of C CTAs, classes with lvl(M) >= cut cluster-wide.
double simulate(const std::vector<Item>& items, const std::map<int64_t, ClassTiming>& tm, int si, int ncl, int cut,
                std::vector<const Item*>* cl_out, std::vector<const Item*>* lo_out) {
  const int C = kClusterSizes[si];
  std::vector<std::pair<double, const Item*>> cl, lo;
  for (const Item& it : items) {
    const ClassTiming& t = tm.at(it.M);
    // line transforms of a refinement pass: n row lines (n / 2 pairs, forward and
    // inverse) and 2 K columns of the half spectrum, K = M / 2 + 1 for the whole class
    const double K = (double)(it.M / 2 + 1);
    const double scale = (2.0 * K + it.n) / (2.0 * K + t.n_probe);
    const bool wide = C > 1 && lvl(it.M) >= cut && t.t[si] > 0;
    const int k = wide ? si : 0;
    const double cost = est_iters(it.n, it.alpha, it.pcg, it.outer) * t.t[k] + it.outer * t.t64[k];
    (wide ? cl : lo).emplace_back(cost * scale, &it);
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
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::map<int64_t, int64_t> rep;  // M -> largest problem of that class
  for (int64_t t = 0; t < count; ++t) {
    const frac_op* op = ops[idx[t]];
    auto it = rep.find(op->M);
    if (it == rep.end() || ops[it->second]->n < op->n) rep[op->M] = idx[t];
  }
  for (auto& kv : rep) FRAC_TRY(prepare_twiddles_len(kv.first));
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
  return op->prob.d == 2 && op->square && opts->precision == FRAC_MIXED_IR && op->M >= (1 << kBatch2dMinLog) &&
         op->M <= (1 << kBatch2dMaxLog);
}

int solve_batch_2d(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                   const frac_solve_opts* opts, const int64_t* idx, cudaStream_t st, frac_batch_plan* plan_out,
                   int pin_size, int pin_cut, BatchPending* pend) {
  if (count <= 0) return FRAC_OK;
  FRAC_TRY(configure_kernel());
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<Item> items;
  std::map<int64_t, int64_t> rep;  // M -> largest problem of that class
  for (int64_t t = 0; t < count; ++t) {
    const frac_op* op = ops[idx[t]];
    const double itol = opts->inner_tol > 0.0 ? opts->inner_tol : auto_inner_tol(op, opts->rtol);
    items.push_back(Item{idx[t], op->M, (int)op->n, op->prob.alpha,
                         opts->precond == FRAC_PRECOND_TAU && op->precond_ok != 0, est_outer(opts->rtol, itol)});
    auto it = rep.find(op->M);
    if (it == rep.end() || ops[it->second]->n < op->n) rep[op->M] = idx[t];
  }
  for (auto& kv : rep) FRAC_TRY(prepare_twiddles_len(kv.first));
  // timings of every class present (measured once per device and FFT length)
  std::map<int64_t, ClassTiming> tm;
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
  bool mx = false;
  for (auto& kv : rep) {
    smem = std::max(smem, smem_bytes(kv.first));
    mx = mx || !is_pow2(kv.first);
  }
  int best_si = 0, best_cut = kBatch2dMaxLog + 1, best_ncl = 0;
  double best = INFINITY;
  for (int si = 0; si < kNumSizes; ++si) {
    const int C = kClusterSizes[si];
    if (pin_size > 0 && C != pin_size) continue;
    const int ncl = active_clusters(C, smem, mx);
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
  SlotSize zcl, zlo;
  for (const Item* it : cl) zcl.add(it->n, it->M);
  for (const Item* it : lo) zlo.add(it->n, it->M);
  const size_t cslot = cl.empty() ? 0 : slot_bytes(zcl), lslot = lo.empty() ? 0 : slot_bytes(zlo);
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
  for (int i = 0; i < n_cslots; ++i) hs.push_back(carve(scratch + (size_t)i * cslot, zcl));
  for (int i = 0; i < n_lslots; ++i) hs.push_back(carve(scratch + (size_t)n_cslots * cslot + (size_t)i * lslot, zlo));
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
  prof::Scope ps("batch2d", st);
  return launch(a, C, grid, smem, mx, st);
}

}  // namespace frac
