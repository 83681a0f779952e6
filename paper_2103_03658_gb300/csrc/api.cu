// C ABI entry points (include/frac.h): argument validation, operator
// lifecycle, staging of host buffers, dispatch to the device kernels.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <initializer_list>
#include <mutex>
#include <new>
#include <vector>

#include "apply.cuh"
#include "batch2d.cuh"

namespace frac {

// c_{d,alpha} = 2^{alpha-1} alpha Gamma((d+alpha)/2) / (pi^{d/2} Gamma(1-alpha/2))
// (definition after Eq. (fL-nD)).
static double c_dalpha(int d, double alpha) {
  return std::pow(2.0, alpha - 1.0) * alpha * std::tgamma((d + alpha) / 2.0) /
         (std::pow(M_PI, d / 2.0) * std::tgamma(1.0 - alpha / 2.0));
}

static int keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  for (int d : done)
    if (d == dev) return FRAC_OK;
  cudaMemPool_t pool;
  FRAC_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  FRAC_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  done.push_back(dev);
  return FRAC_OK;
}

// Non-blocking library streams per device for work that runs beside the caller's stream:
// which = 0 the side stream, 1 the stream a CUDA graph is captured on (the caller's stream
// may be the legacy default stream, which cannot be captured).
static int side_stream(cudaStream_t* out, int which = 0) {
  static std::mutex mu;
  static std::vector<cudaStream_t> per_dev[2];
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  std::vector<cudaStream_t>& v = per_dev[which ? 1 : 0];
  if ((int)v.size() <= dev) v.resize(dev + 1, nullptr);
  if (!v[dev]) FRAC_CUDA_TRY(cudaStreamCreateWithFlags(&v[dev], cudaStreamNonBlocking));
  *out = v[dev];
  return FRAC_OK;
}

static bool is_device_ptr(const void* p) { return ptr_kind(p) == PTR_DEVICE; }

// FRAC_EINVAL (with a detail) unless op was built on the current device and none of
// the given pointers is device memory of another device.
static int check_placement(const frac_op* op, const char* who, std::initializer_list<const void*> ptrs) {
  if (!op_on_current_device(op)) {
    record_detail("%s: the operator was built on device %d, which is not the current device", who, op->device);
    return FRAC_EINVAL;
  }
  for (const void* p : ptrs)
    if (p && ptr_kind(p) == PTR_OTHER_DEVICE) {
      record_detail("%s: a buffer lives on another device than the current one", who);
      return FRAC_EINVAL;
    }
  return FRAC_OK;
}

static int max_logm(int d) { return d == 1 ? 13 : (d == 2 ? 11 : 9); }

static int validate(const frac_problem* p) {
  if (!p) return FRAC_EINVAL;
  if (p->d < 1 || p->d > 3) return FRAC_EINVAL;
  if (!(p->alpha > 0.0 && p->alpha < 2.0)) return FRAC_EINVAL;
  if (p->degree < 0 || p->degree > 4) return FRAC_EINVAL;
  if (!(p->h > 0.0) || !std::isfinite(p->h)) return FRAC_EINVAL;
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return FRAC_EINVAL;
  if (p->gamma != 0.0 && !(p->gamma > p->alpha && p->gamma <= 2.0)) return FRAC_EINVAL;
  if (p->fft_lengths < FRAC_FFT_POW2 || p->fft_lengths > FRAC_FFT_AUTO) return FRAC_EINVAL;
  for (int i = 0; i < p->d; ++i) {
    if (p->n[i] < 1) return FRAC_EINVAL;
    if (p->degree >= 2 && ((p->n[i] + 1) % p->degree) != 0) return FRAC_EINVAL;
  }
  return FRAC_OK;
}

static thread_local char g_detail[256] = "";
static thread_local frac_batch_plan g_last_plan;  // last persistent 2D batch of this thread
static thread_local bool g_have_plan = false;
static thread_local int g_pin_size = 0, g_pin_cut = 11;  // frac_batch_pin_plan

int record_cuda_error(cudaError_t e, const char* file, int line, const char* expr) {
  const char* base = file;
  for (const char* c = file; *c; ++c)
    if (*c == '/') base = c + 1;
  std::snprintf(g_detail, sizeof(g_detail), "%s:%d %s -> %s (%s)", base, line, expr, cudaGetErrorName(e),
                cudaGetErrorString(e));
  return settle(e == cudaErrorMemoryAllocation ? FRAC_ENOMEM : FRAC_ECUDA);
}

void record_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

int record_check_failure(const char* file, int line, long long index) {
  std::snprintf(g_detail, sizeof(g_detail), "%s:%d device bounds check failed at index %lld", file, line, index);
  return FRAC_ECUDA;
}

}  // namespace frac

using namespace frac;

extern "C" {

const char* frac_error_detail(void) { return g_detail; }

const char* frac_strerror(int s) {
  switch (s) {
    case FRAC_OK: return "ok";
    case FRAC_EINVAL: return "invalid argument";
    case FRAC_ENOMEM: return "device allocation failed";
    case FRAC_ENOTSUP: return "not supported by this build";
    case FRAC_ENOCONV: return "solver did not converge within max_iter";
    case FRAC_EBREAKDOWN: return "conjugate-gradient breakdown";
    case FRAC_ETIMEOUT: return "bounded device wait ran out";
    case FRAC_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

// Relative cost of one transform of length M, by the passes it makes through shared
// memory: a power of two takes ceil(log2 M / 4) radix-16 passes on the register
// interface; a mixed length its np passes plus one (the odd passes leave part of
// the threads idle), plus two in 1D (the whole-solve kernel keeps its CG vectors in
// registers across the out-of-line passes).  Calibrated on GB300 FP32 applies:
// 2D 1280 and 640 beat 2048 and 1024, 1440 and 2016 lose to 2048, 3D 432 and 224
// lose to 512 and 256, 1D 6048 and 2240 lose to 8192 and 4096 in the solve.
static double fft_cost(int64_t M, int d) {
  MxPlan p;
  if ((M & (M - 1)) == 0) return (double)M * ((ilog2(M) + 3) / 4);
  if (!mx_plan(M, &p)) return INFINITY;
  return (double)M * (p.np + (d == 1 ? 2 : 1));
}

int frac_fft_length(int64_t n, int32_t d, int32_t fft_lengths, int64_t* M) {
  if (!M || n < 1 || d < 1 || d > 3) return FRAC_EINVAL;
  if (fft_lengths != FRAC_FFT_POW2 && fft_lengths != FRAC_FFT_SMOOTH && fft_lengths != FRAC_FFT_AUTO)
    return FRAC_EINVAL;
  const int64_t cap = int64_t(1) << max_logm(d);
  if (n > cap) return FRAC_ENOTSUP;  // M >= 2 n - 1 > cap (and no overflow below)
  int64_t m = 2;
  while (m < 2 * n - 1) m *= 2;
  if (m > cap) return FRAC_ENOTSUP;  // (also keeps the searches below within the limit)
  if (fft_lengths == FRAC_FFT_SMOOTH) {
    // the smallest 7-smooth length with a >= 4 that keeps M/2 - 1 >= n (the tau
    // system); the power of two when that one is beyond the limit
    if (2 * n + 2 <= cap) {
      const int64_t ms = mx_length_at_least(2 * n + 2);
      if (ms <= cap) m = ms;
    }
  } else if (fft_lengths == FRAC_FFT_AUTO) {
    // the cheapest by fft_cost among the power of two (when it holds the tau system)
    // and the 7-smooth lengths >= 2 n + 2 below twice the power of two
    const bool p2_tau = m / 2 - 1 >= n;
    double best = p2_tau ? fft_cost(m, d) : INFINITY;
    int64_t pick = m;
    for (int64_t c = (2 * n + 2 + 15) / 16 * 16; c <= std::min(cap, p2_tau ? m : 2 * m); c += 16) {
      const double cost = fft_cost(c, d);
      if (cost < best) {
        best = cost;
        pick = c;
      }
    }
    m = pick;
  }
  if (m > cap) return FRAC_ENOTSUP;
  *M = m;
  return FRAC_OK;
}

int frac_coeffs(const frac_problem* prob, frac_op** out, void* stream) {
  if (!out) return FRAC_EINVAL;
  *out = nullptr;
  FRAC_TRY(validate(prob));
  cudaStream_t st = (cudaStream_t)stream;
  const int d = prob->d;
  int64_t Ma[3] = {1, 1, 1}, nmax = 0;
  MxPlan plans[3];
  for (int i = 0; i < d; ++i) {
    FRAC_TRY(frac_fft_length(prob->n[i], d, prob->fft_lengths, &Ma[i]));
    if ((Ma[i] & (Ma[i] - 1)) != 0 && !mx_plan(Ma[i], &plans[i])) return FRAC_ENOTSUP;
    nmax = std::max<int64_t>(nmax, prob->n[i]);
  }
  FRAC_TRY(keep_pool_memory());
  frac_op* op = new (std::nothrow) frac_op();
  if (!op) return FRAC_ENOMEM;
  op->prob = *prob;
  for (int i = d; i < 3; ++i) op->prob.n[i] = 1;
  op->square = 1;
  for (int i = 0; i < 3; ++i) {
    op->na[i] = i < d ? prob->n[i] : 1;
    op->Ma[i] = Ma[i];
    op->Ka[i] = i < d ? Ma[i] / 2 + 1 : 1;
    op->plan[i] = plans[i];
    op->logma[i] = i >= d ? 0 : (plans[i].m ? -1 : ilog2(Ma[i]));
    if (i < d && prob->n[i] != prob->n[0]) op->square = 0;
  }
  op->N = nmax + 1;  // the generator covers [0, L]^d with L the largest extent
  op->n = op->na[0];
  op->M = op->Ma[0];
  op->logm = op->logma[0];
  op->K = op->Ka[0];
  op->nd = op->ngen = op->nsym = 1;
  for (int i = 0; i < d; ++i) {
    op->nd *= op->na[i];
    op->ngen *= (op->N + 1);
    op->nsym *= op->Ka[i];
  }
  op->c = c_dalpha(d, prob->alpha);
  cudaGetDevice(&op->device);
  op->nsym_alloc = d == 1 ? op->nsym : (op->Ka[0] + 3) / 4 * 4 * op->Ka[1] * (d == 3 ? op->Ka[2] : 1);
  op->device_bytes = op->ngen * sizeof(double) + 2 * op->nsym_alloc * (sizeof(double) + sizeof(float));
  int s = FRAC_OK;
  if (cudaMalloc(&op->a, op->ngen * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&op->lam64, op->nsym_alloc * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&op->lam32, op->nsym_alloc * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&op->pinv64, op->nsym_alloc * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&op->pinv32, op->nsym_alloc * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    s = FRAC_ENOMEM;
  }
  for (int i = 0; i < d && s == FRAC_OK; ++i) s = prepare_twiddles_len(op->Ma[i]);
  if (s == FRAC_OK) s = build_coefficients(op, st);
  if (s == FRAC_OK) s = xy_prepare(op);
  if (s != FRAC_OK) {
    frac_op_free(op);
    return s;
  }
  *out = op;
  return FRAC_OK;
}

void frac_op_free(frac_op* op) {
  if (!op) return;
  if (op->a) cudaFree(op->a);
  if (op->lam64) cudaFree(op->lam64);
  if (op->lam32) cudaFree(op->lam32);
  if (op->pinv64) cudaFree(op->pinv64);
  if (op->pinv32) cudaFree(op->pinv32);
  delete op;
}

int frac_op_info(const frac_op* op, frac_op_info_t* info) {
  if (!op || !info) return FRAC_EINVAL;
  info->c_dalpha = op->c;
  info->a0 = op->a0;
  info->far_field = op->far_field;
  info->norm_bound = op->norm_bound;
  info->fft_len = op->M;
  info->n_gen = op->N + 1;
  info->device_bytes = op->device_bytes;
  info->precond_ok = op->precond_ok;
  for (int i = 0; i < 3; ++i) {
    info->n[i] = op->na[i];
    info->fft_lens[i] = op->Ma[i];
  }
  return FRAC_OK;
}

int frac_op_generator(const frac_op* op, double* a, size_t count) {
  if (!op || !a || count != (size_t)op->ngen) return FRAC_EINVAL;
  FRAC_CUDA_TRY(cudaMemcpy(a, op->a, count * sizeof(double), cudaMemcpyDeviceToHost));
  return FRAC_OK;
}

}  // extern "C"

// Library streams per device for the host-buffer pipeline below.
constexpr int kCopyStreams = 3;
static int copy_streams(cudaStream_t* out) {
  static std::mutex mu;
  static std::vector<std::vector<cudaStream_t>> per_dev;
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1);
  if (per_dev[dev].empty()) {
    for (int i = 0; i < kCopyStreams; ++i) {
      cudaStream_t s;
      FRAC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      per_dev[dev].push_back(s);
    }
  }
  for (int i = 0; i < kCopyStreams; ++i) out[i] = per_dev[dev][i];
  return FRAC_OK;
}

static int run_apply(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, void* ws, bool precond,
                     cudaStream_t st) {
  if (precond)
    return dtype == FRAC_F64 ? precond_t<double>(op, (const double*)u, (double*)y, batch, ws, st)
                             : precond_t<float>(op, (const float*)u, (float*)y, batch, ws, st);
  return dtype == FRAC_F64 ? apply_t<double>(op, (const double*)u, (double*)y, batch, ws, st)
                           : apply_t<float>(op, (const float*)u, (float*)y, batch, ws, st);
}

// Host input and output, several fields: a three-stage pipeline over chunks of
// fields on the library's three streams, host-to-device copies on the first, the
// applies on the second, device-to-host copies on the third, through a ring of
// pipe_slots() device input and output buffers.  Events order a chunk's three
// stages and the reuse of a slot: a chunk's input copy waits for the apply that
// last read its input buffer, its apply for the output copy that last read its
// output buffer.  The two copy directions run on separate copy engines and the
// applies (one stream, one workspace) overlap them; the host link bounds the whole
// (the same pipeline with no applies at all takes as long).  Returns after the
// last copy has landed.
constexpr size_t kPipeChunkBytes = 28u << 20;
constexpr int kPipeSlots = 3;
static size_t pipe_chunk_bytes() {  // FRAC_PIPE_CHUNK_MB overrides the chunk size (tuning), read once
  static const size_t v = [] {
    const char* e = std::getenv("FRAC_PIPE_CHUNK_MB");
    const long long mb = e ? std::atoll(e) : 0;
    return mb > 0 ? (size_t)mb << 20 : kPipeChunkBytes;
  }();
  return v;
}
static int pipe_slots() {  // FRAC_PIPE_SLOTS overrides the ring size (tuning, 2..8), read once
  static const int v = [] {
    const char* e = std::getenv("FRAC_PIPE_SLOTS");
    const int k = e ? std::atoi(e) : 0;
    return k >= 2 && k <= 8 ? k : kPipeSlots;
  }();
  return v;
}
static int apply_host_pipelined(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, bool precond,
                                cudaStream_t st) {
  constexpr int kMaxSlots = 8;
  const size_t es = dtype == FRAC_F64 ? sizeof(double) : sizeof(float);
  const size_t fb = (size_t)op->nd * es;
  int64_t nch = std::min<int64_t>(batch, std::max<int64_t>(1, (int64_t)((batch * fb) / pipe_chunk_bytes())));
  nch = std::min<int64_t>(nch, 256);
  const int64_t per = (batch + nch - 1) / nch;
  nch = (batch + per - 1) / per;
  cudaStream_t ss[kCopyStreams];
  FRAC_TRY(copy_streams(ss));
  cudaStream_t s_in = ss[0], s_cmp = ss[1], s_out = ss[2];
  const int K = (int)std::min<int64_t>(pipe_slots(), nch);
  // device buffers (allocated on the caller's stream, freed there after the join)
  void* in[kMaxSlots] = {};
  void* out[kMaxSlots] = {};
  void* ws = nullptr;
  cudaEvent_t ev[3][kMaxSlots] = {};  // input landed, apply done, output landed
  cudaEvent_t fork = nullptr, join[3] = {};
  int s = FRAC_OK;
  const size_t wsb = apply_workspace_bytes(op, dtype, per);
  for (int k = 0; k < K && s == FRAC_OK; ++k)
    if (cudaMallocAsync(&in[k], per * fb, st) != cudaSuccess || cudaMallocAsync(&out[k], per * fb, st) != cudaSuccess)
      s = FRAC_ENOMEM;
  if (s == FRAC_OK && wsb && cudaMallocAsync(&ws, wsb, st) != cudaSuccess) s = FRAC_ENOMEM;
  for (int i = 0; i < 3 && s == FRAC_OK; ++i)
    for (int k = 0; k < K && s == FRAC_OK; ++k)
      if (cudaEventCreateWithFlags(&ev[i][k], cudaEventDisableTiming) != cudaSuccess) s = FRAC_ECUDA;
  if (s == FRAC_OK && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(s_in, fork, 0) != cudaSuccess ||
                       cudaStreamWaitEvent(s_cmp, fork, 0) != cudaSuccess ||
                       cudaStreamWaitEvent(s_out, fork, 0) != cudaSuccess))
    s = FRAC_ECUDA;
  for (int64_t c = 0; c < nch && s == FRAC_OK; ++c) {
    const int k = (int)(c % K);
    const int64_t b0 = c * per, nb = std::min<int64_t>(per, batch - b0);
    const char* src = (const char*)u + b0 * fb;
    char* dst = (char*)y + b0 * fb;
    // stage 1: the slot's input buffer is free once the apply of chunk c - K has read it
    if ((c >= K && cudaStreamWaitEvent(s_in, ev[1][k], 0) != cudaSuccess) ||
        cudaMemcpyAsync(in[k], src, nb * fb, cudaMemcpyHostToDevice, s_in) != cudaSuccess ||
        cudaEventRecord(ev[0][k], s_in) != cudaSuccess) {
      s = FRAC_ECUDA;
      break;
    }
    // stage 2: after the input landed and the output copy of chunk c - K has read the output buffer
    if (cudaStreamWaitEvent(s_cmp, ev[0][k], 0) != cudaSuccess ||
        (c >= K && cudaStreamWaitEvent(s_cmp, ev[2][k], 0) != cudaSuccess)) {
      s = FRAC_ECUDA;
      break;
    }
    s = run_apply(op, in[k], out[k], dtype, nb, ws, precond, s_cmp);
    if (s != FRAC_OK) break;
    // stage 3
    if (cudaEventRecord(ev[1][k], s_cmp) != cudaSuccess || cudaStreamWaitEvent(s_out, ev[1][k], 0) != cudaSuccess ||
        cudaMemcpyAsync(dst, out[k], nb * fb, cudaMemcpyDeviceToHost, s_out) != cudaSuccess ||
        cudaEventRecord(ev[2][k], s_out) != cudaSuccess)
      s = FRAC_ECUDA;
  }
  // join the three streams into the caller's stream, then free there
  if (fork) {
    const cudaStream_t three[3] = {s_in, s_cmp, s_out};
    for (int i = 0; i < 3; ++i)
      if (cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess &&
          cudaEventRecord(join[i], three[i]) == cudaSuccess)
        cudaStreamWaitEvent(st, join[i], 0);
  }
  for (int k = 0; k < K; ++k) {
    if (in[k]) cudaFreeAsync(in[k], st);
    if (out[k]) cudaFreeAsync(out[k], st);
  }
  if (ws) cudaFreeAsync(ws, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == FRAC_OK && e != cudaSuccess) s = FRAC_ECUDA;
  for (int i = 0; i < 3; ++i) {
    for (int k = 0; k < K; ++k)
      if (ev[i][k]) cudaEventDestroy(ev[i][k]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (fork) cudaEventDestroy(fork);
  return settle(s);
}

// Stream-ordered temporaries of one call, freed on its stream on every return
// path; a call that has queued copies from or to the caller's host memory (host_io)
// also waits for its stream before it returns, on an error path too.
struct Temps {
  cudaStream_t st;
  void* p[4] = {};
  int n = 0;
  bool host_io = false;
  template <typename P>
  int get(P** out, size_t bytes) {
    void* q = nullptr;
    FRAC_CUDA_TRY(cudaMallocAsync(&q, bytes, st));
    p[n++] = q;
    *out = static_cast<P*>(q);
    return FRAC_OK;
  }
  ~Temps() {
    for (int i = 0; i < n; ++i) cudaFreeAsync(p[i], st);
    if (host_io && cudaStreamSynchronize(st) != cudaSuccess) (void)cudaGetLastError();
  }
};

// frac_apply (precond = false) and frac_precond (precond = true): device or host buffers.
static int apply_entry(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, void* stream,
                       bool precond) {
  if (!op || batch < 0 || (dtype != FRAC_F32 && dtype != FRAC_F64)) return FRAC_EINVAL;
  if (precond && !op->precond_ok) return FRAC_ENOTSUP;
  if (batch == 0) return FRAC_OK;
  if (!u || !y || u == y) return FRAC_EINVAL;
  FRAC_TRY(check_placement(op, precond ? "frac_precond" : "frac_apply", {u, y}));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = dtype == FRAC_F64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)batch * op->nd * es;
  const bool du = is_device_ptr(u), dy = is_device_ptr(y);
  if ((du && ((uintptr_t)u % es)) || (dy && ((uintptr_t)y % es))) return FRAC_EINVAL;
  if (!du && !dy && batch >= 2 && bytes >= 2 * pipe_chunk_bytes())
    return apply_host_pipelined(op, u, y, dtype, batch, precond, st);
  Temps tmp{st};
  tmp.host_io = !du || !dy;
  void* ws = nullptr;
  const size_t wsb = apply_workspace_bytes(op, dtype, batch);
  if (wsb) FRAC_TRY(tmp.get(&ws, wsb));
  const void* ud = u;
  void* yd = y;
  if (!du) {
    void* tu = nullptr;
    FRAC_TRY(tmp.get(&tu, bytes));
    FRAC_CUDA_TRY(cudaMemcpyAsync(tu, u, bytes, cudaMemcpyHostToDevice, st));
    ud = tu;
  }
  if (!dy) FRAC_TRY(tmp.get(&yd, bytes));
  int s;
  if (precond)
    s = dtype == FRAC_F64 ? precond_t<double>(op, (const double*)ud, (double*)yd, batch, ws, st)
                          : precond_t<float>(op, (const float*)ud, (float*)yd, batch, ws, st);
  else
    s = dtype == FRAC_F64 ? apply_t<double>(op, (const double*)ud, (double*)yd, batch, ws, st)
                          : apply_t<float>(op, (const float*)ud, (float*)yd, batch, ws, st);
  if (s == FRAC_OK && !dy) {
    const cudaError_t e = cudaMemcpyAsync(y, yd, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaMemcpyAsync");
  }
  if (!du || !dy) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (s == FRAC_OK && e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaStreamSynchronize");
  }
  return settle(s);
}

extern "C" {

int frac_apply(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, void* stream) {
  return apply_entry(op, u, y, dtype, batch, stream, false);
}

int frac_precond(const frac_op* op, const void* r, void* z, int dtype, int64_t batch, void* stream) {
  return apply_entry(op, r, z, dtype, batch, stream, true);
}

int frac_boundary(const frac_op* op, const double* g_ext, const double* far, double* b, void* stream) {
  if (!op || !g_ext || !b) return FRAC_EINVAL;
  FRAC_TRY(check_placement(op, "frac_boundary", {g_ext, far, b}));
  cudaStream_t st = (cudaStream_t)stream;
  const int d = op->prob.d;
  int64_t ne = 1;
  for (int i = 0; i < d; ++i) ne *= op->na[i] + 2 * op->N;
  const size_t gbytes = ne * sizeof(double), bbytes = op->nd * sizeof(double);
  const bool dgx = is_device_ptr(g_ext), dfar = far && is_device_ptr(far), db = is_device_ptr(b);
  Temps tmp{st};
  tmp.host_io = !dgx || (far && !dfar) || !db;
  const double *gd = g_ext, *fard = far;
  double* bd = b;
  if (!dgx) {
    double* t = nullptr;
    FRAC_TRY(tmp.get(&t, gbytes));
    FRAC_CUDA_TRY(cudaMemcpyAsync(t, g_ext, gbytes, cudaMemcpyHostToDevice, st));
    gd = t;
  }
  if (far && !dfar) {
    double* t = nullptr;
    FRAC_TRY(tmp.get(&t, bbytes));
    FRAC_CUDA_TRY(cudaMemcpyAsync(t, far, bbytes, cudaMemcpyHostToDevice, st));
    fard = t;
  }
  if (!db) FRAC_TRY(tmp.get(&bd, bbytes));
  int s = boundary_device(op, gd, fard, bd, st);
  if (s == FRAC_OK && !db) {
    const cudaError_t e = cudaMemcpyAsync(b, bd, bbytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaMemcpyAsync");
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == FRAC_OK && e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaStreamSynchronize");
  return settle(s);
}

int frac_solve(const frac_op* op, const double* f, const double* g, double* u, const frac_solve_opts* opts,
               frac_solve_info* info, void* stream) {
  if (!op || !f || !u || !opts || !info) return FRAC_EINVAL;
  if (!(opts->rtol > 0.0) || opts->max_iter < 1) return FRAC_EINVAL;
  if (opts->precision != FRAC_PLAIN_F64 && opts->precision != FRAC_MIXED_IR) return FRAC_EINVAL;
  FRAC_TRY(check_placement(op, "frac_solve", {f, g, u}));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = op->nd * sizeof(double);
  const bool df = is_device_ptr(f), du = is_device_ptr(u), dg = g && is_device_ptr(g);
  const double* fd = f;
  double* ud = u;
  if (!df) {
    for (int64_t i = 0; i < op->nd; ++i)
      if (!std::isfinite(f[i])) return FRAC_EINVAL;
  }
  if (g && !dg) {
    for (int64_t i = 0; i < op->nd; ++i)
      if (!std::isfinite(g[i])) return FRAC_EINVAL;
  }
  Temps tmp{st};
  tmp.host_io = !df || (g && !dg) || !du;
  if (!df || g) {  // device right-hand side: f, or f - g
    double* tf = nullptr;
    FRAC_TRY(tmp.get(&tf, bytes));
    if (!df) FRAC_CUDA_TRY(cudaMemcpyAsync(tf, f, bytes, cudaMemcpyHostToDevice, st));
    if (g) {
      const double* gd = g;
      if (!dg) {
        double* tg = nullptr;
        FRAC_TRY(tmp.get(&tg, bytes));
        FRAC_CUDA_TRY(cudaMemcpyAsync(tg, g, bytes, cudaMemcpyHostToDevice, st));
        gd = tg;
      }
      FRAC_TRY(subtract_device(df ? f : tf, gd, tf, op->nd, st));
    }
    fd = tf;
  }
  if (!du) {
    FRAC_TRY(tmp.get(&ud, bytes));
    if (opts->use_x0) FRAC_CUDA_TRY(cudaMemcpyAsync(ud, u, bytes, cudaMemcpyHostToDevice, st));
  }
  int s = solve_device(op, fd, ud, opts, info, st);
  if (s == FRAC_OK && !du) {
    const cudaError_t e = cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaMemcpyAsync");
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == FRAC_OK && e != cudaSuccess) s = record_cuda_error(e, __FILE__, __LINE__, "cudaStreamSynchronize");
  if (s != FRAC_OK) return settle(s);
  if (std::isnan(info->rel_resid)) {
    info->status = FRAC_EINVAL;  // non-finite data in f
    return FRAC_EINVAL;
  }
  return info->status;
}

int frac_batch_pin_plan(int32_t cluster_size, int32_t first_cluster_logm) {
  if (cluster_size == 0) {
    g_pin_size = 0;
    return FRAC_OK;
  }
  if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 && cluster_size != 16)
    return FRAC_EINVAL;
  if (first_cluster_logm < kBatch2dMinLog || first_cluster_logm > kBatch2dMaxLog + 1) return FRAC_EINVAL;
  g_pin_size = cluster_size;
  g_pin_cut = cluster_size == 1 ? kBatch2dMaxLog + 1 : first_cluster_logm;
  return FRAC_OK;
}

int frac_batch_last_plan(frac_batch_plan* out) {
  if (!out || !g_have_plan) return FRAC_EINVAL;
  *out = g_last_plan;
  return FRAC_OK;
}

int frac_solve_batch(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                     const frac_solve_opts* opts, frac_solve_info* info, void* stream) {
  if (count < 0 || (count > 0 && (!ops || !f || !u || !opts || !info))) return FRAC_EINVAL;
  if (count == 0) return FRAC_OK;
  if (!(opts->rtol > 0.0) || opts->max_iter < 1) return FRAC_EINVAL;
  if (opts->precision != FRAC_PLAIN_F64 && opts->precision != FRAC_MIXED_IR) return FRAC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // 1D problems with device buffers: whole solves, one block each, one launch per FFT length
  std::vector<int64_t> oned, rest;
  for (int64_t i = 0; i < count; ++i) {
    if (!ops[i] || !f[i] || !u[i]) return FRAC_EINVAL;
    if (ops[i]->prob.d == 1 && is_device_ptr(f[i]) && is_device_ptr(u[i])) oned.push_back(i);
    else rest.push_back(i);
  }
  int first = FRAC_OK;
  // 2D problems of the persistent kernel's FFT lengths: one launch
  std::vector<int64_t> wide, others;
  for (int64_t i : rest) {
    if (batch2d_eligible(ops[i], opts) && is_device_ptr(f[i]) && is_device_ptr(u[i])) wide.push_back(i);
    else others.push_back(i);
  }
  rest.swap(others);
  BatchPending p2, p1;
  if (!oned.empty() || !wide.empty()) {
    // Everything that waits on the device or builds tables runs first (the
    // autotuner's timings, twiddles); the uploads, the persistent 2D launch and
    // the 1D launches (on a side stream forked from the capture, so that they run
    // beside the 2D launch) are then captured into one CUDA graph on a library
    // stream, and the graph is launched once on st.
    if (!wide.empty()) FRAC_TRY(batch2d_prepare((int64_t)wide.size(), ops, f, wide.data(), st));
    for (int64_t i : oned) FRAC_TRY(prepare_twiddles_len(ops[i]->M));
    cudaStream_t cap = nullptr;
    FRAC_TRY(side_stream(&cap, 1));
    cudaStream_t s1 = cap;
    if (!oned.empty() && !wide.empty()) FRAC_TRY(side_stream(&s1, 0));
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    struct Release {
      cudaEvent_t *a, *b;
      cudaGraph_t* g;
      cudaGraphExec_t* x;
      ~Release() {
        if (*a) cudaEventDestroy(*a);
        if (*b) cudaEventDestroy(*b);
        if (*x) cudaGraphExecDestroy(*x);
        if (*g) cudaGraphDestroy(*g);
      }
    } rel{&fork, &join, &graph, &exec};
    if (s1 != cap) {
      FRAC_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      FRAC_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    }
    FRAC_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    int cs = FRAC_OK;
    frac_batch_plan plan{};
    if (s1 != cap) {
      if (cudaEventRecord(fork, cap) != cudaSuccess || cudaStreamWaitEvent(s1, fork, 0) != cudaSuccess)
        cs = FRAC_ECUDA;
    }
    if (cs == FRAC_OK && !wide.empty())
      cs = solve_batch_2d((int64_t)wide.size(), ops, f, u, opts, wide.data(), cap, &plan, g_pin_size, g_pin_cut, &p2);
    if (cs == FRAC_OK && !oned.empty()) cs = solve_batch_1d((int64_t)oned.size(), ops, f, u, opts, oned.data(), s1, &p1);
    if (cs == FRAC_OK && s1 != cap) {  // the side stream rejoins the capture
      if (cudaEventRecord(join, s1) != cudaSuccess || cudaStreamWaitEvent(cap, join, 0) != cudaSuccess)
        cs = FRAC_ECUDA;
    }
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);  // always ends the capture
    if (cs != FRAC_OK) return settle(cs);
    FRAC_CUDA_TRY(ec);
    FRAC_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    FRAC_CUDA_TRY(cudaGraphLaunch(exec, st));
    // the results of both branches are complete when st is: collect (and free) on st
    p1.st = st;
    p2.st = st;
    if (!wide.empty()) {
      g_last_plan = plan;
      g_have_plan = true;
      FRAC_TRY(p2.collect(info));
    }
    if (!oned.empty()) FRAC_TRY(p1.collect(info));
  }
  for (const std::vector<int64_t>* v : {&oned, &wide})
    for (int64_t i : *v) {
      if (std::isnan(info[i].rel_resid)) info[i].status = FRAC_EINVAL;
      if (info[i].status == FRAC_ECUDA)
        record_detail("persistent batch: problem %lld failed the kernel's scratch and shared-memory check",
                      (long long)i);
      if (info[i].status != FRAC_OK && first == FRAC_OK) first = info[i].status;
    }
  if (!rest.empty()) {
    // the other problems progress together through a solve engine (their kernels overlap)
    frac_engine* e = nullptr;
    const int ns = (int)std::min<size_t>(8, rest.size());
    FRAC_TRY(frac_engine_create(ns, &e));
    int s = engine_wait_for(e, st);
    std::vector<std::pair<int64_t, int64_t>> ids;  // (job, index)
    for (int64_t i : rest) {
      int64_t job = 0;
      int r = s == FRAC_OK ? frac_engine_submit(e, ops[i], f[i], u[i], opts, &job) : s;
      if (r != FRAC_OK) {
        info[i] = frac_solve_info{r, 0, 0, 0, NAN};
        if (first == FRAC_OK) first = r;
      } else {
        ids.emplace_back(job, i);
      }
    }
    std::vector<frac_job_result> done(ids.size() + 1);
    size_t got = 0;
    while (got < ids.size()) {
      int cnt = 0;
      int r = frac_engine_poll(e, 1, done.data(), (int)done.size(), &cnt);
      if (r != FRAC_OK && first == FRAC_OK) first = r;
      if (cnt == 0 && r != FRAC_OK) break;
      for (int k = 0; k < cnt; ++k)
        for (auto& pr : ids)
          if (pr.first == done[k].job) info[pr.second] = done[k].info;
      got += cnt;
    }
    frac_engine_destroy(e);
    for (int64_t i : rest)
      if (info[i].status != FRAC_OK && first == FRAC_OK) first = info[i].status;
  }
  return settle(first);
}

}  // extern "C"
