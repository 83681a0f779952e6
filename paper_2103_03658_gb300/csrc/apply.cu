// y = A u by circulant embedding and FFT (Sec. 2.1: the Toeplitz structure
// allows an O(N log N) product), A = -c_{d,alpha} T(a).  The scaled symbol Lambda (real, even,
// stored on [0, M/2]^d) already carries -c / M (d = 1) or -c / (2 M^d)
// (d >= 2, the 2 from the two-rows-per-complex packing below).
//
// d = 1: one kernel; two vectors share one complex line (z = u_a + i u_b,
//        A is real so Re and Im stay separate); pad, FFT, * Lambda, iFFT,
//        extract, all in shared memory.
// d = 2: rows (R2C, two rows per complex line, spectra separated in the
//        epilogue) -> columns (pad, FFT, * Lambda, iFFT, extract; in place)
//        -> rows (C2R, two rows per line).
// d = 3: rows -> y-columns (pad, FFT) -> z-columns (pad, FFT, * Lambda, iFFT,
//        extract; in place) -> y-columns (iFFT, extract) -> rows.
#include <cstdio>

#include "apply.cuh"
#include "fft.cuh"
#include "prof.cuh"

namespace frac {

using namespace fft;

// Intermediate spectra are stored column-blocked: entry (row, k) of a slab of
// `n` rows lives at (k / B) (n B) + row B + (k % B), B = 32 bytes / complex
// size (4 for FP32, 2 for FP64).  A tile of B adjacent columns is then one
// contiguous chunk, read and written with one lane per column and
// consecutive lanes on consecutive rows, and every row segment is a full
// 32-byte sector.  Every FFT below keeps the line in registers at entry and
// exit (fft_reg): loads go straight from global memory into registers.
// ---------------------------------------------------------------------------

template <typename T> __host__ __device__ constexpr int blk() { return 32 / (int)sizeof(cplx_t<T>); }

// minimum resident blocks per SM requested from the compiler: at least 512 resident
// threads for FP32 kernels and 256 for FP64 (registers capped at 128 and 255 per thread);
// the row kernels ask for twice that
// (clamped to the 32 resident blocks an SM can hold)
__host__ __device__ constexpr int clamp_blocks(int b) { return b < 1 ? 1 : (b > 32 ? 32 : b); }
template <typename T> __host__ __device__ constexpr int minb(int nt) {
  return clamp_blocks(((int)sizeof(T) == 4 ? 512 : 256) / nt);
}
// the row kernels hold one FFT per thread group and need fewer registers: 1024 / 512
template <typename T> __host__ __device__ constexpr int minb_rows(int nt) {
  return clamp_blocks(((int)sizeof(T) == 4 ? 1024 : 512) / nt);
}
// the column kernels: FP32 fits 64 registers without spills (two 512-thread
// blocks per SM); FP64 needs more than 128 and keeps one block
template <typename T> __host__ __device__ constexpr int minb_cols(int nt) {
  return sizeof(T) == 4 ? minb_rows<T>(nt) : minb<T>(nt);
}

// ---------------------------------------------------------------------------
// d = 1: whole convolution per line (two vectors per complex line)
// ---------------------------------------------------------------------------

template <typename T, int LOGM, int LINES>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb<T>(LINES * tpl(LOGM)))
k_conv1d(const T* __restrict__ u, T* __restrict__ y, int n, int64_t batch, const T* __restrict__ lam,
         const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  const int64_t va = 2 * ((int64_t)blockIdx.x * LINES + line), vb = va + 1;
  const bool ha = va < batch, hb = vb < batch;
  // n <= M/2: entries e >= E/2 (x >= M/2) are zero padding, and only
  // outputs x < n are kept, so both transforms are half-pruned
  C v[E];
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int x = tl + e * TPL;
    T re = (x < n && ha) ? u[va * n + x] : T(0);
    T im = (x < n && hb) ? u[vb * n + x] : T(0);
    v[e] = C{re, im};
  }
  fft_reg<C, LOGM, false, true, false>(v, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    v[e] = cscale(v[e], lam[k <= M / 2 ? k : M - k]);
  }
  fft_reg<C, LOGM, true, false, true>(v, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {
      if (ha) y[va * n + x] = v[e].x;
      if (hb) y[vb * n + x] = v[e].y;
    }
  }
}

// column-blocked layout, slabs of n rows, KB = ceil(K / B) blocks per slab:
// entry (row, k) at rowbase(row) + (k / B) n B + k % B
template <int B>
__device__ __forceinline__ int64_t wrow(int64_t row, int n, int KB) {
  const int64_t slab = row / n, r = row - slab * n;
  return slab * KB * (int64_t)n * B + r * B;
}
template <int B>
__device__ __forceinline__ int64_t wcol(int k, int n) {
  return (int64_t)(k / B) * n * B + (k % B);
}

// Block sum of a per-thread value (FP64), valid in every thread; red needs 32 doubles.
__device__ __forceinline__ double block_sum_all(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Every block stores its total in partials[blockIdx.x]; the last block to
// arrive (counter) sums all of them in index order and calls fin(sum) in
// thread 0, then resets the counter for the next use.
template <typename F>
__device__ __forceinline__ void last_block_reduce(double total, double* partials, unsigned int* counter, double* red,
                                                  F fin) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = total;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum_all(s, red);
  if (threadIdx.x == 0) {
    fin(s);
    *counter = 0;
  }
}

// ---------------------------------------------------------------------------
// Rows, forward: two real rows -> one complex FFT -> two half spectra
// U0 = Z[k] + conj Z[M-k], U1 = -i (Z[k] - conj Z[M-k]), k in [0, M/2]
// (stored without the 1/2 of the separation; the symbol carries it).
// ---------------------------------------------------------------------------

// CG = true: the input is p = r + beta p (beta from st), written back to u (= p)
// on the way in; the block returns at once when st->done is set.
template <typename T, int LOGM, int LINES, bool CG>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb_rows<T>(LINES * tpl(LOGM)))
k_rows_fwd(const T* u, cplx_t<T>* __restrict__ W, int n, int64_t nrows, int KB,
           const cplx_t<T>* __restrict__ tw, const T* __restrict__ r, const CGState* st) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM), B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * LINES + line), r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
  C v[E];
  if constexpr (CG) {
    const T be = (T)st->beta;
    T* p = const_cast<T*>(u);
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {  // x < n <= M/2: e < E/2
      const int x = tl + e * TPL;
      T re = T(0), im = T(0);
      if (x < n && h0) {
        re = r[r0 * n + x] + be * p[r0 * n + x];
        p[r0 * n + x] = re;
      }
      if (x < n && h1) {
        im = r[r1 * n + x] + be * p[r1 * n + x];
        p[r1 * n + x] = im;
      }
      v[e] = C{re, im};
    }
  } else {
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const int x = tl + e * TPL;
      T re = (x < n && h0) ? u[r0 * n + x] : T(0);
      T im = (x < n && h1) ? u[r1 * n + x] : T(0);
      v[e] = C{re, im};
    }
  }
  fft_reg<C, LOGM, false, true, false>(v, buf, tl, tw);  // upper half is zero padding
  // separation needs Z[k] and Z[M-k] for k in [0, M/2]: each thread keeps its
  // lower-half Z[k] in registers and reads the mirror from the upper half,
  // which alone goes through the line buffer
  __syncthreads();
#pragma unroll
  for (int e = E / 2; e < E; ++e) buf[pidx(tl + e * TPL)] = v[e];
  __syncthreads();
  C* W0 = W + wrow<B>(r0, n, KB);
  C* W1 = W + wrow<B>(r1, n, KB);
  auto emit = [&](int k, C z, C zc) {
    const C s = cadd(z, zc), dd = csub(z, zc);
    const int64_t kc = wcol<B>(k, n);
    if (h0) W0[kc] = s;
    if (h1) W1[kc] = C{dd.y, -dd.x};
  };
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int k = tl + e * TPL;  // k < M/2; M - k is in the upper half unless k = 0
    emit(k, v[e], cconj(k == 0 ? v[e] : buf[pidx(M - k)]));
  }
  if (tl == 0) emit(M / 2, v[E / 2], cconj(v[E / 2]));
}

// ---------------------------------------------------------------------------
// Rows, inverse: two half spectra -> one complex line (Hermitian extension)
// -> iFFT -> two real rows (first n entries).
// ---------------------------------------------------------------------------

// CG = true: also per-block partial sums of p.y (p at the same points) into
// partials[blockIdx.x]; the last block to finish sums them in index order and
// sets st->pq, st->alpha (or flags a breakdown).  Returns at once when st->done.
template <typename T, int LOGM, int LINES, bool CG>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb_rows<T>(LINES * tpl(LOGM)))
k_rows_inv(const cplx_t<T>* __restrict__ W, T* __restrict__ y, int n, int64_t nrows, int KB,
           const cplx_t<T>* __restrict__ tw, const T* __restrict__ p, CGState* st, double* partials) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM), B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * LINES + line), r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
  C v[E];
  const C* W0 = W + wrow<B>(h0 ? r0 : 0, n, KB);
  const C* W1 = W + wrow<B>(h1 ? r1 : 0, n, KB);
  // line z = W0 + i W1 extended Hermitian-wise: z[x] = W0[x] + i W1[x] and
  // z[M-x] = conj(W0[x]) + i conj(W1[x]) for x in [0, M/2], so each half
  // spectrum entry is read once; the thread that reads W[x] leaves z[M-x] in
  // the line buffer for its owner
  auto load = [&](int x, C& lo, C& hi) {
    const int64_t kc = wcol<B>(x, n);
    const C v0 = h0 ? W0[kc] : C{0, 0};
    const C v1 = h1 ? W1[kc] : C{0, 0};
    lo = C{v0.x - v1.y, v0.y + v1.x};   // v0 + i v1
    hi = C{v0.x + v1.y, v1.x - v0.y};   // conj(v0) + i conj(v1)
  };
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int x = tl + e * TPL;  // x < M/2
    C hi;
    load(x, v[e], hi);
    if (x > 0) buf[pidx(M - x)] = hi;
  }
  if (tl == 0) {
    C lo, hi;
    load(M / 2, lo, hi);
    buf[pidx(M / 2)] = lo;
  }
  __syncthreads();
#pragma unroll
  for (int e = E / 2; e < E; ++e) v[e] = buf[pidx(tl + e * TPL)];
  fft_reg<C, LOGM, true, false, true>(v, buf, tl, tw);  // only x < n <= M/2 is kept
  T dot = T(0);
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {
      if (h0) {
        y[r0 * n + x] = v[e].x;
        if (CG) dot += v[e].x * p[r0 * n + x];
      }
      if (h1) {
        y[r1 * n + x] = v[e].y;
        if (CG) dot += v[e].y * p[r1 * n + x];
      }
    }
  }
  if constexpr (CG) {
    double* red = reinterpret_cast<double*>(smem_raw);  // the FFT lines are no longer needed
    const double total = block_sum_all(dot, red);
    last_block_reduce(total, partials, &st->count_pq, red, [&](double pq) {
      st->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = FRAC_EBREAKDOWN;
        st->done = 1;
      } else {
        st->alpha = st->rr / pq;
      }
    });
  }
}

// ---------------------------------------------------------------------------
// Columns: one tile of B adjacent columns per block, TPL threads per column
// (lane order: column fastest).  Modes:
//   SYM2 (d = 2): slab o = field, pad n -> M, FFT, * Lambda[kr][k1], iFFT, keep n; in place.
//   YFWD (d = 3): slab o = (b, j3) of W1, pad n -> M, FFT along j2, all M k2 to W2,
//                 W2 column c = k2 Kp + k1 (Kp = KB B), column-blocked with n rows (j3).
//   ZSYM (d = 3): W2 column tile of field o, pad n -> M along j3, FFT, * Lambda[k3r][k2r][k1],
//                 iFFT, keep n; in place.
//   YINV (d = 3): slab o = (b, j3): M entries k2 of W2 columns k1, iFFT, first n (j2) to W1.
// ---------------------------------------------------------------------------

enum ColMode { SYM2 = 0, YFWD = 1, ZSYM = 2, YINV = 3 };

struct ColArgs {
  int n, K, KB;      // interior points, symbol extent M/2+1, column blocks per W1 slab
  int64_t tiles;     // column tiles per slab
  int64_t nb;        // batch (fields)
};

template <typename T, int LOGM, int MODE>
__global__ void __launch_bounds__(blk<T>() * tpl(LOGM), minb_cols<T>(blk<T>() * tpl(LOGM)))
k_cols(const cplx_t<T>* in, cplx_t<T>* out, ColArgs A, const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw,
       const CGState* st) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride_tile(LOGM), B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int cl = threadIdx.x % B, tl = threadIdx.x / B;
  C* buf = sm + cl * LS;
  const int64_t o = blockIdx.x / A.tiles, tile = blockIdx.x % A.tiles;
  const int n = A.n, K = A.K, KB = A.KB, Kp = KB * B;
  const int64_t nB = (int64_t)n * B;
  const int64_t W2slab = (int64_t)M * KB * nB;  // one field of W2
  C v[E];
  // ---- column identity and load
  int k1 = 0, k2r = 0;
  bool live = true;
  if (MODE == SYM2 || MODE == YFWD || MODE == YINV) {
    k1 = (int)tile * B + cl;
    live = k1 < K;
  } else {  // ZSYM: tile indexes W2 column blocks, c = k2 Kp + k1
    const int64_t c = tile * B + cl;
    const int k2 = (int)(c / Kp);
    k1 = (int)(c % Kp);
    k2r = k2 <= M / 2 ? k2 : M - k2;
    live = k1 < K;
  }
  if (MODE == YINV) {
    const int64_t b = o / n, j3 = o % n;
    const C* src = in + b * W2slab + tile * nB + j3 * B + cl;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k2 = tl + e * TPL;
      v[e] = live ? src[(int64_t)k2 * KB * nB] : C{0, 0};
    }
  } else {
    const C* src = (MODE == ZSYM) ? in + o * W2slab + tile * nB + cl : in + (o * KB + tile) * nB + cl;
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {  // j < n <= M/2; the rest is zero padding
      const int j = tl + e * TPL;
      v[e] = (live && j < n) ? src[(int64_t)j * B] : C{0, 0};
    }
  }
  // ---- transforms
  if (MODE != YINV) fft_reg<C, LOGM, false, true, false>(v, buf, tl, tw);
  if (MODE == SYM2 || MODE == ZSYM) {
    const T* lrow = (MODE == SYM2) ? lam + k1 : lam + (int64_t)k2r * K + k1;
    const int64_t kstride = (MODE == SYM2) ? K : (int64_t)K * K;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = tl + e * TPL;
      const int kr = k <= M / 2 ? k : M - k;
      v[e] = cscale(v[e], live ? lrow[kr * kstride] : T(0));
    }
  }
  if (MODE != YFWD) fft_reg<C, LOGM, true, false, true>(v, buf, tl, tw);  // keeps j < n only
  // ---- store
  if (!live) return;
  if (MODE == YFWD) {
    const int64_t b = o / n, j3 = o % n;
    C* dst = out + b * W2slab + tile * nB + j3 * B + cl;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k2 = tl + e * TPL;
      dst[(int64_t)k2 * KB * nB] = v[e];
    }
  } else {
    C* dst = (MODE == ZSYM) ? out + o * W2slab + tile * nB + cl
                            : out + (o * KB + tile) * nB + cl;  // SYM2 in place; YINV to W1 slab o
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const int j = tl + e * TPL;
      if (j < n) dst[(int64_t)j * B] = v[e];
    }
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

template <typename T, int LOGM>
struct Cfg {
  static constexpr int LINE_BYTES = line_stride(LOGM) * (int)sizeof(cplx_t<T>);
  // lines per block for the row and 1D kernels: at most 48 KB of shared memory and 256 threads
  static constexpr int lines_for(int maxbytes, int maxthreads) {
    int l = maxbytes / LINE_BYTES;
    int lim = maxthreads / tpl(LOGM);
    l = l < lim ? l : lim;
    return l < 1 ? 1 : l;
  }
  static constexpr int ROW_LINES = lines_for(48 * 1024, 256);
};

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename T>
static const char* kname(char* buf, const char* what, int logm) {
  std::snprintf(buf, 48, "%s_%s_M%d", what, sizeof(T) == 8 ? "f64" : "f32", 1 << logm);
  return buf;
}

template <typename K>
static int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FRAC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FRAC_OK;
}

template <typename T, int LOGM>
static int launch_conv1d(const T* u, T* y, int64_t n, int64_t batch, const T* lam, cudaStream_t st) {
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  auto kern = k_conv1d<T, LOGM, L>;
  FRAC_TRY(set_smem(kern, sm));
  const int64_t pairs = cdiv(batch, 2);
  char nb[48];
  prof::Scope ps(kname<T>(nb, "conv1d", LOGM), st);
  kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>(u, y, (int)n, batch, lam, tw_table<T>(LOGM));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

struct CgArgs {
  const void* r = nullptr;   // rows_fwd: r of p = r + beta p
  const void* p = nullptr;   // rows_inv: p of the p.q partials
  CGState* st = nullptr;
  double* partials = nullptr;
};

template <typename T, int LOGM, bool CG>
static int launch_rows(bool fwd, const void* in, void* out, int64_t n, int64_t nrows, int KB, const CgArgs& cg,
                       cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  const int64_t pairs = cdiv(nrows, 2);
  char nb[48];
  prof::Scope ps(kname<T>(nb, fwd ? (CG ? "rows_fwd_cg" : "rows_fwd") : (CG ? "rows_inv_cg" : "rows_inv"), LOGM), st);
  if (fwd) {
    auto kern = k_rows_fwd<T, LOGM, L, CG>;
    FRAC_TRY(set_smem(kern, sm));
    kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const T*)in, (C*)out, (int)n, nrows, KB,
                                                               tw_table<T>(LOGM), (const T*)cg.r, cg.st);
  } else {
    auto kern = k_rows_inv<T, LOGM, L, CG>;
    FRAC_TRY(set_smem(kern, sm));
    kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const C*)in, (T*)out, (int)n, nrows, KB,
                                                               tw_table<T>(LOGM), (const T*)cg.p, cg.st, cg.partials);
  }
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int LOGM>
static int64_t rows_grid(int64_t nrows) {
  return cdiv(cdiv(nrows, 2), Cfg<T, LOGM>::ROW_LINES);
}

template <typename T, int LOGM, int MODE>
static int launch_cols(const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam, const CGState* cgst,
                       cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const size_t sm = (size_t)B * line_stride_tile(LOGM) * sizeof(C);
  auto kern = k_cols<T, LOGM, MODE>;
  FRAC_TRY(set_smem(kern, sm));
  const int64_t blocks = nouter * A.tiles;
  static const char* names[4] = {"cols_sym2", "cols_yfwd", "cols_zsym", "cols_yinv"};
  char nb[48];
  prof::Scope ps(kname<T>(nb, names[MODE], LOGM), st);
  kern<<<(unsigned)blocks, B * tpl(LOGM), sm, st>>>((const C*)in, (C*)out, A, lam, tw_table<T>(LOGM), cgst);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

// Size dispatch (LOGM is a template parameter of every kernel).
#define FRAC_DISPATCH_LOGM(logm, LO, HI, CALL)                                 \
  switch (logm) {                                                             \
    case 1: if constexpr (1 >= LO && 1 <= HI) { constexpr int LG = 1; return CALL; } break;   \
    case 2: if constexpr (2 >= LO && 2 <= HI) { constexpr int LG = 2; return CALL; } break;   \
    case 3: if constexpr (3 >= LO && 3 <= HI) { constexpr int LG = 3; return CALL; } break;   \
    case 4: if constexpr (4 >= LO && 4 <= HI) { constexpr int LG = 4; return CALL; } break;   \
    case 5: if constexpr (5 >= LO && 5 <= HI) { constexpr int LG = 5; return CALL; } break;   \
    case 6: if constexpr (6 >= LO && 6 <= HI) { constexpr int LG = 6; return CALL; } break;   \
    case 7: if constexpr (7 >= LO && 7 <= HI) { constexpr int LG = 7; return CALL; } break;   \
    case 8: if constexpr (8 >= LO && 8 <= HI) { constexpr int LG = 8; return CALL; } break;   \
    case 9: if constexpr (9 >= LO && 9 <= HI) { constexpr int LG = 9; return CALL; } break;   \
    case 10: if constexpr (10 >= LO && 10 <= HI) { constexpr int LG = 10; return CALL; } break; \
    case 11: if constexpr (11 >= LO && 11 <= HI) { constexpr int LG = 11; return CALL; } break; \
    case 12: if constexpr (12 >= LO && 12 <= HI) { constexpr int LG = 12; return CALL; } break; \
    case 13: if constexpr (13 >= LO && 13 <= HI) { constexpr int LG = 13; return CALL; } break; \
    default: break;                                                           \
  }                                                                           \
  return FRAC_ENOTSUP;

template <typename T>
static int conv1d_any(int logm, const T* u, T* y, int64_t n, int64_t batch, const T* lam, cudaStream_t st) {
  FRAC_DISPATCH_LOGM(logm, 1, 13, (launch_conv1d<T, LG>(u, y, n, batch, lam, st)));
}
template <typename T, bool CG = false>
static int rows_any(int logm, bool fwd, const void* in, void* out, int64_t n, int64_t nrows, int KB, cudaStream_t st,
                    const CgArgs& cg = CgArgs{}) {
  FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_rows<T, LG, CG>(fwd, in, out, n, nrows, KB, cg, st)));
}
template <typename T>
static int64_t rows_grid_any(int logm, int64_t nrows) {
  switch (logm) {
    case 1: return rows_grid<T, 1>(nrows);
    case 2: return rows_grid<T, 2>(nrows);
    case 3: return rows_grid<T, 3>(nrows);
    case 4: return rows_grid<T, 4>(nrows);
    case 5: return rows_grid<T, 5>(nrows);
    case 6: return rows_grid<T, 6>(nrows);
    case 7: return rows_grid<T, 7>(nrows);
    case 8: return rows_grid<T, 8>(nrows);
    case 9: return rows_grid<T, 9>(nrows);
    case 10: return rows_grid<T, 10>(nrows);
    case 11: return rows_grid<T, 11>(nrows);
    default: return 0;
  }
}
template <typename T, int MODE>
static int cols_any(int logm, const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam,
                    cudaStream_t st, const CGState* cgst = nullptr) {
  if constexpr (MODE == SYM2) {
    FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_cols<T, LG, MODE>(in, out, A, nouter, lam, cgst, st)));
  } else {
    FRAC_DISPATCH_LOGM(logm, 1, 9, (launch_cols<T, LG, MODE>(in, out, A, nouter, lam, cgst, st)));
  }
}

template <typename T>
static void layout(const frac_op* op, int64_t batch, int64_t& KB, int64_t& w1, int64_t& w2) {
  constexpr int B = blk<T>();
  const int64_t n = op->n, M = op->M, K = op->K;
  KB = cdiv(K, B);
  w1 = w2 = 0;
  if (op->prob.d == 2) w1 = batch * KB * n * B;
  if (op->prob.d == 3) {
    w1 = batch * n * KB * n * B;
    w2 = batch * M * KB * n * B;
  }
}

size_t apply_workspace_bytes(const frac_op* op, int dtype, int64_t batch) {
  int64_t KB, w1, w2;
  if (dtype == FRAC_F64) {
    layout<double>(op, batch, KB, w1, w2);
    return (size_t)(w1 + w2) * sizeof(double2);
  }
  layout<float>(op, batch, KB, w1, w2);
  return (size_t)(w1 + w2) * sizeof(float2);
}

template <typename T>
int apply_t(const frac_op* op, const T* u, T* y, int64_t batch, void* ws, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const int d = op->prob.d, logm = op->logm;
  const int64_t n = op->n, M = op->M, K = op->K;
  const T* lam = sym_table<T>(op);
  if (batch <= 0) return FRAC_OK;
  if (d == 1) return conv1d_any<T>(logm, u, y, n, batch, lam, st);
  int64_t KB, w1, w2;
  layout<T>(op, batch, KB, w1, w2);
  C* W1 = (C*)ws;
  if (d == 2) {
    const int64_t nrows = batch * n;
    FRAC_TRY(rows_any<T>(logm, true, u, W1, n, nrows, (int)KB, st));
    ColArgs A{(int)n, (int)K, (int)KB, KB, batch};
    FRAC_TRY((cols_any<T, SYM2>(logm, W1, W1, A, batch, lam, st)));
    FRAC_TRY(rows_any<T>(logm, false, W1, y, n, nrows, (int)KB, st));
    return FRAC_OK;
  }
  C* W2 = W1 + w1;
  const int64_t nrows = batch * n * n;
  FRAC_TRY(rows_any<T>(logm, true, u, W1, n, nrows, (int)KB, st));
  {
    ColArgs A{(int)n, (int)K, (int)KB, KB, batch};
    FRAC_TRY((cols_any<T, YFWD>(logm, W1, W2, A, batch * n, lam, st)));
  }
  {
    ColArgs A{(int)n, (int)K, (int)KB, M * KB, batch};
    FRAC_TRY((cols_any<T, ZSYM>(logm, W2, W2, A, batch, lam, st)));
  }
  {
    ColArgs A{(int)n, (int)K, (int)KB, KB, batch};
    FRAC_TRY((cols_any<T, YINV>(logm, W2, W1, A, batch * n, lam, st)));
  }
  FRAC_TRY(rows_any<T>(logm, false, W1, y, n, nrows, (int)KB, st));
  (void)B;
  return FRAC_OK;
}

template int apply_t<float>(const frac_op*, const float*, float*, int64_t, void*, cudaStream_t);
template int apply_t<double>(const frac_op*, const double*, double*, int64_t, void*, cudaStream_t);

size_t apply_cg_partials(const frac_op* op) {
  int64_t nrows = op->n;
  for (int i = 2; i < op->prob.d; ++i) nrows *= op->n;
  const int64_t a = rows_grid_any<float>(op->logm, nrows), b = rows_grid_any<double>(op->logm, nrows);
  return (size_t)(a > b ? a : b);
}

template <typename T>
int apply_cg_t(const frac_op* op, T* p, const T* r, T* q, void* ws, CGState* cgst, double* partials, cudaStream_t st) {
  using C = cplx_t<T>;
  const int d = op->prob.d, logm = op->logm;
  const int64_t n = op->n, M = op->M, K = op->K;
  const T* lam = sym_table<T>(op);
  if (d < 2) return FRAC_ENOTSUP;
  int64_t KB, w1, w2;
  layout<T>(op, 1, KB, w1, w2);
  C* W1 = (C*)ws;
  CgArgs fwd, inv;
  fwd.r = r;
  fwd.st = cgst;
  inv.p = p;
  inv.st = cgst;
  inv.partials = partials;
  if (d == 2) {
    FRAC_TRY((rows_any<T, true>(logm, true, p, W1, n, n, (int)KB, st, fwd)));
    ColArgs A{(int)n, (int)K, (int)KB, KB, 1};
    FRAC_TRY((cols_any<T, SYM2>(logm, W1, W1, A, 1, lam, st, cgst)));
    FRAC_TRY((rows_any<T, true>(logm, false, W1, q, n, n, (int)KB, st, inv)));
    return FRAC_OK;
  }
  C* W2 = W1 + w1;
  const int64_t nrows = n * n;
  FRAC_TRY((rows_any<T, true>(logm, true, p, W1, n, nrows, (int)KB, st, fwd)));
  ColArgs Ay{(int)n, (int)K, (int)KB, KB, 1};
  FRAC_TRY((cols_any<T, YFWD>(logm, W1, W2, Ay, n, lam, st, cgst)));
  ColArgs Az{(int)n, (int)K, (int)KB, M * KB, 1};
  FRAC_TRY((cols_any<T, ZSYM>(logm, W2, W2, Az, 1, lam, st, cgst)));
  FRAC_TRY((cols_any<T, YINV>(logm, W2, W1, Ay, n, lam, st, cgst)));
  FRAC_TRY((rows_any<T, true>(logm, false, W1, q, n, nrows, (int)KB, st, inv)));
  return FRAC_OK;
}

template int apply_cg_t<float>(const frac_op*, float*, const float*, float*, void*, CGState*, double*, cudaStream_t);
template int apply_cg_t<double>(const frac_op*, double*, const double*, double*, void*, CGState*, double*, cudaStream_t);

}  // namespace frac
