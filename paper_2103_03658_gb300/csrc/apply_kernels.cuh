// Kernels and launch helpers of the FFT apply (internal header of apply.cu and
// precond.cu, which instantiate different parts of it).
//
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
#pragma once

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "apply.cuh"
#include "fft.cuh"
#include "passes.cuh"
#include "prof.cuh"

namespace frac {

using namespace fft;

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

// the mixed-length kernels: blocks per SM asked of the compiler for a block of nt
// threads, so that FP32 kernels fit 64 registers a thread (as the power-of-two
// ones) and FP64 kernels 128
template <typename T> __host__ __device__ constexpr int mx_minb(int nt) {
  return clamp_blocks(65536 / (nt * ((int)sizeof(T) == 4 ? 64 : 128)));
}

// ---------------------------------------------------------------------------
// d = 1: whole convolution per line (two vectors per complex line)
// ---------------------------------------------------------------------------

// ODD: the tau preconditioner (odd extension, entries 1..n kept, lam = its symbol).
// One complex line (vectors va, va + 1) on the thread group of tl; ln: the line policy.
template <typename T, typename LN, bool ODD>
__device__ __forceinline__ void conv1d_pair(const LN& ln, const T* __restrict__ u, T* __restrict__ y, int n,
                                            int64_t batch, const T* __restrict__ lam,
                                            const cplx_t<T>* __restrict__ tw, int64_t va, cplx_t<T>* buf, int tl) {
  using C = cplx_t<T>;
  constexpr int E = LN::E;
  const int M = ln.m(), TPL = ln.tpl();
  const int64_t vb = va + 1;
  const bool ha = va < batch, hb = vb < batch;
  C v[E];
  if constexpr (!ODD) {
    // n <= M/2: entries e >= E/2 (x >= M/2) are zero padding, and only
    // outputs x < n are kept, so both transforms are half-pruned
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const int x = tl + e * TPL;
      T re = (x < n && ha) ? u[va * n + x] : T(0);
      T im = (x < n && hb) ? u[vb * n + x] : T(0);
      v[e] = C{re, im};
    }
    ln.template fft<false, true, false>(v, buf, tl, tw);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      T re = T(0), im = T(0);
      if (x >= 1 && x <= n) {
        if (ha) re = u[va * n + x - 1];
        if (hb) im = u[vb * n + x - 1];
      } else if (x >= M - n) {
        if (ha) re = -u[va * n + M - 1 - x];
        if (hb) im = -u[vb * n + M - 1 - x];
      }
      v[e] = C{re, im};
    }
    ln.template fft<false, false, false>(v, buf, tl, tw);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    v[e] = cscale(v[e], lam[k <= M / 2 ? k : M - k]);
  }
  if constexpr (!ODD) {
    ln.template fft<true, false, true>(v, buf, tl, tw);
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const int x = tl + e * TPL;
      if (x < n) {
        if (ha) y[va * n + x] = v[e].x;
        if (hb) y[vb * n + x] = v[e].y;
      }
    }
  } else {
    ln.template fft<true, false, false>(v, buf, tl, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      if (x >= 1 && x <= n) {
        if (ha) y[va * n + x - 1] = v[e].x;
        if (hb) y[vb * n + x - 1] = v[e].y;
      }
    }
  }
}

template <typename T, int LOGM, int LINES, bool ODD = false>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb<T>(LINES * tpl(LOGM)))
k_conv1d(const T* __restrict__ u, T* __restrict__ y, int n, int64_t batch, const T* __restrict__ lam,
         const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  constexpr int TPL = tpl(LOGM), LS = line_stride(LOGM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  conv1d_pair<T, P2Line<LOGM>, ODD>(P2Line<LOGM>{}, u, y, n, batch, lam, tw, 2 * ((int64_t)blockIdx.x * LINES + line),
                                    sm + line * LS, tl);
}

#ifdef FRAC_MX_TU
// Mixed lengths: blockDim.x / ln.tpl() lines per block.
template <typename T, bool ODD, int NTMAX>
__global__ void __launch_bounds__(NTMAX, mx_minb<T>(NTMAX)) k_conv1d_mx(MxLine ln, const T* __restrict__ u, T* __restrict__ y, int n,
                                                   int64_t batch, const T* __restrict__ lam,
                                                   const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int TPL = ln.tpl(), lines = blockDim.x / TPL;
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  conv1d_pair<T, MxLine, ODD>(ln, u, y, n, batch, lam, tw, 2 * ((int64_t)blockIdx.x * lines + line),
                              sm + line * ln.stride(), tl);
}

#endif  // FRAC_MX_TU

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
// Grid kernels over the passes of passes.cuh: one unit (row pair or column
// tile) per thread group.
// ---------------------------------------------------------------------------

// Row kernel kinds.  Forward: RF_PLAIN (input u), RF_CG (input p = r + beta p,
// beta from st, written back to u = p), RF_ODD (odd extension of u, for the
// preconditioner).  Inverse: RI_PLAIN (y), RI_CG (y = q plus per-block partials
// of p.q; the last block sets st->pq and st->alpha = st->rz / pq), RI_ODD (odd
// extension kept, y = z), RI_ODD_CG (z plus partials of r.z with r = p; the last
// block sets st->beta and st->rz).  CG kinds return at once when st->done.
enum RowKind { RF_PLAIN = 0, RF_CG = 1, RF_ODD = 2, RI_PLAIN = 0, RI_CG = 1, RI_ODD = 2, RI_ODD_CG = 3 };

// One row pair of the forward row pass (kind KIND) on the thread group of tl.
template <typename T, int KIND, typename LN>
__device__ __forceinline__ void rows_fwd_unit(const LN& ln, const T* u, cplx_t<T>* W, int n, int ns, int64_t nrows,
                                              int KB, const cplx_t<T>* __restrict__ tw, const T* __restrict__ r,
                                              const CGState* st, int64_t pair, cplx_t<T>* buf, int tl) {
  if constexpr (KIND == RF_CG) {
    const T be = (T)st->beta;
    T* p = const_cast<T*>(u);
    row_fwd_pair_l<T, LN>(
        ln,
        [&](int64_t row, int x) {
          const T v = r[row * n + x] + be * p[row * n + x];
          p[row * n + x] = v;
          return v;
        },
        W, n, nrows, KB, tw, pair, buf, tl, ns);
  } else {
    row_fwd_pair_l<T, LN, KIND == RF_ODD>(ln, [&](int64_t row, int x) { return u[row * n + x]; }, W, n, nrows, KB, tw,
                                          pair, buf, tl, ns);
  }
}

template <typename T, int LOGM, int LINES, int KIND>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb_rows<T>(LINES * tpl(LOGM)))
k_rows_fwd(const T* u, cplx_t<T>* __restrict__ W, int n, int ns, int64_t nrows, int KB,
           const cplx_t<T>* __restrict__ tw, const T* __restrict__ r, const CGState* st) {
  using C = cplx_t<T>;
  constexpr int TPL = tpl(LOGM), LS = line_stride(LOGM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (KIND == RF_CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  rows_fwd_unit<T, KIND>(P2Line<LOGM>{}, u, W, n, ns, nrows, KB, tw, r, st, (int64_t)blockIdx.x * LINES + line,
                         sm + line * LS, tl);
}

#ifdef FRAC_MX_TU
template <typename T, int KIND>
__global__ void __launch_bounds__(256, mx_minb<T>(256)) k_rows_fwd_mx(MxLine ln, const T* u, cplx_t<T>* __restrict__ W, int n, int ns,
                                                     int64_t nrows, int KB, const cplx_t<T>* __restrict__ tw,
                                                     const T* __restrict__ r, const CGState* st) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (KIND == RF_CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int TPL = ln.tpl(), lines = blockDim.x / TPL, line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  rows_fwd_unit<T, KIND>(ln, u, W, n, ns, nrows, KB, tw, r, st, (int64_t)blockIdx.x * lines + line,
                         sm + line * ln.stride(), tl);
}

#endif  // FRAC_MX_TU

// One row pair of the inverse row pass; returns this thread's part of the CG dot product.
template <typename T, int KIND, typename LN>
__device__ __forceinline__ T rows_inv_unit(const LN& ln, const cplx_t<T>* W, T* __restrict__ y, int n, int ns,
                                           int64_t nrows, int KB, const cplx_t<T>* __restrict__ tw,
                                           const T* __restrict__ p, int64_t pair, cplx_t<T>* buf, int tl) {
  constexpr bool CG = KIND == RI_CG || KIND == RI_ODD_CG;
  constexpr bool ODD = KIND == RI_ODD || KIND == RI_ODD_CG;
  T dot = T(0);
  row_inv_pair_l<T, LN, ODD>(ln, W, n, nrows, KB, tw, pair, buf, tl, [&](int64_t row, int x, T v) {
    y[row * n + x] = v;
    if (CG) dot += v * p[row * n + x];
  }, ns);
  return dot;
}

// The CG kinds' reduction at the end of the inverse row pass (red: the block's
// dynamic shared memory, free once the FFT lines are done).
template <int KIND>
__device__ __forceinline__ void rows_inv_finish(double dot, CGState* st, double* partials, double* red) {
  if constexpr (KIND == RI_CG) {
    const double total = block_sum_all(dot, red);
    last_block_reduce(total, partials, &st->count_pq, red, [&](double pq) {
      st->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = FRAC_EBREAKDOWN;
        st->done = 1;
      } else {
        st->alpha = st->rz / pq;
      }
    });
  } else if constexpr (KIND == RI_ODD_CG) {
    const double total = block_sum_all(dot, red);
    last_block_reduce(total, partials, &st->count_rz, red, [&](double rz) {
      if (!(rz > 0.0) || !isfinite(rz)) {  // P is SPD: r.z > 0 unless r = 0
        st->status = FRAC_EBREAKDOWN;
        st->done = 1;
      } else {
        st->beta = st->rz > 0.0 ? rz / st->rz : 0.0;
        st->rz = rz;
      }
    });
  }
}

template <typename T, int LOGM, int LINES, int KIND>
__global__ void __launch_bounds__(LINES * tpl(LOGM), minb_rows<T>(LINES * tpl(LOGM)))
k_rows_inv(const cplx_t<T>* __restrict__ W, T* __restrict__ y, int n, int ns, int64_t nrows, int KB,
           const cplx_t<T>* __restrict__ tw, const T* __restrict__ p, CGState* st, double* partials) {
  using C = cplx_t<T>;
  constexpr int TPL = tpl(LOGM), LS = line_stride(LOGM);
  constexpr bool CG = KIND == RI_CG || KIND == RI_ODD_CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  const T dot = rows_inv_unit<T, KIND>(P2Line<LOGM>{}, W, y, n, ns, nrows, KB, tw, p,
                                       (int64_t)blockIdx.x * LINES + line, sm + line * LS, tl);
  rows_inv_finish<KIND>(dot, st, partials, reinterpret_cast<double*>(smem_raw));
}

#ifdef FRAC_MX_TU
template <typename T, int KIND>
__global__ void __launch_bounds__(256, mx_minb<T>(256)) k_rows_inv_mx(MxLine ln, const cplx_t<T>* __restrict__ W, T* __restrict__ y,
                                                     int n, int ns, int64_t nrows, int KB,
                                                     const cplx_t<T>* __restrict__ tw, const T* __restrict__ p,
                                                     CGState* st, double* partials) {
  using C = cplx_t<T>;
  constexpr bool CG = KIND == RI_CG || KIND == RI_ODD_CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (CG && st->done) return;
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int TPL = ln.tpl(), lines = blockDim.x / TPL, line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  const T dot = rows_inv_unit<T, KIND>(ln, W, y, n, ns, nrows, KB, tw, p, (int64_t)blockIdx.x * lines + line,
                                       sm + line * ln.stride(), tl);
  rows_inv_finish<KIND>(dot, st, partials, reinterpret_cast<double*>(smem_raw));
}

#endif  // FRAC_MX_TU

// Columns: one tile of B adjacent columns per block (see col_tile).
template <typename T, int LOGM, int MODE, bool ODD>
__global__ void __launch_bounds__(blk<T>() * tpl(LOGM), minb_cols<T>(blk<T>() * tpl(LOGM)))
k_cols(const cplx_t<T>* in, cplx_t<T>* out, ColArgs A, const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw,
       const CGState* st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;
  const int cl = threadIdx.x % B, tl = threadIdx.x / B;
  const int64_t o = blockIdx.x / A.tiles, tile = blockIdx.x % A.tiles;
  col_tile<T, LOGM, MODE, ODD>(in, out, A, lam, tw, o, tile, reinterpret_cast<C*>(smem_raw), cl, tl);
}

// Column passes of the tau preconditioner two columns to a transform (col_pair_tau_l):
// B lines per block, line q = unit B + cl of slab o.
template <typename T, int LOGM, int MODE>
__global__ void __launch_bounds__(blk<T>() * tpl(LOGM), minb_cols<T>(blk<T>() * tpl(LOGM)))
k_cols_tau_pairs(const cplx_t<T>* in, cplx_t<T>* out, ColArgs A, int64_t qtiles, const T* __restrict__ lam,
                 const cplx_t<T>* __restrict__ tw, const CGState* st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;
  const int cl = threadIdx.x % B, tl = threadIdx.x / B;
  const int64_t o = blockIdx.x / qtiles, q = (blockIdx.x % qtiles) * B + cl;
  using LN = P2Line<LOGM, tile_shift(LOGM)>;
  col_pair_tau_l<T, LN, MODE>(LN{}, in, out, A, lam, tw, o, q, reinterpret_cast<C*>(smem_raw), cl, tl);
}

#ifdef FRAC_MX_TU
template <typename T, int MODE, bool ODD, int NTMAX>
__global__ void __launch_bounds__(NTMAX, mx_minb<T>(NTMAX)) k_cols_mx(MxLine ln, const cplx_t<T>* in, cplx_t<T>* out, ColArgs A,
                                                  const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw,
                                                  const CGState* st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;
  const int cl = threadIdx.x % B, tl = threadIdx.x / B;
  const int64_t o = blockIdx.x / A.tiles, tile = blockIdx.x % A.tiles;
  col_tile_l<T, MxLine, MODE, ODD>(ln, in, out, A, lam, tw, o, tile, reinterpret_cast<C*>(smem_raw), cl, tl);
}

// The tau preconditioner's column passes on a mixed length, two columns a transform.
template <typename T, int MODE, int NTMAX>
__global__ void __launch_bounds__(NTMAX, mx_minb<T>(NTMAX))
    k_cols_tau_pairs_mx(MxLine ln, const cplx_t<T>* in, cplx_t<T>* out, ColArgs A, int64_t qtiles,
                        const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, const CGState* st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (st && st->done) return;
  const int cl = threadIdx.x % B, tl = threadIdx.x / B;
  const int64_t o = blockIdx.x / qtiles, q = (blockIdx.x % qtiles) * B + cl;
  col_pair_tau_l<T, MxLine, MODE>(ln, in, out, A, lam, tw, o, q, reinterpret_cast<C*>(smem_raw), cl, tl);
}

#endif  // FRAC_MX_TU

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

template <typename T, int LOGM>
struct Cfg {
  static constexpr int LINE_BYTES = line_stride(LOGM) * (int)sizeof(cplx_t<T>);
  // lines per block for the row and 1D kernels: at most 48 KB of shared memory and 128 threads
  // (one line of M >= 2048 per block: a barrier then waits for 4 warps, not 8; measured 2.5 %
  // faster for the 2D apply than two lines per block, and four lines 7 % slower)
  static constexpr int lines_for(int maxbytes, int maxthreads) {
    int l = maxbytes / LINE_BYTES;
    int lim = maxthreads / tpl(LOGM);
    l = l < lim ? l : lim;
    return l < 1 ? 1 : l;
  }
  static constexpr int ROW_LINES = lines_for(48 * 1024, 128);
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

template <typename T, int LOGM, bool ODD>
static int launch_conv1d(const T* u, T* y, int64_t n, int64_t batch, const T* lam, cudaStream_t st) {
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  auto kern = k_conv1d<T, LOGM, L, ODD>;
  FRAC_TRY(set_smem(kern, sm));
  const int64_t pairs = cdiv(batch, 2);
  char nb[48];
  prof::Scope ps(kname<T>(nb, ODD ? "conv1d_tau" : "conv1d", LOGM), st);
  kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>(u, y, (int)n, batch, lam, tw_table<T>(LOGM));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

struct CgArgs {
  const void* r = nullptr;   // rows_fwd RF_CG: r of p = r + beta p
  const void* p = nullptr;   // rows_inv RI_CG / RI_ODD_CG: the vector dotted with the output
  CGState* st = nullptr;
  double* partials = nullptr;
};

template <typename T, int LOGM, int KIND>
static int launch_rows_fwd(const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB, const CgArgs& cg,
                           cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  const int64_t pairs = cdiv(nrows, 2);
  static const char* names[3] = {"rows_fwd", "rows_fwd_cg", "rows_fwd_tau"};
  char nb[48];
  prof::Scope ps(kname<T>(nb, names[KIND], LOGM), st);
  auto kern = k_rows_fwd<T, LOGM, L, KIND>;
  FRAC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const T*)in, (C*)out, (int)n, (int)ns, nrows, KB,
                                                             tw_table<T>(LOGM), (const T*)cg.r, cg.st);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int LOGM, int KIND>
static int launch_rows_inv(const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB, const CgArgs& cg,
                           cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  const int64_t pairs = cdiv(nrows, 2);
  static const char* names[4] = {"rows_inv", "rows_inv_cg", "rows_inv_tau", "rows_inv_tau_cg"};
  char nb[48];
  prof::Scope ps(kname<T>(nb, names[KIND], LOGM), st);
  auto kern = k_rows_inv<T, LOGM, L, KIND>;
  FRAC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const C*)in, (T*)out, (int)n, (int)ns, nrows, KB,
                                                             tw_table<T>(LOGM), (const T*)cg.p, cg.st, cg.partials);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int LOGM>
static int64_t rows_grid(int64_t nrows) {
  return cdiv(cdiv(nrows, 2), Cfg<T, LOGM>::ROW_LINES);
}

template <typename T, int LOGM, int MODE, bool ODD>
static int launch_cols(const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam, const CGState* cgst,
                       cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const size_t sm = (size_t)B * line_stride_tile(LOGM) * sizeof(C);
  static const char* names[2][4] = {{"cols_sym2", "cols_yfwd", "cols_zsym", "cols_yinv"},
                                    {"cols_sym2_tau", "cols_yfwd_tau", "cols_zsym_tau", "cols_yinv_tau"}};
  char nb[48];
  prof::Scope ps(kname<T>(nb, names[ODD ? 1 : 0][MODE], LOGM), st);
  if constexpr (ODD) {  // tau preconditioner: two columns a transform
    auto kp = k_cols_tau_pairs<T, LOGM, MODE>;
    FRAC_TRY(set_smem(kp, sm));
    // column pairs of a slab: ceil(K / 2), or for ZSYM the W2 blocks' (tiles x B) / 2
    const int64_t qtiles = MODE == ZSYM ? cdiv(A.tiles * B / 2, B) : cdiv(cdiv(A.K, 2), B);
    kp<<<(unsigned)(nouter * qtiles), B * tpl(LOGM), sm, st>>>((const C*)in, (C*)out, A, qtiles, lam,
                                                              tw_table<T>(LOGM), cgst);
  } else {  // (a discarded branch: the full-width kernel is not instantiated for ODD)
    auto kern = k_cols<T, LOGM, MODE, ODD>;
    FRAC_TRY(set_smem(kern, sm));
    const int64_t blocks = nouter * A.tiles;
    kern<<<(unsigned)blocks, B * tpl(LOGM), sm, st>>>((const C*)in, (C*)out, A, lam, tw_table<T>(LOGM), cgst);
  }
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

template <typename T, bool ODD>
static int conv1d_any(int logm, const T* u, T* y, int64_t n, int64_t batch, const T* lam, cudaStream_t st) {
  FRAC_DISPATCH_LOGM(logm, 1, 13, (launch_conv1d<T, LG, ODD>(u, y, n, batch, lam, st)));
}
template <typename T, int KIND>
static int rows_fwd_any(int logm, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                        cudaStream_t st, const CgArgs& cg) {
  FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_rows_fwd<T, LG, KIND>(in, out, n, ns, nrows, KB, cg, st)));
}
template <typename T, int KIND>
static int rows_inv_any(int logm, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                        cudaStream_t st, const CgArgs& cg) {
  FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_rows_inv<T, LG, KIND>(in, out, n, ns, nrows, KB, cg, st)));
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
template <typename T, int MODE, bool ODD>
static int cols_any(int logm, const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam,
                    cudaStream_t st, const CGState* cgst) {
  if constexpr (MODE == SYM2) {
    FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_cols<T, LG, MODE, ODD>(in, out, A, nouter, lam, cgst, st)));
  } else {
    FRAC_DISPATCH_LOGM(logm, 1, 9, (launch_cols<T, LG, MODE, ODD>(in, out, A, nouter, lam, cgst, st)));
  }
}

// ---------------------------------------------------------------------------
// Mixed lengths (op->plan[axis].m set): the same passes on MxLine, runtime M.
// ---------------------------------------------------------------------------

template <typename T> inline const cplx_t<T>* tw_len(int64_t M);
template <> inline const float2* tw_len<float>(int64_t M) { return twiddles32_len(M); }
template <> inline const double2* tw_len<double>(int64_t M) { return twiddles64_len(M); }

template <typename T>
static const char* kname_mx(char* buf, const char* what, int M) {
  std::snprintf(buf, 48, "%s_%s_M%d", what, sizeof(T) == 8 ? "f64" : "f32", M);
  return buf;
}

// lines per block of the mixed row and 1D kernels: as many as fit 128 threads and
// 48 KB of shared memory, at least one
template <typename T>
static int mx_lines(const MxLine& ln) {
  const int by_threads = 128 / ln.tpl();
  const int by_smem = (int)(48 * 1024 / ((size_t)ln.stride() * sizeof(cplx_t<T>)));
  return std::max(1, std::min(by_threads, by_smem));
}

// Launchers of the mixed-length kernels (defined and instantiated in apply_mx_f32.cu and
// apply_mx_f64.cu, so that the mixed kernels compile apart from the power-of-two ones).
template <typename T, bool ODD>
int launch_conv1d_mx(const MxLine& ln, const T* u, T* y, int64_t n, int64_t batch, const T* lam, cudaStream_t st);
template <typename T, int KIND>
int launch_rows_fwd_mx(const MxLine& ln, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                       const CgArgs& cg, cudaStream_t st);
template <typename T, int KIND>
int launch_rows_inv_mx(const MxLine& ln, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                       const CgArgs& cg, cudaStream_t st);
template <typename T, int MODE, bool ODD>
int launch_cols_mx(const MxLine& ln, const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam,
                   const CGState* cgst, cudaStream_t st);

#ifdef FRAC_MX_TU
template <typename T, bool ODD>
int launch_conv1d_mx(const MxLine& ln, const T* u, T* y, int64_t n, int64_t batch, const T* lam,
                            cudaStream_t st) {
  const int L = mx_lines<T>(ln);
  const size_t sm = (size_t)L * ln.stride() * sizeof(cplx_t<T>);
  // blocks of up to 256 threads get up to 255 registers a thread; longer lines take 512
  auto kern = L * ln.tpl() <= 256 ? k_conv1d_mx<T, ODD, 256> : k_conv1d_mx<T, ODD, 512>;
  FRAC_TRY(set_smem(kern, sm));
  char nb[48];
  prof::Scope ps(kname_mx<T>(nb, ODD ? "conv1d_tau" : "conv1d", ln.m()), st);
  kern<<<(unsigned)cdiv(cdiv(batch, 2), L), L * ln.tpl(), sm, st>>>(ln, u, y, (int)n, batch, lam, tw_len<T>(ln.m()));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int KIND>
int launch_rows_fwd_mx(const MxLine& ln, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows,
                              int KB, const CgArgs& cg, cudaStream_t st) {
  using C = cplx_t<T>;
  const int L = mx_lines<T>(ln);
  const size_t sm = (size_t)L * ln.stride() * sizeof(C);
  static const char* names[3] = {"rows_fwd", "rows_fwd_cg", "rows_fwd_tau"};
  char nb[48];
  prof::Scope ps(kname_mx<T>(nb, names[KIND], ln.m()), st);
  auto kern = k_rows_fwd_mx<T, KIND>;
  FRAC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)cdiv(cdiv(nrows, 2), L), L * ln.tpl(), sm, st>>>(ln, (const T*)in, (C*)out, (int)n, (int)ns, nrows,
                                                                     KB, tw_len<T>(ln.m()), (const T*)cg.r, cg.st);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int KIND>
int launch_rows_inv_mx(const MxLine& ln, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows,
                              int KB, const CgArgs& cg, cudaStream_t st) {
  using C = cplx_t<T>;
  const int L = mx_lines<T>(ln);
  const size_t sm = std::max<size_t>((size_t)L * ln.stride() * sizeof(C), 32 * sizeof(double));
  static const char* names[4] = {"rows_inv", "rows_inv_cg", "rows_inv_tau", "rows_inv_tau_cg"};
  char nb[48];
  prof::Scope ps(kname_mx<T>(nb, names[KIND], ln.m()), st);
  auto kern = k_rows_inv_mx<T, KIND>;
  FRAC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)cdiv(cdiv(nrows, 2), L), L * ln.tpl(), sm, st>>>(ln, (const C*)in, (T*)out, (int)n, (int)ns, nrows,
                                                                     KB, tw_len<T>(ln.m()), (const T*)cg.p, cg.st,
                                                                     cg.partials);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int MODE, bool ODD>
int launch_cols_mx(const MxLine& ln, const void* in, void* out, const ColArgs& A, int64_t nouter, const T* lam,
                          const CGState* cgst, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const size_t sm = (size_t)B * ln.stride_tile() * sizeof(C);
  static const char* names[2][4] = {{"cols_sym2", "cols_yfwd", "cols_zsym", "cols_yinv"},
                                    {"cols_sym2_tau", "cols_yfwd_tau", "cols_zsym_tau", "cols_yinv_tau"}};
  char nb[48];
  prof::Scope ps(kname_mx<T>(nb, names[ODD ? 1 : 0][MODE], ln.m()), st);
  if constexpr (ODD) {  // tau preconditioner: two columns a transform (as launch_cols)
    auto kp = B * ln.tpl() <= 256 ? k_cols_tau_pairs_mx<T, MODE, 256> : k_cols_tau_pairs_mx<T, MODE, 512>;
    FRAC_TRY(set_smem(kp, sm));
    const int64_t qtiles = MODE == ZSYM ? cdiv(A.tiles * B / 2, B) : cdiv(cdiv(A.K, 2), B);
    kp<<<(unsigned)(nouter * qtiles), B * ln.tpl(), sm, st>>>(ln, (const C*)in, (C*)out, A, qtiles, lam,
                                                              tw_len<T>(ln.m()), cgst);
  } else {  // (a discarded branch: the full-width kernel is not instantiated for ODD)
    auto kern = B * ln.tpl() <= 256 ? k_cols_mx<T, MODE, ODD, 256> : k_cols_mx<T, MODE, ODD, 512>;
    FRAC_TRY(set_smem(kern, sm));
    kern<<<(unsigned)(nouter * A.tiles), B * ln.tpl(), sm, st>>>(ln, (const C*)in, (C*)out, A, lam,
                                                                  tw_len<T>(ln.m()), cgst);
  }
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

#endif  // FRAC_MX_TU

// Per-axis dispatch: the power-of-two kernels, or the mixed ones where plan[axis].m is set.
template <typename T, bool ODD>
static int conv1d_op(const frac_op* op, const T* u, T* y, int64_t batch, const T* lam, cudaStream_t st) {
  if (op->plan[0].m) return launch_conv1d_mx<T, ODD>(MxLine(op->plan[0]), u, y, op->n, batch, lam, st);
  return conv1d_any<T, ODD>(op->logm, u, y, op->n, batch, lam, st);
}
template <typename T, int KIND>
static int rows_fwd_op(const frac_op* op, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                       cudaStream_t st, const CgArgs& cg) {
  if (op->plan[0].m) return launch_rows_fwd_mx<T, KIND>(MxLine(op->plan[0]), in, out, n, ns, nrows, KB, cg, st);
  return rows_fwd_any<T, KIND>(op->logma[0], in, out, n, ns, nrows, KB, st, cg);
}
template <typename T, int KIND>
static int rows_inv_op(const frac_op* op, const void* in, void* out, int64_t n, int64_t ns, int64_t nrows, int KB,
                       cudaStream_t st, const CgArgs& cg) {
  if (op->plan[0].m) return launch_rows_inv_mx<T, KIND>(MxLine(op->plan[0]), in, out, n, ns, nrows, KB, cg, st);
  return rows_inv_any<T, KIND>(op->logma[0], in, out, n, ns, nrows, KB, st, cg);
}
template <typename T, int MODE, bool ODD>
static int cols_op(const frac_op* op, int axis, const void* in, void* out, const ColArgs& A, int64_t nouter,
                   const T* lam, cudaStream_t st, const CGState* cgst) {
  if (op->plan[axis].m)
    return launch_cols_mx<T, MODE, ODD>(MxLine(op->plan[axis]), in, out, A, nouter, lam, cgst, st);
  return cols_any<T, MODE, ODD>(op->logma[axis], in, out, A, nouter, lam, st, cgst);
}
// blocks of one launch of the row kernels over nrows rows (the partial sums of the CG kinds)
template <typename T>
static int64_t rows_grid_op(const frac_op* op, int64_t nrows) {
  if (op->plan[0].m) return cdiv(cdiv(nrows, 2), mx_lines<T>(MxLine(op->plan[0])));
  return rows_grid_any<T>(op->logm, nrows);
}

// Fused xy passes of the 3D FP32 apply (xy_cluster.cuh, instantiated in apply_xy.cu):
// forward rows + y (kind FK, ODD as the column pass) into W2, and inverse y + rows
// (kind IK) out of it.  xy_enabled: the operator takes them (op->xy_fused, set when it
// was built) and frac_apply_3d_passes has not switched them off.
template <int FK, bool ODD>
int xy_fwd(const frac_op* op, const void* in, void* W2, int64_t batch, const float* lam, const CgArgs& cg,
           const CGState* cgst, cudaStream_t st);
template <int IK, bool ODD>
int xy_inv(const frac_op* op, const void* W2, void* out, int64_t batch, const CgArgs& cg, cudaStream_t st);
bool xy_enabled(const frac_op* op);
// Blocks of one fused launch over `batch` fields (0 when the operator does not take the
// fused passes): the per-block partial sums of the CG epilogues need that many entries.
int64_t xy_grid_blocks(const frac_op* op, int64_t batch);

// Spectrum layout for d >= 2 (axis i: n_i points, FFT length M_i, K_i = M_i/2 + 1;
// axis 0 = x^(1) is the row axis): W1 holds the rows' half spectra column-blocked,
// slabs of n_2 rows (KB = ceil(K_1 / B) blocks); d = 3: W2 holds the y transform,
// per field M_2 x KB column blocks of n_3 rows.
template <typename T>
static void layout(const frac_op* op, int64_t batch, int64_t& KB, int64_t& w1, int64_t& w2) {
  constexpr int B = blk<T>();
  KB = cdiv(op->Ka[0], B);
  w1 = w2 = 0;
  if (op->prob.d == 2) w1 = batch * KB * op->na[1] * B;
  if (op->prob.d == 3) {
    w1 = batch * op->na[2] * KB * op->na[1] * B;
    w2 = batch * op->Ma[1] * KB * op->na[2] * B;
  }
}

// The d >= 2 pipeline: forward rows (kind FK) -> column passes (ODD: odd
// extension, as the preconditioner) with the symbol lam -> inverse rows (kind IK).
template <typename T, int FK, int IK, bool ODD>
static int pipeline(const frac_op* op, const T* lam, const void* in, void* out, int64_t batch, void* ws,
                    const CgArgs& fwd, const CgArgs& inv, const CGState* cgst, cudaStream_t st) {
  using C = cplx_t<T>;
  const int d = op->prob.d;
  const int64_t n1 = op->na[0], n2 = op->na[1], n3 = op->na[2], K1 = op->Ka[0];
  int64_t KB, w1, w2;
  layout<T>(op, batch, KB, w1, w2);
  C* W1 = (C*)ws;
  if (d == 2) {
    const int64_t nrows = batch * n2;
    FRAC_TRY((rows_fwd_op<T, FK>(op, in, W1, n1, n2, nrows, (int)KB, st, fwd)));
    ColArgs A{(int)n2, (int)K1, (int)KB, KB, batch, 0, 0, (int)op->Ka[1]};
    FRAC_TRY((cols_op<T, SYM2, ODD>(op, 1, W1, W1, A, batch, lam, st, cgst)));
    FRAC_TRY((rows_inv_op<T, IK>(op, W1, out, n1, n2, nrows, (int)KB, st, inv)));
    return FRAC_OK;
  }
  C* W2 = W1 + w1;
  if constexpr (std::is_same<T, float>::value) {
    if (xy_enabled(op)) {  // three passes over HBM: xy forward, z (symbol), xy inverse
      FRAC_TRY((xy_fwd<FK, ODD>(op, in, W2, batch, lam, fwd, cgst, st)));
      ColArgs Az{(int)n3, (int)K1, (int)KB, op->Ma[1] * KB, batch, (int)n3, (int)op->Ma[1], (int)op->Ka[1]};
      FRAC_TRY((cols_op<T, ZSYM, ODD>(op, 2, W2, W2, Az, batch, lam, st, cgst)));
      FRAC_TRY((xy_inv<IK, ODD>(op, W2, out, batch, inv, st)));
      return FRAC_OK;
    }
  }
  const int64_t nrows = batch * n3 * n2;
  FRAC_TRY((rows_fwd_op<T, FK>(op, in, W1, n1, n2, nrows, (int)KB, st, fwd)));
  ColArgs Ay{(int)n2, (int)K1, (int)KB, KB, batch, (int)n3, (int)op->Ma[1], (int)op->Ka[1]};
  FRAC_TRY((cols_op<T, YFWD, ODD>(op, 1, W1, W2, Ay, batch * n3, lam, st, cgst)));
  ColArgs Az{(int)n3, (int)K1, (int)KB, op->Ma[1] * KB, batch, (int)n3, (int)op->Ma[1], (int)op->Ka[1]};
  FRAC_TRY((cols_op<T, ZSYM, ODD>(op, 2, W2, W2, Az, batch, lam, st, cgst)));
  FRAC_TRY((cols_op<T, YINV, ODD>(op, 1, W2, W1, Ay, batch * n3, lam, st, cgst)));
  FRAC_TRY((rows_inv_op<T, IK>(op, W1, out, n1, n2, nrows, (int)KB, st, inv)));
  return FRAC_OK;
}

}  // namespace frac
