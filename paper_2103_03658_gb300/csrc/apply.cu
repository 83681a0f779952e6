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

// ---------------------------------------------------------------------------
// d = 1: whole convolution per line
// ---------------------------------------------------------------------------

template <typename T, int LOGM, int LINES>
__global__ void __launch_bounds__(LINES * tpl(LOGM))
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
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    T re = (x < n && ha) ? u[va * n + x] : T(0);
    T im = (x < n && hb) ? u[vb * n + x] : T(0);
    buf[pidx(x)] = C{re, im};
  }
  __syncthreads();
  run<C, LOGM, false>(buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    const int kr = k <= M / 2 ? k : M - k;
    buf[pidx(k)] = cscale(buf[pidx(k)], lam[kr]);
  }
  __syncthreads();
  run<C, LOGM, true>(buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {
      C v = buf[pidx(x)];
      if (ha) y[va * n + x] = v.x;
      if (hb) y[vb * n + x] = v.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Rows, forward: two real rows -> one complex FFT -> two half spectra
// (stored without the 1/2 of the separation; the symbol carries it).
// ---------------------------------------------------------------------------

template <typename T, int LOGM, int LINES>
__global__ void __launch_bounds__(LINES * tpl(LOGM))
k_rows_fwd(const T* __restrict__ u, cplx_t<T>* __restrict__ W, int n, int64_t nrows,
           const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM);
  constexpr int K = M / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * LINES + line), r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    T re = (x < n && h0) ? u[r0 * n + x] : T(0);
    T im = (x < n && h1) ? u[r1 * n + x] : T(0);
    buf[pidx(x)] = C{re, im};
  }
  __syncthreads();
  run<C, LOGM, false>(buf, tl, tw);
  // U0 = Z[k] + conj(Z[M-k]),  U1 = -i (Z[k] - conj(Z[M-k])),  k in [0, M/2]
  for (int k = tl; k < K; k += TPL) {
    const C z = buf[pidx(k)];
    const C zc = cconj(buf[pidx((M - k) & (M - 1))]);
    const C s = cadd(z, zc), dd = csub(z, zc);
    if (h0) W[r0 * K + k] = s;
    if (h1) W[r1 * K + k] = C{dd.y, -dd.x};
  }
}

// ---------------------------------------------------------------------------
// Rows, inverse: two half spectra -> one complex line (Hermitian extension)
// -> iFFT -> two real rows (first n entries).
// ---------------------------------------------------------------------------

template <typename T, int LOGM, int LINES>
__global__ void __launch_bounds__(LINES * tpl(LOGM))
k_rows_inv(const cplx_t<T>* __restrict__ W, T* __restrict__ y, int n, int64_t nrows,
           const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM);
  constexpr int K = M / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * LINES + line), r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    const int k = x <= M / 2 ? x : M - x;
    C v0 = h0 ? W[r0 * K + k] : C{0, 0};
    C v1 = h1 ? W[r1 * K + k] : C{0, 0};
    if (x > M / 2) {
      v0 = cconj(v0);
      v1 = cconj(v1);
    }
    buf[pidx(x)] = C{v0.x - v1.y, v0.y + v1.x};  // v0 + i v1
  }
  __syncthreads();
  run<C, LOGM, true>(buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {
      const C v = buf[pidx(x)];
      if (h0) y[r0 * n + x] = v.x;
      if (h1) y[r1 * n + x] = v.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Columns: TILE adjacent columns per block, one line per column.
// Element j of column c of outer slab o lives at base + o * os + j * es + c.
// MODE 0: pad len_in -> M, FFT, store M.
// MODE 1: pad len_in -> M, FFT, * Lambda, iFFT, store len_out.
// MODE 2: iFFT of all M, store len_out.
// ---------------------------------------------------------------------------

struct ColArgs {
  int64_t ncols, nouter;
  int64_t os_in, es_in, os_out, es_out;
  int len_in, len_out;
  int K;        // symbol extent per axis (M/2 + 1)
  int sym3d;    // 0: Lambda[kr][c] (d = 2); 1: Lambda[kr][c2r][c1], c = c2 K + c1 (d = 3)
};

template <typename T, int LOGM, int TILE, int MODE>
__global__ void __launch_bounds__(TILE * tpl(LOGM))
k_cols(const cplx_t<T>* in, cplx_t<T>* out, ColArgs A, const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), LS = line_stride(LOGM);
  constexpr int NT = TILE * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int64_t tiles = (A.ncols + TILE - 1) / TILE;
  const int64_t o = blockIdx.x / tiles;
  const int64_t c0 = (blockIdx.x % tiles) * TILE;
  const C* src = in + o * A.os_in + c0;
  // load (coalesced over columns)
  const int len_load = (MODE == 2) ? M : A.len_in;
  for (int idx = threadIdx.x; idx < len_load * TILE; idx += NT) {
    const int cl = idx % TILE, j = idx / TILE;
    C v = (c0 + cl < A.ncols) ? src[(int64_t)j * A.es_in + cl] : C{0, 0};
    sm[cl * LS + pidx(j)] = v;
  }
  if (MODE != 2) {
    for (int idx = threadIdx.x; idx < (M - len_load) * TILE; idx += NT) {
      const int cl = idx % TILE, j = len_load + idx / TILE;
      sm[cl * LS + pidx(j)] = C{0, 0};
    }
  }
  __syncthreads();
  const int line = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  C* buf = sm + line * LS;
  if (MODE != 2) run<C, LOGM, false>(buf, tl, tw);
  if (MODE == 1) {
    const int64_t c = c0 + line;
    const int64_t cc = c < A.ncols ? c : 0;
    const T* lrow;
    if (A.sym3d) {
      const int64_t c2 = cc / A.K, c1 = cc % A.K;
      const int64_t c2r = c2 <= M / 2 ? c2 : M - c2;
      lrow = lam + c2r * A.K + c1;  // + kr * K * K
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = tl + e * TPL;
        const int kr = k <= M / 2 ? k : M - k;
        buf[pidx(k)] = cscale(buf[pidx(k)], lrow[(int64_t)kr * A.K * A.K]);
      }
    } else {
      lrow = lam + cc;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = tl + e * TPL;
        const int kr = k <= M / 2 ? k : M - k;
        buf[pidx(k)] = cscale(buf[pidx(k)], lrow[(int64_t)kr * A.K]);
      }
    }
    __syncthreads();
  }
  if (MODE != 0) run<C, LOGM, true>(buf, tl, tw);
  // store (coalesced over columns)
  const int len_store = (MODE == 0) ? M : A.len_out;
  C* dst = out + o * A.os_out + c0;
  for (int idx = threadIdx.x; idx < len_store * TILE; idx += NT) {
    const int cl = idx % TILE, j = idx / TILE;
    if (c0 + cl < A.ncols) dst[(int64_t)j * A.es_out + cl] = sm[cl * LS + pidx(j)];
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

template <typename T, int LOGM>
struct Cfg {
  static constexpr int LINE_BYTES = line_stride(LOGM) * (int)sizeof(cplx_t<T>);
  // lines per block: aim for ~48-64 KB of shared memory and <= 512 threads
  static constexpr int lines_for(int maxbytes) {
    int l = maxbytes / LINE_BYTES;
    int lim = 512 / tpl(LOGM);
    l = l < lim ? l : lim;
    return l < 1 ? 1 : l;
  }
  static constexpr int ROW_LINES = lines_for(64 * 1024);
  static constexpr int TILE = lines_for(72 * 1024) >= 8 ? 8 : lines_for(72 * 1024);
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

template <typename T, int LOGM>
static int launch_rows(bool fwd, const void* in, void* out, int64_t n, int64_t nrows, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int L = Cfg<T, LOGM>::ROW_LINES;
  const size_t sm = (size_t)L * Cfg<T, LOGM>::LINE_BYTES;
  const int64_t pairs = cdiv(nrows, 2);
  char nb[48];
  prof::Scope ps(kname<T>(nb, fwd ? "rows_fwd" : "rows_inv", LOGM), st);
  if (fwd) {
    auto kern = k_rows_fwd<T, LOGM, L>;
    FRAC_TRY(set_smem(kern, sm));
    kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const T*)in, (C*)out, (int)n, nrows, tw_table<T>(LOGM));
  } else {
    auto kern = k_rows_inv<T, LOGM, L>;
    FRAC_TRY(set_smem(kern, sm));
    kern<<<(unsigned)cdiv(pairs, L), L * tpl(LOGM), sm, st>>>((const C*)in, (T*)out, (int)n, nrows, tw_table<T>(LOGM));
  }
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <typename T, int LOGM, int MODE>
static int launch_cols(const void* in, void* out, const ColArgs& A, const T* lam, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int TILE = Cfg<T, LOGM>::TILE;
  const size_t sm = (size_t)TILE * Cfg<T, LOGM>::LINE_BYTES;
  auto kern = k_cols<T, LOGM, TILE, MODE>;
  FRAC_TRY(set_smem(kern, sm));
  const int64_t blocks = A.nouter * cdiv(A.ncols, TILE);
  char nb[48];
  prof::Scope ps(kname<T>(nb, MODE == 0 ? "cols_fwd" : (MODE == 1 ? "cols_sym" : "cols_inv"), LOGM), st);
  kern<<<(unsigned)blocks, TILE * tpl(LOGM), sm, st>>>((const C*)in, (C*)out, A, lam, tw_table<T>(LOGM));
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
template <typename T>
static int rows_any(int logm, bool fwd, const void* in, void* out, int64_t n, int64_t nrows, cudaStream_t st) {
  FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_rows<T, LG>(fwd, in, out, n, nrows, st)));
}
template <typename T, int MODE>
static int cols_any(int logm, const void* in, void* out, const ColArgs& A, const T* lam, cudaStream_t st) {
  FRAC_DISPATCH_LOGM(logm, 1, 11, (launch_cols<T, LG, MODE>(in, out, A, lam, st)));
}

size_t apply_workspace_bytes(const frac_op* op, int dtype, int64_t batch) {
  const size_t cs = dtype == FRAC_F64 ? sizeof(double2) : sizeof(float2);
  const int64_t n = op->n, M = op->M, K = op->K;
  if (op->prob.d == 1) return 0;
  if (op->prob.d == 2) return (size_t)batch * n * K * cs;
  return (size_t)batch * ((size_t)n * n * K + (size_t)n * M * K) * cs;
}

template <typename T>
int apply_t(const frac_op* op, const T* u, T* y, int64_t batch, void* ws, cudaStream_t st) {
  using C = cplx_t<T>;
  const int d = op->prob.d, logm = op->logm;
  const int64_t n = op->n, M = op->M, K = op->K;
  const T* lam = sym_table<T>(op);
  if (batch <= 0) return FRAC_OK;
  if (d == 1) return conv1d_any<T>(logm, u, y, n, batch, lam, st);
  C* W1 = (C*)ws;
  if (d == 2) {
    const int64_t nrows = batch * n;
    FRAC_TRY(rows_any<T>(logm, true, u, W1, n, nrows, st));
    ColArgs A{K, batch, n * K, K, n * K, K, (int)n, (int)n, (int)K, 0};
    FRAC_TRY((cols_any<T, 1>(logm, W1, W1, A, lam, st)));
    FRAC_TRY(rows_any<T>(logm, false, W1, y, n, nrows, st));
    return FRAC_OK;
  }
  // d == 3
  C* W2 = W1 + batch * n * n * K;
  const int64_t nrows = batch * n * n;
  FRAC_TRY(rows_any<T>(logm, true, u, W1, n, nrows, st));
  {  // y forward: outer = (b, j3), columns k1, elements j2
    ColArgs A{K, batch * n, n * K, K, M * K, K, (int)n, (int)M, (int)K, 0};
    FRAC_TRY((cols_any<T, 0>(logm, W1, W2, A, lam, st)));
  }
  {  // z: outer = b, columns (k2, k1), elements j3; symbol; in place
    ColArgs A{M * K, batch, n * M * K, M * K, n * M * K, M * K, (int)n, (int)n, (int)K, 1};
    FRAC_TRY((cols_any<T, 1>(logm, W2, W2, A, lam, st)));
  }
  {  // y inverse: outer = (b, j3), columns k1, elements k2 -> j2 < n
    ColArgs A{K, batch * n, M * K, K, n * K, K, (int)M, (int)n, (int)K, 0};
    FRAC_TRY((cols_any<T, 2>(logm, W2, W1, A, lam, st)));
  }
  FRAC_TRY(rows_any<T>(logm, false, W1, y, n, nrows, st));
  return FRAC_OK;
}

template int apply_t<float>(const frac_op*, const float*, float*, int64_t, void*, cudaStream_t);
template int apply_t<double>(const frac_op*, const double*, double*, int64_t, void*, cudaStream_t);

}  // namespace frac
