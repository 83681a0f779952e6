// Boundary vector of nonhomogeneous exterior data (frac_boundary), Eq. (L2):
// b_i = -c (near_i + far_i) at every interior point, near_i the sum over the
// exterior grid points x_i + o h, o in [-N, N]^d, of a_{|o|} g(x_i + o h) and far_i
// the far-field integrals of g, which the caller supplies.
//
// The near field is a convolution of the extended samples G (g on the grid points
// e in [1-N, n_i+N] per axis, zero at the interior ones; N + 1 the generator's extent,
// its cube spanning the longest axis) with the even generator: in the shifted index
// p = e + N - 1 in [0, E_i - 1], E_i = n_i + 2N, near_i = sum_o a_{|o|} G[p_i + o] with
// p_i = i + N - 1.  On a circulant of side M'_i >= E_i per axis that sum has no
// wrap-around for any p_i (every p_i + o stays in [0, E_i - 1], and |p - q| <= N + n_i - 1
// for output p and input q, so offsets beyond N never reach the kernel's support
// modulo M'_i), so near = IFFT(FFT(G) * Lambda') on the interior window, Lambda' the
// symbol of the generator at sides M'_i (generator_symbol_axes).  d >= 2: FP64 line
// FFTs along each axis of a complex array (M'_0/2 + 1 entries along axis 0, M'_i along
// the others), the first reading G, the last writing b on the interior window only.
// Lines that are still all zero (a coordinate at or beyond E_i on an axis not yet
// transformed) are skipped on the way in, lines whose results the window does not use
// on the way out, and, G being real, the upper half of the axis-0 spectrum, which the
// last pass rebuilds by conjugate symmetry.  d = 1: the N + 2 terms per point summed
// directly (one warp per point).
#include <algorithm>

#include "apply.cuh"
#include "fft.cuh"

namespace frac {
namespace {

// Self-checking accesses (an index outside [0, n) is recorded and skipped; the host
// reports it as FRAC_ECUDA).
__device__ unsigned long long g_bnd_fault_line = 0;
__device__ long long g_bnd_fault_index = 0;
__device__ __noinline__ void bnd_note_fault(int line, long long idx) {
  if (atomicCAS(&g_bnd_fault_line, 0ull, (unsigned long long)line) == 0ull) g_bnd_fault_index = idx;
}
#define BCHK(i, n)                                                                       \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) ? true \
                                                                               : (bnd_note_fault(__LINE__, (long long)(i)), false))

int take_bnd_fault() {
  unsigned long long line = 0;
  long long index = 0;
  FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&line, g_bnd_fault_line, sizeof(line)));
  if (!line) return FRAC_OK;
  FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&index, g_bnd_fault_index, sizeof(index)));
  const unsigned long long zero = 0;
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(g_bnd_fault_line, &zero, sizeof(zero)));
  return record_check_failure("boundary.cu", (int)line, index);
}

enum NfKind { NF_FWD = 0, NF_SYM = 1, NF_INV = 2 };

// One pass of line FFTs along `axis` of the array X (axis 0 fastest; extent K'_0 =
// M'_0/2 + 1 along axis 0, where the first pass keeps only those frequencies of the
// real samples, M'_i along the others).  The lines transformed are those whose
// other coordinates lie in [lo, lo + cnt) on each other axis; `fast` is the other
// axis of smallest stride (the tile axis: L adjacent lines per block), `slow` the
// remaining one (d = 3).  Per axis i: n_i interior points, E_i = n_i + 2N samples
// (p = e + N - 1 for e in [1-N, n_i+N]; the interior window p in [N, N+n_i-1]),
// circulant side M'_i = nextpow2(E_i), symbol extent K'_i = M'_i/2 + 1.
struct NfArgs {
  int d, axis, fast, slow;
  int64_t N;                     // generator intervals (its cube has side N h)
  int64_t n[3], E[3], Mp[3], Kp[3];
  int64_t lo[3], cnt[3];
  int64_t ntf;                   // tiles along `fast`
  int64_t total;                 // K'_0 M'_1 M'_2 entries of X (M'_2 = 1 for d = 2)
  int64_t nG;                    // prod E_i samples
  int64_t nS;                    // prod K'_i symbol entries
  int64_t nb;                    // prod n_i outputs
  int fill;                      // NF_FWD: read G instead of X
  int extract;                   // NF_INV along axis 0: write b on the interior window instead of X
  double negc;                   // -c
  double inv_norm;               // 1 / prod M'_i (unnormalised inverse transforms)
};

template <int LOGM>
__host__ __device__ constexpr int nf_lines_per_block() { return LOGM >= 12 ? 1 : 2; }

template <int LOGM, int KIND>
__global__ void __launch_bounds__(nf_lines_per_block<LOGM>() * fft::tpl(LOGM))
k_nf_lines(double2* X, const double* __restrict__ G, const double* __restrict__ S, const double* __restrict__ far,
           double* __restrict__ b, NfArgs A, const double2* __restrict__ tw) {
  using namespace fft;
  using C = double2;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM), SH = tile_shift(LOGM), LS = line_stride_tile(LOGM);
  constexpr int L = nf_lines_per_block<LOGM>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cl = threadIdx.x % L, tl = threadIdx.x / L;
  C* buf = reinterpret_cast<C*>(smem_raw) + cl * LS;
  const int64_t tile = blockIdx.x % A.ntf, sidx = blockIdx.x / A.ntf;
  const int64_t off = tile * L + cl;
  const bool live = off < A.cnt[A.fast];
  int64_t c[3] = {0, 0, 0};
  c[A.fast] = A.lo[A.fast] + off;
  if (A.d == 3) c[A.slow] = A.lo[A.slow] + sidx;
  const int64_t s1 = A.Kp[0], s2 = A.Kp[0] * A.Mp[1];                  // strides of axes 1, 2 in X
  const int64_t stride = A.axis == 0 ? 1 : (A.axis == 1 ? s1 : s2);
  const int64_t base = c[2] * s2 + c[1] * s1 + c[0];                    // c[axis] = 0
  const int64_t N = A.N;
  C v[E];
  if (KIND == NF_FWD && A.fill) {
    bool others_in = true;
    int64_t gbase = 0, gstride = 1, mul = 1;
    for (int i = 0; i < A.d; ++i) {
      if (i == A.axis) {
        gstride = mul;
      } else {
        gbase += c[i] * mul;
        others_in = others_in && c[i] >= N && c[i] < N + A.n[i];
      }
      mul *= A.E[i];
    }
    const int64_t Ea = A.E[A.axis], na = A.n[A.axis];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      double x = 0.0;
      if (live && j < Ea && !(others_in && j >= N && j < N + na)) {
        const int64_t idx = gbase + j * gstride;
        if (BCHK(idx, A.nG)) x = G[idx];
      }
      v[e] = C{x, 0.0};
    }
  } else if (KIND == NF_INV && A.extract) {
    // axis 0 of a real result: only k0 < K'_0 was carried through the other axes;
    // the rest is the conjugate, X[M'_0 - k0]
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      const bool lo_half = j < A.Kp[0];
      C x{0.0, 0.0};
      if (live) {
        const int64_t idx = base + (lo_half ? j : M - j) * stride;
        if (BCHK(idx, A.total)) x = X[idx];
      }
      v[e] = lo_half ? x : C{x.x, -x.y};
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      C x{0.0, 0.0};
      if (live) {
        const int64_t idx = base + j * stride;
        if (BCHK(idx, A.total)) x = X[idx];
      }
      v[e] = x;
    }
  }
  if (KIND != NF_INV) fft_reg<C, LOGM, false, false, false, SH>(v, buf, tl, tw);
  if (KIND == NF_SYM) {
    int64_t sb = 0, sstride = 1, mul = 1;
    for (int i = 0; i < A.d; ++i) {
      if (i == A.axis) {
        sstride = mul;
      } else {
        const int64_t k = c[i], kr = k <= A.Mp[i] / 2 ? k : A.Mp[i] - k;
        sb += kr * mul;
      }
      mul *= A.Kp[i];
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL, jr = j <= M / 2 ? j : M - j;
      double sv = 0.0;
      if (live) {
        const int64_t idx = sb + jr * sstride;
        if (BCHK(idx, A.nS)) sv = S[idx];
      }
      v[e] = cscale(v[e], sv);
    }
  }
  if (KIND != NF_FWD) fft_reg<C, LOGM, true, false, false, SH>(v, buf, tl, tw);
  if (!live) return;
  if (KIND == NF_INV && A.extract) {  // axis 0; the other coordinates lie in the window (launch range)
    int64_t ob = 0;
    for (int i = A.d - 1; i >= 1; --i) ob = ob * A.n[i] + (c[i] - N);
    ob *= A.n[0];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      if (j >= N && j < N + A.n[0]) {
        const int64_t o = ob + (j - N);
        if (BCHK(o, A.nb)) b[o] = A.negc * (v[e].x * A.inv_norm + (far ? far[o] : 0.0));
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      if (A.axis == 0 && j >= A.Kp[0]) continue;  // the conjugate half is not stored
      const int64_t idx = base + j * stride;
      if (BCHK(idx, A.total)) X[idx] = v[e];
    }
  }
}

template <int LOGM, int KIND>
int nf_launch(NfArgs A, double2* X, const double* G, const double* S, const double* far, double* b,
              cudaStream_t st) {
  constexpr int L = nf_lines_per_block<LOGM>();
  constexpr int threads = L * fft::tpl(LOGM);
  const size_t sm = (size_t)L * fft::line_stride_tile(LOGM) * sizeof(double2);
  A.ntf = (A.cnt[A.fast] + L - 1) / L;
  const int64_t blocks = A.ntf * (A.d == 3 ? A.cnt[A.slow] : 1);
  if (blocks == 0) return FRAC_OK;
  if (blocks > INT32_MAX) return FRAC_ENOTSUP;
  FRAC_CUDA_TRY(cudaFuncSetAttribute(k_nf_lines<LOGM, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_nf_lines<LOGM, KIND><<<(unsigned)blocks, threads, sm, st>>>(X, G, S, far, b, A, twiddles64(LOGM));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <int LOGM>
int nf_pass_t(int kind, const NfArgs& A, double2* X, const double* G, const double* S, const double* far, double* b,
              cudaStream_t st) {
  switch (kind) {
    case NF_FWD: return nf_launch<LOGM, NF_FWD>(A, X, G, S, far, b, st);
    case NF_SYM: return nf_launch<LOGM, NF_SYM>(A, X, G, S, far, b, st);
    default: return nf_launch<LOGM, NF_INV>(A, X, G, S, far, b, st);
  }
}

constexpr int kNfMinLog = 3, kNfMaxLog = 12;

int nf_pass(int logm, int kind, const NfArgs& A, double2* X, const double* G, const double* S, const double* far,
            double* b, cudaStream_t st) {
  switch (logm) {
    case 3: return nf_pass_t<3>(kind, A, X, G, S, far, b, st);
    case 4: return nf_pass_t<4>(kind, A, X, G, S, far, b, st);
    case 5: return nf_pass_t<5>(kind, A, X, G, S, far, b, st);
    case 6: return nf_pass_t<6>(kind, A, X, G, S, far, b, st);
    case 7: return nf_pass_t<7>(kind, A, X, G, S, far, b, st);
    case 8: return nf_pass_t<8>(kind, A, X, G, S, far, b, st);
    case 9: return nf_pass_t<9>(kind, A, X, G, S, far, b, st);
    case 10: return nf_pass_t<10>(kind, A, X, G, S, far, b, st);
    case 11: return nf_pass_t<11>(kind, A, X, G, S, far, b, st);
    case 12: return nf_pass_t<12>(kind, A, X, G, S, far, b, st);
    default: return FRAC_ENOTSUP;
  }
}

// d = 1: one warp per interior point i (p = i + N - 1); the lanes stride over the
// offsets o in [-N, N], skipping the interior window, and a butterfly of shuffles
// sums the lanes (the same order on every run).
__global__ void k_nf_direct_1d(const double* __restrict__ a, const double* __restrict__ G,
                               const double* __restrict__ far, double* __restrict__ b, int64_t N, double negc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t n = N - 1;
  if (w >= n) return;  // uniform across the warp
  const int64_t p = w + N;
  double s = 0.0;
  for (int64_t o = -N + lane; o <= N; o += 32) {
    const int64_t q = p + o, ao = o < 0 ? -o : o;
    if (q >= N && q <= 2 * N - 2) continue;
    if (BCHK(q, 3 * N - 1) && BCHK(ao, N + 1)) s += a[ao] * G[q];
  }
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (lane == 0) b[w] = negc * (s + (far ? far[w] : 0.0));
}

__global__ void k_subtract(const double* f, const double* __restrict__ g, double* r,
                           int64_t count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) r[i] = f[i] - g[i];
}

}  // namespace

int subtract_device(const double* f, const double* g, double* r, int64_t count, cudaStream_t st) {
  if (count == 0) return FRAC_OK;
  k_subtract<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(f, g, r, count);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

// g_ext, far and b on the device: prod_i (n_i + 2N), prod n_i (or NULL) and prod n_i
// doubles, axis 0 fastest; N = op->N (the generator's cube, N = max n_i + 1).
int boundary_device(const frac_op* op, const double* g_ext, const double* far, double* b, cudaStream_t st) {
  const int d = op->prob.d;
  const int64_t N = op->N;
  const double negc = -op->c;
  if (N < 2) return FRAC_EINVAL;
  if (d == 1) {
    if (op->na[0] != N - 1) return FRAC_EINVAL;
    const int64_t threads = (N - 1) * 32;
    k_nf_direct_1d<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(op->a, g_ext, far, b, N, negc);
    FRAC_CUDA_TRY(cudaGetLastError());
    FRAC_CUDA_TRY(cudaStreamSynchronize(st));
    return take_bnd_fault();
  }
  NfArgs A{};
  A.d = d;
  A.N = N;
  int logm[3] = {0, 0, 0};
  double full = 1.0;
  A.nG = A.nS = A.nb = 1;
  for (int i = 0; i < 3; ++i) {
    A.n[i] = A.E[i] = A.Mp[i] = A.Kp[i] = 1;
    if (i >= d) continue;
    A.n[i] = op->na[i];
    A.E[i] = op->na[i] + 2 * N;
    logm[i] = ilog2(A.E[i]);
    if (logm[i] < kNfMinLog || logm[i] > kNfMaxLog) return FRAC_ENOTSUP;
    A.Mp[i] = int64_t(1) << logm[i];
    A.Kp[i] = A.Mp[i] / 2 + 1;
    full *= (double)A.Mp[i];
    A.nG *= A.E[i];
    A.nS *= A.Kp[i];
    A.nb *= A.n[i];
  }
  A.total = A.Kp[0] * A.Mp[1] * A.Mp[2];
  A.negc = negc;
  A.inv_norm = 1.0 / full;
  for (int i = 0; i < d; ++i) FRAC_TRY(prepare_twiddles(logm[i]));
  double2* X = nullptr;
  double *S = nullptr, *tmp = nullptr;
  struct Free {
    double2** x;
    double** s;
    double** t;
    cudaStream_t st;
    ~Free() {
      if (*x) cudaFreeAsync(*x, st);
      if (*s) cudaFreeAsync(*s, st);
      if (*t) cudaFreeAsync(*t, st);
    }
  } fr{&X, &S, &tmp, st};
  FRAC_CUDA_TRY(cudaMallocAsync(&S, A.nS * sizeof(double), st));
  FRAC_CUDA_TRY(cudaMallocAsync(&tmp, A.nS * sizeof(double), st));
  FRAC_TRY(generator_symbol_axes(op, logm, S, tmp, st));
  FRAC_CUDA_TRY(cudaFreeAsync(tmp, st));
  tmp = nullptr;
  FRAC_CUDA_TRY(cudaMallocAsync(&X, A.total * sizeof(double2), st));
  FRAC_CUDA_TRY(cudaMemsetAsync(X, 0, A.total * sizeof(double2), st));

  auto pass = [&](int kind, int axis, const int64_t lo[3], const int64_t cnt[3], int fill, int extract) {
    NfArgs P = A;
    P.axis = axis;
    P.fast = axis == 0 ? 1 : 0;
    P.slow = 3 - axis - P.fast;  // d = 3 only
    for (int i = 0; i < 3; ++i) {
      P.lo[i] = lo[i];
      P.cnt[i] = i < d ? cnt[i] : 1;
    }
    P.fill = fill;
    P.extract = extract;
    return nf_pass(logm[axis], kind, P, X, g_ext, S, far, b, st);
  };
  // other-axis ranges: [0, E_i) where G has samples, [0, M'_i) everywhere, [N, N + n_i) the
  // interior window; along axis 0 after its forward transform only k0 < K'_0 (G is real: the
  // rest is conjugate-symmetric and the last pass rebuilds it)
  const int64_t z = 0, w = N;
  if (d == 2) {
    const int64_t lo0[3] = {z, z, z}, cnt0[3] = {0, A.E[1], 1};      // axis 0 from G: rows y < E_1
    const int64_t lo1[3] = {z, z, z}, cnt1[3] = {A.Kp[0], 0, 1};     // axis 1 with the symbol
    const int64_t lo2[3] = {z, w, z}, cnt2[3] = {0, A.n[1], 1};      // axis 0 inverse: window rows
    FRAC_TRY(pass(NF_FWD, 0, lo0, cnt0, 1, 0));
    FRAC_TRY(pass(NF_SYM, 1, lo1, cnt1, 0, 0));
    FRAC_TRY(pass(NF_INV, 0, lo2, cnt2, 0, 1));
  } else {
    const int64_t lo0[3] = {z, z, z}, cnt0[3] = {0, A.E[1], A.E[2]};        // axis 0 from G
    const int64_t lo1[3] = {z, z, z}, cnt1[3] = {A.Kp[0], 0, A.E[2]};       // axis 1: planes z < E_2
    const int64_t lo2[3] = {z, z, z}, cnt2[3] = {A.Kp[0], A.Mp[1], 0};      // axis 2 with the symbol
    const int64_t lo3[3] = {z, z, w}, cnt3[3] = {A.Kp[0], 0, A.n[2]};       // axis 1 inverse: window planes
    const int64_t lo4[3] = {z, w, w}, cnt4[3] = {0, A.n[1], A.n[2]};        // axis 0 inverse to b
    FRAC_TRY(pass(NF_FWD, 0, lo0, cnt0, 1, 0));
    FRAC_TRY(pass(NF_FWD, 1, lo1, cnt1, 0, 0));
    FRAC_TRY(pass(NF_SYM, 2, lo2, cnt2, 0, 0));
    FRAC_TRY(pass(NF_INV, 1, lo3, cnt3, 0, 0));
    FRAC_TRY(pass(NF_INV, 0, lo4, cnt4, 0, 1));
  }
  FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  FRAC_TRY(take_coeff_fault());
  return take_bnd_fault();
}

}  // namespace frac
