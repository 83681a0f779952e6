// Whole 1D solves inside one thread block (M <= 8192): the FFT line lives in
// shared memory, each thread keeps its 16 entries of the CG vectors in
// registers, every scalar of CG and of the iterative refinement stays in the
// block.  One launch solves any number of problems of one FFT length (one
// block per problem), so a batch of 1D problems costs one launch per size
// class instead of several launches per CG iteration.
//
//   plain : CG with the FP64 apply.
//   mixed : r = f - A64 u (FP64), FP32 CG on A d = r / ||r|| to a relative
//           reduction inner_tol, u += ||r|| d, until ||f - A64 u|| <= rtol ||f||.
#include <cmath>
#include <cstdio>

#include "apply.cuh"
#include "fft.cuh"
#include "prof.cuh"
#include "solve1d.cuh"

namespace frac {

using namespace fft;

namespace {

// Block-wide FP64 sum; every thread gets the result.
template <int NT>
__device__ __forceinline__ double block_allsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // previous use of red[] finished
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  constexpr int NW = (NT + 31) / 32;
#pragma unroll
  for (int i = 0; i < NW; ++i) s += red[i];
  return s;
}

// (A v) for one real vector with the register-interface FFT: v is zero beyond n
// <= M/2 (the first pass skips that half) and only entries below n are kept (the
// last pass skips the other half).  `load(e, x)` gives v at grid point x = tl + e TPL
// (e < E/2); on return y[e].x holds (A v) at x = tl + e TPL for e < E/2.
template <typename T, int LOGM, typename Load>
__device__ __forceinline__ void conv_line(cplx_t<T> (&y)[elems(LOGM)], cplx_t<T>* buf, int n,
                                          const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, Load load) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM);
  const int tl = threadIdx.x;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    y[e] = C{(e < E / 2 && x < n) ? load(e, x) : T(0), T(0)};
  }
  fft_reg<C, LOGM, false, true, false>(y, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    const int kr = k <= M / 2 ? k : M - k;
    y[e] = cscale(y[e], lam[kr]);
  }
  fft_reg<C, LOGM, true, false, true>(y, buf, tl, tw);
}

// z = P r with the tau preconditioner on the line `buf`: the odd extension of
// the vector (entry x at x + 1, its negative at M - 1 - x), FFT, * pinv, iFFT;
// z at entry x is left in buf[pidx(x + 1)].x.
template <typename T, int LOGM, typename Load>
__device__ __forceinline__ void precond_line(cplx_t<T>* buf, int n, const T* __restrict__ pinv,
                                             const cplx_t<T>* __restrict__ tw, Load load) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LOGM, E = elems(LOGM), TPL = tpl(LOGM);
  const int tl = threadIdx.x;
  __syncthreads();  // earlier readers of buf are done
#pragma unroll
  for (int e = 0; e < E; ++e) buf[pidx(tl + e * TPL)] = C{T(0), T(0)};
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {  // n <= M/2 - 1: the two images never meet
      const T v = load(e, x);
      buf[pidx(x + 1)] = C{v, T(0)};
      buf[pidx(M - 1 - x)] = C{-v, T(0)};
    }
  }
  __syncthreads();
  C v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = buf[pidx(tl + e * TPL)];
  fft_reg<C, LOGM, false, false, false>(v, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    const int kr = k <= M / 2 ? k : M - k;
    v[e] = cscale(v[e], pinv[kr]);
  }
  fft_reg<C, LOGM, true, false, false>(v, buf, tl, tw);
  __syncthreads();  // the last pass's reads of buf are done
#pragma unroll
  for (int e = 0; e < E; ++e) buf[pidx(tl + e * TPL)] = v[e];
  __syncthreads();
}

}  // namespace

template <int LOGM, bool MIXED>
__global__ void __launch_bounds__(tpl(LOGM))
k_solve1d(const Solve1dTask* __restrict__ tasks, int ntasks, const float2* __restrict__ tw32,
          const double2* __restrict__ tw64) {
  constexpr int E = elems(LOGM), TPL = tpl(LOGM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  if (blockIdx.x >= ntasks) return;
  const Solve1dTask T = tasks[blockIdx.x];
  const int n = T.n, tl = threadIdx.x;
  double2* buf64 = reinterpret_cast<double2*>(smem_raw);
  float2* buf32 = reinterpret_cast<float2*>(smem_raw);
  double* __restrict__ U = T.u;
  const double* __restrict__ F = T.f;

  if (!T.use_x0) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      if (x < n) U[x] = 0.0;
    }
  }
  double fn2 = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    const double fv = x < n ? F[x] : 0.0;
    fn2 += fv * fv;
  }
  fn2 = block_allsum<TPL>(fn2, red);

  int iters = 0, outer = 0, status = FRAC_OK;
  // r64 = f - A64 u into r (registers), returns ||r||^2
  double2 y64[E];
  auto residual = [&](double (&r)[E]) {
    conv_line<double, LOGM>(y64, buf64, n, T.lam64, tw64, [&](int, int x) { return U[x]; });
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      r[e] = (e < E / 2 && x < n) ? F[x] - y64[e].x : 0.0;
      s += r[e] * r[e];
    }
    return block_allsum<TPL>(s, red);
  };
  // the first residual when u starts at 0: f itself (no FP64 convolution)
  auto from_f = [&](double (&r)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      r[e] = (e < E / 2 && x < n) ? F[x] : 0.0;
    }
    return fn2;
  };
  const double tol2 = T.rtol * T.rtol * fn2;
  double rn2 = 0.0;

  if (fn2 == 0.0) {
    rn2 = 0.0;
  } else if constexpr (!MIXED) {
    // FP64 CG (preconditioned when T.pcg), restarted from the true residual if
    // the recursive one drifts
    double r[E], p[E];
    rn2 = T.use_x0 ? residual(r) : from_f(r);
    // rz = r.z with z = P r (pcg) or z = r; the new direction p = z + beta p
    auto precond_rz = [&]() -> double {
      precond_line<double, LOGM>(buf64, n, T.pinv64, tw64, [&](int e, int) { return r[e]; });
      double s = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int x = tl + e * TPL;
        if (x < n) s += r[e] * buf64[pidx(x + 1)].x;
      }
      return block_allsum<TPL>(s, red);
    };
    for (int restart = 0; restart < 8 && rn2 > tol2 && iters < T.max_iter; ++restart) {
      double rz = T.pcg ? precond_rz() : rn2;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int x = tl + e * TPL;
        p[e] = T.pcg ? (x < n ? buf64[pidx(x + 1)].x : 0.0) : r[e];
      }
      double rr = rn2;
      while (rr > tol2 && iters < T.max_iter) {
        conv_line<double, LOGM>(y64, buf64, n, T.lam64, tw64, [&](int e, int) { return p[e]; });
        double pq = 0.0;
#pragma unroll
        for (int e = 0; e < E / 2; ++e) pq += p[e] * y64[e].x;  // p = 0 beyond n
        pq = block_allsum<TPL>(pq, red);
        if (!(pq > 0.0) || !isfinite(pq)) {
          status = FRAC_EBREAKDOWN;
          break;
        }
        const double al = rz / pq;
        double rr1 = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int x = tl + e * TPL;
          if (e < E / 2 && x < n) {  // the convolution is nonzero beyond n; r and p stay zero there
            U[x] += al * p[e];
            r[e] -= al * y64[e].x;
          }
          rr1 += r[e] * r[e];
        }
        rr1 = block_allsum<TPL>(rr1, red);
        rr = rr1;
        ++iters;
        if (!(rr > tol2)) break;
        const double rz1 = T.pcg ? precond_rz() : rr1;
        const double be = rz1 / rz;
        rz = rz1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int x = tl + e * TPL;
          const double z = T.pcg ? (x < n ? buf64[pidx(x + 1)].x : 0.0) : r[e];
          p[e] = z + be * p[e];
        }
      }
      if (status != FRAC_OK) break;
      rn2 = residual(r);
    }
  } else {
    static_assert(MIXED, "");
    const double inner2 = T.inner_tol * T.inner_tol;
    float x[E], r[E], p[E];
    // residual in FP64, then scaled to unit norm in FP32 for the next inner solve
    auto refresh = [&](bool zero_u) {
      double r64[E];
      const double nn = zero_u ? from_f(r64) : residual(r64);
      const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) r[e] = (float)(r64[e] * sc);
      return nn;
    };
    rn2 = refresh(!T.use_x0);
    double prev = INFINITY;
    auto precond_rz = [&]() -> double {
      precond_line<float, LOGM>(buf32, n, T.pinv32, tw32, [&](int e, int) { return r[e]; });
      float s = 0.0f;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int xx = tl + e * TPL;
        if (xx < n) s += r[e] * buf32[pidx(xx + 1)].x;
      }
      return block_allsum<TPL>((double)s, red);
    };
    while (rn2 > tol2 && iters < T.max_iter && outer < 100) {
      double rr = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        x[e] = 0.0f;
        rr += (double)r[e] * r[e];
      }
      rr = block_allsum<TPL>(rr, red);
      double rz = T.pcg ? precond_rz() : rr;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int xx = tl + e * TPL;
        p[e] = T.pcg ? (xx < n ? buf32[pidx(xx + 1)].x : 0.0f) : r[e];
      }
      const double stop = inner2 * rr;
      while (rr > stop && iters < T.max_iter) {
        float2 y32[E];
        conv_line<float, LOGM>(y32, buf32, n, T.lam32, tw32, [&](int e, int) { return p[e]; });
        float pqf = 0.0f;
#pragma unroll
        for (int e = 0; e < E / 2; ++e) pqf += p[e] * y32[e].x;
        const double pq = block_allsum<TPL>((double)pqf, red);
        if (!(pq > 0.0) || !isfinite(pq)) break;  // inner breakdown: refine from here
        const float al = (float)(rz / pq);
        float rr1f = 0.0f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (e < E / 2 && tl + e * TPL < n) {  // r and p stay zero beyond n
            x[e] += al * p[e];
            r[e] -= al * y32[e].x;
          }
          rr1f += r[e] * r[e];
        }
        const double rr1 = block_allsum<TPL>((double)rr1f, red);
        rr = rr1;
        ++iters;
        if (!(rr > stop)) break;
        const double rz1 = T.pcg ? precond_rz() : rr1;
        const float be = (float)(rz1 / rz);
        rz = rz1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int xx = tl + e * TPL;
          const float z = T.pcg ? (xx < n ? buf32[pidx(xx + 1)].x : 0.0f) : r[e];
          p[e] = z + be * p[e];
        }
      }
      const double sc = sqrt(rn2);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int xx = tl + e * TPL;
        if (xx < n) U[xx] += sc * (double)x[e];
      }
      rn2 = refresh(false);
      ++outer;
      if (!(rn2 < prev) && outer > 3) break;  // refinement stagnated
      prev = rn2;
    }
  }
  if (tl == 0) {
    frac_solve_info out;
    out.iters = iters;
    out.outer = outer;
    out.precond = T.pcg;
    out.rel_resid = fn2 > 0.0 ? sqrt(rn2 / fn2) : (fn2 == 0.0 ? 0.0 : NAN);  // NaN: non-finite f
    if (status == FRAC_OK && !(out.rel_resid <= T.rtol)) status = FRAC_ENOCONV;
    if (!isfinite(out.rel_resid)) status = FRAC_EINVAL;
    out.status = status;
    *T.info = out;
  }
}

template <int LOGM, bool MIXED>
static int launch_solve1d(const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  constexpr int LS = line_stride(LOGM);
  const size_t smem = (size_t)LS * (MIXED ? sizeof(double2) : sizeof(double2));
  auto kern = k_solve1d<LOGM, MIXED>;
  if (smem > 48 * 1024)
    FRAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  char nb[48];
  std::snprintf(nb, sizeof(nb), "solve1d_%s_M%d", MIXED ? "mixed" : "f64", 1 << LOGM);
  prof::Scope ps(nb, st);
  kern<<<ntasks, tpl(LOGM), smem, st>>>(d_tasks, ntasks, twiddles32(LOGM), twiddles64(LOGM));
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

template <int LOGM>
static int launch_any(bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  return mixed ? launch_solve1d<LOGM, true>(d_tasks, ntasks, st) : launch_solve1d<LOGM, false>(d_tasks, ntasks, st);
}

int solve1d_launch(int logm, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return FRAC_OK;
  FRAC_TRY(prepare_twiddles(logm));
  switch (logm) {
    case 1: return launch_any<1>(mixed, d_tasks, ntasks, st);
    case 2: return launch_any<2>(mixed, d_tasks, ntasks, st);
    case 3: return launch_any<3>(mixed, d_tasks, ntasks, st);
    case 4: return launch_any<4>(mixed, d_tasks, ntasks, st);
    case 5: return launch_any<5>(mixed, d_tasks, ntasks, st);
    case 6: return launch_any<6>(mixed, d_tasks, ntasks, st);
    case 7: return launch_any<7>(mixed, d_tasks, ntasks, st);
    case 8: return launch_any<8>(mixed, d_tasks, ntasks, st);
    case 9: return launch_any<9>(mixed, d_tasks, ntasks, st);
    case 10: return launch_any<10>(mixed, d_tasks, ntasks, st);
    case 11: return launch_any<11>(mixed, d_tasks, ntasks, st);
    case 12: return launch_any<12>(mixed, d_tasks, ntasks, st);
    case 13: return launch_any<13>(mixed, d_tasks, ntasks, st);
    default: return FRAC_ENOTSUP;
  }
}

}  // namespace frac
