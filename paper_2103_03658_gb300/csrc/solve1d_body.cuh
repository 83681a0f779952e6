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
#pragma once

#include <cmath>
#include <cstdio>

#include "apply.cuh"
#include "fft.cuh"
#include "fft_mixed.cuh"
#include "prof.cuh"
#include "solve1d.cuh"

namespace frac {

using namespace fft;

namespace {

// Block-wide FP64 sum; every thread gets the result.  NT: the block size (0: taken
// from blockDim.x; a block whose size is not a multiple of 32 ends in a partial warp,
// whose missing lanes the shuffle mask leaves out).
template <int NT>
__device__ __forceinline__ double block_allsum(double v, double* red) {
  const int nt = NT > 0 ? NT : (int)blockDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int live = nt - (w << 5);
  const unsigned mask = live >= 32 ? 0xffffffffu : ((1u << live) - 1u);
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(mask, v, o);
    if ((l ^ o) < live) v += t;
  }
  __syncthreads();  // previous use of red[] finished
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (nt + 31) / 32;
#pragma unroll 4
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Threads per block of a line policy known at compile time (0: a mixed length).
template <typename LN> struct line_threads { static constexpr int value = 0; };
template <int L, int S> struct line_threads<P2Line<L, S>> { static constexpr int value = tpl(L); };

// (A v) for one real vector with the register-interface FFT: v is zero beyond n
// <= M/2 (the first pass skips that half) and only entries below n are kept (the
// last pass skips the other half).  `load(e, x)` gives v at grid point x = tl + e TPL
// (e < E/2); on return y[e].x holds (A v) at x = tl + e TPL for e < E/2.
template <typename T, typename LN, typename Load>
__device__ __forceinline__ void conv_line(const LN& ln, cplx_t<T> (&y)[LN::E], cplx_t<T>* buf, int n,
                                          const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, Load load) {
  using C = cplx_t<T>;
  constexpr int E = LN::E;
  const int M = ln.m(), TPL = ln.tpl();
  const int tl = threadIdx.x;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    y[e] = C{(e < E / 2 && x < n) ? load(e, x) : T(0), T(0)};
  }
  ln.template fft<false, true, false>(y, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    const int kr = k <= M / 2 ? k : M - k;
    y[e] = cscale(y[e], lam[kr]);
  }
  ln.template fft<true, false, true>(y, buf, tl, tw);
}

// z = P r with the tau preconditioner on the line `buf`: the odd extension of
// the vector (entry x at x + 1, its negative at M - 1 - x), FFT, * pinv, iFFT;
// z at entry x is left in buf[ln.pad(x + 1)].x.
template <typename T, typename LN, typename Load>
__device__ __forceinline__ void precond_line(const LN& ln, cplx_t<T>* buf, int n, const T* __restrict__ pinv,
                                             const cplx_t<T>* __restrict__ tw, Load load) {
  using C = cplx_t<T>;
  constexpr int E = LN::E;
  const int M = ln.m(), TPL = ln.tpl();
  const int tl = threadIdx.x;
  __syncthreads();  // earlier readers of buf are done
#pragma unroll
  for (int e = 0; e < E; ++e) buf[ln.pad(tl + e * TPL)] = C{T(0), T(0)};
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = tl + e * TPL;
    if (x < n) {  // n <= M/2 - 1: the two images never meet
      const T v = load(e, x);
      buf[ln.pad(x + 1)] = C{v, T(0)};
      buf[ln.pad(M - 1 - x)] = C{-v, T(0)};
    }
  }
  __syncthreads();
  C v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = buf[ln.pad(tl + e * TPL)];
  ln.template fft<false, false, false>(v, buf, tl, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = tl + e * TPL;
    const int kr = k <= M / 2 ? k : M - k;
    v[e] = cscale(v[e], pinv[kr]);
  }
  ln.template fft<true, false, false>(v, buf, tl, tw);
  __syncthreads();  // the last pass's reads of buf are done
#pragma unroll
  for (int e = 0; e < E; ++e) buf[ln.pad(tl + e * TPL)] = v[e];
  __syncthreads();
}

}  // namespace

// One whole solve per block on the line policy ln (block size ln.tpl()).
template <typename LN, bool MIXED>
__device__ __forceinline__ void solve1d_block(const LN& ln, const Solve1dTask* __restrict__ tasks, int ntasks,
                                              const float2* __restrict__ tw32, const double2* __restrict__ tw64,
                                              unsigned char* smem_raw, double* red) {
  constexpr int E = LN::E, NT = line_threads<LN>::value;
  const int TPL = ln.tpl();
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
  fn2 = block_allsum<NT>(fn2, red);

  int iters = 0, outer = 0, status = FRAC_OK;
  // r64 = f - A64 u into r (registers), returns ||r||^2
  double2 y64[E];
  auto residual = [&](double (&r)[E]) {
    conv_line<double>(ln, y64, buf64, n, T.lam64, tw64, [&](int, int x) { return U[x]; });
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      r[e] = (e < E / 2 && x < n) ? F[x] - y64[e].x : 0.0;
      s += r[e] * r[e];
    }
    return block_allsum<NT>(s, red);
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
      precond_line<double>(ln, buf64, n, T.pinv64, tw64, [&](int e, int) { return r[e]; });
      double s = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int x = tl + e * TPL;
        if (x < n) s += r[e] * buf64[ln.pad(x + 1)].x;
      }
      return block_allsum<NT>(s, red);
    };
    for (int restart = 0; restart < 8 && rn2 > tol2 && iters < T.max_iter; ++restart) {
      double rz = T.pcg ? precond_rz() : rn2;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int x = tl + e * TPL;
        p[e] = T.pcg ? (x < n ? buf64[ln.pad(x + 1)].x : 0.0) : r[e];
      }
      double rr = rn2;
      while (rr > tol2 && iters < T.max_iter) {
        conv_line<double>(ln, y64, buf64, n, T.lam64, tw64, [&](int e, int) { return p[e]; });
        double pq = 0.0;
#pragma unroll
        for (int e = 0; e < E / 2; ++e) pq += p[e] * y64[e].x;  // p = 0 beyond n
        pq = block_allsum<NT>(pq, red);
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
        rr1 = block_allsum<NT>(rr1, red);
        rr = rr1;
        ++iters;
        if (!(rr > tol2)) break;
        const double rz1 = T.pcg ? precond_rz() : rr1;
        const double be = rz1 / rz;
        rz = rz1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int x = tl + e * TPL;
          const double z = T.pcg ? (x < n ? buf64[ln.pad(x + 1)].x : 0.0) : r[e];
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
      precond_line<float>(ln, buf32, n, T.pinv32, tw32, [&](int e, int) { return r[e]; });
      float s = 0.0f;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int xx = tl + e * TPL;
        if (xx < n) s += r[e] * buf32[ln.pad(xx + 1)].x;
      }
      return block_allsum<NT>((double)s, red);
    };
    while (rn2 > tol2 && iters < T.max_iter && outer < 100) {
      double rr = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        x[e] = 0.0f;
        rr += (double)r[e] * r[e];
      }
      rr = block_allsum<NT>(rr, red);
      double rz = T.pcg ? precond_rz() : rr;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int xx = tl + e * TPL;
        p[e] = T.pcg ? (xx < n ? buf32[ln.pad(xx + 1)].x : 0.0f) : r[e];
      }
      const double stop = inner2 * rr;
      while (rr > stop && iters < T.max_iter) {
        float2 y32[E];
        conv_line<float>(ln, y32, buf32, n, T.lam32, tw32, [&](int e, int) { return p[e]; });
        float pqf = 0.0f;
#pragma unroll
        for (int e = 0; e < E / 2; ++e) pqf += p[e] * y32[e].x;
        const double pq = block_allsum<NT>((double)pqf, red);
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
        const double rr1 = block_allsum<NT>((double)rr1f, red);
        rr = rr1;
        ++iters;
        if (!(rr > stop)) break;
        const double rz1 = T.pcg ? precond_rz() : rr1;
        const float be = (float)(rz1 / rz);
        rz = rz1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int xx = tl + e * TPL;
          const float z = T.pcg ? (xx < n ? buf32[ln.pad(xx + 1)].x : 0.0f) : r[e];
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

}  // namespace frac
