// Mixed-radix line FFT for lengths M = 2^a 3^b 5^c 7^d with a >= 4 (Sec. 2.2:
// the FFT length of an axis only has to hold the circulant embedding, and a
// 7-smooth length wastes less padding than the next power of two), and the
// line policies through which the passes of passes.cuh and the 1D solver use
// either transform.
//
// The mixed transform keeps the register interface of fft_reg: on entry and
// exit thread tl of a line holds entries tl + e TPL (e < 16) with TPL = M / 16.
// In between, every pass goes through the line's shared buffer (padded index
// i + i / 16): pass p of radix R with Ns = the product of the earlier radices
// takes butterfly j in [0, M/R) from x[j + r M/R], multiplies element r by
// w_M^{r (j mod Ns) M / (Ns R)}, does an R-point DFT and writes element r to
// (j / Ns) Ns R + (j mod Ns) + r Ns (the Stockham order, valid for any sequence of
// radices; natural order after the last pass).  The sequence (MxPlan): a
// power-of-two pass of radix 8 or 16 first, taken straight from the registers,
// then one radix-3, 5 or 7 pass per odd factor and the other power-of-two passes
// through the shared buffer, and the smallest power-of-two pass last, written
// straight into the registers (as fft_reg does at both ends).  Power-of-two
// passes give every thread 16 / R butterflies; an odd pass ceil(16 / R), the last
// of them idle on part of the threads.
#pragma once

#include <cstdint>

#include "fft.cuh"

namespace frac {
namespace fft {

// cos and sin of 2 pi m / R (R = 3, 5, 7; m in [0, R)), from the values on (0, pi).
__host__ __device__ constexpr double cos_odd_half(int R, int m) {
  return R == 3 ? -0.5
       : R == 5 ? (m == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
                : (m == 1 ? 0.623489801858733530525 : m == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double sin_odd_half(int R, int m) {
  return R == 3 ? 0.8660254037844386467637
       : R == 5 ? (m == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
                : (m == 1 ? 0.7818314824680298087084 : m == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758);
}
__host__ __device__ constexpr double cos_odd(int R, int m) {
  return m % R == 0 ? 1.0 : (m % R) <= R / 2 ? cos_odd_half(R, m % R) : cos_odd_half(R, R - m % R);
}
__host__ __device__ constexpr double sin_odd(int R, int m) {
  return m % R == 0 ? 0.0 : (m % R) <= R / 2 ? sin_odd_half(R, m % R) : -sin_odd_half(R, R - m % R);
}

// In-register R-point DFT for odd R (3, 5, 7), natural order in and out, by the
// pairs x_j +- x_{R-j}: X_k = x_0 + sum_j (x_j + x_{R-j}) cos(2 pi j k / R)
// -+ i sum_j (x_j - x_{R-j}) sin(2 pi j k / R), j = 1 .. (R-1)/2, and X_{R-k}
// with the sine part's sign flipped (- for the forward transform).
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_odd(C* x) {
  using T = decltype(x[0].x);
  constexpr int H = (R - 1) / 2;
  C s[H + 1], d[H + 1];
  C X0 = x[0];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    s[j] = cadd(x[j], x[R - j]);
    d[j] = csub(x[j], x[R - j]);
    X0 = cadd(X0, s[j]);
  }
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    C a = x[0], b = C{T(0), T(0)};
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      const T c = (T)cos_odd(R, j * k), sn = (T)sin_odd(R, j * k);
      a = C{a.x + c * s[j].x, a.y + c * s[j].y};
      b = C{b.x + sn * d[j].x, b.y + sn * d[j].y};
    }
    // forward: X_k = a - i b, X_{R-k} = a + i b; inverse: the other way round
    const C mib = C{b.y, -b.x};  // -i b
    x[INV ? R - k : k] = cadd(a, mib);
    x[INV ? k : R - k] = csub(a, mib);
  }
  x[0] = X0;
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_mx(C* x) {
  if constexpr ((R & (R - 1)) == 0)
    dft<R, INV>(x);
  else
    dft_odd<R, INV>(x);
}

__device__ __forceinline__ int mx_pad(int i) { return i + (i >> 4); }

// One pass of radix R over the line in buf (see the header).
// j / Ns for j < 2^14 and Ns <= 2^13 as the high word of j * inv, inv = ceil(2^32 / Ns)
// (exact in that range; Ns = 1 is j itself).
__device__ __forceinline__ unsigned mx_div(unsigned j, unsigned Ns, unsigned inv) {
  return Ns == 1 ? j : __umulhi(j, inv);
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void mx_pass(C* buf, int tl, int TPL, int M, int Ns, const C* __restrict__ tw) {
  constexpr int NB = (16 + R - 1) / R;
  const int nbf = M / R, tws = M / (Ns * R);
  const unsigned inv = 0xffffffffu / (unsigned)Ns + 1u;
  C w[NB * R];
  // for an odd R, nbf = M / R is a multiple of 16 (as M is), so pad(j + r nbf) =
  // pad(j) + r (nbf + nbf / 16): one address per butterfly
  const int rstep = nbf + (nbf >> 4);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
    if (NB * R == 16 || j < nbf) {
      if constexpr (R % 2 == 1) {
        const C* src = buf + mx_pad(j);
#pragma unroll
        for (int r = 0; r < R; ++r) w[b * R + r] = src[r * rstep];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) w[b * R + r] = buf[mx_pad(j + r * nbf)];
      }
    }
  }
  __syncthreads();  // every read of this pass done before its writes
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
    if (NB * R == 16 || j < nbf) {
      const int q = (int)mx_div((unsigned)j, (unsigned)Ns, inv), k = j - q * Ns;
      if (Ns > 1) {
        if constexpr (sizeof(decltype(w[0].x)) == 4) {
          // FP32: one table load, the other powers by binary splitting (as in fft.cuh)
          C wp[R];
          wp[1] = tw[k * tws];
          if (INV) wp[1].y = -wp[1].y;
#pragma unroll
          for (int r = 2; r < R; ++r) wp[r] = cmul(wp[r >> 1], wp[r - (r >> 1)]);
#pragma unroll
          for (int r = 1; r < R; ++r) w[b * R + r] = cmul(w[b * R + r], wp[r]);
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) {
            C t = tw[r * k * tws];
            if (INV) t.y = -t.y;
            w[b * R + r] = cmul(w[b * R + r], t);
          }
        }
      }
      dft_mx<R, INV>(w + b * R);
      const int base = q * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[mx_pad(base + r * Ns)] = w[b * R + r];
    }
  }
  __syncthreads();  // writes visible to the next pass
}

// The middle passes of the plan over the line in buf (everything but the first and
// last power-of-two passes), starting at Ns = plan.first.  Kernels with many
// transforms (the whole 1D solve) call it out of line, so that the radices of a
// runtime plan are compiled once per element type and direction (the line is in
// shared memory across the call); the apply kernels, with one or two transforms
// each, define FRAC_MX_PASSES_INLINE and inline it.
#ifdef FRAC_MX_PASSES_INLINE
#define FRAC_MX_PASSES_ATTR __forceinline__
#else
#define FRAC_MX_PASSES_ATTR __noinline__
#endif
template <bool INV, typename C>
__device__ FRAC_MX_PASSES_ATTR void mx_passes(C* buf, int tl, int TPL, MxPlan plan, const C* __restrict__ tw) {
  // one loop per radix keeps the register allocation of each pass to itself
  const int M = plan.m;
  int Ns = plan.first;
#pragma unroll 1
  for (int i = 0; i < plan.count[0]; ++i, Ns *= 3) mx_pass<3, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[1]; ++i, Ns *= 5) mx_pass<5, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[2]; ++i, Ns *= 7) mx_pass<7, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[3]; ++i, Ns *= 16) mx_pass<16, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[4]; ++i, Ns *= 8) mx_pass<8, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[5]; ++i, Ns *= 4) mx_pass<4, INV>(buf, tl, TPL, M, Ns, tw);
#pragma unroll 1
  for (int i = 0; i < plan.count[6]; ++i, Ns *= 2) mx_pass<2, INV>(buf, tl, TPL, M, Ns, tw);
}

// First pass (radix R = plan.first, Ns = 1, no twiddles) straight from the register
// interface: butterfly j = tl + b TPL (b < 16 / R) takes its inputs j + r M/R from
// v[b + r (16 / R)] and writes element r to j R + r.  ZIN: inputs r >= R/2 are zero.
template <int R, bool INV, bool ZIN, typename C>
__device__ __forceinline__ void mx_first(C (&v)[16], C* buf, int tl, int TPL) {
  constexpr int NB = 16 / R;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    C w[R];
#pragma unroll
    for (int r = 0; r < (ZIN ? R / 2 : R); ++r) w[r] = v[b + r * NB];
    if constexpr (ZIN)
      dft_zin<R, INV>(w);
    else
      dft<R, INV>(w);
    const int j = tl + b * TPL;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[mx_pad(j * R + r)] = w[r];
  }
}

// Last pass (radix R = plan.last, Ns = M / R) into the register interface: butterfly
// j = tl + b TPL (b < 16 / R; k = j) reads j + r M/R, multiplies element r by
// w_M^{r j}, and its outputs j + r M/R are the thread's v[b + r (16 / R)].  ZOUT:
// only outputs r < R/2 (entries below M/2) are stored.
template <int R, bool INV, bool ZOUT, typename C>
__device__ __forceinline__ void mx_last(C (&v)[16], const C* buf, int tl, int TPL, int M,
                                        const C* __restrict__ tw) {
  constexpr int NB = 16 / R;
  const int step = M / R;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
    C w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = buf[mx_pad(j + r * step)];
    if constexpr (sizeof(decltype(w[0].x)) == 4) {
      C wp[R];
      wp[1] = tw[j];
      if (INV) wp[1].y = -wp[1].y;
#pragma unroll
      for (int r = 2; r < R; ++r) wp[r] = cmul(wp[r >> 1], wp[r - (r >> 1)]);
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = cmul(w[r], wp[r]);
    } else {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C t = tw[r * j];
        if (INV) t.y = -t.y;
        w[r] = cmul(w[r], t);
      }
    }
    dft<R, INV>(w);
#pragma unroll
    for (int r = 0; r < (ZOUT ? R / 2 : R); ++r) v[b + r * NB] = w[r];
  }
}

// Line of a mixed length: M, its plan and TPL = M / 16 threads.
struct MxLine {
  static constexpr int E = 16;
  MxPlan plan;
  int tpl_;
  __host__ __device__ explicit MxLine(const MxPlan& p) : plan(p), tpl_(p.m / 16) {}
  __host__ __device__ int m() const { return plan.m; }
  __host__ __device__ int tpl() const { return tpl_; }
  __device__ static int pad(int i) { return mx_pad(i); }
  // entries of one line buffer (odd: consecutive lines in different banks)
  __host__ __device__ int stride() const { return plan.m + (plan.m >> 4) + 1; }
  // column tiles: lanes of B lines interleaved, stride 4 mod 16 (see line_stride_tile)
  __host__ __device__ int stride_tile() const {
    const int s = plan.m + (plan.m >> 4);
    return s + ((4 - (s & 15)) & 15);
  }
  // FFT of the line held in registers (the interface and the ZIN / ZOUT meaning of
  // fft_reg): the first pass from registers, the middle passes through buf, the last
  // pass into registers (or, with a single power-of-two pass, all 16 entries read
  // back from buf).
  template <bool INV, bool ZIN, bool ZOUT, typename C>
  __device__ void fft(C (&v)[E], C* buf, int tl, const C* __restrict__ tw) const {
    const int TPL = tpl_;
    __syncthreads();  // earlier users of buf are done
    if (plan.first == 16)
      mx_first<16, INV, ZIN>(v, buf, tl, TPL);
    else
      mx_first<8, INV, ZIN>(v, buf, tl, TPL);
    __syncthreads();
    mx_passes<INV>(buf, tl, TPL, plan, tw);
    if (plan.last == 16) {
      mx_last<16, INV, ZOUT>(v, buf, tl, TPL, plan.m, tw);
    } else if (plan.last == 8) {
      mx_last<8, INV, ZOUT>(v, buf, tl, TPL, plan.m, tw);
    } else if (plan.last == 4) {
      mx_last<4, INV, ZOUT>(v, buf, tl, TPL, plan.m, tw);
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = buf[mx_pad(tl + e * TPL)];
    }
  }
};

// Line of 2^LOGM entries on the register-interface FFT of fft.cuh (pad shift SH).
template <int LOGM, int SH = 4>
struct P2Line {
  static constexpr int E = elems(LOGM);
  __host__ __device__ static constexpr int m() { return 1 << LOGM; }
  __host__ __device__ static constexpr int tpl() { return fft::tpl(LOGM); }
  __device__ static constexpr int pad(int i) { return pidx<SH>(i); }
  __host__ __device__ static constexpr int stride() { return line_stride(LOGM); }
  __host__ __device__ static constexpr int stride_tile() { return line_stride_tile(LOGM); }
  template <bool INV, bool ZIN, bool ZOUT, typename C>
  __device__ static void fft(C (&v)[E], C* buf, int tl, const C* __restrict__ tw) {
    fft_reg<C, LOGM, INV, ZIN, ZOUT, SH>(v, buf, tl, tw);
  }
};

}  // namespace fft
}  // namespace frac
