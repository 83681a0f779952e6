// Shared-memory Stockham FFT of one line (length M = 2^LOGM) per group of
// threads, radix 2..16 passes with register butterflies.
//
// Layout: each line lives in shared memory with padded index pidx(i) =
// i + i/16 (breaks the power-of-two strides of the butterfly writes into
// distinct banks) and a line stride LS = line_stride(M) (odd, so that the same
// element of consecutive lines falls in different banks when a tile of
// columns is loaded with one lane per line).
//
// Pass p of radix R = 2^b with sub-transform length Ns (product of the
// earlier radices): butterfly j in [0, M/R) reads x[j + r M/R], multiplies
// element r by w^{r (j mod Ns)} with w = exp(-+2 pi i/(Ns R)), does an R-point
// DFT in registers and writes element r to (j / Ns) Ns R + (j mod Ns) + r Ns.
// After the last pass the line holds the DFT in natural order.
#pragma once

#include <utility>

#include "common.cuh"

namespace frac {
namespace fft {

__host__ __device__ constexpr int npasses(int logm) { return logm <= 0 ? 0 : (logm + 3) / 4; }
__host__ __device__ constexpr int pass_bits(int logm, int p) {
  return logm / npasses(logm) + (p < logm % npasses(logm) ? 1 : 0);
}
__host__ __device__ constexpr int pass_ns_bits(int logm, int p) {
  return p == 0 ? 0 : pass_ns_bits(logm, p - 1) + pass_bits(logm, p - 1);
}
// elements held by one thread, and threads per line
__host__ __device__ constexpr int elems(int logm) { return logm >= 4 ? 16 : (1 << logm); }
__host__ __device__ constexpr int tpl(int logm) { return (1 << logm) / elems(logm); }
__host__ __device__ constexpr int line_stride(int logm) {
  return (1 << logm) + ((1 << logm) >> 4) + 1;
}

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// cos(2 pi k / 16) for k in [0, 16)
__host__ __device__ constexpr double cos16_0_8(int k) {
  return k == 0 ? 1.0 : k == 1 ? 0.92387953251128675613 : k == 2 ? 0.70710678118654752440
       : k == 3 ? 0.38268343236508977173 : k == 4 ? 0.0 : k == 5 ? -0.38268343236508977173
       : k == 6 ? -0.70710678118654752440 : k == 7 ? -0.92387953251128675613 : -1.0;
}
__host__ __device__ constexpr double cos16(int k) { return k <= 8 ? cos16_0_8(k) : cos16_0_8(16 - k); }
// sin(2 pi k / 16) = cos(2 pi (k - 4) / 16)
__host__ __device__ constexpr double sin16(int k) { return cos16((k + 12) & 15); }

// v * exp(s 2 pi i K / 16), s = -1 forward, +1 inverse
template <int K, bool INV, typename C>
__device__ __forceinline__ C mul_w16(C v) {
  using T = decltype(v.x);
  constexpr int k = K & 15;
  if constexpr (k == 0) {
    return v;
  } else if constexpr (k == 4) {  // forward: -i, inverse: +i
    return INV ? C{-v.y, v.x} : C{v.y, -v.x};
  } else if constexpr (k == 8) {
    return C{-v.x, -v.y};
  } else if constexpr (k == 12) {  // forward: +i, inverse: -i
    return INV ? C{v.y, -v.x} : C{-v.y, v.x};
  } else {
    constexpr double cr = cos16(k);
    constexpr double si = sin16(k);
    const T c = (T)cr;
    const T s = INV ? (T)si : (T)(-si);
    return C{v.x * c - v.y * s, v.x * s + v.y * c};
  }
}

template <int R, bool INV, typename C, int... Ks>
__device__ __forceinline__ void combine(C* x, const C* e, const C* o, std::integer_sequence<int, Ks...>) {
  C t[R / 2];
  ((t[Ks] = mul_w16<Ks * (16 / R), INV>(o[Ks])), ...);
  ((x[Ks] = cadd(e[Ks], t[Ks])), ...);
  ((x[Ks + R / 2] = csub(e[Ks], t[Ks])), ...);
}

// In-register R-point DFT (R = 1, 2, 4, 8, 16), natural order in and out.
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft(C* x) {
  if constexpr (R == 2) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (R > 2) {
    constexpr int H = R / 2;
    C e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    dft<H, INV>(e);
    dft<H, INV>(o);
    combine<R, INV>(x, e, o, std::make_integer_sequence<int, H>{});
  }
}

// One Stockham pass on this thread's line; tl = thread index within the line.
template <typename C, int LOGM, int P, bool INV>
__device__ __forceinline__ void pass(C* __restrict__ buf, int tl, const C* __restrict__ tw) {
  constexpr int M = 1 << LOGM;
  constexpr int RB = pass_bits(LOGM, P);
  constexpr int R = 1 << RB;
  constexpr int NSB = pass_ns_bits(LOGM, P);
  constexpr int Ns = 1 << NSB;
  constexpr int E = elems(LOGM);
  constexpr int TPL = tpl(LOGM);
  constexpr int NB = E / R;
  constexpr int TWS = M / (Ns * R);  // twiddle table stride
  C v[E];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = buf[pidx(j + r * (M / R))];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
    const int k = j & (Ns - 1);
    if constexpr (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * TWS];
        if (INV) w.y = -w.y;
        v[b * R + r] = cmul(v[b * R + r], w);
      }
    }
    dft<R, INV>(v + b * R);
    const int base = ((j >> NSB) << (NSB + RB)) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pidx(base + r * Ns)] = v[b * R + r];
  }
  __syncthreads();
}

template <typename C, int LOGM, bool INV, int P = 0>
__device__ __forceinline__ void run(C* __restrict__ buf, int tl, const C* __restrict__ tw) {
  if constexpr (P < npasses(LOGM)) {
    pass<C, LOGM, P, INV>(buf, tl, tw);
    run<C, LOGM, INV, P + 1>(buf, tl, tw);
  }
}

}  // namespace fft
}  // namespace frac
