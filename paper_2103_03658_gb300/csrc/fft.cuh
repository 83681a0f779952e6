// Shared-memory Stockham FFT of one line (length M = 2^LOGM) per group of
// threads, radix 2..16 passes with register butterflies.
//
// Layout: each line lives in shared memory with padded index pidx(i) =
// i + i/16 (breaks the power-of-two strides of the butterfly writes into
// distinct banks) and a line stride LS = line_stride(M) (odd, so that the same
// element of consecutive lines falls in different banks when a tile of
// columns is loaded with one lane per line).  Column tiles (lanes of 4 or 2
// lines interleaved) pad every 2^tile_shift(M) entries instead, with their own
// stride line_stride_tile(M).
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
// Padding shift of the lines of a column tile: one pad entry every 2^SH entries.
// SH = 4 unless the first pass has radix 8 or less (M = 32, 64, 512): its
// butterflies then write R-entry runs at j R, and with a pad every 16 entries
// two lanes of a half-warp land on the same bank slot; one pad per R entries
// (SH = log2 R) spreads them.
__host__ __device__ constexpr int tile_shift(int logm) {
  return npasses(logm) > 1 && pass_bits(logm, 0) < 4 ? pass_bits(logm, 0) : 4;
}
// Line stride for tiles whose lanes interleave 4 (FP32) or 2 (FP64) lines with the
// line index fastest: a stride of 4 mod 16 puts the 16 lanes of a half-warp
// (4 lines x 4 consecutive entries) in 16 distinct 8-byte bank slots.
__host__ __device__ constexpr int line_stride_tile(int logm) {
  return (1 << logm) + ((1 << logm) >> tile_shift(logm)) +
         ((4 - (((1 << logm) + ((1 << logm) >> tile_shift(logm))) & 15)) & 15);
}

template <int SH = 4>
__device__ __forceinline__ int pidx(int i) { return i + (i >> SH); }

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

template <int R, bool INV, typename C, int... Is>
__device__ __forceinline__ void split_half(const C* x, C* a, C* b, std::integer_sequence<int, Is...>) {
  ((a[Is] = x[Is]), ...);
  ((b[Is] = mul_w16<Is * (16 / R), INV>(x[Is])), ...);
}

// R-point DFT of a vector whose upper half x[R/2 .. R-1] is zero (those
// entries are not read).  Decimation in frequency: with the upper half zero,
// the even outputs are the R/2-point DFT of x[0 .. R/2-1] and the odd outputs
// that of x[i] w_R^i.
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_zin(C* x) {
  if constexpr (R == 2) {
    x[1] = x[0];
  } else if constexpr (R > 2) {
    constexpr int H = R / 2;
    C a[H], b[H];
    split_half<R, INV>(x, a, b, std::make_integer_sequence<int, H>{});
    dft<H, INV>(a);
    dft<H, INV>(b);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      x[2 * k] = a[k];
      x[2 * k + 1] = b[k];
    }
  }
}

// One Stockham pass on this thread's line; tl = thread index within the line.
template <typename C, int LOGM, int P, bool INV>
__device__ __forceinline__ void pass(C* buf, int tl, const C* __restrict__ tw) {
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

// ---------------------------------------------------------------------------
// Register-interface FFT: on entry and on exit thread tl of a line holds the
// E entries tl + e TPL (e = 0..E-1) of the line in v[e]; only the passes in
// between exchange through the line's shared-memory buffer.  Butterfly b of
// a pass of radix R (j = tl + b TPL) takes its inputs j + r M/R from
// v[b + r NB] in the first pass and leaves its outputs j + r M/R in
// v[b + r NB] in the last pass (NB = E / R), so no permutation is needed at
// either end.  The caller must not touch `buf` between the entry __syncthreads
// and the return.
//
// The line buffer `buf` is shared memory that other threads write between the
// barriers of a pass; it must not be declared __restrict__: a restrict-qualified
// pointer lets the compiler assume that the barrier does not change what it points
// to and move accesses across it (inlined into the persistent batch kernel, that
// produced wrong transforms for M = 32).
//
// Zero-padded transforms: ZIN states that entries M/2 .. M-1 of the input are
// zero (v[e] for e >= E/2 is not read); ZOUT that only outputs 0 .. M/2-1 are
// wanted (v[e] for e >= E/2 is left undefined).  A convolution of n <= M/2
// points embedded in length M meets both, and the first and last passes then
// skip the butterflies' dead halves.
// ---------------------------------------------------------------------------

template <typename C, int LOGM, int P, bool INV, bool ZIN, bool ZOUT, int SH>
__device__ __forceinline__ void reg_pass(C (&v)[elems(LOGM)], C* buf, int tl, const C* __restrict__ tw) {
  constexpr int M = 1 << LOGM;
  constexpr int NP = npasses(LOGM);
  constexpr int RB = pass_bits(LOGM, P);
  constexpr int R = 1 << RB;
  constexpr int NSB = pass_ns_bits(LOGM, P);
  constexpr int Ns = 1 << NSB;
  constexpr int E = elems(LOGM);
  constexpr int TPL = tpl(LOGM);
  constexpr int NB = E / R;
  constexpr int TWS = M / (Ns * R);
  constexpr bool FIRST = (P == 0), LAST = (P == NP - 1);
  constexpr int Q = 1 << SH;  // pad block: pidx<SH>(i) = i + i / Q
  C w[E];
  if constexpr (FIRST) {
    // butterfly j < M/R reads j + r M/R, which lies in the zero half iff r >= R/2
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int r = 0; r < (ZIN ? R / 2 : R); ++r) w[b * R + r] = v[b + r * NB];
  } else {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = tl + b * TPL;
      if constexpr ((M / R) % Q == 0) {  // pidx(j + c) = pidx(j) + pidx(c) for c a multiple of Q
        const C* src = buf + pidx<SH>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) w[b * R + r] = src[r * (M / R) + ((r * (M / R)) >> SH)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) w[b * R + r] = buf[pidx<SH>(j + r * (M / R))];
      }
    }
    if constexpr (!LAST) __syncthreads();  // every read of this pass done before its writes
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tl + b * TPL;
    const int k = j & (Ns - 1);
    if constexpr (Ns > 1) {
      if constexpr (sizeof(decltype(w[0].x)) == 4) {
        // FP32: one table load, the other powers by binary splitting
        // (w^r = w^{r/2} w^{r - r/2}, at most four products deep)
        C wp[R];
        wp[1] = tw[k * TWS];
        if (INV) wp[1].y = -wp[1].y;
#pragma unroll
        for (int r = 2; r < R; ++r) wp[r] = cmul(wp[r >> 1], wp[r - (r >> 1)]);
#pragma unroll
        for (int r = 1; r < R; ++r) w[b * R + r] = cmul(w[b * R + r], wp[r]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C t = tw[r * k * TWS];
          if (INV) t.y = -t.y;
          w[b * R + r] = cmul(w[b * R + r], t);
        }
      }
    }
    if constexpr (FIRST && ZIN)
      dft_zin<R, INV>(w + b * R);
    else
      dft<R, INV>(w + b * R);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < (ZOUT ? R / 2 : R); ++r) v[b + r * NB] = w[b * R + r];
    } else {
      const int base = ((j >> NSB) << (NSB + RB)) + k;
      if constexpr (Ns % Q == 0) {
        C* dst = buf + pidx<SH>(base);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * Ns + ((r * Ns) >> SH)] = w[b * R + r];
      } else if constexpr (Ns == 1 && Q % R == 0) {  // base = j R: base + r stays in one Q-block
        C* dst = buf + pidx<SH>(base);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r] = w[b * R + r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pidx<SH>(base + r * Ns)] = w[b * R + r];
      }
    }
  }
  if constexpr (!LAST) __syncthreads();  // writes visible to the next pass
}

template <typename C, int LOGM, bool INV, bool ZIN, bool ZOUT, int SH, int P = 0>
__device__ __forceinline__ void reg_passes(C (&v)[elems(LOGM)], C* buf, int tl, const C* __restrict__ tw) {
  if constexpr (P < npasses(LOGM)) {
    reg_pass<C, LOGM, P, INV, ZIN, ZOUT, SH>(v, buf, tl, tw);
    reg_passes<C, LOGM, INV, ZIN, ZOUT, SH, P + 1>(v, buf, tl, tw);
  }
}

// FFT of the line held in registers (see above); `buf` is the line's shared
// buffer, used only when there is more than one pass: line_stride(LOGM)
// entries with SH = 4, line_stride_tile(LOGM) with SH = tile_shift(LOGM).
template <typename C, int LOGM, bool INV, bool ZIN = false, bool ZOUT = false, int SH = 4>
__device__ __forceinline__ void fft_reg(C (&v)[elems(LOGM)], C* buf, int tl, const C* __restrict__ tw) {
  if constexpr (npasses(LOGM) > 1) __syncthreads();  // earlier users of buf are done
  reg_passes<C, LOGM, INV, ZIN, ZOUT, SH>(v, buf, tl, tw);
}

template <typename C, int LOGM, bool INV, int P = 0>
__device__ __forceinline__ void run(C* buf, int tl, const C* __restrict__ tw) {
  if constexpr (P < npasses(LOGM)) {
    pass<C, LOGM, P, INV>(buf, tl, tw);
    run<C, LOGM, INV, P + 1>(buf, tl, tw);
  }
}

}  // namespace fft
}  // namespace frac
