// The three passes of the d >= 2 FFT apply (Sec. 2.1: the Toeplitz product by
// circulant embedding and FFT), as device functions over one unit of work: a
// pair of rows (forward and inverse row passes) or a tile of B adjacent
// columns (column passes).  The grid kernels of apply.cu run one unit per
// thread group; the persistent batched solver (batch2d.cu) loops over units.
//
// Every function calls __syncthreads(): all threads of the block must call it
// together, with units out of range passed in as empty ones (they load zeros
// and store nothing).  The spectrum pointers are deliberately not __restrict__:
// in the persistent solver other threads of the same launch write a spectrum
// that these functions then read after a barrier, and a const __restrict__
// pointer would let the compiler read it through the non-coherent path or
// move those reads ahead of the barrier.  The grid kernels declare their own
// parameters __restrict__ where the data is written by an earlier launch.
//
// Intermediate spectra are stored column-blocked: entry (row, k) of a slab of
// `n` rows lives at (k / B) (n B) + row B + (k % B), B = 32 bytes / complex
// size (4 for FP32, 2 for FP64).  A tile of B adjacent columns is then one
// contiguous chunk, read and written with one lane per column and
// consecutive lanes on consecutive rows, and every row segment is a full
// 32-byte sector.  Every FFT keeps the line in registers at entry and exit
// (fft_reg): loads go straight from global memory into registers.
#pragma once

#include "fft.cuh"
#include "fft_mixed.cuh"

namespace frac {

template <typename T> __host__ __device__ constexpr int blk() { return 32 / (int)sizeof(cplx_t<T>); }

// column-blocked layout, slabs of n rows (n: the extent of the next axis),
// KB = ceil(K / B) blocks per slab: entry (row, k) at rowbase(row) + (k / B) n B + k % B
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

// ---------------------------------------------------------------------------
// Rows, forward: two real rows r0 = 2 pair, r1 = r0 + 1 (of nrows) -> one
// complex FFT -> two half spectra U0 = Z[k] + conj Z[M-k], U1 = -i (Z[k] -
// conj Z[M-k]), k in [0, M/2] (stored without the 1/2 of the separation; the
// symbol carries it).  in(row, x) gives the real input at x < n of a row < nrows
// (called once per such point).  ln: the line policy (fft_mixed.cuh: P2Line for
// M = 2^LOGM, MxLine for a 7-smooth M); buf: this group's line buffer
// (ln.stride() entries); tl: thread index within the group of ln.tpl().  The
// LOGM form is the power-of-two line.
// ---------------------------------------------------------------------------
// The same with the half spectra handed to a sink(k, U0, U1, h0, h1) (the entries k in
// [0, M/2] of rows r0 and r1; h0, h1: whether r0, r1 are rows below nrows, whose entry
// the sink stores) instead of stored into W.  make_sink() gives the sink once the
// transform is done (so that its addressing is not live across the FFT).
template <typename T, typename LN, bool ODD = false, typename In, typename MakeSink>
__device__ __forceinline__ void row_fwd_pair_s(const LN& ln, In in, MakeSink make_sink, int n, int64_t nrows,
                                               const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                               int tl) {
  using C = cplx_t<T>;
  using namespace fft;
  constexpr int E = LN::E;
  const int M = ln.m(), TPL = ln.tpl();
  const int64_t r0 = 2 * pair, r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
  C v[E];
  if constexpr (!ODD) {
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {  // x < n <= M/2: e < E/2
      const int x = tl + e * TPL;
      const T re = (x < n && h0) ? in(r0, x) : T(0);
      const T im = (x < n && h1) ? in(r1, x) : T(0);
      v[e] = C{re, im};
    }
    ln.template fft<false, true, false>(v, buf, tl, tw);  // upper half is zero padding
  } else {
    // odd extension (n <= M/2 - 1): entry j at x = j + 1, -entry j at x = M - 1 - j,
    // zero at x = 0, M/2 and between; in() is called twice per point here
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      T re = T(0), im = T(0);
      if (x >= 1 && x <= n) {
        if (h0) re = in(r0, x - 1);
        if (h1) im = in(r1, x - 1);
      } else if (x >= M - n) {
        if (h0) re = -in(r0, M - 1 - x);
        if (h1) im = -in(r1, M - 1 - x);
      }
      v[e] = C{re, im};
    }
    ln.template fft<false, false, false>(v, buf, tl, tw);
  }
  // separation needs Z[k] and Z[M-k] for k in [0, M/2]: each thread keeps its
  // lower-half Z[k] in registers and reads the mirror from the upper half,
  // which alone goes through the line buffer
  __syncthreads();
#pragma unroll
  for (int e = E / 2; e < E; ++e) buf[ln.pad(tl + e * TPL)] = v[e];
  __syncthreads();
  auto sink = make_sink();
  auto emit = [&](int k, C z, C zc) {
    const C s = cadd(z, zc), dd = csub(z, zc);
    sink(k, s, C{dd.y, -dd.x}, h0, h1);
  };
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int k = tl + e * TPL;  // k < M/2; M - k is in the upper half unless k = 0
    emit(k, v[e], cconj(k == 0 ? v[e] : buf[ln.pad(M - k)]));
  }
  if (tl == 0) emit(M / 2, v[E / 2], cconj(v[E / 2]));
}

template <typename T, typename LN, bool ODD = false, typename In>
__device__ __forceinline__ void row_fwd_pair_l(const LN& ln, In in, cplx_t<T>* W, int n, int64_t nrows, int KB,
                                               const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                               int tl, int ns = 0) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const int64_t r0 = 2 * pair, r1 = r0 + 1;
  if (ns <= 0) ns = n;  // rows per slab of W (the next axis' extent; n on square grids)
  row_fwd_pair_s<T, LN, ODD>(
      ln, in,
      [&]() {
        C* W0 = W + wrow<B>(r0 < nrows ? r0 : 0, ns, KB);
        C* W1 = W + wrow<B>(r1 < nrows ? r1 : 0, ns, KB);
        return [=](int k, C z0, C z1, bool h0, bool h1) {
          const int64_t kc = wcol<B>(k, ns);
          if (h0) W0[kc] = z0;
          if (h1) W1[kc] = z1;
        };
      },
      n, nrows, tw, pair, buf, tl);
}
template <typename T, int LOGM, bool ODD = false, typename In>
__device__ __forceinline__ void row_fwd_pair(In in, cplx_t<T>* W, int n, int64_t nrows, int KB,
                                             const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                             int tl, int ns = 0) {
  row_fwd_pair_l<T, fft::P2Line<LOGM>, ODD>(fft::P2Line<LOGM>{}, in, W, n, nrows, KB, tw, pair, buf, tl, ns);
}

// ---------------------------------------------------------------------------
// Rows, inverse: two half spectra -> one complex line (Hermitian extension)
// -> iFFT -> two real rows; out(row, x, value) receives the first n entries
// of each row < nrows (ODD: entries 1..n, as x = 0..n-1).
// ---------------------------------------------------------------------------
// The same with the half spectra read through src(x, v0, v1, h0, h1) (sets v0, v1 to the
// entries x in [0, M/2] of rows r0, r1, zero for a row not below nrows: h0, h1 false)
// instead of from W.
template <typename T, typename LN, bool ODD = false, typename Src, typename Out>
__device__ __forceinline__ void row_inv_pair_s(const LN& ln, Src src, int n, int64_t nrows,
                                               const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                               int tl, Out out) {
  using C = cplx_t<T>;
  using namespace fft;
  constexpr int E = LN::E;
  const int M = ln.m(), TPL = ln.tpl();
  const int64_t r0 = 2 * pair, r1 = r0 + 1;
  const bool h0 = r0 < nrows, h1 = r1 < nrows;
  C v[E];
  // line z = W0 + i W1 extended Hermitian-wise: z[x] = W0[x] + i W1[x] and
  // z[M-x] = conj(W0[x]) + i conj(W1[x]) for x in [0, M/2], so each half
  // spectrum entry is read once; the thread that reads W[x] leaves z[M-x] in
  // the line buffer for its owner
  auto load = [&](int x, C& lo, C& hi) {
    C v0, v1;
    src(x, v0, v1, h0, h1);
    lo = C{v0.x - v1.y, v0.y + v1.x};  // v0 + i v1
    hi = C{v0.x + v1.y, v1.x - v0.y};  // conj(v0) + i conj(v1)
  };
  __syncthreads();  // earlier users of buf are done
#pragma unroll
  for (int e = 0; e < E / 2; ++e) {
    const int x = tl + e * TPL;  // x < M/2
    C hi;
    load(x, v[e], hi);
    if (x > 0) buf[ln.pad(M - x)] = hi;
  }
  if (tl == 0) {
    C lo, hi;
    load(M / 2, lo, hi);
    buf[ln.pad(M / 2)] = lo;
  }
  __syncthreads();
#pragma unroll
  for (int e = E / 2; e < E; ++e) v[e] = buf[ln.pad(tl + e * TPL)];
  if constexpr (!ODD) {
    ln.template fft<true, false, true>(v, buf, tl, tw);  // only x < n <= M/2 is kept
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
      const int x = tl + e * TPL;
      if (x < n) {
        if (h0) out(r0, x, v[e].x);
        if (h1) out(r1, x, v[e].y);
      }
    }
  } else {
    ln.template fft<true, false, false>(v, buf, tl, tw);  // odd extension: entries 1..n are kept
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = tl + e * TPL;
      if (x >= 1 && x <= n) {
        if (h0) out(r0, x - 1, v[e].x);
        if (h1) out(r1, x - 1, v[e].y);
      }
    }
  }
}
template <typename T, typename LN, bool ODD = false, typename Out>
__device__ __forceinline__ void row_inv_pair_l(const LN& ln, const cplx_t<T>* W, int n, int64_t nrows, int KB,
                                               const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                               int tl, Out out, int ns = 0) {
  using C = cplx_t<T>;
  constexpr int B = blk<T>();
  const int64_t r0 = 2 * pair, r1 = r0 + 1;
  if (ns <= 0) ns = n;  // rows per slab of W
  const C* W0 = W + wrow<B>(r0 < nrows ? r0 : 0, ns, KB);
  const C* W1 = W + wrow<B>(r1 < nrows ? r1 : 0, ns, KB);
  row_inv_pair_s<T, LN, ODD>(
      ln,
      [&](int x, C& v0, C& v1, bool h0, bool h1) {
        const int64_t kc = wcol<B>(x, ns);
        v0 = h0 ? W0[kc] : C{0, 0};
        v1 = h1 ? W1[kc] : C{0, 0};
      },
      n, nrows, tw, pair, buf, tl, out);
}
template <typename T, int LOGM, bool ODD = false, typename Out>
__device__ __forceinline__ void row_inv_pair(const cplx_t<T>* W, int n, int64_t nrows, int KB,
                                             const cplx_t<T>* __restrict__ tw, int64_t pair, cplx_t<T>* buf,
                                             int tl, Out out, int ns = 0) {
  row_inv_pair_l<T, fft::P2Line<LOGM>, ODD>(fft::P2Line<LOGM>{}, W, n, nrows, KB, tw, pair, buf, tl, out, ns);
}

// ---------------------------------------------------------------------------
// Columns: one tile of B adjacent columns, TPL threads per column (lane order:
// column fastest, cl = column in the tile, tl = thread in the column).  Modes:
//   SYM2 (d = 2): slab o = field, pad n -> M, FFT, * Lambda[kr][k1], iFFT, keep n; in place.
//   YFWD (d = 3): slab o = (b, j3) of W1, pad n -> M, FFT along j2, all M k2 to W2,
//                 W2 column c = k2 Kp + k1 (Kp = KB B), column-blocked with n rows (j3).
//   ZSYM (d = 3): W2 column tile of field o, pad n -> M along j3, FFT, * Lambda[k3r][k2r][k1],
//                 iFFT, keep n; in place.
//   YINV (d = 3): slab o = (b, j3): M entries k2 of W2 columns k1, iFFT, first n (j2) to W1.
// A tile whose column k1 >= K is empty.  sm: the tile's B line buffers of
// ln.stride_tile() entries each (line_stride_tile(LOGM) for M = 2^LOGM).  ODD: the odd extension of the n
// entries (the sine-transform embedding of the tau preconditioner) instead of
// zero padding, and entries 1..n kept.
// ---------------------------------------------------------------------------

enum ColMode { SYM2 = 0, YFWD = 1, ZSYM = 2, YINV = 3 };

struct ColArgs {
  int n, K, KB;      // interior points along this pass's axis, k1 extent K_1 = M_1/2+1, column blocks per slab
  int64_t tiles;     // column tiles per slab
  int64_t nb;        // batch (fields)
  int nz = 0;        // d = 3: z extent n_3 (slabs (b, j3) of W1; rows j3 of a W2 column block)
  int My = 0, Ky = 0;  // d = 3: y FFT length M_2 and its symbol extent K_2 = M_2/2+1;
                       // SYM2: Ky = K_2, the symbol's rows (the symbol is stored in column tiles)
};

// src_tile (YFWD) / dst_tile (YINV): when given, the tile's n rows of B lanes are read
// from / written to there (row j at j B) instead of the W1 slab in global memory (the
// fused xy passes keep that slab in distributed shared memory).
template <typename T, typename LN, int MODE, bool ODD = false>
__device__ __forceinline__ void col_tile_l(const LN& ln, const cplx_t<T>* in, cplx_t<T>* out, const ColArgs& A,
                                           const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, int64_t o,
                                           int64_t tile, cplx_t<T>* sm, int cl, int tl,
                                           const cplx_t<T>* src_tile = nullptr, cplx_t<T>* dst_tile = nullptr) {
  using C = cplx_t<T>;
  using namespace fft;
  constexpr int E = LN::E, B = blk<T>();
  const int M = ln.m(), TPL = ln.tpl(), LS = ln.stride_tile();
  C* buf = sm + cl * LS;
  const int n = A.n, K = A.K, KB = A.KB, Kp = KB * B;
  const int64_t nB = (int64_t)n * B;              // W1 slab rows (SYM2, YFWD, YINV: j2) / W2 rows (ZSYM: j3)
  const int64_t zB = (int64_t)A.nz * B;           // W2 rows per column block (j3)
  const int64_t W2slab = (int64_t)A.My * KB * zB;  // one field of W2
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
    k2r = k2 <= A.My / 2 ? k2 : A.My - k2;
    live = k1 < K;
  }
  if (MODE == YINV) {
    const int64_t b = o / A.nz, j3 = o % A.nz;
    const C* src = in + b * W2slab + tile * zB + j3 * B + cl;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k2 = tl + e * TPL;
      v[e] = live ? src[(int64_t)k2 * KB * zB] : C{0, 0};
    }
  } else if constexpr (!ODD) {
    const C* src = (MODE == ZSYM) ? in + o * W2slab + tile * nB + cl
                 : src_tile       ? src_tile + cl
                                  : in + (o * KB + tile) * nB + cl;
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {  // j < n <= M/2; the rest is zero padding
      const int j = tl + e * TPL;
      v[e] = (live && j < n) ? src[(int64_t)j * B] : C{0, 0};
    }
  } else {  // odd extension: row j at j + 1, its negative at M - 1 - j
    const C* src = (MODE == ZSYM) ? in + o * W2slab + tile * nB + cl
                 : src_tile       ? src_tile + cl
                                  : in + (o * KB + tile) * nB + cl;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      C w = C{0, 0};
      if (live && j >= 1 && j <= n) {
        w = src[(int64_t)(j - 1) * B];
      } else if (live && j >= M - n) {
        w = src[(int64_t)(M - 1 - j) * B];
        w = C{-w.x, -w.y};
      }
      v[e] = w;
    }
  }
  // ---- transforms
  if (MODE != YINV) ln.template fft<false, !ODD, false>(v, buf, tl, tw);
  if (MODE == SYM2 || MODE == ZSYM) {
    // the symbol in column tiles, so that the B lanes of a row read one contiguous run:
    // SYM2 entry (kr, k1) at (k1 / B) K_2 B + kr B + k1 % B; ZSYM entry (k3r, k2r, k1) at
    // ((k2r KB + k1 / B) K_3 + k3r) B + k1 % B with K_3 = M / 2 + 1 (this pass's axis)
    const T* lrow = (MODE == SYM2) ? lam + (int64_t)tile * A.Ky * B + cl
                                   : lam + ((int64_t)k2r * KB + k1 / B) * (M / 2 + 1) * B + (k1 % B);
    const int64_t kstride = B;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = tl + e * TPL;
      const int kr = k <= M / 2 ? k : M - k;
      v[e] = cscale(v[e], live ? lrow[kr * kstride] : T(0));
    }
  }
  if (MODE != YFWD) ln.template fft<true, false, !ODD>(v, buf, tl, tw);  // keeps j < n (ODD: 1..n) only
  // ---- store
  if (!live) return;
  if (MODE == YFWD) {
    const int64_t b = o / A.nz, j3 = o % A.nz;
    C* dst = out + b * W2slab + tile * zB + j3 * B + cl;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k2 = tl + e * TPL;
      dst[(int64_t)k2 * KB * zB] = v[e];
    }
  } else {
    C* dst = (MODE == ZSYM) ? out + o * W2slab + tile * nB + cl
             : dst_tile       ? dst_tile + cl
                              : out + (o * KB + tile) * nB + cl;  // SYM2 in place; YINV to W1 slab o
    if constexpr (!ODD) {
#pragma unroll
      for (int e = 0; e < E / 2; ++e) {
        const int j = tl + e * TPL;
        if (j < n) dst[(int64_t)j * B] = v[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = tl + e * TPL;
        if (j >= 1 && j <= n) dst[(int64_t)(j - 1) * B] = v[e];
      }
    }
  }
}
// Column passes of the tau preconditioner (all on the odd extension), two columns per
// transform.  The odd-extension spectra are purely imaginary or purely real: after the
// row pass every entry of W (W1 in 3D) is i s(j, k1) with s real; the 3D y pass maps
// such columns to purely real ones r(k2, c) of W2, the z pass keeps W2 real, and the
// inverse y pass maps them back to imaginary ones.  So the full-width passes spend a
// complex transform on one real column.  Here line q carries columns c = 2q and c + 1
// (one tile, B even) as z = s(., c) + i s(., c + 1): with the odd extension the
// transform of each real part is purely imaginary (an odd-symmetric real spectrum
// transforms back to a purely imaginary one), so the two columns separate again into
// the real and imaginary parts:
//   SYM2, ZSYM: z(j) -> forward -> imaginary part column c, real part c + 1, each scaled
//               by its own symbol entry -> inverse -> s'(j, c) + i s'(j, c + 1), stored
//               back as i s' (SYM2) or s' (ZSYM);
//   YFWD:       z(j2) from the imaginary parts of W1 -> forward -> the full-width pass's
//               real outputs -Im (column c) and Re (c + 1), to W2 at every k2;
//   YINV:       z(k2) from the real parts of W2 -> inverse -> i s''(c) - s''(c + 1), so
//               Im to column c and -Re to c + 1 of W1 (as i s'').
// The results equal the full-width passes' up to rounding (which leaves a rounding-size
// second part there); a column past the half spectrum (k1 >= K) is empty.  sm: the
// block's B line buffers (ln.stride_tile() entries each); cl: this lane's line in the
// block; o: the slab (the field; (b, j3) for YFWD and YINV).
template <typename T, bool IM>
__device__ __forceinline__ cplx_t<T> part_pair(const cplx_t<T>* p) {
  // the imaginary (IM) or real parts of p[0] and p[1], one vector load for FP32
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    return IM ? cplx_t<T>{q.y, q.w} : cplx_t<T>{q.x, q.z};
  } else {
    return IM ? cplx_t<T>{p[0].y, p[1].y} : cplx_t<T>{p[0].x, p[1].x};
  }
}

// p[0] = a and, when both, p[1] = b (one vector store for FP32; p 2-entry aligned).
template <typename T>
__device__ __forceinline__ void store_pair(cplx_t<T>* p, cplx_t<T> a, cplx_t<T> b, bool both) {
  if constexpr (sizeof(T) == 4) {
    if (both)
      *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
    else
      p[0] = a;
  } else {
    p[0] = a;
    if (both) p[1] = b;
  }
}

template <typename T, typename LN, int MODE>
__device__ __forceinline__ void col_pair_tau_l(const LN& ln, const cplx_t<T>* in, cplx_t<T>* out, const ColArgs& A,
                                               const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, int64_t o,
                                               int64_t q, cplx_t<T>* sm, int cl, int tl) {
  using C = cplx_t<T>;
  constexpr int E = LN::E, B = blk<T>();
  constexpr bool IN_IM = MODE == SYM2 || MODE == YFWD;  // the input columns' nonzero part
  static_assert(B % 2 == 0, "a column pair lies in one tile");
  const int M = ln.m(), TPL = ln.tpl(), LS = ln.stride_tile();
  C* buf = sm + cl * LS;
  const int n = A.n, K = A.K, KB = A.KB;
  const int64_t nB = (int64_t)n * B, zB = (int64_t)A.nz * B, W2slab = (int64_t)A.My * KB * zB;
  const int64_t c = 2 * q, tile = c / B;
  const int lt = (int)(c % B);
  // k1 of the first column; W1 slab rows (SYM2, YFWD in, YINV out: j2) or W2 column
  // (ZSYM: j3 rows; YFWD out, YINV in: k2 rows); the symbol's (k1, kr = 0) entry
  int64_t k1 = c, w1 = (o * KB + tile) * nB, w2 = 0, sbase = 0;
  if constexpr (MODE == SYM2) {
    sbase = tile * A.Ky * B + lt;  // entry (kr, k1) at (k1 / B) K_2 B + kr B + k1 % B
  } else if constexpr (MODE == ZSYM) {  // W2 column c = k2 Kp + k1 (Kp = KB B) of field o
    const int64_t Kp = (int64_t)KB * B, k2 = c / Kp;
    k1 = c % Kp;
    const int64_t k2r = k2 <= A.My / 2 ? k2 : A.My - k2;
    w2 = o * W2slab + tile * nB;
    // entry (k3r, k2r, k1) at ((k2r KB + k1 / B) K_3 + k3r) B + k1 % B, K_3 = M / 2 + 1
    sbase = (k2r * KB + k1 / B) * (M / 2 + 1) * B + k1 % B;
  } else {  // YFWD, YINV: slab o = (b, j3); W2 entry k2 of the tile's columns at k2 KB zB
    w2 = (o / A.nz) * W2slab + tile * zB + (o % A.nz) * B;
  }
  const bool la = k1 < K, lb = k1 + 1 < K;
  C v[E];
  if constexpr (MODE == YINV) {
    const C* src = in + (la ? w2 : 0) + lt;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k2 = tl + e * TPL;
      const C pr = la ? part_pair<T, false>(src + (int64_t)k2 * KB * zB) : C{0, 0};
      v[e] = C{pr.x, lb ? pr.y : T(0)};
    }
  } else {
    const C* src = in + (la ? (MODE == ZSYM ? w2 : w1) : 0) + lt;
#pragma unroll
    for (int e = 0; e < E; ++e) {  // odd extension: row j at j + 1, its negative at M - 1 - j
      const int j = tl + e * TPL;
      const bool pos = j >= 1 && j <= n, neg = !pos && j >= M - n;
      C w = C{0, 0};
      if (la && (pos || neg)) {
        const C pr = part_pair<T, IN_IM>(src + (int64_t)(pos ? j - 1 : M - 1 - j) * B);
        const T sg = pos ? T(1) : T(-1);
        w = C{sg * pr.x, lb ? sg * pr.y : T(0)};
      }
      v[e] = w;
    }
  }
  if constexpr (MODE != YINV) ln.template fft<false, false, false>(v, buf, tl, tw);
  if constexpr (MODE == SYM2 || MODE == ZSYM) {
    const T* lrow = lam + (la ? sbase : 0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = tl + e * TPL;
      const int kr = k <= M / 2 ? k : M - k;
      // both entries in one aligned load (k1 even; the tiles are padded to B columns, so
      // entry k1 + 1 exists even past K, and an empty column's factor is zero)
      const C s2 = la ? *reinterpret_cast<const C*>(lrow + (int64_t)kr * B) : C{0, 0};
      v[e] = C{v[e].x * (lb ? s2.y : T(0)), v[e].y * s2.x};
    }
  }
  if constexpr (MODE != YFWD) ln.template fft<true, false, false>(v, buf, tl, tw);
  if (!la) return;
  if constexpr (MODE == YFWD) {
    C* dst = out + w2 + lt;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t k2 = tl + e * TPL;
      store_pair<T>(dst + k2 * KB * zB, C{-v[e].y, T(0)}, C{v[e].x, T(0)}, lb);
    }
  } else {
    C* dst = out + (MODE == ZSYM ? w2 : w1) + lt;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tl + e * TPL;
      if (j >= 1 && j <= n) {
        C a, b;
        if constexpr (MODE == SYM2) {
          a = C{T(0), v[e].x};
          b = C{T(0), v[e].y};
        } else if constexpr (MODE == ZSYM) {
          a = C{v[e].x, T(0)};
          b = C{v[e].y, T(0)};
        } else {  // YINV
          a = C{T(0), v[e].y};
          b = C{T(0), -v[e].x};
        }
        store_pair<T>(dst + (int64_t)(j - 1) * B, a, b, lb);
      }
    }
  }
}

template <typename T, int LOGM, int MODE, bool ODD = false>
__device__ __forceinline__ void col_tile(const cplx_t<T>* in, cplx_t<T>* out, const ColArgs& A,
                                         const T* __restrict__ lam, const cplx_t<T>* __restrict__ tw, int64_t o,
                                         int64_t tile, cplx_t<T>* sm, int cl, int tl) {
  using LN = fft::P2Line<LOGM, fft::tile_shift(LOGM)>;
  col_tile_l<T, LN, MODE, ODD>(LN{}, in, out, A, lam, tw, o, tile, sm, cl, tl);
}

}  // namespace frac
