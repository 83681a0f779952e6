// Coefficient generation on the device, FP64:
//   weight integrals omega_k^p (Eq. (wi-1D), Eq. (2D-scheme0) and its 3D analogue;
//   tempered kernel of Remark 2.2), stencil a_k with the origin rule, centre
//   coefficient a_0, far field F_d (host), and the symbol of the circulant
//   embedding (separable cosine sums, each axis by an FP64 FFT).
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fft_mixed.cuh"

namespace frac {

// ---------------------------------------------------------------------------
// Gauss-Legendre rules on [-1, 1] (Newton iteration on P_q, host, FP64)
// ---------------------------------------------------------------------------

constexpr int kNumRules = 9;
constexpr int kRuleTotal = 84;
// rule r: q points, stored from offset rule_off(r)
__host__ __device__ constexpr int rule_q(int r) {
  return r == 0 ? 4 : r == 1 ? 5 : r == 2 ? 6 : r == 3 ? 8 : r == 4 ? 10 : r == 5 ? 12 : r == 6 ? 16 : r == 7 ? 20 : 3;
}
// (no recursion: a recursive device function called with a runtime argument
// would need stack beyond the kernel's static frame)
__host__ __device__ constexpr int rule_off(int r) {
  return r == 0 ? 0 : r == 1 ? 4 : r == 2 ? 9 : r == 3 ? 15 : r == 4 ? 23 : r == 5 ? 33 : r == 6 ? 45 : r == 7 ? 61 : 81;
}
__host__ __device__ constexpr bool rule_table_ok(int r) {
  return r == kNumRules ? true : (rule_off(r) + rule_q(r) == (r + 1 == kNumRules ? kRuleTotal : rule_off(r + 1)) &&
                                  rule_table_ok(r + 1));
}
static_assert(rule_table_ok(0), "rule offsets");

__constant__ double c_gl_x[kRuleTotal];
__constant__ double c_gl_w[kRuleTotal];
__constant__ double c_gl32_x[32];  // angular rule of the far field
__constant__ double c_gl32_w[32];
constexpr int kSeriesMax = 40;
__constant__ double c_inv[kSeriesMax + 1];    // 1 / j (entry 0 unused)
__constant__ double c_bhalf[kSeriesMax + 1];  // binom(1/2, j)

// Self-checking accesses: an index outside [0, n) is recorded (first source
// line and index) and the access is skipped; the host reads the record after
// the coefficient build and reports it as FRAC_ECUDA with the line.
__device__ unsigned long long g_fault_line = 0;
__device__ long long g_fault_index = 0;
__device__ __noinline__ void note_fault(int line, long long idx) {
  if (atomicCAS(&g_fault_line, 0ull, (unsigned long long)line) == 0ull) g_fault_index = idx;
}
#define CHK(i, n) \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) ? true : (note_fault(__LINE__, (long long)(i)), false))

static void legendre_rule(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation for the derivative at the converged node
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= q; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static int upload_rules() {
  static std::mutex mu;
  static std::vector<int> done;  // devices already initialised
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  for (int d : done)
    if (d == dev) return FRAC_OK;
  double hx[kRuleTotal], hw[kRuleTotal];
  for (int r = 0; r < kNumRules; ++r) legendre_rule(rule_q(r), hx + rule_off(r), hw + rule_off(r));
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_gl_x, hx, sizeof(hx)));
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_gl_w, hw, sizeof(hw)));
  double x32[32], w32[32];
  legendre_rule(32, x32, w32);
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_gl32_x, x32, sizeof(x32)));
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_gl32_w, w32, sizeof(w32)));
  double inv[kSeriesMax + 1], bh[kSeriesMax + 1];
  inv[0] = 0.0;
  bh[0] = 1.0;
  for (int j = 1; j <= kSeriesMax; ++j) {
    inv[j] = 1.0 / j;
    bh[j] = bh[j - 1] * (1.5 - j) / j;
  }
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_inv, inv, sizeof(inv)));
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(c_bhalf, bh, sizeof(bh)));
  done.push_back(dev);
  return FRAC_OK;
}

// ---------------------------------------------------------------------------
// Twiddle tables exp(-2 pi i t / M) (host FP64 with octant symmetry)
// ---------------------------------------------------------------------------

static void host_twiddles(int64_t M, std::vector<double2>& out) {
  out.resize(M);
  for (int64_t t = 0; t < M; ++t) {
    // angle 2 pi t / M reduced to [0, pi/4] by symmetry
    int64_t t8 = t * 8;  // octant = t8 / M
    int64_t oct = t8 / M;
    int64_t r = t8 - oct * M;  // remainder, angle within octant = (r / M) * pi/4
    double th, c, s;
    if (oct & 1) {
      th = (double)(M - r) / (double)M * (M_PI / 4.0);
    } else {
      th = (double)r / (double)M * (M_PI / 4.0);
    }
    double ct = std::cos(th), st = std::sin(th);
    // base angle: oct * pi/4 + (oct odd ? pi/4 - th : th)
    switch (oct & 7) {
      case 0: c = ct; s = st; break;
      case 1: c = st; s = ct; break;
      case 2: c = -st; s = ct; break;
      case 3: c = -ct; s = st; break;
      case 4: c = -ct; s = -st; break;
      case 5: c = -st; s = -ct; break;
      case 6: c = st; s = -ct; break;
      default: c = ct; s = -st; break;
    }
    out[t] = double2{c, -s};  // exp(-i angle)
  }
}

struct TwTables {
  std::mutex mu;
  // per device, per logm
  std::vector<std::vector<double2*>> t64;
  std::vector<std::vector<float2*>> t32;
};
static TwTables g_tw;

static int ensure_twiddles(int logm) {
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw.mu);
  if ((int)g_tw.t64.size() <= dev) {
    g_tw.t64.resize(dev + 1);
    g_tw.t32.resize(dev + 1);
  }
  auto& a64 = g_tw.t64[dev];
  auto& a32 = g_tw.t32[dev];
  if ((int)a64.size() <= logm) {
    a64.resize(logm + 1, nullptr);
    a32.resize(logm + 1, nullptr);
  }
  if (a64[logm]) return FRAC_OK;
  int64_t M = int64_t(1) << logm;
  std::vector<double2> h;
  host_twiddles(M, h);
  std::vector<float2> hf(M);
  for (int64_t t = 0; t < M; ++t) hf[t] = float2{(float)h[t].x, (float)h[t].y};
  double2* d64 = nullptr;
  float2* d32 = nullptr;
  FRAC_CUDA_TRY(cudaMalloc(&d64, M * sizeof(double2)));
  FRAC_CUDA_TRY(cudaMalloc(&d32, M * sizeof(float2)));
  FRAC_CUDA_TRY(cudaMemcpy(d64, h.data(), M * sizeof(double2), cudaMemcpyHostToDevice));
  FRAC_CUDA_TRY(cudaMemcpy(d32, hf.data(), M * sizeof(float2), cudaMemcpyHostToDevice));
  a64[logm] = d64;
  a32[logm] = d32;
  return FRAC_OK;
}

int prepare_twiddles(int logm) { return ensure_twiddles(logm); }

// Tables of the mixed lengths, keyed by (device, M).
struct TwLenTables {
  std::mutex mu;
  std::map<std::pair<int, int64_t>, std::pair<double2*, float2*>> t;
};
static TwLenTables g_twl;

int prepare_twiddles_len(int64_t M) {
  if (M >= 2 && (M & (M - 1)) == 0) return ensure_twiddles(ilog2(M));
  int dev = 0;
  FRAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_twl.mu);
  if (g_twl.t.count({dev, M})) return FRAC_OK;
  std::vector<double2> h;
  host_twiddles(M, h);
  std::vector<float2> hf(M);
  for (int64_t t = 0; t < M; ++t) hf[t] = float2{(float)h[t].x, (float)h[t].y};
  double2* d64 = nullptr;
  float2* d32 = nullptr;
  FRAC_CUDA_TRY(cudaMalloc(&d64, M * sizeof(double2)));
  FRAC_CUDA_TRY(cudaMalloc(&d32, M * sizeof(float2)));
  FRAC_CUDA_TRY(cudaMemcpy(d64, h.data(), M * sizeof(double2), cudaMemcpyHostToDevice));
  FRAC_CUDA_TRY(cudaMemcpy(d32, hf.data(), M * sizeof(float2), cudaMemcpyHostToDevice));
  g_twl.t[{dev, M}] = {d64, d32};
  return FRAC_OK;
}

const double2* twiddles64_len(int64_t M) {
  if (M >= 2 && (M & (M - 1)) == 0) return twiddles64(ilog2(M));
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_twl.mu);
  auto it = g_twl.t.find({dev, M});
  return it == g_twl.t.end() ? nullptr : it->second.first;
}
const float2* twiddles32_len(int64_t M) {
  if (M >= 2 && (M & (M - 1)) == 0) return twiddles32(ilog2(M));
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_twl.mu);
  auto it = g_twl.t.find({dev, M});
  return it == g_twl.t.end() ? nullptr : it->second.second;
}

const double2* twiddles64(int logm) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tw.mu);
  return g_tw.t64[dev][logm];
}
const float2* twiddles32(int logm) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tw.mu);
  return g_tw.t32[dev][logm];
}

// ---------------------------------------------------------------------------
// Far field F_d = int over R_+^d \ [0, L]^d of |xi|^{-d-alpha} e^{-lambda |xi|}
// (the u(x) part of Eq. (L2); 1D: 1/(alpha L^alpha) when lambda = 0).
// Largest-coordinate split: xi = rho (1, s), rho > L, s in [0,1]^{d-1}:
// F_d = d int_s c(s)^{-d-alpha} int_L^inf rho^{-1-alpha} e^{-lambda c rho} d rho ds,
// s by a 32-point Gauss-Legendre rule per coordinate.  The rho-integral with
// rho = L / t is L^{-alpha} int_0^1 t^{alpha-1} e^{-lambda c L / t} dt, integrated
// by a 20-point Gauss-Legendre rule on the graded panels [2^{-j-1}, 2^{-j}]
// until e^{-lambda c L / t} underflows (closed form L^{-alpha} / alpha when
// lambda c L is negligible).  k_far_terms writes one term per (angle, panel);
// k_centre sums them.
// ---------------------------------------------------------------------------

constexpr int kFarPanels = 80;

__device__ __forceinline__ int far_angles(int d) { return d == 1 ? 1 : (d == 2 ? 32 : 32 * 32); }

__global__ void k_far_terms(int d, double alpha, double lambda, double L, double* __restrict__ terms, int64_t count) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int a = (int)(idx / kFarPanels), j = (int)(idx % kFarPanels);
  double c = 1.0, wa = 1.0;
  if (d >= 2) {
    const int i0 = a % 32, i1 = a / 32;
    const double s0 = 0.5 * (c_gl32_x[i0] + 1.0);
    const double s1 = d == 3 && i1 < 32 ? 0.5 * (c_gl32_x[i1] + 1.0) : 0.0;
    c = sqrt(1.0 + s0 * s0 + s1 * s1);
    wa = d * 0.5 * c_gl32_w[i0] * (d == 3 && i1 < 32 ? 0.5 * c_gl32_w[i1] : 1.0) * pow(c, -(double)d - alpha);
  }
  const double x = lambda * c * L;
  double v = 0.0;
  if (x < 1e-14) {
    if (j == 0) v = pow(L, -alpha) / alpha;
  } else if (j == 0 || ldexp(x, j - 1) <= 800.0) {  // panel j follows one that did not underflow
    const double hi = ldexp(1.0, -j), lo = ldexp(1.0, -j - 1);
    const int off = rule_off(7), q = rule_q(7);
    double part = 0.0;
    for (int g = 0; g < q && CHK(off + g, kRuleTotal); ++g) {
      const double t = 0.5 * (hi + lo) + 0.5 * (hi - lo) * c_gl_x[off + g];
      part += c_gl_w[off + g] * pow(t, alpha - 1.0) * exp(-x / t);
    }
    v = pow(L, -alpha) * part * 0.5 * (hi - lo);
  }
  terms[idx] = wa * v;
}

// ---------------------------------------------------------------------------
// Weight integrals omega_k = int phi_k(xi) mu(xi) dxi (Eq. (wi-1D), Eq. (2D-scheme0)): per
// element a Gauss-Legendre rule of q points per axis, q chosen by the
// element's distance to the origin; the origin element by exact radial
// moments (1D) or a Duffy split (d >= 2).
// ---------------------------------------------------------------------------

struct WParams {
  int d, p;
  int64_t N;
  double h, alpha, lambda, beta;  // beta = d + alpha - gamma: mu_gamma = |xi|^{-beta} e^{-lambda |xi|}
  double gamma;                   // splitting parameter in (alpha, 2] (Eq. (eq0))
};

struct AxisEl {
  double lo, hi;     // element interval
  double r0, r1;     // roots of the local basis function (product form; p <= 2)
  double scale;
  int nroots;
  int origin_l;      // local index on the origin element, or -1 if lo > 0
  double r2, r3;     // further roots (p = 3, 4; d = 1 only)
};

// Elements of the support of the 1D basis function of node k (at most 2).
__device__ int axis_elements(const WParams& P, int64_t k, AxisEl* el) {
  const double h = P.h;
  const int64_t N = P.N;
  const double L = N * h;
  int ne = 0;
  if (P.p == 0) {
    if (!CHK(0, 2)) return 0;
    el[0] = AxisEl{fmax(0.0, (k - 0.5) * h), fmin(L, (k + 0.5) * h), 0, 0, 1.0, 0, k == 0 ? 0 : -1};
    ne = 1;
  } else if (P.p == 1) {
    if (k >= 1 && CHK(ne, 2)) el[ne++] = AxisEl{(k - 1) * h, k * h, (k - 1) * h, 0, 1.0 / h, 1, k == 1 ? 1 : -1};
    if (k < N && CHK(ne, 2)) el[ne++] = AxisEl{k * h, (k + 1) * h, (k + 1) * h, 0, -1.0 / h, 1, k == 0 ? 0 : -1};
  } else if (P.p == 2) {
    if (k & 1) {
      if (CHK(ne, 2)) el[ne++] = AxisEl{(k - 1) * h, (k + 1) * h, (k - 1) * h, (k + 1) * h, -1.0 / (h * h), 2, k == 1 ? 1 : -1};
    } else {
      if (k >= 2 && CHK(ne, 2)) el[ne++] = AxisEl{(k - 2) * h, k * h, (k - 2) * h, (k - 1) * h, 0.5 / (h * h), 2, k == 2 ? 2 : -1};
      if (k <= N - 2 && CHK(ne, 2)) el[ne++] = AxisEl{k * h, (k + 2) * h, (k + 1) * h, (k + 2) * h, 0.5 / (h * h), 2, k == 0 ? 0 : -1};
    }
  } else {  // p = 3, 4 (d = 1): Lagrange polynomial of node k on the elements [p m h, (p m + p) h]
    const int p = P.p;
    const int64_t m_lo = (k % p == 0) ? k / p - 1 : k / p, m_hi = k / p;
    for (int64_t m = m_lo; m <= m_hi; ++m) {
      if (m < 0 || (m + 1) * p > N || !CHK(ne, 2)) continue;
      const int t = (int)(k - p * m);  // local index
      double roots[4] = {0, 0, 0, 0}, scale = 1.0;
      int nr = 0;
      for (int s2 = 0; s2 <= p; ++s2) {
        if (s2 == t) continue;
        if (CHK(nr, 4)) roots[nr++] = (p * m + s2) * h;
        scale /= (double)(t - s2) * h;
      }
      el[ne++] = AxisEl{p * m * h, (p * m + p) * h, roots[0], roots[1], scale, nr, m == 0 ? t : -1, roots[2], roots[3]};
    }
  }
  return ne;
}

__device__ __forceinline__ double basis_val(const AxisEl& e, double x) {
  double v = e.scale;
  if (e.nroots >= 1) v *= (x - e.r0);
  if (e.nroots >= 2) v *= (x - e.r1);
  if (e.nroots >= 3) v *= (x - e.r2);
  if (e.nroots >= 4) v *= (x - e.r3);
  return v;
}

__device__ __forceinline__ double mu_r2(double r2, const WParams& P) {
  // |xi|^{2-d-alpha} e^{-lambda |xi|}
  double lg = log(r2);
  if (P.lambda == 0.0) return exp(-0.5 * P.beta * lg);
  return exp(-0.5 * P.beta * lg - P.lambda * sqrt(r2));
}

__device__ int pick_rule(double ratio) {
  // ratio = distance of the element's nearest corner to the origin / element width
  if (ratio < 1.0) return 7;   // q = 20
  if (ratio < 2.0) return 6;   // 16
  if (ratio < 4.0) return 5;   // 12
  if (ratio < 8.0) return 4;   // 10
  if (ratio < 16.0) return 3;  // 8
  if (ratio < 32.0) return 2;  // 6
  if (ratio < 64.0) return 1;  // 5
  if (ratio < 128.0) return 0; // 4
  return 8;                    // 3: error ~ (1 / (2 ratio))^6 < 4e-15 relative
}

// Rule for bases of degree p >= 3 (d >= 2): the degree-p product leaves 2q - p orders of the
// kernel's Taylor series to a q-point rule, so each distance class takes more points than
// pick_rule gives for p <= 2 (the error ~ (1 / (2 ratio))^{2q - p} stays below 1e-16).
__device__ int pick_rule_high(double ratio) {
  if (ratio < 2.0) return 7;    // q = 20
  if (ratio < 8.0) return 6;    // 16
  if (ratio < 32.0) return 5;   // 12
  if (ratio < 128.0) return 4;  // 10
  if (ratio < 512.0) return 3;  // 8
  return 2;                     // 6
}
__device__ __forceinline__ int pick_rule_p(double ratio, int p) { return p >= 3 ? pick_rule_high(ratio) : pick_rule(ratio); }

// Monomial coefficients (in t = xi / h) of the local basis on the origin element.
__device__ void origin_poly(int p, int l, double* c) {
  c[0] = c[1] = c[2] = 0.0;
  if (p == 0) {
    c[0] = 1.0;
  } else if (p == 1) {
    if (l == 0) { c[0] = 1.0; c[1] = -1.0; } else { c[1] = 1.0; }
  } else {
    if (l == 0) { c[0] = 1.0; c[1] = -1.5; c[2] = 0.5; }
    else if (l == 1) { c[1] = 2.0; c[2] = -1.0; }
    else { c[1] = -0.5; c[2] = 0.5; }
  }
}

// int_0^H r^{a-1} e^{-b r} dr = H^a sum_j (-b H)^j / (j! (a + j))  (power series of the lower
// incomplete gamma function; b H <= a few on every element that reaches the origin)
__device__ double radial_moment(double a, double b, double H) {
  double Ha = pow(H, a);
  if (b == 0.0) return Ha / a;
  double x = -b * H, term = 1.0, sum = 1.0 / a;
  for (int j = 1; j < 200; ++j) {
    term *= x / j;
    double t = term / (a + j);
    sum += t;
    if (fabs(t) < 1e-18 * fabs(sum)) break;
  }
  return Ha * sum;
}

// Monomial coefficients (in t = xi / h, ascending) of the Lagrange basis of local
// node l on the nodes t = 0..p, any p <= 4: prod_{s != l} (t - s) / (l - s).
__device__ void origin_poly_lagrange(int p, int l, double* c) {
  for (int m = 0; m <= 4; ++m) c[m] = m == 0 ? 1.0 : 0.0;
  int deg = 0;
  for (int s = 0; s <= p; ++s) {
    if (s == l) continue;
    const double inv = 1.0 / (double)(l - s);
    for (int m = deg + 1; m >= 1; --m)
      if (CHK(m, 5)) c[m] = (c[m - 1] - s * c[m]) * inv;
    c[0] = -s * c[0] * inv;
    ++deg;
  }
}

// int_0^H phi_l(xi) mu(xi) dxi on the 1D origin element: exact radial moments of the
// monomials of the local basis.
__device__ double origin_element_1d(const WParams& P, int l, double H) {
  double cf[5];
  if (P.p <= 2) {
    origin_poly(P.p, l, cf);
  } else {
    origin_poly_lagrange(P.p, l, cf);
  }
  const double ih = 1.0 / P.h;
  double s = 0.0, scale = 1.0;
  for (int m = 0; m <= P.p; ++m, scale *= ih) s += cf[m] * scale * radial_moment(P.gamma - P.alpha + m, P.lambda, H);
  return s;
}

// Origin element [0, H]^d (d >= 2) of prod_i phi_{l_i}(xi_i) mu(xi): Duffy split into the d
// pyramids {xi_i = max}, xi = r (s with s_i = 1), exact radial moments in r, tensor
// Gauss-Legendre (16 points per angular coordinate) in s.  duffy_angle evaluates what angle
// a shares across all basis products (direction, weight x |s|^{-beta}, radial moments);
// duffy_product the sum over the pyramids for one product l.
constexpr int kDuffyRule = 6;  // rule index of q = 16
constexpr int kDuffyMoments = 13;  // radial moments m = 0 .. p d (p <= 4, d <= 3)
struct DuffyAngle {
  double s[2];
  double base;
  double R[kDuffyMoments];
};

__device__ void duffy_angle(const WParams& P, int a, double H, DuffyAngle& A) {
  const int d = P.d, q = rule_q(kDuffyRule), off = rule_off(kDuffyRule);
  const int ia = a % q, ib = a / q;
  double ws = 1.0;
  A.s[0] = A.s[1] = 0.0;
  if (CHK(off + ia, kRuleTotal)) {
    A.s[0] = 0.5 * (c_gl_x[off + ia] + 1.0);
    ws *= 0.5 * c_gl_w[off + ia];
  }
  if (d == 3 && CHK(off + ib, kRuleTotal)) {
    A.s[1] = 0.5 * (c_gl_x[off + ib] + 1.0);
    ws *= 0.5 * c_gl_w[off + ib];
  }
  const double cs = sqrt(1.0 + A.s[0] * A.s[0] + A.s[1] * A.s[1]);
  for (int m = 0; m <= P.p * d && CHK(m, kDuffyMoments); ++m)
    A.R[m] = radial_moment(P.gamma - P.alpha + m, P.lambda * cs, H);
  A.base = ws * pow(cs, -P.beta);
}

__device__ double duffy_product(const WParams& P, const int* l, const DuffyAngle& A) {
  constexpr int NM = kDuffyMoments;
  const int d = P.d, p = P.p;
  const double ih = 1.0 / P.h;
  double cf[3][5];
  for (int i = 0; i < d && CHK(i, 3); ++i) {
    if (p <= 2) {
      origin_poly(p, l[i], cf[i]);
      cf[i][3] = cf[i][4] = 0.0;
    } else {
      origin_poly_lagrange(p, l[i], cf[i]);
    }
    double sc = ih;  // coefficients of xi^m
    for (int m = 1; m <= 4; ++m, sc *= ih) cf[i][m] *= sc;
  }
  double tot = 0.0;
  for (int i = 0; i < d; ++i) {  // pyramid: axis i largest
    double poly[NM] = {1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int deg = 0, col = 0;
    for (int j = 0; j < d && CHK(j, 3); ++j) {
      const double t = (j == i) ? 1.0 : (CHK(col, 2) ? A.s[col++] : 0.0);
      double pj[5];
      double tp = 1.0;
      for (int m = 0; m < 5; ++m, tp *= t) pj[m] = cf[j][m] * tp;
      double np[NM] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int m1 = 0; m1 <= deg; ++m1)
        for (int m2 = 0; m2 <= p; ++m2)
          if (CHK(m1 + m2, NM) && CHK(m1, NM) && CHK(m2, 5)) np[m1 + m2] += poly[m1] * pj[m2];
      deg += p;
      for (int m = 0; m < NM; ++m) poly[m] = np[m];
    }
    double acc = 0.0;
    for (int m = 0; m <= deg && CHK(m, NM); ++m) acc += poly[m] * A.R[m];
    tot += acc;
  }
  return A.base * tot;
}

__global__ void k_weights_1d(WParams P, double* __restrict__ omega, int64_t count) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  AxisEl el[2];
  const int ne = axis_elements(P, idx, el);
  double total = 0.0;
  for (int e = 0; e < ne && CHK(e, 2); ++e) {
    const AxisEl& E = el[e];
    if (E.origin_l >= 0) {
      total += origin_element_1d(P, E.origin_l, E.hi - E.lo);
      continue;
    }
    // p = 3, 4: a degree-p basis leaves 2q - p orders of the kernel's Taylor series to the
    // rule, so the distance-chosen q (tuned for p <= 2) falls short far out; 20 points on
    // every element (1D weights are a few per node)
    const int rule = P.p >= 3 ? 7 : pick_rule(sqrt(E.lo * E.lo) / (E.hi - E.lo));
    if (!CHK(rule, kNumRules)) continue;
    const int q = rule_q(rule), off = rule_off(rule);
    if (!CHK(off + q - 1, kRuleTotal)) continue;
    const double c = 0.5 * (E.hi + E.lo), hw = 0.5 * (E.hi - E.lo);
    double acc = 0.0;
    for (int g = 0; g < q; ++g) {
      const double x = c + hw * c_gl_x[off + g];
      acc += hw * c_gl_w[off + g] * basis_val(E, x) * mu_r2(x * x, P);
    }
    total += acc;
  }
  if (CHK(idx, count)) omega[idx] = total;
}

// ---------------------------------------------------------------------------
// Weights for d >= 2 in three steps, each element integrated once:
//   k_near_elements: the elements near the origin (densest rules, Duffy-split
//     origin element), spread over several blocks each;
//   k_elements: one thread per element, the integrals of all its local basis
//     products (tensor Gauss-Legendre, q per axis from the distance to the
//     origin), eint[e * NL + c];
//   k_gather: one thread per node, the sum of its elements' contributions in a
//     fixed order.
// Elements per axis: p = 0: e = k (one node); p = 1: [e h, (e+1) h], nodes e,
// e+1; p = 2: [2e h, (2e+2) h], nodes 2e, 2e+1, 2e+2.
// ---------------------------------------------------------------------------

// 1D element e of degree p: interval and the local basis function l (product form)
__device__ AxisEl elem_axis(const WParams& P, int e, int l) {
  const double h = P.h, L = P.N * h;
  if (P.p == 0) return AxisEl{fmax(0.0, (e - 0.5) * h), fmin(L, (e + 0.5) * h), 0, 0, 1.0, 0, e == 0 ? 0 : -1};
  if (P.p == 1) {
    const double a = e * h;
    if (l == 0) return AxisEl{a, a + h, a + h, 0, -1.0 / h, 1, e == 0 ? 0 : -1};
    return AxisEl{a, a + h, a, 0, 1.0 / h, 1, e == 0 ? 1 : -1};
  }
  if (P.p == 2) {
    const double a = 2 * e * h;
    if (l == 0) return AxisEl{a, a + 2 * h, a + h, a + 2 * h, 0.5 / (h * h), 2, e == 0 ? 0 : -1};
    if (l == 1) return AxisEl{a, a + 2 * h, a, a + 2 * h, -1.0 / (h * h), 2, e == 0 ? 1 : -1};
    return AxisEl{a, a + 2 * h, a, a + h, 0.5 / (h * h), 2, e == 0 ? 2 : -1};
  }
  // p = 3, 4: Lagrange polynomial of local node l on the nodes p e + s, s = 0..p
  const int p = P.p;
  double roots[4] = {0, 0, 0, 0}, scale = 1.0;
  int nr = 0;
  for (int s2 = 0; s2 <= p; ++s2) {
    if (s2 == l) continue;
    if (CHK(nr, 4)) roots[nr++] = ((double)p * e + s2) * h;
    scale /= (double)(l - s2) * h;
  }
  return AxisEl{(double)p * e * h, ((double)p * e + p) * h, roots[0], roots[1], scale, nr, e == 0 ? l : -1, roots[2],
                roots[3]};
}

// ---------------------------------------------------------------------------
// Near-origin elements (d >= 2): the elements e in [0, E)^d carry the densest
// rules (q up to 20 per axis, the Duffy-split origin element), so they are
// integrated up front with kNearSplit blocks each: block s takes every
// kNearSplit-th quadrature point (or, on the origin element, every
// kNearSplit-th (angle, product group) pair), and writes per-product partial
// sums tab[(element * kNearSplit + s) * nloc + c]; the tiled kernel adds the
// kNearSplit partials in order.  Deterministic: fixed split, fixed reduction tree.
// ---------------------------------------------------------------------------

constexpr int kNearSplit = 8;
constexpr int kNearGroups = 8;   // product groups per Duffy angle
constexpr int kNearE[4] = {0, 0, 16, 8};

template <int D, int PD>
__global__ void __launch_bounds__(256) k_near_elements(WParams P, int E, double* __restrict__ tab) {
  constexpr int N1 = PD + 1, NL = (D == 2) ? N1 * N1 : N1 * N1 * N1;
  __shared__ double red[8][NL];
  const int eidx = blockIdx.x / kNearSplit, sp = blockIdx.x % kNearSplit;
  const int el[3] = {eidx % E, (eidx / E) % E, D == 3 ? eidx / (E * E) : 0};
  double acc[NL];
#pragma unroll
  for (int c = 0; c < NL; ++c) acc[c] = 0.0;
  AxisEl ax[3][N1];
  bool origin = true;
  double lo2 = 0.0, width = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int l = 0; l < N1; ++l) ax[i][l] = elem_axis(P, el[i], l);
    origin = origin && el[i] == 0;
    lo2 += ax[i][0].lo * ax[i][0].lo;
    width = fmax(width, ax[i][0].hi - ax[i][0].lo);
  }
  const int stride = kNearSplit * blockDim.x;
  if (origin) {
    // Degrees p <= 2: the Duffy split on the whole element.  p >= 3: the Duffy split on
    // the cell [0, h]^D at the origin only (the monomial expansion over the whole element,
    // side p h, would multiply terms by up to p^{p D} and cancel to 1e-11), and the
    // element's other p^D - 1 cells, where the integrand is smooth, by a 20-point tensor
    // Gauss-Legendre rule with the basis functions in product form.
    const int q = rule_q(kDuffyRule), nang = (D == 2) ? q : q * q;
    const double H = PD >= 3 ? P.h : ax[0][0].hi - ax[0][0].lo;
    for (int u = sp + kNearSplit * threadIdx.x; u < nang * kNearGroups; u += stride) {
      const int a = u % nang, g = u / nang;
      DuffyAngle A;
      duffy_angle(P, a, H, A);
      if constexpr (PD <= 2) {
#pragma unroll
        for (int c = 0; c < NL; ++c) {
          if (c % kNearGroups != g) continue;
          const int l[3] = {c % N1, (c / N1) % N1, D == 3 ? c / (N1 * N1) : 0};
          acc[c] += duffy_product(P, l, A);
        }
      } else {  // up to 125 products: a loop, not 125 inlined copies
#pragma unroll 1
        for (int c = g; c < NL; c += kNearGroups) {
          const int l[3] = {c % N1, (c / N1) % N1, D == 3 ? c / (N1 * N1) : 0};
          acc[c] += duffy_product(P, l, A);
        }
      }
    }
    if constexpr (PD >= 3) {
      constexpr int QS = 20, NCELL = (D == 2) ? PD * PD : PD * PD * PD, NPTS = (D == 2) ? QS * QS : QS * QS * QS;
      const int off = rule_off(7);  // q = 20
      for (int j = sp + kNearSplit * threadIdx.x; j < (NCELL - 1) * NPTS; j += stride) {
        const int cell = 1 + j / NPTS, pt = j % NPTS;
        const int ci[3] = {cell % PD, (cell / PD) % PD, D == 3 ? cell / (PD * PD) : 0};
        const int gq[3] = {pt % QS, (pt / QS) % QS, D == 3 ? pt / (QS * QS) : 0};
        double wb[3][N1], r2 = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const int gi = CHK(off + gq[i], kRuleTotal) ? off + gq[i] : off;
          const double x = (ci[i] + 0.5 * (c_gl_x[gi] + 1.0)) * P.h;
          const double w = 0.5 * P.h * c_gl_w[gi];
          r2 += x * x;
#pragma unroll
          for (int l = 0; l < N1; ++l) wb[i][l] = w * basis_val(ax[i][l], x);
        }
        const double m = mu_r2(r2, P);
#pragma unroll
        for (int c = 0; c < NL; ++c) {
          double v = m * wb[0][c % N1] * wb[1][(c / N1) % N1];
          if (D == 3) v *= wb[2][c / (N1 * N1)];
          acc[c] += v;
        }
      }
    }
  } else {
    const int rule = pick_rule_p(sqrt(lo2) / width, PD);
    const int q = rule_q(rule), off = rule_off(rule);
    const int npts = (D == 2) ? q * q : q * q * q;
    double cen[3], hw[3];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      cen[i] = 0.5 * (ax[i][0].hi + ax[i][0].lo);
      hw[i] = 0.5 * (ax[i][0].hi - ax[i][0].lo);
    }
    for (int j = sp + kNearSplit * threadIdx.x; j < npts; j += stride) {
      const int g[3] = {j % q, (j / q) % q, D == 3 ? j / (q * q) : 0};
      double wb[3][N1], r2 = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const int gi = CHK(off + g[i], kRuleTotal) ? off + g[i] : off;
        const double x = cen[i] + hw[i] * c_gl_x[gi];
        const double w = hw[i] * c_gl_w[gi];
        r2 += x * x;
#pragma unroll
        for (int l = 0; l < N1; ++l) wb[i][l] = w * basis_val(ax[i][l], x);
      }
      const double m = mu_r2(r2, P);
#pragma unroll
      for (int c = 0; c < NL; ++c) {
        double v = m * wb[0][c % N1] * wb[1][(c / N1) % N1];
        if (D == 3) v *= wb[2][c / (N1 * N1)];
        acc[c] += v;
      }
    }
  }
  // block sum per product: warps by shuffles, then the 8 warp sums in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NL; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0 && CHK(warp, 8)) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < NL) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5) && w < 8; ++w) t += red[w][threadIdx.x];
    tab[((int64_t)eidx * kNearSplit + sp) * NL + threadIdx.x] = t;
  }
}

// The integrand mu(|xi|) prod_i phi_{l_i}(xi_i) is symmetric under permutations of the
// axes (mu is radial and every axis carries the same basis), so the integrals of a
// permuted element are those of the sorted one with the local indices permuted: only
// the elements with e_0 <= e_1 (<= e_2) are integrated, numbered by
// canon_index(e) = T3(e_2) + T2(e_1) + e_0 (3D) or T2(e_1) + e_0 (2D), with the
// tetrahedral T3(m) = m (m+1) (m+2) / 6 and triangular T2(m) = m (m+1) / 2 numbers.
__host__ __device__ __forceinline__ int64_t tri2(int64_t m) { return m * (m + 1) / 2; }
__host__ __device__ __forceinline__ int64_t tri3(int64_t m) { return m * (m + 1) * (m + 2) / 6; }
__host__ __device__ __forceinline__ int64_t canon_count(int d, int64_t ne) { return d == 2 ? tri2(ne) : tri3(ne); }

// the largest m with f(m) <= t for an increasing f, from an estimate (corrected both ways)
template <typename F>
__device__ __forceinline__ int64_t inv_increasing(int64_t t, int64_t guess, F f) {
  int64_t m = guess < 0 ? 0 : guess;
  while (m > 0 && f(m) > t) --m;
  while (f(m + 1) <= t) ++m;
  return m;
}

// canonical element number t -> (e_0 <= e_1 [<= e_2])
template <int D>
__device__ __forceinline__ void canon_element(int64_t t, int* el) {
  if (D == 2) {
    const int64_t e1 = inv_increasing(t, (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5), tri2);
    el[1] = (int)e1;
    el[0] = (int)(t - tri2(e1));
    el[2] = 0;
  } else {
    const int64_t e2 = inv_increasing(t, (int64_t)cbrt(6.0 * (double)t) - 1, tri3);
    const int64_t rem = t - tri3(e2);
    const int64_t e1 = inv_increasing(rem, (int64_t)((sqrt(8.0 * (double)rem + 1.0) - 1.0) * 0.5), tri2);
    el[2] = (int)e2;
    el[1] = (int)e1;
    el[0] = (int)(rem - tri2(e1));
  }
}

template <int D, int PD>
__global__ void __launch_bounds__(256) k_elements(WParams P, int64_t ne, const double* __restrict__ near, int E,
                                                  double* __restrict__ eint) {
  constexpr int N1 = PD + 1, NL = (D == 2) ? N1 * N1 : N1 * N1 * N1, NW = (D == 2) ? N1 : N1 * N1;
  const int64_t total = canon_count(D, ne);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int el[3];
  canon_element<D>(t, el);
  double acc[NL];
#pragma unroll
  for (int c = 0; c < NL; ++c) acc[c] = 0.0;
  bool in_near = true;
#pragma unroll
  for (int i = 0; i < D; ++i) in_near = in_near && el[i] < E;
  if (in_near) {
    const int64_t nidx = el[0] + E * (el[1] + (D == 3 ? E * el[2] : 0));
#pragma unroll
    for (int c = 0; c < NL; ++c)
      for (int sp = 0; sp < kNearSplit; ++sp) acc[c] += near[(nidx * kNearSplit + sp) * NL + c];
  } else {
    AxisEl ax[3][N1];
    double lo2 = 0.0, width = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int l = 0; l < N1; ++l) ax[i][l] = elem_axis(P, el[i], l);
      lo2 += ax[i][0].lo * ax[i][0].lo;
      width = fmax(width, ax[i][0].hi - ax[i][0].lo);
    }
    const int rule = pick_rule_p(sqrt(lo2) / width, PD);
    const int q = rule_q(rule), off = rule_off(rule);
    if (CHK(q - 1, 20) && CHK(off + q - 1, kRuleTotal)) {
      double cen[3], hw[3];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        cen[i] = 0.5 * (ax[i][0].hi + ax[i][0].lo);
        hw[i] = 0.5 * (ax[i][0].hi - ax[i][0].lo);
      }
      // Away from the origin mu is evaluated through its Taylor series in delta = r^2 / c^2 - 1
      // about the element centre c: mu(r^2) = mu(c^2) exp(-(beta/2) log(1 + delta)
      // - lambda c (sqrt(1 + delta) - 1)) = mu(c^2) sum_k h_k delta^k, the h_k from the series
      // of the exponent g by h_k = (1/k) sum_{j<=k} j g_j h_{k-j}.  The degree covers both
      // factors to 1e-17 over the element (|delta|^k for the power, (lambda c |delta|)^k / k!
      // for the tempering) plus 4; elements with |delta| > 0.15 or a degree above kSeriesMax
      // keep the direct evaluation.  Checked against 40-digit evaluations: relative error
      // below 6e-16 for beta in (0, 3), lambda c up to 35, the level of the direct log/exp.
      // The series replaces a log and an exp (and a sqrt) per point by a short Horner chain.
      double c2 = 0.0, hi2 = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        c2 += cen[i] * cen[i];
        hi2 += ax[i][0].hi * ax[i][0].hi;
      }
      const double inv_c2 = 1.0 / c2;
      const double dmax = fmax(c2 - lo2, hi2 - c2) * inv_c2;
      int deg = 0;
      double hser[kSeriesMax + 1], muc = 1.0;
      const double c = sqrt(c2);
      if (D == 3 && dmax > 0.0 && dmax <= 0.15) {  // (2D elements have too few points to pay for the setup)
        // k1 >= log(1e-17) / log(dmax) without a log: dmax = m 2^e, m in [1, 2), and
        // log2(m) <= (m - 1) / ln 2, so -log2(dmax) >= -e - (m - 1) / ln 2; 1e-17 > 2^-56.5
        int e2;
        const double m2 = 2.0 * frexp(dmax, &e2);
        const int k1 = (int)ceil(56.5 / (double)(1 - e2 - (m2 - 1.0) * 1.4426950408889634));
        int k2 = 0;
        for (double t = 1.0, x = P.lambda * c * dmax; t > 1e-17 && k2 < kSeriesMax; t *= x * c_inv[k2]) ++k2;
        deg = (k1 > k2 ? k1 : k2) + 4;
        if (deg > kSeriesMax) deg = 0;
      }
      if (deg > 0) {
        double jg[kSeriesMax + 1];  // j g_j, g_j = -(beta/2) (-1)^{j+1} / j - lambda c binom(1/2, j)
        const double hb = -0.5 * P.beta, lc = P.lambda * c;
        for (int j = 1; j <= deg; ++j) jg[j] = ((j & 1) ? hb : -hb) - j * lc * c_bhalf[j];
        hser[0] = 1.0;
        for (int k = 1; k <= deg; ++k) {
          double t = 0.0;
          for (int j = 1; j <= k; ++j) t = fma(jg[j], hser[k - j], t);
          hser[k] = t * c_inv[k];
        }
        muc = mu_r2(c2, P);
      }
      // axis 0 (innermost): squared nodes and weighted basis values
      double X0[20], W0[N1][20];
      for (int g = 0; g < q; ++g) {
        const double x = cen[0] + hw[0] * c_gl_x[off + g], w = hw[0] * c_gl_w[off + g];
        X0[g] = x * x;
#pragma unroll
        for (int l = 0; l < N1; ++l) W0[l][g] = w * basis_val(ax[0][l], x);
      }
      for (int g2 = 0; g2 < (D == 3 ? q : 1); ++g2) {
        double x2s = 0.0, wb2[N1];
#pragma unroll
        for (int l = 0; l < N1; ++l) wb2[l] = 1.0;
        if (D == 3) {
          const double x = cen[2] + hw[2] * c_gl_x[off + g2], w = hw[2] * c_gl_w[off + g2];
          x2s = x * x;
#pragma unroll
          for (int l = 0; l < N1; ++l) wb2[l] = w * basis_val(ax[2][l], x);
        }
        for (int g1 = 0; g1 < q; ++g1) {
          const double x = cen[1] + hw[1] * c_gl_x[off + g1], w = hw[1] * c_gl_w[off + g1];
          const double r12 = x * x + x2s;
          double w21[NW];  // products of the outer axes' weighted basis values, (l2, l1) with l1 fastest
#pragma unroll
          for (int j = 0; j < NW; ++j) w21[j] = w * basis_val(ax[1][j % N1], x) * wb2[j / N1];
          for (int g0 = 0; g0 < q; ++g0) {
            double m;
            if (deg > 0) {
              const double dl = fma(X0[g0] + r12, inv_c2, -1.0);
              m = hser[deg];
              for (int k = deg - 1; k >= 0; --k) m = fma(m, dl, hser[k]);
            } else {
              m = mu_r2(X0[g0] + r12, P);
            }
#pragma unroll
            for (int l0 = 0; l0 < N1; ++l0) {
              const double ml = m * W0[l0][g0];
#pragma unroll
              for (int j = 0; j < NW; ++j) acc[j * N1 + l0] += ml * w21[j];
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NL; ++c) acc[c] *= muc;
    }
  }
#pragma unroll
  for (int c = 0; c < NL; ++c) eint[t * NL + c] = acc[c];
}

// omega_k = sum over the elements containing node k of the integral of k's local basis product
template <int D>
__global__ void k_gather(WParams P, int64_t ne, const double* __restrict__ eint, double* __restrict__ omega,
                         int64_t count) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int p = P.p, nl1 = p + 1, nloc = (D == 2) ? nl1 * nl1 : nl1 * nl1 * nl1;
  const int64_t N1 = P.N + 1;
  int64_t k[3] = {idx % N1, (idx / N1) % N1, D == 3 ? idx / (N1 * N1) : 0};
  // per axis: elements containing node k and the local index of k in them
  int64_t ee[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  int ll[3][2] = {{0, 0}, {0, 0}, {0, 0}}, nc[3] = {1, 1, 1};
  for (int i = 0; i < D; ++i) {
    nc[i] = 0;
    if (p == 0) { ee[i][0] = k[i]; ll[i][0] = 0; nc[i] = 1; }
    else if (p == 1) {
      if (k[i] >= 1) { ee[i][nc[i]] = k[i] - 1; ll[i][nc[i]++] = 1; }
      if (k[i] < P.N) { ee[i][nc[i]] = k[i]; ll[i][nc[i]++] = 0; }
    } else {  // elements of p intervals: an inner node in one, a shared node in two
      const int64_t m = k[i] / p, t = k[i] - m * p;
      if (t != 0) { ee[i][0] = m; ll[i][0] = (int)t; nc[i] = 1; }
      else {
        if (k[i] >= p) { ee[i][nc[i]] = m - 1; ll[i][nc[i]++] = p; }
        if (k[i] <= P.N - p) { ee[i][nc[i]] = m; ll[i][nc[i]++] = 0; }
      }
    }
  }
  const int64_t total = canon_count(D, ne);
  double tot = 0.0;
  for (int a = 0; a < nc[0]; ++a)
    for (int b = 0; b < nc[1]; ++b)
      for (int cc = 0; cc < (D == 3 ? nc[2] : 1); ++cc) {
        // sort (element, local index) pairs by element: the canonical element and its local product
        int64_t es[3] = {ee[0][a], ee[1][b], D == 3 ? ee[2][cc] : 0};
        int ls[3] = {ll[0][a], ll[1][b], D == 3 ? ll[2][cc] : 0};
        for (int i = 1; i < D; ++i)
          for (int j = i; j > 0 && es[j - 1] > es[j]; --j) {
            const int64_t te = es[j];
            es[j] = es[j - 1];
            es[j - 1] = te;
            const int tl = ls[j];
            ls[j] = ls[j - 1];
            ls[j - 1] = tl;
          }
        const int64_t e = D == 2 ? tri2(es[1]) + es[0] : tri3(es[2]) + tri2(es[1]) + es[0];
        const int lc = ls[0] + nl1 * (ls[1] + (D == 3 ? nl1 * ls[2] : 0));
        if (CHK(e, total) && CHK(lc, nloc)) tot += eint[e * nloc + lc];
      }
  omega[idx] = tot;
}

// ---------------------------------------------------------------------------
// Stencil: a_k = 2^{z(k)} omega_k / (h^2 |k|^2) (k != 0), plus the origin rule
// a_{j e_i} += 2^{d-1} e_j omega_0 / (d (j h)^2), e = (1) for p <= 1 and
// (4/3, -1/3) for p = 2.  Writes a_k, and per-block partial sums (Kahan) of
// 2^{d-z(k)} a_k over k != 0 for the centre coefficient.
// ---------------------------------------------------------------------------

__global__ void k_stencil(WParams P, const double* __restrict__ omega, double* __restrict__ a,
                          double* __restrict__ partial, int64_t count) {
  __shared__ double sh[32];
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (idx < count && idx > 0) {
    const int d = P.d;
    const int64_t N1 = P.N + 1;
    int64_t k[3] = {0, 0, 0}, rem = idx;
    int z = 0, nzaxis = -1;
    double k2 = 0.0;
    for (int i = 0; i < d; ++i) {
      k[i] = rem % N1;
      rem /= N1;
      if (k[i] == 0) ++z; else nzaxis = i;
      k2 += (double)k[i] * (double)k[i];
    }
    // a_k = 2^{z(k)} omega_k / |xi_k|^gamma; the origin rule (zeta = floor(gamma / 2)) only at gamma = 2
    const double xi2 = P.h * P.h * k2;
    double v = CHK(idx, count) ? ldexp(omega[idx], z) / (P.gamma == 2.0 ? xi2 : pow(xi2, 0.5 * P.gamma)) : 0.0;
    if (z == d - 1 && P.gamma == 2.0) {  // on an axis: k = j e_i
      const int64_t j = k[nzaxis];
      // origin rule: second differences combined to order 2 (p <= 1), 4 (p = 2), 6 (p = 3), 8 (p = 4)
      double e = 0.0;
      if (P.p <= 1) e = (j == 1) ? 1.0 : 0.0;
      else if (P.p == 2) e = (j == 1) ? 4.0 / 3.0 : (j == 2 ? -1.0 / 3.0 : 0.0);
      else if (P.p == 3) e = (j == 1) ? 1.5 : (j == 2 ? -0.6 : (j == 3 ? 0.1 : 0.0));
      else e = (j == 1) ? 1.6 : (j == 2 ? -0.8 : (j == 3 ? 8.0 / 35.0 : (j == 4 ? -1.0 / 35.0 : 0.0)));
      if (e != 0.0) v += ldexp(1.0, d - 1) * e * omega[0] / (d * (j * P.h) * (j * P.h));
    }
    if (CHK(idx, count)) a[idx] = v;
    contrib = ldexp(v, d - z);
  }
  // block sum with pairwise tree (deterministic)
  for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = contrib;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && CHK(blockIdx.x, gridDim.x)) partial[blockIdx.x] = v;
  }
}

// a_0 = -sum(partials) - 2^d F_d, Kahan-compensated, one block.
// Compensated sum of x[0..n) by the block (1024 threads): each thread a strided
// Kahan sum, then the (sum, compensation) pairs merged in a fixed binary tree
// (TwoSum of the sums, the compensations added).  Result in thread 0.
__device__ double block_sum_compensated(const double* __restrict__ x, int64_t n, double* sh_s, double* sh_c) {
  double s = 0.0, c = 0.0;  // value s - c
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double y = (CHK(i, n) ? x[i] : 0.0) - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
      const double a = sh_s[threadIdx.x], b = sh_s[threadIdx.x + stride];
      const double t = a + b, bb = t - a, e = (a - (t - bb)) + (b - bb);  // t + e = a + b exactly
      sh_s[threadIdx.x] = t;
      sh_c[threadIdx.x] = sh_c[threadIdx.x] + sh_c[threadIdx.x + stride] - e;
    }
    __syncthreads();
  }
  const double r = sh_s[0] - sh_c[0];
  __syncthreads();
  return r;
}

// a_0 = -sum(partials) - 2^d F_d, F_d = sum of the far-field terms (also stored in far_out)
__global__ void __launch_bounds__(1024) k_centre(const double* __restrict__ partial, int64_t nparts,
                                                 const double* __restrict__ terms, int64_t nterms, int d, double* a,
                                                 double* far_out) {
  __shared__ double sh_s[1024], sh_c[1024];
  const double S = block_sum_compensated(partial, nparts, sh_s, sh_c);
  const double F = block_sum_compensated(terms, nterms, sh_s, sh_c);
  if (threadIdx.x == 0) {
    a[0] = -S - ldexp(F, d);
    far_out[0] = F;
  }
}

// ---------------------------------------------------------------------------
// Symbol: Lambda_raw[k] = sum_{j in (-(n-1)..n-1)^d} a_{|j|} e^{-2 pi i j.k/M}
//       = prod-separable cosine sums  sum_{j=0}^{n-1} w_j a_j cos(2 pi j k / M),
// w_0 = 1, w_j = 2; computed axis by axis, k in [0, M/2].
// ---------------------------------------------------------------------------

// compact copy of the [0, n_1) x .. x [0, n_d) block of the generator
__global__ void k_gen_block(const double* __restrict__ a, double* __restrict__ out, int d, int64_t N1, int64_t n0,
                            int64_t n1, int64_t n2, int64_t count) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  int64_t rem = idx, src = 0, mul = 1;
  for (int i = 0; i < d; ++i) {
    const int64_t ni = i == 0 ? n0 : (i == 1 ? n1 : n2);
    const int64_t ki = rem % ni;
    rem /= ni;
    src += ki * mul;
    mul *= N1;
  }
  int64_t tot = 1;
  for (int i = 0; i < d; ++i) tot *= N1;
  if (CHK(src, tot)) out[idx] = a[src];
}

// One axis of the symbol by FFT, in: (A, n, B) -> out: (A, K, B).  Line (a, b) is
// even-extended to length M (x_j = a_{min(j, M - j)} when that index is below n,
// else 0; n <= M/2 so the two halves never overlap), whose DFT is the cosine sum
// sum_j w_j a_j cos(2 pi j k / M) above.  The DFT of a real even sequence is real, so
// two lines share one complex transform (one as the real part, one as the imaginary
// part).  A block takes 2 LB consecutive lines (consecutive b: coalesced when B > 1,
// along the line when B = 1), loads them in bit-reversed order into shared memory
// (M x LB complex slots), runs log2 M in-place radix-2 stages with the FP64 twiddle
// table tw[t] = e^{-2 pi i t / M}, and writes k in [0, K).
constexpr int kSymFftMaxSmem = 8192 * (int)sizeof(double2);  // M x LB <= 8192 slots

__global__ void __launch_bounds__(256) k_sym_fft(const double* __restrict__ in, double* __restrict__ out, int64_t A,
                                                 int64_t n, int64_t B, int64_t K, int logm, int LB,
                                                 const double2* __restrict__ tw) {
  extern __shared__ __align__(16) double2 sx[];
  const int64_t M = (int64_t)1 << logm, lines = A * B, L0 = (int64_t)blockIdx.x * 2 * LB;
  const int64_t nl = 2 * LB;
  const int64_t nsh = M * LB;
  for (int64_t idx = threadIdx.x; idx < nl * M; idx += blockDim.x) {
    const int64_t l = (B == 1) ? idx / M : idx % nl, j = (B == 1) ? idx % M : idx / nl;
    const int64_t L = L0 + l, jj = j <= M - j ? j : M - j;
    double v = 0.0;
    if (L < lines && jj < n) {
      const int64_t a = L / B, b = L % B, src = (a * n + jj) * B + b;
      if (CHK(src, lines * n)) v = in[src];
    }
    const int64_t pos = (int64_t)(__brev((unsigned)j) >> (32 - logm));
    const int64_t slot = pos * LB + (l % LB);
    if (CHK(slot, nsh)) {
      if (l < LB) sx[slot].x = v;
      else sx[slot].y = v;
    }
  }
  __syncthreads();
  for (int s = 0; s < logm; ++s) {
    const int64_t half = (int64_t)1 << s;
    for (int64_t t = threadIdx.x; t < (M / 2) * LB; t += blockDim.x) {
      const int64_t i = t % LB, bf = t / LB, k = bf & (half - 1);
      const int64_t p0 = ((bf >> s) << (s + 1)) + k, p1 = p0 + half;
      const int64_t ti = k << (logm - 1 - s);
      if (!CHK(p1 * LB + i, nsh) || !CHK(ti, M)) continue;
      const double2 w = tw[ti], x0 = sx[p0 * LB + i], y = sx[p1 * LB + i];
      const double2 x1 = make_double2(y.x * w.x - y.y * w.y, y.x * w.y + y.y * w.x);
      sx[p0 * LB + i] = make_double2(x0.x + x1.x, x0.y + x1.y);
      sx[p1 * LB + i] = make_double2(x0.x - x1.x, x0.y - x1.y);
    }
    __syncthreads();
  }
  for (int64_t idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
    const int64_t l = (B == 1) ? idx / K : idx % nl, k = (B == 1) ? idx % K : idx / nl;
    const int64_t L = L0 + l;
    if (L >= lines || !CHK(k * LB + (l % LB), nsh)) continue;
    const double2 v = sx[k * LB + (l % LB)];
    const int64_t a = L / B, b = L % B, dst = (a * K + k) * B + b;
    if (CHK(dst, lines * K)) out[dst] = l < LB ? v.x : v.y;
  }
}

// The same for an axis of mixed length M (a 7-smooth M that is not a power of two):
// thread group g of ln.tpl() threads transforms lines 2 q and 2 q + 1 (q = blockIdx.x G
// + g) as the real and imaginary parts of one complex line with the mixed-radix FFT.
__global__ void __launch_bounds__(512, 1) k_sym_fft_mx(const double* __restrict__ in, double* __restrict__ out, int64_t A, int64_t n,
                             int64_t B, int64_t K, fft::MxLine ln, const double2* __restrict__ tw) {
  extern __shared__ __align__(16) double2 sxm[];
  const int TPL = ln.tpl(), M = ln.m(), G = blockDim.x / TPL;
  const int g = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  const int64_t lines = A * B, L0 = 2 * ((int64_t)blockIdx.x * G + g);
  double2 v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int j = tl + e * TPL, jj = j <= M - j ? j : M - j;
    double re = 0.0, im = 0.0;
    if (jj < n) {
      if (L0 < lines) {
        const int64_t src = ((L0 / B) * n + jj) * B + L0 % B;
        if (CHK(src, lines * n)) re = in[src];
      }
      if (L0 + 1 < lines) {
        const int64_t src = (((L0 + 1) / B) * n + jj) * B + (L0 + 1) % B;
        if (CHK(src, lines * n)) im = in[src];
      }
    }
    v[e] = double2{re, im};
  }
  ln.fft<false, false, false>(v, sxm + g * ln.stride(), tl, tw);
#pragma unroll
  for (int e = 0; e <= 8; ++e) {
    const int64_t k = tl + e * TPL;
    if (k >= K) continue;
    if (L0 < lines) {
      const int64_t dst = ((L0 / B) * K + k) * B + L0 % B;
      if (CHK(dst, lines * K)) out[dst] = v[e].x;
    }
    if (L0 + 1 < lines) {
      const int64_t dst = (((L0 + 1) / B) * K + k) * B + (L0 + 1) % B;
      if (CHK(dst, lines * K)) out[dst] = v[e].y;
    }
  }
}

// Launches one axis of the symbol (k_sym_fft, or k_sym_fft_mx when plan.m is set).
static int sym_axis(const double* src, double* dst, int64_t A, int64_t n, int64_t B, int64_t K, int64_t M,
                    const MxPlan& plan, cudaStream_t st) {
  if (plan.m == 0) {
    const int logm = ilog2(M);
    // 2 LB lines per block, M x LB complex slots (64 KB; one 128 KB line at M = 8192)
    const int LB = (int)std::max<int64_t>(1, std::min<int64_t>(8, 4096 / M));
    const size_t fsm = (size_t)M * LB * sizeof(double2);
    if (fsm > (size_t)kSymFftMaxSmem) return FRAC_ENOTSUP;
    FRAC_TRY(ensure_twiddles(logm));
    k_sym_fft<<<(unsigned)((A * B + 2 * LB - 1) / (2 * LB)), 256, fsm, st>>>(src, dst, A, n, B, K, logm, LB,
                                                                            twiddles64(logm));
  } else {
    const fft::MxLine ln(plan);
    const int G = std::max(1, 256 / ln.tpl());
    const size_t fsm = (size_t)G * ln.stride() * sizeof(double2);
    if (fsm > 200 * 1024) return FRAC_ENOTSUP;
    FRAC_TRY(prepare_twiddles_len(M));
    FRAC_CUDA_TRY(cudaFuncSetAttribute(k_sym_fft_mx, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    const int64_t pairs = (A * B + 1) / 2;
    k_sym_fft_mx<<<(unsigned)((pairs + G - 1) / G), G * ln.tpl(), fsm, st>>>(src, dst, A, n, B, K, ln,
                                                                             twiddles64_len(M));
  }
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

__global__ void k_scale_symbol(const double* __restrict__ raw, double* __restrict__ l64, float* __restrict__ l32,
                               double scale, int64_t count, double* __restrict__ partial_max) {
  __shared__ double sh[32];
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double m = 0.0;
  if (idx < count && CHK(idx, count)) {
    double v = raw[idx] * scale;
    l64[idx] = v;
    l32[idx] = (float)v;
    m = fabs(raw[idx]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partial_max[blockIdx.x] = v;
  }
}

// Symbol of the tau preconditioner: the sine transform of size M/2 - 1 per axis
// diagonalises the tau matrix of the (zero-extended) Toeplitz operator with the
// circulant-embedding eigenvalues mu at k in [1, M/2 - 1]^d as its eigenvalues, so
// tau^{-1} is the same FFT pipeline on the odd extension with 1/mu.  The stored
// symbol is scale * mu (scale = 1/M for d = 1, 1/(2 M^d) otherwise, the
// normalisation of the FFT pipeline), so 1/mu in that normalisation is
// 1 / (stored * s2) with s2 = M^2 (d = 1) or (2 M^d)^2.  Zero where some k_i is
// 0 or M/2 (the odd extension has no spectrum there); per-block minimum of the
// stored symbol over the other entries for the positivity check.
// Symbols from the plain layout (axis 0 = k1 fastest) -> the column tiles the column
// passes read, B entries of k1 side by side and the column axis next:
//   d = 2: entry (k2, k1) at (k1 / B) K2 B + k2 B + k1 % B;
//   d = 3: entry (k3, k2, k1) at ((k2 KB + k1 / B) K3 + k3) B + k1 % B, KB = ceil(K1 / B).
// Padding columns k1 >= K1 get 0.  K3 = 1 for d = 2 (then k2 is the column axis).
template <typename T, int B>
__global__ void k_tile_symbol(const T* __restrict__ plain, T* __restrict__ tiled, int64_t K1, int64_t K2,
                              int64_t K3, int d, int64_t count) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int64_t KB = (K1 + B - 1) / B, c = idx % B;
  if (d == 2) {
    const int64_t k2 = (idx / B) % K2, t = idx / (B * K2), k1 = t * B + c;
    tiled[idx] = k1 < K1 ? plain[k2 * K1 + k1] : T(0);
  } else {
    const int64_t k3 = (idx / B) % K3, t = (idx / (B * K3)) % KB, k2 = idx / (B * K3 * KB), k1 = t * B + c;
    tiled[idx] = k1 < K1 ? plain[(k3 * K2 + k2) * K1 + k1] : T(0);
  }
}

__global__ void k_precond_symbol(const double* __restrict__ l64, double* __restrict__ p64, float* __restrict__ p32,
                                 int64_t K0, int64_t K1, int64_t K2, int d, double s2, int64_t count,
                                 double* __restrict__ partial_min) {
  __shared__ double sh[32];
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double m = INFINITY;
  if (idx < count) {
    int64_t r = idx;
    bool edge = false;
    for (int i = 0; i < d; ++i) {
      const int64_t K = i == 0 ? K0 : (i == 1 ? K1 : K2);
      const int64_t k = r % K;
      r /= K;
      edge = edge || k == 0 || k == K - 1;
    }
    double v = 0.0;
    if (!edge) {
      const double mu = l64[idx];
      m = mu;
      v = mu > 0.0 ? 1.0 / (mu * s2) : 0.0;
    }
    p64[idx] = v;
    p32[idx] = (float)v;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : INFINITY;
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partial_min[blockIdx.x] = v;
  }
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int build_coefficients(frac_op* op, cudaStream_t st) {
  FRAC_TRY(upload_rules());
  for (int i = 0; i < op->prob.d; ++i) FRAC_TRY(prepare_twiddles_len(op->Ma[i]));
  const frac_problem& pr = op->prob;
  WParams P;
  P.d = pr.d;
  P.p = pr.degree;
  P.N = op->N;
  P.h = pr.h;
  P.alpha = pr.alpha;
  P.lambda = pr.lambda;
  P.gamma = pr.gamma > 0.0 ? pr.gamma : 2.0;
  P.beta = pr.d + pr.alpha - P.gamma;
  const int d = pr.d;
  const int64_t ngen = op->ngen;
  const double L = op->N * pr.h;

  double *omega = nullptr, *partial = nullptr, *near = nullptr, *eint = nullptr;
  const int TB = 256;
  const int64_t nblk = ceil_div(ngen, TB);
  FRAC_CUDA_TRY(cudaMallocAsync(&omega, ngen * sizeof(double), st));
  FRAC_CUDA_TRY(cudaMallocAsync(&partial, nblk * sizeof(double), st));
  if (d == 1) {
    k_weights_1d<<<(unsigned)nblk, TB, 0, st>>>(P, omega, ngen);
  } else {
    // near-origin elements [0, E)^d first, spread over kNearSplit blocks each
    const int64_t ne_axis = pr.degree == 0 ? op->N + 1 : op->N / pr.degree;
    const int E = (int)std::min<int64_t>(kNearE[d], ne_axis);
    int64_t nnear = 1;
    for (int i = 0; i < d; ++i) nnear *= E;
    const int64_t nel = canon_count(d, ne_axis);  // elements up to a permutation of the axes
    const int nl1 = pr.degree + 1;
    const int nloc = d == 2 ? nl1 * nl1 : nl1 * nl1 * nl1;
    FRAC_CUDA_TRY(cudaMallocAsync(&near, (size_t)nnear * kNearSplit * nloc * sizeof(double), st));
    FRAC_CUDA_TRY(cudaMallocAsync(&eint, (size_t)nel * nloc * sizeof(double), st));
    const unsigned nb = (unsigned)(nnear * kNearSplit), eb = (unsigned)ceil_div(nel, 256);
#define FRAC_ELEM_CASE(DD, PP)                                                \
  case DD * 5 + PP:                                                           \
    k_near_elements<DD, PP><<<nb, 256, 0, st>>>(P, E, near);                  \
    k_elements<DD, PP><<<eb, 256, 0, st>>>(P, ne_axis, near, E, eint);        \
    break;
    switch (d * 5 + pr.degree) {
      FRAC_ELEM_CASE(2, 0)
      FRAC_ELEM_CASE(2, 1)
      FRAC_ELEM_CASE(2, 2)
      FRAC_ELEM_CASE(2, 3)
      FRAC_ELEM_CASE(2, 4)
      FRAC_ELEM_CASE(3, 0)
      FRAC_ELEM_CASE(3, 1)
      FRAC_ELEM_CASE(3, 2)
      FRAC_ELEM_CASE(3, 3)
      FRAC_ELEM_CASE(3, 4)
      default:
        return FRAC_EINVAL;
    }
#undef FRAC_ELEM_CASE
    FRAC_CUDA_TRY(cudaGetLastError());
    if (d == 2) k_gather<2><<<(unsigned)nblk, TB, 0, st>>>(P, ne_axis, eint, omega, ngen);
    else k_gather<3><<<(unsigned)nblk, TB, 0, st>>>(P, ne_axis, eint, omega, ngen);
  }
  FRAC_CUDA_TRY(cudaGetLastError());
  k_stencil<<<(unsigned)nblk, TB, 0, st>>>(P, omega, op->a, partial, ngen);
  FRAC_CUDA_TRY(cudaGetLastError());
  const int64_t nterms = (int64_t)(d == 1 ? 1 : (d == 2 ? 32 : 1024)) * kFarPanels;
  double *terms = nullptr, *far_dev = nullptr;
  FRAC_CUDA_TRY(cudaMallocAsync(&terms, (nterms + 1) * sizeof(double), st));
  far_dev = terms + nterms;
  k_far_terms<<<(unsigned)ceil_div(nterms, TB), TB, 0, st>>>(d, pr.alpha, pr.lambda, L, terms, nterms);
  FRAC_CUDA_TRY(cudaGetLastError());
  k_centre<<<1, 1024, 0, st>>>(partial, nblk, terms, nterms, d, op->a, far_dev);
  FRAC_CUDA_TRY(cudaGetLastError());

  // symbol: axis by axis, shape (A, n_i, B) -> (A, K_i, B) with A = prod_{j > i} n_j, B = prod_{j < i} K_j
  int64_t sz = 1;
  for (int i = 0; i < d; ++i) sz *= op->na[i];
  int64_t maxsz = sz;
  {
    int64_t s = sz;
    for (int i = 0; i < d; ++i) {
      s = s / op->na[i] * op->Ka[i];
      if (s > maxsz) maxsz = s;
    }
  }
  double *bufA = nullptr, *bufB = nullptr;
  FRAC_CUDA_TRY(cudaMallocAsync(&bufA, maxsz * sizeof(double), st));
  FRAC_CUDA_TRY(cudaMallocAsync(&bufB, maxsz * sizeof(double), st));
  k_gen_block<<<(unsigned)ceil_div(sz, TB), TB, 0, st>>>(op->a, bufA, d, op->N + 1, op->na[0], op->na[1], op->na[2],
                                                          sz);
  FRAC_CUDA_TRY(cudaGetLastError());
  // one value for every build (builds on several host threads must not lower it under one another)
  FRAC_CUDA_TRY(cudaFuncSetAttribute(k_sym_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymFftMaxSmem));
  int64_t B = 1;
  for (int i = 0; i < d; ++i) {
    int64_t A = 1;
    for (int j = i + 1; j < d; ++j) A *= op->na[j];
    FRAC_TRY(sym_axis(bufA, bufB, A, op->na[i], B, op->Ka[i], op->Ma[i], op->plan[i], st));
    std::swap(bufA, bufB);
    B *= op->Ka[i];
  }
  // bufA holds Lambda_raw on [0, K)^d
  const int64_t ns = op->nsym;
  double Md = 1.0;
  for (int i = 0; i < d; ++i) Md *= (double)op->Ma[i];
  const double scale = -op->c / (d == 1 ? Md : 2.0 * Md);
  const int64_t nb2 = ceil_div(ns, TB);
  double* pmax = nullptr;
  FRAC_CUDA_TRY(cudaMallocAsync(&pmax, nb2 * sizeof(double), st));
  k_scale_symbol<<<(unsigned)nb2, TB, 0, st>>>(bufA, op->lam64, op->lam32, scale, ns, pmax);
  FRAC_CUDA_TRY(cudaGetLastError());
  std::vector<double> hmax(nb2);
  FRAC_CUDA_TRY(cudaMemcpyAsync(hmax.data(), pmax, nb2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  double* pmin = nullptr;
  FRAC_CUDA_TRY(cudaMallocAsync(&pmin, nb2 * sizeof(double), st));
  const double s2 = d == 1 ? Md * Md : (2.0 * Md) * (2.0 * Md);
  k_precond_symbol<<<(unsigned)nb2, TB, 0, st>>>(op->lam64, op->pinv64, op->pinv32, op->Ka[0], op->Ka[1], op->Ka[2], d,
                                                 s2, ns, pmin);
  FRAC_CUDA_TRY(cudaGetLastError());
  std::vector<double> hmin(nb2);
  FRAC_CUDA_TRY(cudaMemcpyAsync(hmin.data(), pmin, nb2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  FRAC_CUDA_TRY(cudaFreeAsync(pmin, st));
  if (d >= 2) {  // the column passes read the symbols in column tiles (one run per tile row)
    const int64_t K1 = op->Ka[0], K2 = op->Ka[1], K3 = d == 3 ? op->Ka[2] : 1;
    void* tmp = nullptr;
    FRAC_CUDA_TRY(cudaMallocAsync(&tmp, ns * sizeof(double), st));
    auto tile = [&](auto* arr, auto bconst) -> int {
      using T = std::remove_pointer_t<decltype(arr)>;
      constexpr int B = decltype(bconst)::value;
      const int64_t cnt = (K1 + B - 1) / B * B * K2 * K3;
      FRAC_CUDA_TRY(cudaMemcpyAsync(tmp, arr, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
      k_tile_symbol<T, B><<<(unsigned)ceil_div(cnt, TB), TB, 0, st>>>((const T*)tmp, arr, K1, K2, K3, d, cnt);
      FRAC_CUDA_TRY(cudaGetLastError());
      return FRAC_OK;
    };
    FRAC_TRY(tile(op->lam64, std::integral_constant<int, 2>{}));
    FRAC_TRY(tile(op->pinv64, std::integral_constant<int, 2>{}));
    FRAC_TRY(tile(op->lam32, std::integral_constant<int, 4>{}));
    FRAC_TRY(tile(op->pinv32, std::integral_constant<int, 4>{}));
    FRAC_CUDA_TRY(cudaFreeAsync(tmp, st));
  }
  FRAC_CUDA_TRY(cudaMemcpyAsync(&op->a0, op->a, sizeof(double), cudaMemcpyDeviceToHost, st));
  FRAC_CUDA_TRY(cudaMemcpyAsync(&op->far_field, far_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  FRAC_CUDA_TRY(cudaFreeAsync(omega, st));
  if (near) FRAC_CUDA_TRY(cudaFreeAsync(near, st));
  if (eint) FRAC_CUDA_TRY(cudaFreeAsync(eint, st));
  FRAC_CUDA_TRY(cudaFreeAsync(terms, st));
  FRAC_CUDA_TRY(cudaFreeAsync(partial, st));
  FRAC_CUDA_TRY(cudaFreeAsync(bufA, st));
  FRAC_CUDA_TRY(cudaFreeAsync(bufB, st));
  FRAC_CUDA_TRY(cudaFreeAsync(pmax, st));
  FRAC_CUDA_TRY(cudaStreamSynchronize(st));
  {
    unsigned long long line = 0;
    long long index = 0;
    FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&line, g_fault_line, sizeof(line)));
    if (line) {
      FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&index, g_fault_index, sizeof(index)));
      const unsigned long long zero = 0;
      FRAC_CUDA_TRY(cudaMemcpyToSymbol(g_fault_line, &zero, sizeof(zero)));
      return record_check_failure("coeffs.cu", (int)line, index);
    }
  }
  double m = 0.0;
  for (double v : hmax) m = v > m ? v : m;
  op->norm_bound = op->c * m;
  double mn = INFINITY;
  for (double v : hmin) mn = v < mn ? v : mn;
  bool fits = true;
  for (int i = 0; i < d; ++i) fits = fits && op->na[i] <= op->Ma[i] / 2 - 1;
  op->precond_ok = fits && mn > 0.0 ? 1 : 0;
  // condition estimate: largest over smallest symbol entry (the scaled symbol is m |scale| at most)
  op->kappa_est = mn > 0.0 ? m * std::fabs(scale) / mn : INFINITY;
  return FRAC_OK;
}


// Symbol of the generator on a box of sides M'_i = 2^logm[i]: the unnormalised DFT
// of a_{|o|} placed at o mod M'_i (per axis) for o in [-N, N]^d, on k in
// prod_i [0, M'_i/2 + 1) (axis 0 fastest; the rest follows by k_i -> M'_i - k_i).
// The even extension of each axis needs N + 1 <= M'_i/2.  Axis by axis with
// k_sym_fft, ping-ponging between `tmp` and `out` so that the last axis writes
// `out` (both prod_i (M'_i/2 + 1) doubles).
int generator_symbol_axes(const frac_op* op, const int* logm, double* out, double* tmp, cudaStream_t st) {
  const int d = op->prob.d;
  const int64_t n1 = op->N + 1;
  FRAC_CUDA_TRY(cudaFuncSetAttribute(k_sym_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymFftMaxSmem));
  double* bufs[2] = {(d % 2) ? out : tmp, (d % 2) ? tmp : out};
  const double* src = op->a;  // the whole (N + 1)^d generator, axis 0 fastest
  int64_t B = 1;
  for (int i = 0; i < d; ++i) {
    const int64_t M = int64_t(1) << logm[i], K = M / 2 + 1;
    if (2 * n1 > M) return FRAC_EINVAL;
    const int LB = (int)std::max<int64_t>(1, std::min<int64_t>(8, 4096 / M));
    const size_t fsm = (size_t)M * LB * sizeof(double2);
    if (fsm > (size_t)kSymFftMaxSmem) return FRAC_ENOTSUP;
    FRAC_TRY(ensure_twiddles(logm[i]));
    int64_t A = 1;
    for (int j = i + 1; j < d; ++j) A *= n1;
    double* dst = bufs[i % 2];
    k_sym_fft<<<(unsigned)ceil_div(A * B, 2 * LB), 256, fsm, st>>>(src, dst, A, n1, B, K, logm[i], LB,
                                                                     twiddles64(logm[i]));
    FRAC_CUDA_TRY(cudaGetLastError());
    src = dst;
    B *= K;
  }
  return FRAC_OK;
}

// Reads and clears the record of a failed self-check in this file's kernels.
int take_coeff_fault() {
  unsigned long long line = 0;
  long long index = 0;
  FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&line, g_fault_line, sizeof(line)));
  if (!line) return FRAC_OK;
  FRAC_CUDA_TRY(cudaMemcpyFromSymbol(&index, g_fault_index, sizeof(index)));
  const unsigned long long zero = 0;
  FRAC_CUDA_TRY(cudaMemcpyToSymbol(g_fault_line, &zero, sizeof(zero)));
  return record_check_failure("coeffs.cu", (int)line, index);
}

}  // namespace frac
