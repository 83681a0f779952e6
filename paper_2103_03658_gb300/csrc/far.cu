// Far field of nonhomogeneous exterior data: the g part of Eq. (L2),
//   far_i = sum over the 2^d reflections m of the integral over Upsilon_+^c
//           (R_+^d outside [0, L]^d) of g(x_i + m o xi) |xi|^{-d-alpha} e^{-lambda |xi|} dxi,
// by a fixed quadrature rule whose nodes xi_q do not depend on the grid point:
// the caller evaluates g at the points x_i + m o xi_q that the library lists
// (frac_far_points, on the device) and the library forms the weighted sums
// (frac_far_sum).  The C ABI cannot carry a function, so the evaluation of g is
// handed back to the caller between the two calls (reverse communication).
//
// Rule: the region is the union of the d pyramids in which coordinate k is the
// largest, xi = rho (1, s) with coordinate k in front, rho > L, s in [0, 1]^{d-1},
// dxi = rho^{d-1} drho ds; with rho = L / t,
//   int_L^inf rho^{-1-alpha} G(rho) drho = L^{-alpha} int_0^1 t^{alpha-1} G(L / t) dt,
// so t takes an nr-point Gauss-Jacobi rule for the weight t^{alpha-1} (exact for
// the power singularity of the kernel) and every s_j an ns-point Gauss-Legendre
// rule; |xi|^{-d-alpha} = rho^{-d-alpha} |(1, s)|^{-d-alpha}.  The rules come from
// the eigenvalues of the Jacobi matrices of the two families (Golub and Welsch,
// Math. Comp. 23 (1969)), computed here in FP64 on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace frac {
namespace {

// Eigenvalues of the symmetric tridiagonal matrix (diag a[0..n), off-diagonal
// b[0..n-1)) and the squares of the first components of its normalised
// eigenvectors, by implicit QL sweeps with Wilkinson shifts; the first row of
// the accumulated rotations is all that is kept.
bool tridiag_first_row(std::vector<double>& a, std::vector<double> b, std::vector<double>& z2) {
  const int n = (int)a.size();
  b.resize(n, 0.0);
  std::vector<double> z(n, 0.0);  // first row of the eigenvector matrix
  z[0] = 1.0;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::fabs(a[m]) + std::fabs(a[m + 1]);
        if (std::fabs(b[m]) + dd == dd) break;  // negligible against its neighbours in FP64
      }
      if (m == l) break;
      if (iter == 60) return false;
      // Wilkinson shift from the leading 2x2 block
      double g = (a[l + 1] - a[l]) / (2.0 * b[l]);
      double r = std::hypot(g, 1.0);
      g = a[m] - a[l] + b[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * b[i];
        const double bb = c * b[i];
        r = std::hypot(f, g);
        b[i + 1] = r;
        if (r == 0.0) {  // the off-diagonal entry vanished: deflate
          a[i + 1] -= p;
          b[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = a[i + 1] - p;
        r = (a[i] - g) * s + 2.0 * c * bb;
        p = s * r;
        a[i + 1] = g + p;
        g = c * r - bb;
        f = z[i + 1];
        z[i + 1] = s * z[i] + c * f;
        z[i] = c * z[i] - s * f;
      }
      if (r == 0.0 && i >= l) continue;
      a[l] -= p;
      b[l] = g;
      b[m] = 0.0;
    }
  }
  z2.resize(n);
  for (int k = 0; k < n; ++k) z2[k] = z[k] * z[k];
  return true;
}

// Gauss rule of the weight (1 - x)^ja (1 + x)^jb on [-1, 1] (Legendre: 0, 0).
bool jacobi_rule(int q, double ja, double jb, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> a(q), b(q > 1 ? q - 1 : 0);
  const double ab = ja + jb;
  for (int k = 0; k < q; ++k) {
    const double s = 2.0 * k + ab;
    a[k] = k == 0 ? (jb - ja) / (ab + 2.0) : (jb * jb - ja * ja) / (s * (s + 2.0));
  }
  for (int k = 1; k < q; ++k) {
    const double s = 2.0 * k + ab;
    const double num = 4.0 * k * (k + ja) * (k + jb) * (k + ab);
    b[k - 1] = std::sqrt(num / (s * s * (s + 1.0) * (s - 1.0)));
  }
  std::vector<double> z2;
  if (!tridiag_first_row(a, b, z2)) return false;
  // total mass of the weight: 2^{ja+jb+1} Gamma(ja+1) Gamma(jb+1) / Gamma(ja+jb+2)
  const double mu0 = std::pow(2.0, ab + 1.0) * std::tgamma(ja + 1.0) * std::tgamma(jb + 1.0) / std::tgamma(ab + 2.0);
  std::vector<int> ord(q);
  for (int k = 0; k < q; ++k) ord[k] = k;
  for (int i = 1; i < q; ++i)  // ascending nodes
    for (int j = i; j > 0 && a[ord[j]] < a[ord[j - 1]]; --j) std::swap(ord[j], ord[j - 1]);
  x.resize(q);
  w.resize(q);
  for (int k = 0; k < q; ++k) {
    x[k] = a[ord[k]];
    w[k] = mu0 * z2[ord[k]];
  }
  return true;
}

__global__ void k_far_points(const double* __restrict__ xi, int64_t nq, int d, int64_t n0, int64_t n1, double h,
                             double lo0, double lo1, double lo2, int64_t first, int64_t count,
                             double* __restrict__ pts) {
  const int64_t per = ((int64_t)1 << d) * nq;  // values per grid point
  const int64_t total = count * per;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / per, r = t - p * per;
    const int m = (int)(r / nq);
    const int64_t q = r - (int64_t)m * nq;
    const int64_t flat = first + p;  // axis 0 fastest
    const int64_t j0 = flat % n0, j1 = (flat / n0) % n1, j2 = flat / (n0 * n1);
    const double x[3] = {lo0 + (double)(j0 + 1) * h, lo1 + (double)(j1 + 1) * h, lo2 + (double)(j2 + 1) * h};
    for (int k = 0; k < d; ++k) {
      const double sg = (m >> k) & 1 ? -1.0 : 1.0;
      pts[t * d + k] = x[k] + sg * xi[q * d + k];
    }
  }
}

// far[p] = sum over the 2^d reflections and the nq nodes of w_q g, one block per
// point, per-thread sums in a fixed order then a fixed-shape tree: deterministic.
__global__ void __launch_bounds__(256) k_far_sum(const double* __restrict__ w, int64_t nq, int d,
                                                 const double* __restrict__ g, int64_t count,
                                                 double* __restrict__ far) {
  __shared__ double red[256];
  const int64_t per = ((int64_t)1 << d) * nq;
  for (int64_t p = blockIdx.x; p < count; p += gridDim.x) {
    const double* gp = g + p * per;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < per; r += blockDim.x) s += w[r % nq] * gp[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) far[p] = red[0];
    __syncthreads();
  }
}

}  // namespace

// The node set of the library's far-field rule (host).
int far_rule(int d, double alpha, double lam, double L, int nr, int ns, std::vector<double>& xi,
             std::vector<double>& w) {
  if (d < 1 || d > 3 || !(alpha > 0.0 && alpha < 2.0) || !(lam >= 0.0) || !std::isfinite(lam) || !(L > 0.0) ||
      !std::isfinite(L) || nr < 1 || nr > 512 || ns < 1 || ns > 512)
    return FRAC_EINVAL;
  std::vector<double> tx, tw, sx, sw;
  if (!jacobi_rule(nr, 0.0, alpha - 1.0, tx, tw)) return FRAC_ECUDA;
  if (d > 1 && !jacobi_rule(ns, 0.0, 0.0, sx, sw)) return FRAC_ECUDA;
  const double La = std::pow(L, -alpha), half_a = std::pow(0.5, alpha);
  int64_t nang = 1;
  for (int k = 1; k < d; ++k) nang *= ns;
  xi.clear();
  w.clear();
  xi.reserve((size_t)d * nang * nr * d);
  w.reserve((size_t)d * nang * nr);
  for (int lead = 0; lead < d; ++lead)  // pyramid: coordinate `lead` is the largest
    for (int64_t a = 0; a < nang; ++a) {
      double s[3] = {0, 0, 0}, ws = 1.0, c2 = 1.0;
      int64_t rem = a;
      for (int k = 0; k < d - 1; ++k) {
        const int i = (int)(rem % ns);
        rem /= ns;
        s[k] = 0.5 * (sx[i] + 1.0);
        ws *= 0.5 * sw[i];
        c2 += s[k] * s[k];
      }
      const double cs = std::sqrt(c2);
      for (int it = 0; it < nr; ++it) {
        const double t = 0.5 * (tx[it] + 1.0), rho = L / t;
        int k = 0;
        for (int ax = 0; ax < d; ++ax) xi.push_back(ax == lead ? rho : rho * s[k++]);
        w.push_back(La * half_a * tw[it] * ws * std::pow(cs, -(double)d - alpha) * std::exp(-lam * rho * cs));
      }
    }
  return FRAC_OK;
}

}  // namespace frac

using namespace frac;

extern "C" int frac_far_nodes(int32_t d, double alpha, double lambda, double L, int32_t nr, int32_t ns, double* xi,
                              double* w, int64_t* count) {
  if (!count) return FRAC_EINVAL;
  std::vector<double> X, W;
  FRAC_TRY(far_rule(d, alpha, lambda, L, nr, ns, X, W));
  *count = (int64_t)W.size();
  if (xi) std::copy(X.begin(), X.end(), xi);
  if (w) std::copy(W.begin(), W.end(), w);
  return FRAC_OK;
}

extern "C" int frac_far_points(const frac_op* op, const double* lo, const double* xi, int64_t nq, int64_t first,
                               int64_t count, double* pts, void* stream) {
  if (!op || !lo || !xi || !pts || nq < 1 || first < 0 || count < 0 || first + count > op->nd) return FRAC_EINVAL;
  if (count == 0) return FRAC_OK;
  if (!op_on_current_device(op) || ptr_kind(xi) != PTR_DEVICE || ptr_kind(pts) != PTR_DEVICE) {
    record_detail("frac_far_points: xi and pts must be device buffers of the operator's device");
    return FRAC_EINVAL;
  }
  const int d = op->prob.d;
  const int64_t total = count * ((int64_t)1 << d) * nq;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 64);
  k_far_points<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      xi, nq, d, op->na[0], op->na[1], op->prob.h, lo[0], d > 1 ? lo[1] : 0.0, d > 2 ? lo[2] : 0.0, first, count,
      pts);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}

extern "C" int frac_far_sum(const frac_op* op, const double* w, int64_t nq, const double* g, int64_t count,
                            double* far, void* stream) {
  if (!op || !w || !g || !far || nq < 1 || count < 0 || count > op->nd) return FRAC_EINVAL;
  if (count == 0) return FRAC_OK;
  if (!op_on_current_device(op) || ptr_kind(w) != PTR_DEVICE || ptr_kind(g) != PTR_DEVICE ||
      ptr_kind(far) != PTR_DEVICE) {
    record_detail("frac_far_sum: w, g and far must be device buffers of the operator's device");
    return FRAC_EINVAL;
  }
  const int64_t blocks = std::min<int64_t>(count, 152 * 16);
  k_far_sum<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(w, nq, op->prob.d, g, count, far);
  FRAC_CUDA_TRY(cudaGetLastError());
  return FRAC_OK;
}
