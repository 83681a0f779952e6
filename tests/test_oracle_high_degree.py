"""Oracle pins for Lagrange bases of degree p = 3 and 4 (the paper says higher
degrees raise the accuracy further and gives no scheme; the library has none on the
GPU yet).  Weights: the degree-p interpolation reproduces polynomials of degree <= p,
so sum_k omega_k P(xi_k) = int_0^L P(xi) mu(xi) dxi exactly (closed form in 1D,
polar quadrature of the constant in 2D).  Origin rules: the moment conditions of the
second-difference combinations.  Accuracy: convergence on u = 1/(1+x^2) with the
same data outside (the setting of Table 3-1-3): order 4 for p = 3 (the order p = 2
already reaches by superconvergence, with a smaller constant at large alpha) and 6
for p = 4."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import frac_oracle as O


@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("alpha", [0.4, 1.3, 1.8])
def test_weights_integrate_polynomials_of_degree_p_exactly_1d(p, alpha):
    N = 6 * p
    h = 2.0 / N
    L = N * h
    w = O.weights(1, N, h, alpha, p)
    xi = h * np.arange(N + 1)
    for m in range(p + 1):                          # mu = xi^{1-alpha} (gamma = 2, d = 1)
        exact = L ** (m + 2 - alpha) / (m + 2 - alpha)
        assert abs(np.dot(w, xi ** m) - exact) <= 1e-12 * exact, (m, np.dot(w, xi ** m), exact)


@pytest.mark.parametrize("p", [3, 4])
def test_weights_constant_moment_2d(p):
    alpha, N = 1.1, 2 * p
    h = 2.0 / N
    L = N * h
    w = O.weights(2, N, h, alpha, p, q=16)
    # int over [0, L]^2 of |xi|^{-alpha}: polar, r up to L / max(cos, sin)
    f = lambda t: (L / max(math.cos(t), math.sin(t))) ** (2 - alpha) / (2 - alpha)  # noqa: E731
    exact = integrate.quad(f, 0.0, math.pi / 4, epsabs=0, epsrel=1e-13, limit=200)[0] * 2
    assert abs(w.sum() - exact) <= 1e-10 * exact


@pytest.mark.parametrize("p,order", [(0, 2), (1, 2), (2, 4), (3, 6), (4, 8)])
def test_origin_rule_moment_conditions(p, order):
    e = np.array(O.ORIGIN_RULE[p])
    j = np.arange(1, len(e) + 1)
    assert abs(e.sum() - 1.0) < 1e-15
    for m in range(1, order // 2):
        assert abs(np.sum(e * j ** (2 * m))) < 1e-13, m


@pytest.mark.parametrize("p,alpha,rate", [(3, 0.5, 3.8), (3, 1.7, 3.7), (4, 0.5, 5.8), (4, 1.7, 5.6)])
def test_convergence_order_on_smooth_data(p, alpha, rate):
    g = lambda P: 1.0 / (1.0 + P[..., 0] ** 2)  # noqa: E731
    errs = []
    for N in (48, 96, 192):
        N = N // p * p
        a, c, h = O.build_operator(1, N, alpha, p)
        x = O.interior_points(N)
        b = O.boundary_vector(1, N, h, alpha, a, c, g)
        errs.append(np.max(np.abs(O.apply_dense(a, c, 1.0 / (1.0 + x * x)) + b - O.fl_lorentzian_1d(alpha, x))))
    assert math.log2(errs[1] / errs[2]) >= rate, errs


def test_p4_beats_p2_at_equal_grid():
    alpha, N = 1.2, 96
    g = lambda P: 1.0 / (1.0 + P[..., 0] ** 2)  # noqa: E731
    err = {}
    for p in (2, 4):
        a, c, h = O.build_operator(1, N, alpha, p)
        x = O.interior_points(N)
        b = O.boundary_vector(1, N, h, alpha, a, c, g)
        err[p] = np.max(np.abs(O.apply_dense(a, c, 1.0 / (1.0 + x * x)) + b - O.fl_lorentzian_1d(alpha, x)))
    assert err[4] < 1e-2 * err[2], err


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_weights_integrate_tensor_monomials_2d(p):
    """sum_k omega_k xi_1^a xi_2^b = int over [0, L]^2 of xi_1^a xi_2^b |xi|^{-alpha} for
    a, b <= p (the tensor Lagrange interpolation reproduces them); reference by a polar
    integral, r in closed form and theta by adaptive quadrature."""
    alpha, N = 0.7, 2 * p if p > 1 else 3
    h = 2.0 / N
    L = N * h
    w = O.weights(2, N, h, alpha, p, q=16)
    K = np.indices(w.shape) * h
    for a, b in {(0, 0), (1, 0), (p, 1), (p, p), (0, p)}:
        def f(t, a=a, b=b):
            R = L / max(math.cos(t), math.sin(t))
            return math.cos(t) ** a * math.sin(t) ** b * R ** (a + b + 2 - alpha) / (a + b + 2 - alpha)
        exact = sum(integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
                    for lo, hi in ((0.0, math.pi / 4), (math.pi / 4, math.pi / 2)))
        got = float(np.sum(w * K[0] ** a * K[1] ** b))
        assert abs(got - exact) <= 1e-10 * exact, (p, a, b, got, exact)
