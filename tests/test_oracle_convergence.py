"""Pins of the oracle where the paper prints no numbers: 3D and 2D (p = 0, 2)
apply errors against the closed form of (-Delta)^{alpha/2}(1-|x|^2)_+^s, and
the tempered operator (Remark 2.2) against a direct quadrature of its
definition.  Rates follow Remark 3.2: O(h^2) for p <= 1, O(h^4) for p = 2."""
import math
import warnings

import numpy as np
import pytest
from scipy import integrate

from oracle import frac_oracle as O


def _rates(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("p,alpha", [(1, 0.5), (1, 1.5), (2, 0.5), (2, 1.5), (0, 1.0)])
def test_3d_apply_converges_to_closed_form(p, alpha):
    s = 6.5
    errs = []
    for N in (8, 16, 32):
        a, c, h = O.build_operator(3, N, alpha, p, q=10)
        n = N - 1
        u = np.clip(1 - O.radius2(N, 3), 0, None) ** s
        y = O.apply_rows(a, c, u, np.array([[n // 2] * 3]))[0]
        errs.append(abs(y - O.fl_ball_power(3, alpha, s, 0.0)))
    r = _rates(errs)
    want = 4.0 if p == 2 else 2.0
    assert all(ri > want - 0.25 for ri in r), (errs, r)


@pytest.mark.parametrize("p,alpha", [(0, 0.7), (0, 1.6), (2, 0.4), (2, 1.0), (2, 1.6)])
def test_2d_apply_converges_to_closed_form(p, alpha):
    """Off-centre point (0, 0.5).  For d >= 2, Phi(x, xi) depends on the
    direction of xi as xi -> 0, so its interpolation on the origin element is
    accurate only to O(h^2) there, an O(h^{4-alpha}) contribution after
    weighting by mu; with p = 2 that caps the rate at 4 - alpha (the leading
    anisotropic term cancels by symmetry).  p <= 1 keeps O(h^2)."""
    s = 6.5
    errs = []
    for N in (16, 32, 64, 128):
        a, c, h = O.build_operator(2, N, alpha, p)
        n = N - 1
        r2 = O.radius2(N, 2)
        u = np.clip(1 - r2, 0, None) ** s
        rows = np.array([[n // 2, 3 * N // 4 - 1]])
        y = O.apply_rows(a, c, u, rows)
        errs.append(abs(y[0] - O.fl_ball_power(2, alpha, s, r2[tuple(rows.T)])[0]))
    r = _rates(errs)
    want = (4.0 - alpha) if p == 2 else 2.0
    assert all(abs(ri - want) < 0.3 for ri in r[1:]), (errs, r)


def _tempered_exact(alpha, lam, x, s=4):
    """-c int_0^inf (u(x+xi) - 2u(x) + u(x-xi)) e^{-lam xi} xi^{-1-alpha} dxi, u = (1-x^2)_+^s."""
    u = lambda z: max(0.0, 1 - z * z) ** s  # noqa: E731
    f = lambda xi: (u(x + xi) - 2 * u(x) + u(x - xi)) * math.exp(-lam * xi) * xi ** (-1 - alpha)  # noqa: E731
    pts = [0.0] + sorted({1 - abs(x), 1 + abs(x)})
    kw = dict(epsabs=1e-15, epsrel=1e-13, limit=400)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        v = sum(integrate.quad(f, pts[i], pts[i + 1], **kw)[0] for i in range(len(pts) - 1))
        v += integrate.quad(lambda xi: -2 * u(x) * math.exp(-lam * xi) * xi ** (-1 - alpha),
                            pts[-1], np.inf, **kw)[0]
    return -O.c_dalpha(1, alpha) * v


@pytest.mark.parametrize("p", [0, 1, 2])
@pytest.mark.parametrize("alpha,lam", [(0.6, 0.5), (1.5, 1.0)])
def test_tempered_1d_apply_converges_to_definition(p, alpha, lam):
    errs = []
    for N in (16, 32, 64, 128):
        a, c, h = O.build_operator(1, N, alpha, p, lam)
        x = O.interior_points(N)
        y = O.apply_dense(a, c, np.clip(1 - x * x, 0, None) ** 4)
        idx = (N // 2 - 1, 3 * N // 4 - 1)
        errs.append(max(abs(y[i] - _tempered_exact(alpha, lam, x[i])) for i in idx))
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[0] / errs[-1] > (1000 if p == 2 else 40), errs


def test_tempered_lambda_zero_is_fractional_laplacian():
    """lambda -> 0 recovers the fractional Laplacian (Example 3.2.2)."""
    for d, p in ((1, 2), (2, 1)):
        N = 8
        a0 = O.stencil(d, N, 2.0 / N, 0.9, p, 0.0)
        a1 = O.stencil(d, N, 2.0 / N, 0.9, p, 1e-9)
        assert np.allclose(a0, a1, rtol=1e-7, atol=0)


def test_synth_rhs_matches_oracle_closed_form():
    """Inside the unit ball the workload right-hand side (polynomial, s = 1 +
    alpha/2) equals the oracle's 2F1 closed form, which holds for |x| < 1 only;
    the cube corners outside the ball are checked against the definition below."""
    import synth
    for d in (1, 2, 3):
        for alpha in (0.4, 1.6):
            n = 15
            f = synth.ball_power_rhs(d, n, alpha)
            r2 = synth.radius2(d, n)
            inside = r2 < 1.0
            assert inside.sum() > n ** d // 2
            ref = O.fl_ball_power(d, alpha, 1 + alpha / 2, r2[inside])
            assert np.allclose(f[inside], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d,alpha", [(2, 0.7), (3, 0.7), (3, 1.6)])
def test_synth_rhs_outside_ball_matches_definition(d, alpha):
    """At the cube corners (|x| > 1, where u = 0) the workload right-hand side
    must equal -c int_{|y|<1} u(y) |x-y|^{-d-alpha} dy (Eq. (fL-nD)); brute-force
    cubature over the ball in polar / spherical coordinates here."""
    import synth
    s = 1 + alpha / 2
    c = O.c_dalpha(d, alpha)
    fn = synth._outside_ball(d, alpha, s)
    for r in (1.05, 1.3):
        if d == 2:
            g = lambda ph, rho: rho * (1 - rho * rho) ** s * (r * r + rho * rho - 2 * r * rho * math.cos(ph)) ** (-(2 + alpha) / 2)  # noqa: E731
            ref = -c * integrate.dblquad(g, 0, 1, 0, 2 * math.pi, epsabs=0, epsrel=1e-9)[0]
        else:
            g = lambda th, rho: 2 * math.pi * rho * rho * math.sin(th) * (1 - rho * rho) ** s * (r * r + rho * rho - 2 * r * rho * math.cos(th)) ** (-(3 + alpha) / 2)  # noqa: E731
            ref = -c * integrate.dblquad(g, 0, 1, 0, math.pi, epsabs=0, epsrel=1e-9)[0]
        assert abs(float(fn(r)) - ref) <= 1e-5 * abs(ref), (r, float(fn(r)), ref)
