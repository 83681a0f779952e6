"""Pins of the oracle's weight integrals and stencil against closed forms,
exactness identities and an independent quadrature (no GPU)."""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import frac_oracle as O


# ---------------------------------------------------------------------------
# Independent reference: int over [0, L]^d of P(xi) |xi|^{2-d-alpha} e^{-lam |xi|},
# P homogeneous of degree k, in polar / spherical coordinates with QUADPACK.
# ---------------------------------------------------------------------------

def _radial(alpha, lam, k, R):
    a = 2.0 - alpha + k          # r^{d-1} r^{2-d-alpha} r^k = r^{a-1}
    if lam == 0.0:
        return R ** a / a
    v, _ = integrate.quad(lambda r: math.exp(-lam * r), 0.0, R, weight="alg", wvar=(a - 1.0, 0.0),
                          epsabs=0.0, epsrel=1e-13)
    return v


def cube_moment(d, alpha, lam, L, P, k):
    q = dict(epsabs=0.0, epsrel=1e-12, limit=200)
    if d == 1:
        return P(np.array([1.0])) * _radial(alpha, lam, k, L)
    if d == 2:
        def f(t):
            dv = np.array([math.cos(t), math.sin(t)])
            return P(dv) * _radial(alpha, lam, k, L / max(dv))
        return sum(integrate.quad(f, lo, hi, **q)[0] for lo, hi in ((0, math.pi / 4), (math.pi / 4, math.pi / 2)))
    assert lam == 0.0

    def f(ph, th):
        dv = np.array([math.sin(ph) * math.cos(th), math.sin(ph) * math.sin(th), math.cos(ph)])
        return P(dv) * _radial(alpha, lam, k, L / max(dv)) * math.sin(ph)
    tot = 0.0
    for lo, hi in ((0, math.pi / 4), (math.pi / 4, math.pi / 2)):
        phs = lambda th: math.atan(1.0 / max(math.cos(th), math.sin(th)))  # noqa: E731
        tot += integrate.dblquad(f, lo, hi, 0.0, phs, epsabs=0.0, epsrel=1e-11)[0]
        tot += integrate.dblquad(f, lo, hi, phs, math.pi / 2, epsabs=0.0, epsrel=1e-11)[0]
    return tot


def _nodes(N, h, d):
    return [g * h for g in np.indices((N + 1,) * d)]


# ---------------------------------------------------------------------------
# 1D closed forms (Appendix) versus the oracle's quadrature of Eq. (wi-1D)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [0, 1, 2])
@pytest.mark.parametrize("alpha", [0.3, 1.0, 1.7])
@pytest.mark.parametrize("N", [4, 16, 64])
def test_appendix_closed_forms(p, alpha, N):
    h = 2.0 / N
    w = O.weights(1, N, h, alpha, p)
    wa = O.weights_1d_appendix(N, h, alpha, p)
    # the closed forms are differences of powers xi^{sigma} that cancel to
    # O(k^{-(p+1)}) of their terms; the quadrature does not cancel (checked
    # against 40-digit mpmath in test_weights_1d_against_mpmath)
    k = np.arange(N + 1)
    scale = np.maximum(np.abs(wa), np.abs(wa[1]))   # omega_0 (p = 2) also cancels
    tol = 64 * np.finfo(float).eps * (k + 1.0) ** (p + 1) * scale
    assert np.all(np.abs(w - wa) <= tol)


def test_appendix_as_printed_is_wrong_for_p2():
    """The printed even-k formula (xi_{k-1/2}, xi_{k+1/2}) disagrees with Eq. (wi-1D);
    the corrected one (xi_{k-3/2}, xi_{k+3/2}) is what the oracle pins above."""
    N, alpha = 8, 0.7
    h = 2.0 / N
    s0 = 2 - alpha
    s1, s2 = s0 + 1, s0 + 2
    k = 4
    xi = lambda t: t * h  # noqa: E731
    printed = ((xi(k + 2) ** s2 - xi(k - 2) ** s2) / s2
               - 2.0 / s1 * (xi(k - 0.5) * (xi(k) ** s1 - xi(k - 2) ** s1) + xi(k + 0.5) * (xi(k + 2) ** s1 - xi(k) ** s1))
               + 1.0 / s0 * (xi(k - 2) * xi(k - 1) * (xi(k) ** s0 - xi(k - 2) ** s0)
                             + xi(k + 2) * xi(k + 1) * (xi(k + 2) ** s0 - xi(k) ** s0))) / (2 * h * h)
    w = O.weights(1, N, h, alpha, 2)
    assert abs(printed - w[k]) > 0.1 * abs(w[k])


# ---------------------------------------------------------------------------
# Partition of unity and moment exactness:  sum_k omega_k P(xi_k) = int P mu
# for every P the degree-p tensor interpolation reproduces.
# ---------------------------------------------------------------------------

MOMENT_CASES = [(d, p, alpha, lam, N)
                for d in (1, 2, 3) for p in (0, 1, 2) for alpha, lam in ((0.4, 0.0), (1.6, 0.0), (1.1, 0.7))
                for N in (2, 8) if not (d == 3 and lam > 0)]


@pytest.mark.parametrize("d,p,alpha,lam,N", MOMENT_CASES)
def test_weight_moments(d, p, alpha, lam, N):
    L, h = 2.0, 2.0 / N
    w = O.weights(d, N, h, alpha, p, lam)
    X = _nodes(N, h, d)
    tol = 1e-11 if d < 3 else 1e-9
    ref0 = cube_moment(d, alpha, lam, L, lambda v: 1.0, 0)
    assert abs(w.sum() - ref0) <= tol * ref0
    if p >= 1:
        ref1 = cube_moment(d, alpha, lam, L, lambda v: v[0], 1)
        assert abs(np.sum(w * X[0]) - ref1) <= tol * ref1
    if p == 2:
        ref2 = cube_moment(d, alpha, lam, L, lambda v: v[0] ** 2, 2)
        assert abs(np.sum(w * X[0] ** 2) - ref2) <= tol * ref2
        if d >= 2:
            ref11 = cube_moment(d, alpha, lam, L, lambda v: v[0] * v[1], 2)
            assert abs(np.sum(w * X[0] * X[1]) - ref11) <= tol * ref11


@pytest.mark.parametrize("d", [2, 3])
def test_weights_permutation_symmetric(d):
    w = O.weights(d, 6, 2.0 / 6, 0.9, 2, 0.3)
    for perm in itertools.permutations(range(d)):
        assert np.allclose(w, np.transpose(w, perm), rtol=5e-14, atol=0)


def test_weights_quadrature_order_converged():
    for d, p in ((2, 0), (2, 2), (3, 1)):
        N = 6
        w20 = O.weights(d, N, 2.0 / N, 1.3, p, 0.5, q=20)
        w30 = O.weights(d, N, 2.0 / N, 1.3, p, 0.5, q=30)
        assert np.max(np.abs(w20 - w30)) <= 1e-14 * np.max(np.abs(w30))


def test_weights_1d_against_mpmath():
    """omega_k^2 by exact antiderivatives of polynomial * xi^{1-alpha} in
    40-digit arithmetic (no cancellation at that precision)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    N, al = 64, 1.7
    w = O.weights(1, N, 2.0 / N, al, 2)
    H = mpmath.mpf(2) / N
    a = 1 - mpmath.mpf(al)
    for k in (0, 1, 2, 33, 62, 63, 64):
        ref = mpmath.mpf(0)
        for m in range(N // 2):
            if not 2 * m <= k <= 2 * m + 2:
                continue
            pts = [2 * m * H, (2 * m + 1) * H, (2 * m + 2) * H]
            t = k - 2 * m
            o = [pts[s] for s in range(3) if s != t]
            den = (pts[t] - o[0]) * (pts[t] - o[1])
            coef = [o[0] * o[1] / den, -(o[0] + o[1]) / den, 1 / den]   # ascending powers
            for j, cj in enumerate(coef):
                e = a + j + 1
                ref += cj * (pts[2] ** e - pts[0] ** e) / e
        assert abs(w[k] - float(ref)) <= 1e-14 * abs(float(ref)), (k, w[k], float(ref))


def test_weights_2d_against_mpmath():
    """A few 2D tempered p = 1 weights by mpmath tanh-sinh quadrature, element
    by element (the origin element in polar coordinates, radial part exact)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 20
    N, alpha, lam = 4, 0.7, 0.5
    h = 2.0 / N
    w = O.weights(2, N, h, alpha, 1, lam)
    H = mpmath.mpf(h)
    al, la = mpmath.mpf(alpha), mpmath.mpf(lam)

    def hat(k, x):
        return max(mpmath.mpf(0), 1 - abs(x / H - k))

    for k in [(1, 1), (2, 3), (4, 0)]:
        def f(x, y):
            r = mpmath.sqrt(x * x + y * y)
            return hat(k[0], x) * hat(k[1], y) * r ** (-al) * mpmath.exp(-la * r)
        ref = 0
        for i in (k[0] - 1, k[0]):
            for j in (k[1] - 1, k[1]):
                if 0 <= i < N and 0 <= j < N:
                    ref += mpmath.quad(f, [i * H, (i + 1) * H], [j * H, (j + 1) * H])
        assert abs(w[k] - float(ref)) <= 1e-13 * abs(float(ref)), (k, w[k], float(ref))


# ---------------------------------------------------------------------------
# Stencil identities
# ---------------------------------------------------------------------------

def _offset_sum(a, N, h, fn):
    """sum over o in [-N, N]^d, o != 0, of a_{|o|} fn(|o h|^2)."""
    d = a.ndim
    K = np.indices(a.shape)
    mult = 2.0 ** np.sum(K > 0, axis=0)
    r2 = np.sum(K * K, axis=0) * h * h
    m = r2 > 0
    return float(np.sum((mult * a * fn(r2))[m]))


STENCIL_CASES = [(d, p, alpha, lam) for d in (1, 2, 3) for p in (0, 1, 2)
                 for alpha, lam in ((0.5, 0.0), (1.5, 0.0), (1.2, 0.9)) if not (d == 3 and lam > 0)]


@pytest.mark.parametrize("d,p,alpha,lam", STENCIL_CASES)
def test_stencil_quadratic_exactness(d, p, alpha, lam):
    """u = |x|^2: Phi(x, xi) = 2^d for every xi, so the near field is exactly
    2^d int_{[0,L]^d} mu (this fixes the 2^{z(k)} multiplicities and the total
    weight of the origin rule in every d)."""
    N = 4
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, p, lam)
    lhs = _offset_sum(a, N, h, lambda r2: r2)
    ref = 2 ** d * cube_moment(d, alpha, lam, 2.0, lambda v: 1.0, 0)
    assert abs(lhs - ref) <= 2e-9 * ref


@pytest.mark.parametrize("d", [1, 2, 3])
def test_stencil_quartic_exactness_p2(d):
    """u = |x|^4 at x = 0: Phi(0, xi) = 2^d |xi|^2, reproduced by quadratic
    interpolation; the origin rule (4/3, -1/3) gives Phi(0, 0) = 0 exactly."""
    N, alpha = 4, 0.8
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, 2)
    lhs = _offset_sum(a, N, h, lambda r2: r2 * r2)
    ref = 2 ** d * cube_moment(d, alpha, 0.0, 2.0, lambda v: float(np.sum(v * v)), 2)
    assert abs(lhs - ref) <= 2e-9 * ref


def test_planted_origin_rule_mistake_is_caught(monkeypatch):
    """Plant e = (1,) for p = 2 in the oracle: the quartic identity must fail."""
    monkeypatch.setitem(O.ORIGIN_RULE, 2, (1.0,))
    N, alpha, d = 4, 0.8, 2
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, 2)
    lhs = _offset_sum(a, N, h, lambda r2: r2 * r2)
    ref = 2 ** d * cube_moment(d, alpha, 0.0, 2.0, lambda v: float(np.sum(v * v)), 2)
    assert abs(lhs - ref) > 1e-3 * ref


def test_constant_annihilated():
    for d, p, lam in ((1, 1, 0.0), (2, 2, 0.4), (3, 0, 0.0)):
        N = 6
        a = O.stencil(d, N, 2.0 / N, 1.1, p, lam)
        K = np.indices(a.shape)
        mult = 2.0 ** np.sum(K > 0, axis=0)
        F = O.far_field(d, 1.1, 2.0, lam)
        assert abs(np.sum(mult * a) + 2 ** d * F) <= 1e-12 * abs(a[(0,) * d])


def test_far_field_closed_form_1d_and_tempered_quad():
    assert abs(O.far_field(1, 0.7, 2.0) - 1 / (0.7 * 2 ** 0.7)) < 1e-15
    # tempered: b^alpha Gamma(-alpha, b L) with Gamma(s, x), s < 0, from
    # scipy's Gamma(s + 2, x) by Gamma(s + 1, x) = s Gamma(s, x) + x^s e^{-x}
    from scipy import special
    for al, lam in ((0.7, 0.3), (1.6, 1.9), (0.2, 0.05)):
        b, L = lam, 2.0
        x, s = b * L, -al
        g2 = special.gammaincc(s + 2, x) * special.gamma(s + 2)
        g1 = (g2 - x ** (s + 1) * math.exp(-x)) / (s + 1)
        ref = b ** al * (g1 - x ** s * math.exp(-x)) / s
        assert abs(O.far_field(1, al, L, lam) - ref) <= 1e-12 * ref
    # alpha = 1: b Gamma(-1, x) = b (e^{-x}/x - E1(x)), x = b L = 1
    ref = 0.5 * (math.exp(-1.0) - special.exp1(1.0))
    assert abs(O.far_field(1, 1.0, 2.0, 0.5) - ref) <= 1e-12 * ref
    # 2D, polar: int_0^{pi/2} int_{R(t)}^inf r^{-1-alpha} = int (R(t))^{-alpha}/alpha dt
    al = 1.3
    ref = sum(integrate.quad(lambda t: (2.0 / max(math.cos(t), math.sin(t))) ** (-al) / al, lo, hi,
                             epsabs=0, epsrel=1e-13)[0] for lo, hi in ((0, math.pi / 4), (math.pi / 4, math.pi / 2)))
    assert abs(O.far_field(2, al, 2.0) - ref) <= 1e-12 * ref


def test_alpha_one_p0_equals_p1_1d():
    """At alpha = 1 the p = 0 and p = 1 matrices coincide (Sec. 3.1, Example 3.2.1)."""
    for N in (8, 32):
        a0 = O.stencil(1, N, 2.0 / N, 1.0, 0)
        a1 = O.stencil(1, N, 2.0 / N, 1.0, 1)
        assert np.allclose(a0, a1, rtol=1e-13, atol=0)


@pytest.mark.parametrize("d,N", [(1, 64), (2, 12), (3, 6)])
@pytest.mark.parametrize("p", [0, 1, 2])
def test_operator_spd(d, N, p):
    for alpha, lam in ((0.2, 0.0), (1.9, 0.0), (1.0, 1.5)):
        a, c, h = O.build_operator(d, N, alpha, p, lam)
        A = O.operator_matrix(a, c, N - 1)
        assert np.array_equal(A, A.T)
        np.linalg.cholesky(A)


def test_2d_matrix_from_printed_index_ranges():
    """Assemble A^{(2)} from the explicit sums of Eq. (2D-scheme) and compare
    with the multilevel Toeplitz matrix built from the generator."""
    N, alpha = 6, 1.3
    a, c, h = O.build_operator(2, N, alpha, 1)
    n = N - 1
    A = np.zeros((n * n, n * n))
    idx = lambda i, j: (i - 1) * n + (j - 1)  # noqa: E731
    for i in range(1, N):
        for j in range(1, N):
            row = idx(i, j)
            A[row, row] += a[0, 0]
            for k in range(0, i):
                for l in range(0, j):
                    if k + l:
                        A[row, idx(i - k, j - l)] += a[k, l]
                for l in range(1, N - j):
                    A[row, idx(i - k, j + l)] += a[k, l]
            for k in range(1, N - i):
                for l in range(0, j):
                    A[row, idx(i + k, j - l)] += a[k, l]
                for l in range(1, N - j):
                    A[row, idx(i + k, j + l)] += a[k, l]
    assert np.allclose(-c * A, O.operator_matrix(a, c, n), rtol=1e-15, atol=0)


@pytest.mark.parametrize("d,N,p", [(1, 8, 0), (1, 8, 2), (2, 6, 1), (2, 6, 2), (3, 4, 0), (3, 4, 1), (3, 4, 2)])
def test_definition_level_sum(d, N, p):
    """Evaluate Eq. (FL3) / Eq. (2D-scheme0) directly: sum_k omega_k Phi(x_i, xi_k)
    with Phi from grid values (g = 0 outside), the origin rule, and the far
    field -2^d F_d u; compare with the folded Toeplitz apply."""
    alpha, lam = 1.2, 0.3
    h = 2.0 / N
    n = N - 1
    w = O.weights(d, N, h, alpha, p, lam)
    a = O.stencil(d, N, h, alpha, p, lam, omega=w)
    c = O.c_dalpha(d, alpha)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((n,) * d)
    U = np.zeros((3 * N + 1,) * d)           # grid values on index range [-N, 2N]
    U[tuple(slice(N + 1, N + 1 + n) for _ in range(d))] = u

    def val(idx):
        return U[tuple(t + N for t in idx)]

    def Phi(i, off):
        s = sum(val(tuple(i[t] + sg[t] * off[t] for t in range(d))) for sg in itertools.product((1, -1), repeat=d))
        return (s - 2 ** d * val(i)) / (h * h * sum(t * t for t in off))

    F = O.far_field(d, alpha, N * h, lam)
    y = np.zeros((n,) * d)
    for ii in itertools.product(range(n), repeat=d):
        i = tuple(t + 1 for t in ii)
        acc = 0.0
        for k in itertools.product(range(N + 1), repeat=d):
            if any(k):
                acc += w[k] * Phi(i, k)
        for ax in range(d):
            for j, ej in enumerate(O.ORIGIN_RULE[p], start=1):
                off = [0] * d
                off[ax] = j
                acc += O.zeta(2.0) * w[(0,) * d] * ej * Phi(i, tuple(off)) / d
        acc += -(2 ** d) * F * val(i)
        y[ii] = -c * acc
    assert np.allclose(y, O.apply_dense(a, c, u), rtol=0, atol=1e-12 * np.max(np.abs(y)))


# ---------------------------------------------------------------------------
# Degrees 3 and 4: moments up to degree p in every d, and the stencil identity
# one even degree up (the origin rules of order 6 and 8 give Phi(0, 0) exactly).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,p,alpha", [(1, 3, 0.4), (1, 4, 1.6), (2, 3, 1.1), (2, 4, 0.4), (3, 3, 1.6), (3, 4, 1.1)])
def test_weight_moments_high_degree(d, p, alpha):
    N = p
    L, h = 2.0, 2.0 / N
    w = O.weights(d, N, h, alpha, p, q=16 if d < 3 else 12)
    X = _nodes(N, h, d)
    tol = 1e-11 if d < 3 else 1e-9
    for k in range(p + 1):
        ref = cube_moment(d, alpha, 0.0, L, lambda v, k=k: v[0] ** k, k)
        assert abs(np.sum(w * X[0] ** k) - ref) <= tol * ref, k
    if d >= 2:
        ref = cube_moment(d, alpha, 0.0, L, lambda v: v[0] ** p * v[1] ** (p - 1), 2 * p - 1)
        assert abs(np.sum(w * X[0] ** p * X[1] ** (p - 1)) - ref) <= tol * ref


@pytest.mark.parametrize("d", [1, 2, 3])
def test_stencil_sextic_exactness_p4(d):
    """u = |x|^6 at x = 0: Phi(0, xi) = 2^d |xi|^4, reproduced by quartic interpolation; the
    eighth-order origin rule gives Phi(0, 0) = 0 exactly (sum e_j j^4 = 0)."""
    N, alpha = 4, 0.8
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, 4, q=16 if d < 3 else 12)
    lhs = _offset_sum(a, N, h, lambda r2: r2 ** 3)
    ref = 2 ** d * cube_moment(d, alpha, 0.0, 2.0, lambda v: float(np.sum(v * v)) ** 2, 4)
    assert abs(lhs - ref) <= 2e-9 * ref


def test_planted_origin_rule_mistake_is_caught_p4(monkeypatch):
    """Plant the fourth-order rule of p = 2 for p = 4: the sextic identity must fail (it
    needs sum e_j j^4 = 0; the eighth-order condition sum e_j j^6 = 0 is pinned by the
    moment conditions of the rules)."""
    monkeypatch.setitem(O.ORIGIN_RULE, 4, O.ORIGIN_RULE[2] + (0.0, 0.0))
    N, alpha, d = 4, 0.8, 1
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, 4)
    lhs = _offset_sum(a, N, h, lambda r2: r2 ** 3)
    ref = 2 ** d * cube_moment(d, alpha, 0.0, 2.0, lambda v: float(np.sum(v * v)) ** 2, 4)
    assert abs(lhs - ref) > 1e-6 * ref


# ---------------------------------------------------------------------------
# The origin element by an independent rule (spherical / polar coordinates with
# QUADPACK, not the Duffy split of the oracle), in 2D and 3D
# ---------------------------------------------------------------------------

def _lagrange_1d(p, h, j):
    """Ascending coefficients of the Lagrange polynomial of node j h on the nodes
    0, h, .., p h (degree p)."""
    c = np.array([1.0])
    for t in range(p + 1):
        if t != j:
            c = np.convolve(c, np.array([-t * h, 1.0])) / ((j - t) * h)
    return c


def _origin_node_polar(d, N, alpha, lam, p, k):
    """omega_k for a node k that only the origin element [0, max(p, 1) h]^d supports,
    as sum over total degrees m of int P_m(xi) |xi|^{2-d-alpha} e^{-lam |xi|} with P_m
    the degree-m part of the basis product (cube_moment: radial part exact or adaptive,
    angles by QUADPACK)."""
    h = 2.0 / N
    pe = max(p, 1)
    polys = [_lagrange_1d(pe, h, int(ki)) for ki in k]
    coef = {}
    for mono in itertools.product(*[range(len(c)) for c in polys]):
        coef[mono] = np.prod([polys[i][m] for i, m in enumerate(mono)])
    tot = 0.0
    for deg in range(sum(len(c) - 1 for c in polys) + 1):
        terms = [(m, v) for m, v in coef.items() if sum(m) == deg and v != 0.0]
        if not terms:
            continue

        def P(dv, terms=terms):
            return sum(v * np.prod(dv ** np.array(m)) for m, v in terms)
        tot += cube_moment(d, alpha, lam, pe * h, P, deg)
    return tot


@pytest.mark.parametrize("d,p,alpha,lam,k", [
    (3, 1, 1.3, 0.0, (0, 0, 0)), (3, 1, 0.4, 0.0, (0, 0, 0)),
    (3, 2, 1.6, 0.0, (0, 0, 0)), (3, 2, 0.7, 0.0, (1, 0, 0)), (3, 2, 1.2, 0.0, (1, 1, 0)),
    (3, 2, 1.9, 0.0, (1, 1, 1)),
    (2, 2, 1.2, 0.0, (0, 0)), (2, 2, 0.5, 0.8, (1, 0)), (2, 2, 1.8, 1.5, (1, 1)),
    (2, 1, 0.9, 0.6, (0, 0)),
])
def test_origin_element_against_polar_quadrature(d, p, alpha, lam, k):
    """The nodes that only the origin element supports (k = 0 for p <= 1, k_i in {0, 1}
    for p = 2): the oracle's Duffy-split weights against spherical (3D) / polar (2D)
    coordinates integrated by QUADPACK, to 1e-12 relative (they agree to ~1e-15)."""
    N = 8
    w = O.weights(d, N, 2.0 / N, alpha, p, lam)
    ref = _origin_node_polar(d, N, alpha, lam, p, k)
    assert abs(w[tuple(k)] - ref) <= 1e-12 * abs(ref), (w[tuple(k)], ref)


def _origin_node_mp(d, N, alpha, p, k, dps=34):
    """omega_k for a node of the origin element of degree p (gamma = 2, lambda = 0) in dps-digit
    arithmetic: the Duffy split of [0, p h]^d with the radial integral of every monomial in
    closed form and the angles by mpmath quadrature (the monomial expansion cancels by up to
    p^{p d} relative, harmless at 34 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    h = mpmath.mpf(2) / N
    H, al = p * h, mpmath.mpf(alpha)

    def lag(j):
        c = [mpmath.mpf(1)]
        for t in range(p + 1):
            if t != j:
                nc = [mpmath.mpf(0)] * (len(c) + 1)
                for i, v in enumerate(c):
                    nc[i] += v * (-t * h)
                    nc[i + 1] += v
                c = [v / ((j - t) * h) for v in nc]
        return c

    polys = [lag(int(ki)) for ki in k]
    tot = mpmath.mpf(0)
    for lead in range(d):
        def f(*s, lead=lead):
            it = iter(s)
            coords = [mpmath.mpf(1) if j == lead else next(it) for j in range(d)]
            P = [mpmath.mpf(1)]
            for j in range(d):
                pj = [polys[j][m] * coords[j] ** m for m in range(p + 1)]
                nP = [mpmath.mpf(0)] * (len(P) + p)
                for a_, va in enumerate(P):
                    for b_, vb in enumerate(pj):
                        nP[a_ + b_] += va * vb
                P = nP
            rad = sum(v * H ** (2 - al + m) / (2 - al + m) for m, v in enumerate(P))
            return rad * mpmath.sqrt(1 + sum(x * x for x in s)) ** (-(d + al - 2))
        tot += mpmath.quad(f, *([[0, 1]] * (d - 1)))
    return float(tot)


@pytest.mark.parametrize("d,p,alpha,k,tol", [
    (2, 3, 0.6, (2, 1), 1e-14), (2, 4, 1.3, (3, 1), 1e-14), (2, 4, 1.9, (0, 0), 1e-14), (3, 4, 0.7, (3, 2, 1), 1e-13),
])
def test_origin_element_high_degree_against_high_precision(d, p, alpha, k, tol):
    """Degrees 3, 4: the origin element's weights (the oracle cuts it into cells of side h
    and integrates the one at the origin by the Duffy split) against the Duffy split of the
    whole element carried out in 34-digit arithmetic; in FP64 that whole-element expansion
    loses up to 6e-11 to cancellation, the cell split does not."""
    N = 4 * p
    w = O.weights(d, N, 2.0 / N, alpha, p)
    ref = _origin_node_mp(d, N, alpha, p, k)
    assert abs(w[k] - ref) <= tol * abs(ref), (w[k], ref)
