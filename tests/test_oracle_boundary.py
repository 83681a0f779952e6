"""Oracle pins for the boundary vector of nonhomogeneous exterior data (Eq. (L2)):
its near-field part (the generator against the exterior grid samples) and its
far-field part (integrals of g over the far region).

* Constants are annihilated: with u = 1 inside and g = 1 outside, the scheme's
  value at every interior point is -c (sum of all a_{|o|}, o in [-N, N]^d, plus
  the far integrals), and a_0 is defined so that the sum of all a_{|o|} is
  -2^d F_d; so T 1 + near(1) = -2^d F_d at every point.  A wrong offset, a
  missing or doubled term in the near-field sum breaks this.
* The far part of g = 1 is 2^d F_d, computed by a different quadrature
  (``far_field``) than ``boundary_far``'s rays.
* Brute force: the near field as a loop over every exterior grid point within
  reach of each interior point (not over offsets).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import frac_oracle as O


@pytest.mark.parametrize("d,N,p,alpha,lam", [(1, 8, 1, 1.2, 0.0), (1, 12, 2, 0.6, 0.0), (2, 6, 1, 1.5, 0.0),
                                             (2, 5, 0, 0.8, 0.7), (3, 4, 1, 1.1, 0.0)])
def test_near_field_of_constant_completes_the_generator_sum(d, N, p, alpha, lam):
    if p == 2 and N % 2:
        pytest.skip("p = 2 needs N even")
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, p, lam, q=20 if d < 3 else 12)
    G = O.extended_samples(d, N, h, lambda P: np.ones(P.shape[:-1]))
    near = O.boundary_near(a, G)
    n = N - 1
    T1 = (O.toeplitz_matrix(a, n) @ np.ones(n ** d)).reshape((n,) * d)
    F = O.far_field(d, alpha, N * h, lam)
    assert np.allclose(T1 + near, -(2.0 ** d) * F, rtol=0, atol=1e-12 * np.abs(a).sum())


@pytest.mark.parametrize("d,alpha,lam", [(1, 0.5, 0.0), (1, 1.7, 0.0), (2, 1.2, 0.0), (2, 0.9, 0.5), (3, 1.4, 0.0)])
def test_far_part_of_constant_is_the_far_field_constant(d, alpha, lam):
    N = 4
    h = 2.0 / N
    far = O.boundary_far(d, N, h, alpha, lambda P: np.ones(P.shape[:-1]), lam, nq=48 if d == 3 else 96)
    F = O.far_field(d, alpha, N * h, lam)
    assert np.allclose(far, (2.0 ** d) * F, rtol=1e-9, atol=0)


@pytest.mark.parametrize("d,N", [(1, 6), (2, 4), (3, 3)])
def test_near_field_equals_brute_force_over_exterior_points(d, N):
    rng = np.random.default_rng(11 + d)
    a = rng.standard_normal((N + 1,) * d)
    G = rng.standard_normal((3 * N - 1,) * d)
    ext = np.arange(1 - N, 2 * N)
    for e in itertools.product(range(len(ext)), repeat=d):     # interior samples are never read
        if all(1 <= ext[t] <= N - 1 for t in e):
            G[e] = 0.0
    n = N - 1
    ref = np.zeros((n,) * d)
    for i in itertools.product(range(1, N), repeat=d):
        s = 0.0
        for e in itertools.product(range(len(ext)), repeat=d):
            x = tuple(int(ext[t]) for t in e)
            if all(1 <= xt <= N - 1 for xt in x):
                continue                                        # interior: the unknown, not g
            o = tuple(abs(x[t] - i[t]) for t in range(d))
            if max(o) <= N:
                s += a[o] * G[e]
        ref[tuple(t - 1 for t in i)] = s
    assert np.allclose(O.boundary_near(a, G), ref, rtol=1e-13, atol=1e-13)


def test_boundary_vector_is_minus_c_near_plus_far():
    d, N, alpha = 2, 6, 1.3
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, 1)
    c = O.c_dalpha(d, alpha)
    g = lambda P: np.exp(-np.sum(P * P, axis=-1))  # noqa: E731
    b = O.boundary_vector(d, N, h, alpha, a, c, g)
    near = O.boundary_near(a, O.extended_samples(d, N, h, g))
    far = O.boundary_far(d, N, h, alpha, g)
    assert np.allclose(b, -c * (near + far), rtol=1e-15, atol=0)


@pytest.mark.parametrize("d,shape,p,alpha", [(2, (7, 3), 1, 1.2), (2, (4, 9), 0, 0.7), (3, (5, 2, 3), 1, 1.5)])
def test_rectangular_near_field_completes_the_generator_sum(d, shape, p, alpha):
    """Rectangular grids (N_2 < N_1): the generator's cube has side N h with N = max n_i + 1,
    so g is sampled on [1-N, n_i+N] per axis; constants are still annihilated."""
    N = max(shape) + 1
    h = 2.0 / N
    a = O.stencil(d, N, h, alpha, p, q=12)
    G = O.extended_samples(d, N, h, lambda P: np.ones(P.shape[:-1]), shape=shape)
    assert G.shape == tuple(m + 2 * N for m in shape)
    near = O.boundary_near(a, G)
    T1 = (O.toeplitz_matrix(a, shape) @ np.ones(int(np.prod(shape)))).reshape(shape)
    F = O.far_field(d, alpha, N * h)
    assert np.allclose(T1 + near, -(2.0 ** d) * F, rtol=0, atol=1e-12 * np.abs(a).sum())
    far = O.boundary_far(d, N, h, alpha, lambda P: np.ones(P.shape[:-1]), nq=48, shape=shape)
    assert np.allclose(far, (2.0 ** d) * F, rtol=1e-9, atol=0)


def test_rectangular_near_field_equals_brute_force():
    d, shape = 2, (4, 2)
    N = max(shape) + 1
    rng = np.random.default_rng(3)
    a = rng.standard_normal((N + 1,) * d)
    G = rng.standard_normal(tuple(m + 2 * N for m in shape))
    exts = [np.arange(1 - N, m + N + 1) for m in shape]
    for e in itertools.product(*[range(len(x)) for x in exts]):
        if all(1 <= exts[t][e[t]] <= shape[t] for t in range(d)):
            G[e] = 0.0
    ref = np.zeros(shape)
    for i in itertools.product(*[range(1, m + 1) for m in shape]):
        s = 0.0
        for e in itertools.product(*[range(len(x)) for x in exts]):
            x = tuple(int(exts[t][e[t]]) for t in range(d))
            if all(1 <= x[t] <= shape[t] for t in range(d)):
                continue
            o = tuple(abs(x[t] - i[t]) for t in range(d))
            if max(o) <= N:
                s += a[o] * G[e]
        ref[tuple(t - 1 for t in i)] = s
    assert np.allclose(O.boundary_near(a, G), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d,shape", [(1, (5,)), (2, (4, 4)), (2, (6, 3)), (3, (2, 4, 3))])
def test_synth_extended_points_match_the_oracle_samples(d, shape):
    """The inputs' extended grid (synth) and the oracle's sampling points are the same points:
    a positive g that tells the axes apart, sampled both ways, agrees off the interior."""
    import synth
    N = max(shape) + 1
    h = 2.0 / N
    wts = np.arange(1, d + 1, dtype=float) ** 2
    g = lambda P: np.sum(P * P * wts, axis=-1) + 1.0 + 0.1 * P[..., 0]  # noqa: E731  (positive)
    G = O.extended_samples(d, N, h, g, shape=shape)
    P = synth.extended_points(d, shape if d > 1 else shape[0])
    S = g(P)
    mask = G != 0.0
    assert S.shape == G.shape
    assert np.allclose(S[mask], G[mask], rtol=0, atol=1e-13)
    assert np.count_nonzero(~mask) == int(np.prod(shape))      # exactly the interior is zeroed


@pytest.mark.parametrize("alpha,lam", [(0.5, 0.0), (1.5, 0.0), (1.2, 0.8)])
def test_far_part_1d_against_adaptive_quadrature(alpha, lam):
    """1D: far_i = sum over s = +-1 of int_L^inf g(x_i + s rho) rho^{-1-alpha} e^{-lam rho} d rho,
    by QUADPACK on the half line (independent of the oracle's t = L / rho substitution)."""
    from scipy import integrate
    N = 8
    h = 2.0 / N
    L = N * h
    g = lambda P: 1.0 / (1.0 + P[..., 0] ** 2)  # noqa: E731
    far = O.boundary_far(1, N, h, alpha, g, lam)
    x = -1.0 + h * np.arange(1, N)
    for i, xi in enumerate(x):
        ref = 0.0
        for s in (-1.0, 1.0):
            f = lambda r, s=s, xi=xi: r ** (-1.0 - alpha) * math.exp(-lam * r) / (1.0 + (xi + s * r) ** 2)  # noqa: E731
            ref += integrate.quad(f, L, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]
        assert abs(far[i] - ref) <= 1e-10 * ref, (i, far[i], ref)
