"""The library's far-field rule for exterior data (frac_far_nodes: host only, no GPU):
its nodes and weights against scipy's Gauss-Jacobi and Gauss-Legendre rules, its weights
summing to the far-field constant F_d of Eq. (L2) (g = 1) computed by the oracle's own,
different quadrature, every node outside the cube [0, L]^d, and argument checks."""
import math

import numpy as np
import pytest
from scipy import special

import paper_2103_03658_gb300 as fg
from oracle import frac_oracle as O


@pytest.mark.parametrize("alpha,lam", [(0.3, 0.0), (1.0, 0.0), (1.9, 0.0), (0.7, 1.3)])
def test_rule_1d_is_gauss_jacobi_in_t(alpha, lam):
    """1D: xi = L / t, t = (x + 1) / 2 with x the Gauss-Jacobi nodes of the weight
    (1 + x)^{alpha - 1} (scipy's nodes, to their absolute accuracy); the weights are
    L^{-alpha} 2^{-alpha} w_J e^{-lambda xi} (scipy's weights carry errors near 1e-12, so
    the bar is 1e-11 of the largest; the exactness test below holds them to 1e-14)."""
    L, nr = 2.0, 40
    xi, w = fg.far_nodes(1, alpha, lam, L, nr=nr, ns=1)
    x, wj = special.roots_jacobi(nr, 0.0, alpha - 1.0)
    t = 0.5 * (x + 1.0)
    order = np.argsort(t)
    got = np.argsort(L / xi[:, 0])
    # t = L / xi to the absolute accuracy of the nodes x (t near 0 is a difference x + 1)
    assert np.allclose(L / xi[got, 0], t[order], rtol=0, atol=1e-14)
    ref_w = (L ** -alpha * 0.5 ** alpha * wj * np.exp(-lam * L / t))[order]
    assert np.allclose(w[got], ref_w, rtol=0, atol=1e-11 * np.max(ref_w))


@pytest.mark.parametrize("alpha", [0.3, 1.0, 1.9])
def test_rule_1d_is_exact_for_powers_of_t(alpha):
    """With G(rho) = (L / rho)^j = t^j (lambda = 0) the rule must give
    L^{-alpha} int_0^1 t^{alpha - 1 + j} dt = L^{-alpha} / (alpha + j) exactly for
    j <= 2 nr - 1 (Gauss exactness), here to 2e-14 for j = 0..30."""
    L, nr = 1.5, 40
    xi, w = fg.far_nodes(1, alpha, 0.0, L, nr=nr, ns=1)
    t = L / xi[:, 0]
    for j in range(31):
        ref = L ** -alpha / (alpha + j)
        assert abs(math.fsum(w * t ** j) - ref) <= 2e-14 * ref, j


def test_rule_2d_angles_are_gauss_legendre():
    """2D, pyramid of the first coordinate: xi = rho (1, s) with s the Gauss-Legendre nodes
    on [0, 1]; the weight's angular factor is w_s |(1, s)|^{-2-alpha}."""
    alpha, L, nr, ns = 1.3, 2.0, 8, 12
    xi, w = fg.far_nodes(2, alpha, 0.0, L, nr=nr, ns=ns)
    first = xi[: ns * nr]                      # lead coordinate 0: xi_0 = rho
    s = np.unique(np.round(first[:, 1] / first[:, 0], 12))
    xs, _ = special.roots_legendre(ns)
    assert np.allclose(np.sort(s), np.sort(0.5 * (xs + 1.0)), rtol=0, atol=1e-12)
    assert len(w) == 2 * ns * nr


@pytest.mark.parametrize("d,alpha,lam,nr,ns,tol", [
    (1, 0.5, 0.0, 96, 1, 1e-14), (1, 1.5, 0.8, 96, 1, 1e-13),
    (2, 0.4, 0.0, 96, 48, 1e-13), (2, 1.7, 0.0, 96, 48, 1e-13), (2, 1.1, 1.2, 96, 48, 1e-12),
    (3, 0.8, 0.0, 48, 24, 1e-12), (3, 1.6, 0.5, 48, 24, 1e-11),
])
def test_weights_sum_to_far_field_constant(d, alpha, lam, nr, ns, tol):
    """g = 1: sum_m sum_q w_q = 2^d F_d, F_d the far-field constant of Eq. (L2) from the
    oracle (48-point angles, radial integral by QUADPACK or in closed form)."""
    L = 2.0 + 2.0 / 63
    _, w = fg.far_nodes(d, alpha, lam, L, nr=nr, ns=ns)
    F = O.far_field(d, alpha, L, lam)
    assert abs(math.fsum(w) - F) <= tol * F, (math.fsum(w), F)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_nodes_lie_in_the_far_region(d):
    L = 1.7
    xi, w = fg.far_nodes(d, 1.2, 0.0, L, nr=16, ns=6)
    assert np.all(np.max(xi, axis=1) >= L * (1 - 1e-15)) and np.all(xi >= 0) and np.all(w > 0)


def test_bad_arguments_are_rejected():
    for args in [(0, 1.0, 0.0, 2.0, 8, 8), (4, 1.0, 0.0, 2.0, 8, 8), (1, 0.0, 0.0, 2.0, 8, 8),
                 (1, 2.0, 0.0, 2.0, 8, 8), (1, 1.0, -1.0, 2.0, 8, 8), (1, 1.0, 0.0, 0.0, 8, 8),
                 (1, 1.0, 0.0, 2.0, 0, 8), (2, 1.0, 0.0, 2.0, 8, 0), (1, 1.0, float("nan"), 2.0, 8, 8)]:
        with pytest.raises(fg.FracError):
            fg.far_nodes(*args)
