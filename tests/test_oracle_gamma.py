"""Oracle pins for the splitting parameter gamma in (alpha, 2] (Eq. (eq0), Eq. (gamma2)):
the 1D weights against the Appendix closed forms with sigma_0 = gamma - alpha (the paper
states them for any gamma), gamma = 2 as the default, and the accuracy rates of the
1D operator on u = 1/(1+x^2) with its extended Dirichlet data (the setting of Fig. 3-1-3,
exact values from the pseudo-differential definition): O(h^{2-alpha}) for p = 0, 1 at
gamma = 1 + alpha/2 as the text states, and -- a finding -- O(h^{2-alpha}) also for p = 2,
where the text states O(h^{3-alpha}): below gamma = 2 the difference quotient carries the
singular part u'' xi^{2-gamma}, whose interpolation error weighted by mu_gamma is of order
h^{2-alpha} on every element for every p (the figure prints no numbers to compare)."""
import math

import numpy as np
import pytest

from oracle import frac_oracle as O


@pytest.mark.parametrize("p", [0, 1, 2])
@pytest.mark.parametrize("alpha,gamma", [(0.6, 1.3), (0.6, 0.8), (1.5, 1.75), (1.2, 1.9)])
def test_1d_weights_match_appendix_closed_forms(p, alpha, gamma):
    N = 16
    h = 2.0 / N
    w = O.weights(1, N, h, alpha, p, gamma=gamma)
    ref = O.weights_1d_appendix(N, h, alpha, p, gamma=gamma)
    assert np.allclose(w, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_gamma_two_is_the_default():
    for d, p in ((1, 2), (2, 1), (3, 0)):
        N = 6
        a = O.stencil(d, N, 2.0 / N, 1.1, p, 0.4, q=12)
        b = O.stencil(d, N, 2.0 / N, 1.1, p, 0.4, q=12, gamma=2.0)
        assert np.array_equal(a, b)
    assert O.zeta(2.0) == 1 and O.zeta(1.99) == 0 and O.zeta(0.7) == 0


def _err(N, alpha, p, gamma):
    h = 2.0 / N
    a = O.stencil(1, N, h, alpha, p, 0.0, gamma=gamma)
    c = O.c_dalpha(1, alpha)
    x = O.interior_points(N)
    u = 1.0 / (1.0 + x * x)
    b = O.boundary_vector(1, N, h, alpha, a, c, lambda P: 1.0 / (1.0 + P[..., 0] ** 2))
    return np.max(np.abs(O.apply_dense(a, c, u) + b - O.fl_lorentzian_1d(alpha, x)))


@pytest.mark.parametrize("alpha", [0.6, 1.5])
@pytest.mark.parametrize("p", [0, 1, 2])
def test_rates_at_gamma_one_plus_half_alpha(alpha, p):
    gamma = 1.0 + alpha / 2.0
    es = [_err(N, alpha, p, gamma) for N in (32, 64, 128)]
    rates = [math.log2(es[i] / es[i + 1]) for i in range(2)]
    for r in rates:
        assert abs(r - (2.0 - alpha)) <= 0.12, (rates, es)


@pytest.mark.parametrize("alpha", [0.6, 1.5])
def test_gamma_two_is_more_accurate(alpha):
    """Sec. 3.1: gamma = 2 gives the smallest errors for every basis."""
    for p in (0, 1, 2):
        assert _err(64, alpha, p, 2.0) < _err(64, alpha, p, 1.0 + alpha / 2.0)
