"""Pins of the oracle's per-node weights and of the two norm bounds that scale
every apply tolerance (no GPU).

* ``weights_at`` (the weights of single nodes, the only oracle source for the
  largest 3D generators) against ``weights`` (the whole array) at seeded nodes,
  including the origin, the axes and the far corner, plain and tempered,
  gamma = 2 and gamma < 2, p = 0, 1, 2, d = 2, 3.
* ``norm_bound`` (the row-sum bound) and ``spectral_bound`` (the largest
  eigenvalue magnitude of the circulant embedding) against the spectral norm of
  the dense operator: both must bound ||A||_2 from above, and neither may exceed
  it by more than a small factor, or every tolerance scaled by it would loosen.
"""
import numpy as np
import pytest

from oracle import frac_oracle as O


@pytest.mark.parametrize("d,N,p,alpha,lam,gamma", [
    (2, 8, 0, 1.3, 0.0, 2.0), (2, 8, 1, 0.4, 1.2, 2.0), (2, 8, 2, 1.7, 0.0, 2.0), (2, 8, 1, 0.8, 0.0, 1.3),
    (3, 6, 1, 1.1, 0.5, 2.0), (3, 6, 2, 0.6, 0.0, 2.0), (3, 6, 0, 1.9, 0.0, 2.0), (3, 8, 2, 0.5, 0.7, 1.2),
])
def test_weights_at_equals_weights(d, N, p, alpha, lam, gamma):
    h = 2.0 / N
    w = O.weights(d, N, h, alpha, p, lam, gamma=gamma)
    rng = np.random.default_rng(17 * N + d + p)
    nodes = [(0,) * d, (N,) * d, (1,) + (0,) * (d - 1), (0,) * (d - 1) + (2,), (N,) + (1,) * (d - 1)]
    nodes += [tuple(int(v) for v in rng.integers(0, N + 1, d)) for _ in range(16)]
    got = O.weights_at(d, N, h, alpha, p, lam, nodes, gamma=gamma)
    ref = np.array([w[k] for k in nodes])
    assert np.all(np.abs(got - ref) <= 2e-15 * np.abs(ref)), np.max(np.abs(got - ref) / np.abs(ref))


def test_weights_first_axis_ranges_sum_to_whole():
    """The partial sums over ranges of the first element index add up to the whole array."""
    d, N, p, alpha = 3, 6, 2, 1.1
    h = 2.0 / N
    w = O.weights(d, N, h, alpha, p, 0.4)
    ne = N // 2
    parts = sum(O.weights(d, N, h, alpha, p, 0.4, first=range(lo, min(lo + 2, ne))) for lo in range(0, ne, 2))
    assert np.max(np.abs(parts - w)) <= 1e-15 * np.max(np.abs(w))


BOUND_CASES = [(d, n, p, alpha, lam) for d, n in ((1, 40), (1, 7), (2, 12), (2, 5), (3, 6), (3, 3))
               for p, alpha, lam in ((0, 0.3, 0.0), (1, 1.0, 0.0), (2, 1.9, 0.0), (1, 1.5, 1.0))
               if not (p == 2 and (n + 1) % 2)]


@pytest.mark.parametrize("d,n,p,alpha,lam", BOUND_CASES)
def test_norm_bounds_bracket_the_spectral_norm(d, n, p, alpha, lam):
    """||A||_2 <= spectral_bound <= norm_bound <= 1.5 ||A||_2 (measured ratios: row-sum
    bound 1.04-1.42, circulant bound 1.001-1.2 at these sizes)."""
    a, c, _ = O.build_operator(d, n + 1, alpha, p, lam)
    A = O.operator_matrix(a, c, n)
    nA = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    nb = O.norm_bound(a, c, n)
    sb = O.spectral_bound(a, c, n)
    assert nA * (1 - 1e-12) <= sb <= nb * (1 + 1e-12)
    assert nb <= 1.5 * nA
    assert sb <= 1.25 * nA


def test_norm_bound_without_multiplicities_is_caught():
    """A row-sum bound that counts each offset once (dropping the 2^{d - z(k)} mirror
    images) falls below ||A||_2: the lower-bound check above would catch it."""
    d, n, p, alpha = 2, 12, 1, 1.0
    a, c, _ = O.build_operator(d, n + 1, alpha, p)
    nA = float(np.max(np.abs(np.linalg.eigvalsh(O.operator_matrix(a, c, n)))))
    wrong = c * float(np.sum(np.abs(a[:n, :n])))
    assert wrong < nA
