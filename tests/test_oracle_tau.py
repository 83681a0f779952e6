"""Oracle pins for the tau preconditioner (the paper names no solver; the
library offers tau-preconditioned CG).  The oracle's sine-transform
implementation is checked against the definition of the tau algebra:
tau(T_m) = T_m - H_m with the Hankel correction H_m, which the sine transform
diagonalises with the symbol as eigenvalues; the multilevel case against the
Kronecker product of 1D tau matrices; and preconditioned CG against a dense
solve."""
import numpy as np
import pytest

from oracle import frac_oracle as O


def _toeplitz(t):
    m = len(t)
    return np.array([[t[abs(i - j)] for j in range(m)] for i in range(m)])


@pytest.mark.parametrize("m", [1, 2, 3, 5, 9, 16])
def test_sine_transform_diagonalises_tau_matrix(m):
    t = np.random.default_rng(m).standard_normal(m)
    S = O.sine_matrix(m)
    assert np.allclose(S @ S, np.eye(m), atol=1e-13)              # orthogonal and symmetric
    k = np.arange(1, m + 1)
    lam = t[0] + 2 * (np.cos(np.pi * np.outer(k, np.arange(1, m)) / (m + 1)) @ t[1:])
    tau = _toeplitz(t) - O.tau_hankel_1d(t)
    assert np.allclose(S @ np.diag(lam) @ S, tau, atol=1e-12 * np.abs(t).sum())


@pytest.mark.parametrize("n", [5, 7, 12])
def test_tau_precond_1d_is_restricted_tau_inverse(n):
    """P v = R tau(T_m)^{-1} R^T v with T_m the zero-extended Toeplitz matrix of
    the operator's generator (m = M/2 - 1 >= n), tau from its definition."""
    N = n + 1
    a = O.stencil(1, N, 2.0 / N, 1.3, 1)
    c = O.c_dalpha(1, 1.3)
    m = O.fft_len(n) // 2 - 1
    t = np.zeros(m)
    t[:n] = a[:n]
    tau = -c * (_toeplitz(t) - O.tau_hankel_1d(t))
    v = np.random.default_rng(1).standard_normal(n)
    ref = np.linalg.solve(tau, np.concatenate([v, np.zeros(m - n)]))[:n]
    assert np.allclose(O.tau_precond(a, c, v), ref, rtol=1e-11, atol=0)


def test_tau_precond_2d_is_kronecker_of_1d_tau():
    """A separable generator a_{j1 j2} = b_{j1} b'_{j2} has the two-level tau
    matrix tau(T_b) (x) tau(T_b'); the oracle's 2D preconditioner (c = -1) must
    invert it on the leading block."""
    n = 6
    m = O.fft_len(n) // 2 - 1
    rng = np.random.default_rng(3)
    b1 = np.concatenate([[4.0], -rng.uniform(0.1, 0.5, n - 1)])
    b2 = np.concatenate([[3.0], -rng.uniform(0.1, 0.4, n - 1)])
    a = np.zeros((n + 2, n + 2))
    a[:n, :n] = np.outer(b1, b2)
    t1 = np.zeros(m)
    t1[:n] = b1
    t2 = np.zeros(m)
    t2[:n] = b2
    tau = np.kron(_toeplitz(t1) - O.tau_hankel_1d(t1), _toeplitz(t2) - O.tau_hankel_1d(t2))
    v = rng.standard_normal((n, n))
    w = np.zeros((m, m))
    w[:n, :n] = v
    ref = np.linalg.solve(tau, w.reshape(-1)).reshape(m, m)[:n, :n]
    assert np.allclose(O.tau_precond(a, -1.0, v), ref, rtol=1e-10, atol=1e-13)


def test_tau_precond_refuses_power_of_two_sizes():
    with pytest.raises(ValueError):
        O.tau_precond(np.ones(10), 1.0, np.ones(8))     # n = 8: M = 16, m = 7 < n


@pytest.mark.parametrize("d,n,p,alpha,lam", [(1, 63, 1, 0.5, 0.0), (1, 63, 2, 1.9, 0.0), (1, 100, 0, 1.5, 1.0),
                                             (2, 15, 1, 1.6, 0.0), (2, 20, 0, 1.0, 1.5), (3, 7, 2, 1.2, 0.0)])
def test_tau_pcg_solves_and_converges_fast(d, n, p, alpha, lam):
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    f = np.cos(np.linspace(0.0, 2.0, n ** d)).reshape((n,) * d) + 0.2
    u, it = O.solve_pcg(a, c, f, rtol=1e-10)
    _, it0 = O.solve_cg(a, c, f, rtol=1e-10)
    uref = O.solve_dense(a, c, f)
    assert np.linalg.norm(u - uref) <= 1e-8 * np.linalg.norm(uref)
    assert it <= 20 and it < it0
