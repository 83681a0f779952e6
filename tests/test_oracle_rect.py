"""Oracle pins for rectangular grids (N_2 < N_1, Sec. 2.2: N_1 = N spans the longer
side, N_2 the smallest count with a_2 + N_2 h >= b_2).  The generator is the one of the
square [0, L]^d with L the longer extent; the matrix is the block-Toeplitz-Toeplitz-block
A^{(2)} printed after Eq. (2D-scheme) with N_2 - 1 block rows of size N_1 - 1.  Pinned
against that block structure built entry by entry, against the square grid's matrix
(whose principal submatrix it must be), and, for the tau preconditioner, against the
Kronecker product of 1D tau matrices of different sizes."""
import numpy as np
import pytest

from oracle import frac_oracle as O


def _gen(d, N, alpha=1.3, p=1, lam=0.0):
    return O.stencil(d, N, 2.0 / N, alpha, p, lam, q=12), O.c_dalpha(d, alpha)


@pytest.mark.parametrize("n1,n2", [(7, 4), (9, 9), (6, 2), (8, 1)])
def test_rect_matrix_is_the_printed_block_toeplitz_form(n1, n2):
    """A^{(2)} = [A_{|j-l|}]_{j,l < N_2 - 1}, A_m the (N_1-1)x(N_1-1) Toeplitz matrix of the
    generator row a_{m, .}; unknowns ordered x^(1) fastest within a block (block vector u_j^(1))."""
    N = max(n1, n2) + 1
    a, c = _gen(2, N)
    A = O.operator_matrix(a, c, (n2, n1))
    ref = np.zeros((n1 * n2, n1 * n2))
    for j in range(n2):
        for l in range(n2):
            m = abs(j - l)
            blk = np.array([[a[m, abs(i1 - i2)] for i2 in range(n1)] for i1 in range(n1)])
            ref[j * n1:(j + 1) * n1, l * n1:(l + 1) * n1] = -c * blk
    assert np.array_equal(A, ref)


@pytest.mark.parametrize("shape", [(3, 7), (7, 3), (2, 5, 4), (5, 2, 3)])
def test_rect_operator_is_principal_submatrix_of_square(shape):
    d = len(shape)
    n = max(shape)
    a, c = _gen(d, n + 1)
    A = O.operator_matrix(a, c, shape)
    Asq = O.operator_matrix(a, c, n)
    idx = np.ravel_multi_index(np.indices(shape).reshape(d, -1), (n,) * d)
    assert np.array_equal(A, Asq[np.ix_(idx, idx)])
    u = np.random.default_rng(1).standard_normal(shape)
    assert np.allclose(O.apply_dense(a, c, u), (A @ u.reshape(-1)).reshape(shape), rtol=0, atol=1e-12)
    rows = np.array([[0] * d, [s - 1 for s in shape], [s // 2 for s in shape]])
    ref = (A @ u.reshape(-1)).reshape(shape)
    assert np.allclose(O.apply_rows(a, c, u, rows), [ref[tuple(r)] for r in rows], rtol=1e-13, atol=1e-13)


def _toeplitz(t):
    m = len(t)
    return np.array([[t[abs(i - j)] for j in range(m)] for i in range(m)])


def test_rect_tau_precond_is_kronecker_of_1d_tau_of_two_sizes():
    """Separable generator b_{j2} b'_{j1}: tau(T_b, m_2) (x) tau(T_b', m_1) with m_i = M_i/2 - 1."""
    n1, n2 = 11, 5
    m1, m2 = O.fft_len(n1) // 2 - 1, O.fft_len(n2) // 2 - 1
    assert (m1, m2) == (15, 7)
    rng = np.random.default_rng(4)
    b2 = np.concatenate([[4.0], -rng.uniform(0.1, 0.5, n2 - 1)])
    b1 = np.concatenate([[3.0], -rng.uniform(0.05, 0.3, n1 - 1)])
    N = max(n1, n2) + 2
    a = np.zeros((N, N))
    a[:n2, :n1] = np.outer(b2, b1)
    t2 = np.zeros(m2)
    t2[:n2] = b2
    t1 = np.zeros(m1)
    t1[:n1] = b1
    tau = np.kron(_toeplitz(t2) - O.tau_hankel_1d(t2), _toeplitz(t1) - O.tau_hankel_1d(t1))
    v = rng.standard_normal((n2, n1))
    w = np.zeros((m2, m1))
    w[:n2, :n1] = v
    ref = np.linalg.solve(tau, w.reshape(-1)).reshape(m2, m1)[:n2, :n1]
    assert np.allclose(O.tau_precond(a, -1.0, v), ref, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("shape,p", [((9, 21), 1), ((21, 9), 0), ((5, 11, 7), 2)])
def test_rect_pcg_matches_dense_solve(shape, p):
    d = len(shape)
    N = max(shape) + 1
    a, c = O.stencil(d, N, 2.0 / N, 1.5, p, 0.0, q=12), O.c_dalpha(d, 1.5)
    f = np.cos(np.linspace(0.0, 3.0, int(np.prod(shape)))).reshape(shape) + 0.3
    u, it = O.solve_pcg(a, c, f, rtol=1e-11)
    uref = O.solve_dense(a, c, f)
    assert np.linalg.norm(u - uref) <= 1e-9 * np.linalg.norm(uref)
    _, it0 = O.solve_cg(a, c, f, rtol=1e-11)
    assert it < it0
