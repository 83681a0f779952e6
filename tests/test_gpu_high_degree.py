"""GPU parity, Lagrange bases of degree 3 and 4 (origin rules of order 6 and 8; the
oracle's higher-degree scheme) in 1D, 2D and 3D: the generator against the oracle's
(1e-13 of its largest entry, the bar of the lower degrees), the applies against the
oracle's dense sum, solves whose residual the oracle recomputes, and the accuracy the
oracle shows on u = 1/(1+x^2) with its exterior data (the GPU's apply and boundary
vector, the far integrals of g from the oracle)."""
import math

import numpy as np
import pytest

import synth
from oracle import frac_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _op(n, p, alpha, lam=0.0, gamma=2.0):
    import paper_2103_03658_gb300 as fg
    return fg.FracOp(1, n, alpha, degree=p, lam=lam, gamma=gamma)


CASES = [(2, 3, 1.2, 0.0, 2.0), (5, 3, 0.4, 0.0, 2.0), (47, 3, 1.7, 0.9, 2.0), (1022, 3, 1.5, 0.0, 2.0),
         (3, 4, 0.8, 0.0, 2.0), (7, 4, 1.9, 0.0, 2.0), (63, 4, 0.3, 1.5, 2.0), (4095, 4, 1.2, 0.0, 2.0),
         (35, 3, 1.0, 0.0, 1.5), (39, 4, 1.4, 0.3, 1.8)]


@pytest.mark.parametrize("n,p,alpha,lam,gamma", CASES)
def test_generator_matches_oracle(n, p, alpha, lam, gamma):
    N = n + 1
    a_ref = O.stencil(1, N, 2.0 / N, alpha, p, lam, gamma=gamma)
    op = _op(n, p, alpha, lam, gamma)
    a_gpu = op.generator()
    assert np.max(np.abs(a_gpu - a_ref)) <= 1e-13 * np.max(np.abs(a_ref))
    op.close()


@pytest.mark.parametrize("n,p,alpha", [(47, 3, 1.3), (63, 4, 0.7), (255, 4, 1.8)])
def test_apply_matches_oracle(n, p, alpha):
    N = n + 1
    a = O.stencil(1, N, 2.0 / N, alpha, p)
    c = O.c_dalpha(1, alpha)
    u = np.random.default_rng(n).standard_normal((3, n))
    op = _op(n, p, alpha)
    y = op.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    for b in range(3):
        ref = O.apply_dense(a, c, u[b])
        assert np.linalg.norm(y[b] - ref) <= 1e-12 * O.norm_bound(a, c, n) * np.linalg.norm(u[b])
    op.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("n,p,alpha", [(299, 3, 1.5), (1023, 4, 0.9)])
def test_solve_residual_recomputed_by_oracle(n, p, alpha, precision):
    N = n + 1
    a = O.stencil(1, N, 2.0 / N, alpha, p)
    c = O.c_dalpha(1, alpha)
    f = synth.smooth_field(1, n, 11 + n) + 0.5
    op = _op(n, p, alpha)
    u, info = op.solve(torch.tensor(f, device="cuda"), rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    res = np.linalg.norm(f - O.apply_dense(a, c, u.cpu().numpy())) / np.linalg.norm(f)
    assert res <= 1.05e-10 + 1e-13 * O.norm_bound(a, c, n) * np.linalg.norm(u.cpu().numpy()) / np.linalg.norm(f)
    op.close()


@pytest.mark.parametrize("p,alpha,bound", [(3, 1.7, 1e-8), (4, 0.5, 2e-12), (4, 1.7, 1e-10)])
def test_accuracy_on_smooth_exterior_data(p, alpha, bound):
    """N = 192, u = 1/(1+x^2): max |A u + b - (-Delta)^{alpha/2} u| at the level the oracle
    reaches (p = 3: 2.8e-9 at alpha 1.7; p = 4: 1.8e-13 at 0.5, 1.0e-11 at 1.7)."""
    N = 192
    n = N - 1
    h = 2.0 / N
    g = lambda P: 1.0 / (1.0 + P[..., 0] ** 2)  # noqa: E731
    far = O.boundary_far(1, N, h, alpha, g)
    op = _op(n, p, alpha)
    b = op.boundary(g(synth.extended_points(1, n)), far=far)
    x = synth.interior_grid(n)
    Au = op.apply(torch.tensor(1.0 / (1.0 + x * x), device="cuda")).cpu().numpy()
    err = np.max(np.abs(Au + b - O.fl_lorentzian_1d(alpha, x)))
    assert err <= bound, err
    op.close()


# ---------------------------------------------------------------------------
# d = 2, 3
# ---------------------------------------------------------------------------

def _opd(d, n, p, alpha, lam=0.0):
    import paper_2103_03658_gb300 as fg
    return fg.FracOp(d, n, alpha, degree=p, lam=lam)


DCASES = [(2, 2, 3, 1.1, 0.0), (2, 11, 3, 0.6, 0.0), (2, 23, 3, 1.8, 0.7), (2, 3, 4, 1.3, 0.0), (2, 23, 4, 0.4, 0.0),
          (2, 39, 4, 1.5, 1.2), (3, 2, 3, 0.9, 0.0), (3, 11, 3, 1.5, 0.0), (3, 7, 4, 0.7, 0.0), (3, 11, 4, 1.2, 0.8)]


@pytest.mark.parametrize("d,n,p,alpha,lam", DCASES)
def test_generator_matches_oracle_2d_3d(d, n, p, alpha, lam):
    N = n + 1
    a_ref = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12)
    op = _opd(d, n, p, alpha, lam)
    a_gpu = op.generator()
    assert np.max(np.abs(a_gpu - a_ref)) <= 1e-13 * np.max(np.abs(a_ref)), np.max(np.abs(a_gpu - a_ref))
    op.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,n,p,alpha", [(2, 23, 3, 1.3), (2, 35, 4, 0.7), (3, 11, 3, 1.6), (3, 7, 4, 0.9)])
def test_apply_matches_oracle_2d_3d(d, n, p, alpha, dtype):
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    nrm = O.norm_bound(a, c, n)
    U = np.random.default_rng(7 * n + p).standard_normal((2,) + (n,) * d)
    op = _opd(d, n, p, alpha)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = op.apply(torch.tensor(U, dtype=tdt, device="cuda")).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(2):
        uu = U[b] if dtype == "f64" else U[b].astype(np.float32).astype(np.float64)
        ref = O.apply_dense(a, c, uu)
        assert np.linalg.norm(y[b] - ref) <= tol * nrm * np.linalg.norm(uu)
    op.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("d,n,p,alpha", [(2, 35, 3, 1.5), (3, 11, 4, 0.9)])
def test_solve_residual_recomputed_by_oracle_2d_3d(d, n, p, alpha, precision):
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    f = synth.smooth_field(d, n, 5 + n) + 0.5
    op = _opd(d, n, p, alpha)
    u, info = op.solve(torch.tensor(f, device="cuda"), rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    uu = u.cpu().numpy()
    res = np.linalg.norm(f - O.apply_dense(a, c, uu)) / np.linalg.norm(f)
    assert res <= 1.05e-10 + 1e-13 * O.norm_bound(a, c, n) * np.linalg.norm(uu) / np.linalg.norm(f)
    op.close()
