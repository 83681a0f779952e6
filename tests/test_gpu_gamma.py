"""GPU parity for the splitting parameter gamma in (alpha, 2) (Eq. (eq0); zeta = 0 below 2):
generator (1e-13 of max |a|), FP64 apply (normwise 1e-12) and solves (oracle residual),
against the oracle with the same gamma, as in test_gpu_apply and test_gpu_solve."""
import numpy as np
import pytest

from oracle import frac_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [(1, 63, 0, 0.6, 1.3, 0.0), (1, 127, 2, 1.5, 1.75, 0.5), (1, 31, 1, 0.3, 0.5, 0.0),
         (2, 15, 1, 1.2, 1.6, 0.0), (2, 21, 2, 0.7, 1.35, 1.0), (2, 30, 0, 1.8, 1.9, 0.0),
         (3, 7, 1, 0.9, 1.45, 0.0), (3, 9, 2, 1.4, 1.7, 0.3), (3, 20, 1, 0.5, 1.8, 0.0)]


@pytest.mark.parametrize("d,n,p,alpha,gamma,lam", CASES)
def test_gamma_generator_and_apply_match_oracle(d, n, p, alpha, gamma, lam):
    import paper_2103_03658_gb300 as fg
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12, gamma=gamma)
    c = O.c_dalpha(d, alpha)
    op = fg.FracOp(d, n, alpha, degree=p, lam=lam, gamma=gamma)
    a_gpu = op.generator()
    assert np.max(np.abs(a_gpu - a)) <= 1e-13 * np.max(np.abs(a))
    u = np.random.default_rng(n + d).standard_normal((2,) + (n,) * d)
    y = op.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    nrm = O.norm_bound(a, c, n)
    for b in range(2):
        ref = O.apply_dense(a, c, u[b])
        assert np.linalg.norm(y[b] - ref) <= 1e-12 * nrm * np.linalg.norm(u[b])
    # the same operator without gamma differs (gamma = 2 keeps the origin term)
    op2 = fg.FracOp(d, n, alpha, degree=p, lam=lam)
    assert np.max(np.abs(op2.generator() - a_gpu)) > 1e-6 * np.max(np.abs(a))
    op.close()
    op2.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("d,n,p,alpha,gamma", [(1, 255, 1, 1.2, 1.6), (2, 31, 2, 0.8, 1.4), (3, 15, 0, 1.5, 1.75)])
def test_gamma_solve_residual_recomputed_by_oracle(d, n, p, alpha, gamma, precision):
    import paper_2103_03658_gb300 as fg
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, 0.0, q=20 if d < 3 else 12, gamma=gamma)
    c = O.c_dalpha(d, alpha)
    f = np.cos(np.linspace(0.0, 3.0, n ** d)).reshape((n,) * d) + 0.4
    op = fg.FracOp(d, n, alpha, degree=p, gamma=gamma)
    u, info = op.solve(torch.tensor(f, device="cuda"), rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    uh = u.cpu().numpy()
    res = np.linalg.norm(f.reshape(-1) - O.operator_matrix(a, c, n) @ uh.reshape(-1)) / np.linalg.norm(f)
    da = np.abs(op.generator() - a)
    K = np.indices(da.shape)
    slack = c * float(np.sum(2.0 ** np.sum(K > 0, axis=0) * da)) * np.linalg.norm(uh) / np.linalg.norm(f)
    assert res <= 1e-10 * 1.05 + 2 * slack, (res, slack)
    op.close()
