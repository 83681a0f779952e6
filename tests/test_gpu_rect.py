"""GPU parity on rectangular grids (unequal n_i, Sec. 2.2): generator, apply (FP64 and
FP32), tau preconditioner and solves against the oracle, with the bars of the square
tests (test_gpu_apply, test_gpu_precond, test_gpu_solve): apply normwise error
||y - y_ref|| / (||A||_2 ||u||) <= 1e-12 (FP64) / 1e-5 (FP32), ||A||_2 bounded by the
oracle's row-sum bound; preconditioner the same with ||P||_2 = 1 / min symbol; solves:
the oracle's residual of the returned u <= rtol plus the generator slack.  FracOp takes
n = (n_1, .., n_d) with x^(1) fastest; arrays have shape (n_d, .., n_1)."""
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


def _oracle(d, ns, p, alpha, lam):
    N = max(ns) + 1
    return O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12), O.c_dalpha(d, alpha)


CASES = [(2, (17, 9), 1, 1.2, 0.0, 2), (2, (9, 17), 0, 0.6, 0.7, 1), (2, (31, 20), 1, 1.9, 0.0, 1),
         (2, (63, 5), 2, 1.4, 0.0, 2), (2, (100, 63), 1, 0.3, 1.2, 1), (2, (1, 7), 1, 1.0, 0.0, 1),
         (3, (9, 7, 5), 1, 0.8, 0.0, 2), (3, (5, 9, 7), 2, 1.6, 0.4, 1), (3, (17, 12, 8), 0, 1.1, 0.0, 1),
         (3, (3, 1, 9), 1, 1.5, 0.0, 1)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,ns,p,alpha,lam,batch", CASES)
def test_rect_apply_matches_oracle(d, ns, p, alpha, lam, batch, dtype):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(d, ns, alpha, degree=p, lam=lam)
    shape = tuple(reversed(ns))
    assert op.shape == shape and op.info()["n"] == ns
    a, c = _oracle(d, ns, p, alpha, lam)
    if dtype == "f64":
        scale = np.max(np.abs(a))
        assert np.max(np.abs(op.generator() - a)) <= 1e-13 * scale
    nrm = O.norm_bound(a, c, shape)
    rng = np.random.default_rng(sum(ns) + 7 * d)
    U = rng.standard_normal((batch,) + shape)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = op.apply(torch.tensor(U, dtype=tdt, device="cuda")).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(batch):
        ub = U[b] if dtype == "f64" else U[b].astype(np.float32).astype(np.float64)
        ref = O.apply_dense(a, c, ub)
        err = np.linalg.norm(y[b] - ref) / (nrm * np.linalg.norm(ub))
        assert err <= tol, (b, err)
    op.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,ns,p,alpha,lam", [(2, (17, 9), 1, 1.2, 0.0), (2, (9, 31), 2, 1.7, 0.5),
                                              (3, (9, 7, 5), 1, 0.8, 0.0), (3, (5, 11, 7), 0, 1.4, 0.0)])
def test_rect_precond_matches_oracle(d, ns, p, alpha, lam, dtype):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(d, ns, alpha, degree=p, lam=lam)
    assert op.info()["precond_ok"] == 1
    shape = tuple(reversed(ns))
    a, c = _oracle(d, ns, p, alpha, lam)
    ms = tuple(O.fft_len(x) // 2 - 1 for x in shape)
    pnorm = 1.0 / np.min(O.tau_symbol(a, c, shape, ms))
    r = np.random.default_rng(3).standard_normal(shape)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    z = op.precond(torch.tensor(r, dtype=tdt, device="cuda")).double().cpu().numpy()
    rr = r if dtype == "f64" else r.astype(np.float32).astype(np.float64)
    err = np.linalg.norm(z - O.tau_precond(a, c, rr)) / (pnorm * np.linalg.norm(rr))
    assert err <= (1e-12 if dtype == "f64" else 1e-5), err
    op.close()


def test_rect_precond_refused_when_an_axis_is_a_power_of_two():
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(2, (15, 8), 1.0, degree=1)
    assert op.info()["precond_ok"] == 0
    with pytest.raises(fg.FracError):
        op.precond(torch.ones(op.shape, dtype=torch.float64, device="cuda"))
    op.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("d,ns,p,alpha,lam", [(2, (45, 21), 1, 1.5, 0.0), (2, (21, 63), 2, 0.7, 0.9),
                                              (3, (15, 9, 11), 1, 1.2, 0.0), (2, (30, 16), 0, 1.8, 0.0)])
def test_rect_solve_residual_recomputed_by_oracle(d, ns, p, alpha, lam, precision):
    import paper_2103_03658_gb300 as fg
    shape = tuple(reversed(ns))
    a, c = _oracle(d, ns, p, alpha, lam)
    rng = np.random.default_rng(11)
    f = np.cos(np.linspace(0.0, 4.0, int(np.prod(shape)))).reshape(shape) + 0.2 * rng.standard_normal(shape)
    op = fg.FracOp(d, ns, alpha, degree=p, lam=lam)
    fd = torch.tensor(f, device="cuda")
    u, info = op.solve(fd, rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    uh = u.cpu().numpy()
    A = O.operator_matrix(a, c, shape)
    res = np.linalg.norm(f.reshape(-1) - A @ uh.reshape(-1)) / np.linalg.norm(f)
    da = np.abs(op.generator() - a)
    K = np.indices(da.shape)
    slack = c * float(np.sum(2.0 ** np.sum(K > 0, axis=0) * da)) * np.linalg.norm(uh) / np.linalg.norm(f)
    assert res <= 1e-10 * 1.05 + 2 * slack, (res, slack)
    op.close()


def test_rect_batch_and_engine_take_rectangular_problems():
    """A rectangular 2D problem is not eligible for the persistent square-grid launch: the
    batch routes it through the solve engine beside square ones."""
    import paper_2103_03658_gb300 as fg
    probs = [(2, (63, 31), 1, 1.1, 0.0), (2, 63, 1, 1.1, 0.0), (3, (9, 15, 7), 2, 0.5, 0.3)]
    ops = [fg.FracOp(d, n, al, degree=p, lam=lam) for d, n, p, al, lam in probs]
    fs = [torch.tensor(synth.smooth_field(2, 63, 3)[: op.shape[0], : op.shape[1]] + 0.5, device="cuda")
          if op.d == 2 else torch.ones(op.shape, dtype=torch.float64, device="cuda") for op in ops]
    fs = [f.contiguous() for f in fs]
    us = [torch.empty_like(f) for f in fs]
    infos = fg.solve_batch(ops, fs, us, rtol=1e-10)
    for op, f, u, info in zip(ops, fs, us, infos):
        assert info["status"] == 0 and info["rel_resid"] <= 1e-10
        r = f - op.apply(u)
        assert float(r.norm() / f.norm()) <= 1e-10 * 1.01
    for op in ops:
        op.close()
