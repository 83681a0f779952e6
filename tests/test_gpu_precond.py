"""GPU parity, the tau preconditioner (frac_precond) and tau-preconditioned CG.

Bars: z = P r against the oracle's dense sine-transform preconditioner,
normwise ||z - z_ref|| <= tol * ||P||_2 ||r|| with ||P||_2 = 1 / min(symbol)
(1e-12 FP64, 1e-5 FP32, as for the apply); solves: the oracle's residual of the
returned u <= rtol plus the generator slack (as in test_gpu_solve), and the
solution equal to the unpreconditioned solve's within what the 1e-10 residuals
of both allow.
"""
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


def _op(d, n, p, alpha, lam=0.0):
    import paper_2103_03658_gb300 as fg
    return fg.FracOp(d, n, alpha, degree=p, lam=lam)


# n = 2^k - 1 (tau system of exactly the problem's size) and other n (restricted)
CASES = [(1, 3, 1, 1.2, 0.0, 1), (1, 7, 2, 0.4, 0.0, 3), (1, 100, 0, 1.5, 1.0, 2), (1, 1023, 1, 1.9, 0.0, 2),
         (2, 3, 1, 1.0, 0.0, 1), (2, 15, 2, 1.6, 0.3, 2), (2, 20, 0, 0.5, 1.5, 1), (2, 63, 1, 1.2, 0.0, 2),
         (3, 3, 1, 0.7, 0.0, 1), (3, 9, 2, 1.6, 0.0, 2), (3, 15, 1, 0.4, 0.8, 1),
         # several column tiles and slabs per pass, the last column pair half empty
         (2, 127, 1, 0.9, 0.0, 3), (3, 31, 1, 0.4, 0.0, 2)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,n,p,alpha,lam,batch", CASES)
def test_precond_matches_oracle(d, n, p, alpha, lam, batch, dtype):
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    op = _op(d, n, p, alpha, lam)
    assert op.info()["precond_ok"] == 1
    m = O.fft_len(n) // 2 - 1
    pnorm = 1.0 / np.min(O.tau_symbol(a, c, n, m))
    rng = np.random.default_rng(7 * n + d)
    R = rng.standard_normal((batch,) + (n,) * d)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    z = op.precond(torch.tensor(R, dtype=tdt, device="cuda")).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(batch):
        rr = R[b] if dtype == "f64" else R[b].astype(np.float32).astype(np.float64)
        ref = O.tau_precond(a, c, rr)
        err = np.linalg.norm(z[b] - ref) / (pnorm * np.linalg.norm(rr))
        assert err <= tol, (b, err)
    if dtype == "f64":  # symmetric: <v, P r> = <P v, r>
        v = rng.standard_normal((n,) * d)
        Pv = op.precond(torch.tensor(v, device="cuda")).cpu().numpy()
        Pr = op.precond(torch.tensor(R[0], device="cuda")).cpu().numpy()
        assert abs(np.vdot(v, Pr) - np.vdot(Pv, R[0])) <= 1e-12 * pnorm * np.linalg.norm(v) * np.linalg.norm(R[0])
    op.close()


def test_precond_not_available_for_power_of_two_sizes():
    """n a power of two (n = 1 included) has M/2 - 1 < n: no tau system contains
    the problem; frac_precond refuses and the solvers fall back to plain CG."""
    import paper_2103_03658_gb300 as fg
    for d, n in ((1, 1), (1, 16), (2, 8), (3, 4)):
        op = _op(d, n, 1, 1.0)
        assert op.info()["precond_ok"] == 0
        with pytest.raises(fg.FracError):
            op.precond(torch.ones((n,) * d, dtype=torch.float64, device="cuda"))
        f = torch.ones((n,) * d, dtype=torch.float64, device="cuda")
        u, info = op.solve(f, rtol=1e-10)
        assert info["status"] == 0 and info["precond"] == 0
        op.close()


SOLVE_CASES = [(1, 1023, 1, 1.5, 0.0), (1, 301, 2, 1.9, 1.2), (2, 31, 1, 1.2, 0.0), (2, 45, 2, 0.5, 0.7),
               (2, 100, 0, 1.8, 0.0), (3, 15, 2, 1.6, 0.3), (3, 21, 1, 0.4, 0.0)]


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("d,n,p,alpha,lam", SOLVE_CASES)
def test_pcg_solve_residual_recomputed_by_oracle(d, n, p, alpha, lam, precision):
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    f = synth.smooth_field(d, n, 2103 + n) + 0.5
    op = _op(d, n, p, alpha, lam)
    fd = torch.tensor(f, device="cuda")
    u, info = op.solve(fd, rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10 and info["precond"] == 1
    u0, info0 = op.solve(fd, rtol=1e-10, precision=precision, precond="none")
    assert info0["status"] == 0 and info0["precond"] == 0
    assert info["iters"] < info0["iters"] or info0["iters"] <= 12, (info, info0)
    uh = u.cpu().numpy()
    if n ** d <= 40000:
        A = O.operator_matrix(a, c, n)
        res = np.linalg.norm(f.reshape(-1) - A @ uh.reshape(-1)) / np.linalg.norm(f)
        da = np.abs(op.generator() - a)
        K = np.indices(da.shape)
        slack = c * float(np.sum(2.0 ** np.sum(K > 0, axis=0) * da)) * np.linalg.norm(uh) / np.linalg.norm(f)
        assert res <= 1e-10 * 1.05 + 2 * slack, (res, slack)
    kappa = op.info()["norm_bound"] * float(u.norm()) / float(fd.norm())
    assert float((u - u0).norm() / u0.norm()) <= 4e-10 * max(kappa, 1.0)
    op.close()


def test_pcg_engine_and_batch_use_the_preconditioner():
    import paper_2103_03658_gb300 as fg
    probs = [(1, 255, 1, 0.7, 0.0), (2, 63, 2, 1.3, 0.4), (2, 100, 0, 1.9, 0.0), (3, 15, 1, 0.5, 0.0)]
    ops = [_op(*q) for q in probs]
    fs = [torch.tensor(synth.smooth_field(q[0], q[1], 5 + i) + 1.0, device="cuda") for i, q in enumerate(probs)]
    us = [torch.empty_like(f) for f in fs]
    infos = fg.solve_batch(ops, fs, us, rtol=1e-10)
    for op, f, u, info in zip(ops, fs, us, infos):
        assert info["status"] == 0 and info["rel_resid"] <= 1e-10 and info["precond"] == 1
        r = f - op.apply(u)
        assert float(r.norm() / f.norm()) <= 1e-10 * 1.01
    eng = fg.Engine(4)
    jobs = [eng.submit(op, f, rtol=1e-10) for op, f in zip(ops, fs)]
    got = {}
    while len(got) < len(jobs):
        for job, info, _ms, u in eng.poll(block=True):
            got[job] = (info, u)
    for (job, _), op, f in zip(jobs, ops, fs):
        info, u = got[job]
        assert info["status"] == 0 and info["precond"] == 1
        r = f - op.apply(u)
        assert float(r.norm() / f.norm()) <= 1e-10 * 1.01
    eng.close()
    for op in ops:
        op.close()
