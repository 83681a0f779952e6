"""GPU: the 3D FP32 apply with its x and y transforms fused on thread-block clusters
(frac_apply_3d_passes(1)) against the five-pencil-pass schedule (0, the default).  Both run
the same device functions on the same values; the compiler may fuse multiplies and adds
differently in the two kernels, so the applies and the tau preconditioner agree to FP32
rounding (the apply normwise 2e-6 of ||A|| ||u||, the preconditioner 1e-3 of ||P u||, FP32
rounding times the spread of its symbol), and whole mixed-precision solves
(their FP32 CG runs the fused passes with the CG epilogues) to the solve tolerance; each
schedule is deterministic.  The fused schedule is also checked against the oracle here
(the default's parity is in test_gpu_apply, test_gpu_precond and test_gpu_solve)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _both(fn):
    import paper_2103_03658_gb300 as fg
    try:
        fg.apply_3d_passes(True)
        a = fn()
        fg.apply_3d_passes(False)
        b = fn()
    finally:
        fg.apply_3d_passes(False)  # the default
    return a, b


@pytest.mark.parametrize("n,p,alpha,lam", [(21, 1, 1.3, 0.0), ((31, 31, 9), 2, 0.8, 0.6)])
def test_fused_xy_apply_matches_oracle(n, p, alpha, lam):
    """The fused schedule against the oracle's dense apply (FP32 bar: 1e-5 of ||A|| ||u||)."""
    import paper_2103_03658_gb300 as fg
    from oracle import frac_oracle as O
    ns = n if isinstance(n, tuple) else (n,) * 3
    N = max(ns) + 1
    a = O.stencil(3, N, 2.0 / N, alpha, p, lam, q=12)
    c = O.c_dalpha(3, alpha)
    op = fg.FracOp(3, n, alpha, degree=p, lam=lam)
    assert op.info()["fft_lens"][0] == op.info()["fft_lens"][1]
    rng = np.random.default_rng(9)
    u = rng.standard_normal(op.shape).astype(np.float32).astype(np.float64)
    try:
        fg.apply_3d_passes(True)
        y = op.apply(torch.tensor(u, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    finally:
        fg.apply_3d_passes(False)
    rows = np.array([(0, 0, 0), tuple(s - 1 for s in op.shape)] +
                    [tuple(int(rng.integers(0, s)) for s in op.shape) for _ in range(60)])
    ref = O.apply_rows(a, c, u, rows)
    nrm = O.norm_bound(a, c, op.shape)
    err = np.linalg.norm(y[tuple(rows.T)] - ref) / (nrm * np.linalg.norm(u) * np.sqrt(len(rows) / u.size))
    assert err <= 1e-5, err
    op.close()


# (n per axis, degree, alpha, lambda, fields); n = (n1, n2, n3) with x, y lengths equal
CASES = [(255, 1, 1.6, 0.0, 2), (127, 2, 0.7, 0.5, 3), ((63, 63, 40), 1, 1.2, 0.0, 2), (21, 0, 1.9, 0.0, 4),
         ((31, 17, 63), 1, 0.4, 0.0, 1)]


@pytest.mark.parametrize("n,p,alpha,lam,batch", CASES)
def test_fused_xy_apply_and_precond_equal_five_passes(n, p, alpha, lam, batch):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(3, n, alpha, degree=p, lam=lam)
    rng = np.random.default_rng(5)
    u = torch.tensor(rng.standard_normal((batch,) + op.shape), dtype=torch.float32, device="cuda")
    nrm = op.info()["norm_bound"]
    y_fused, y_five = _both(lambda: op.apply(u))
    assert bool(torch.isfinite(y_fused).all())
    err = float((y_fused - y_five).double().norm() / (nrm * u.double().norm()))
    assert err <= 2e-6, err
    assert torch.equal(y_fused, _both(lambda: op.apply(u))[0])  # deterministic
    if op.info()["precond_ok"]:
        z_fused, z_five = _both(lambda: op.precond(u))
        # relative to ||z||: FP32 rounding times the tau symbol's spread (up to 1e3 here);
        # a wrong transform would differ at O(1)
        rel = float((z_fused - z_five).double().norm() / z_five.double().norm())
        assert rel <= 1e-3, rel
    op.close()


@pytest.mark.parametrize("n,alpha", [(63, 1.6), (127, 0.4)])
def test_fused_xy_solves_equal_five_pass_solves(n, alpha):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(3, n, alpha, degree=1)
    f = torch.tensor(synth.ball_power_rhs(3, n, alpha), device="cuda")
    (u1, i1), (u2, i2) = _both(lambda: op.solve(f, rtol=1e-10, precision="mixed"))
    assert i1["status"] == 0 and i1["rel_resid"] <= 1e-10 and i2["status"] == 0
    kappa = op.info()["norm_bound"] * float(u2.norm()) / float(f.norm())
    assert float((u1 - u2).norm() / u2.norm()) <= 4e-10 * max(kappa, 1.0)
    op.close()
