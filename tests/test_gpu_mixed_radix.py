"""GPU parity for mixed-radix FFT lengths (fft="smooth": M_i the smallest 2^a 3^b 5^c 7^d
>= 2 n_i + 2 with a >= 4; Sec. 2.1 only needs a circulant embedding of length >= 2 n_i - 1):
the apply (FP64 and FP32), the tau preconditioner of size m_i = M_i/2 - 1, the solves
(whole-solve 1D kernel, engine and graph paths for d = 2, 3) and batches against the
oracle, with the bars of the power-of-two tests: apply ||y - y_ref|| / (||A||_2 ||u||) <=
1e-12 (FP64) / 1e-5 (FP32), ||A||_2 bounded by the oracle's row-sum bound; preconditioner
the same with ||P||_2 = 1 / min tau symbol; solves: the oracle's residual of the returned u
<= rtol plus the generator slack.  The same operator on power-of-two lengths is a second,
independent embedding of the same matrix: both applies agree to FP64 rounding."""
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


def _op(d, n, p, alpha, lam=0.0, fft="smooth"):
    import paper_2103_03658_gb300 as fg
    return fg.FracOp(d, n, alpha, degree=p, lam=lam, fft=fft)


_GEN = {}


def _oracle(d, ns, p, alpha, lam):
    key = (d, ns, p, alpha, lam)
    if key not in _GEN:
        N = max(ns) + 1
        _GEN[key] = (O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12), O.c_dalpha(d, alpha))
    return _GEN[key]


def _is_pow2(m):
    return m & (m - 1) == 0


# (d, n or per-axis n, degree, alpha, lambda, batch); every case has a non-power-of-two axis
APPLY_CASES = [
    (1, 23, 1, 1.2, 0.0, 3),      # M = 48 = 16 * 3
    (1, 39, 2, 0.6, 0.7, 2),      # 80 = 16 * 5
    (1, 99, 0, 1.5, 0.0, 3),      # 224 = 32 * 7
    (1, 1001, 1, 1.9, 0.0, 2),    # 2016 = 32 * 63
    (1, 2999, 2, 0.4, 1.1, 1),    # 6000 = 2^4 * 3 * 5^3
    (2, 23, 1, 1.2, 0.0, 2),
    (2, 39, 2, 1.6, 0.4, 1),
    (2, 99, 1, 0.8, 0.0, 1),      # sampled rows
    (2, (39, 23), 1, 1.0, 0.0, 2),  # M = (80, 48)
    (2, (31, 45), 0, 1.4, 0.0, 1),  # M = (64, 96): the row axis a power of two
    (3, 21, 1, 1.3, 0.0, 1),      # 48^3
    (3, 23, 1, 0.7, 0.0, 1),      # 48^3, sampled rows
    (3, (19, 23, 11), 2, 1.6, 0.2, 1),  # (48, 48, 32)
]


def _fields(shape, batch, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch,) + shape)


def _rows(shape, count, seed):
    rng = np.random.default_rng(seed)
    rows = [tuple(0 for _ in shape), tuple(s - 1 for s in shape), tuple(s // 2 for s in shape)]
    rows += [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(count)]
    return np.array(rows)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,n,p,alpha,lam,batch", APPLY_CASES)
def test_mixed_apply_matches_oracle(d, n, p, alpha, lam, batch, dtype):
    ns = tuple(n) if isinstance(n, tuple) else (n,) * d
    op = _op(d, n, p, alpha, lam)
    info = op.info()
    import paper_2103_03658_gb300 as fg
    assert info["fft_lens"] == tuple(fg.fft_length(v, d, "smooth") for v in ns)
    shape = tuple(reversed(ns))
    a, c = _oracle(d, ns, p, alpha, lam)
    if dtype == "f64":
        assert np.max(np.abs(op.generator() - a)) <= 1e-13 * np.max(np.abs(a))
    nrm = O.norm_bound(a, c, shape)
    U = _fields(shape, batch, 31 * sum(ns) + d)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = op.apply(torch.tensor(U, dtype=tdt, device="cuda")).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(batch):
        ub = U[b] if dtype == "f64" else U[b].astype(np.float32).astype(np.float64)
        if np.prod(shape) <= 6000:
            ref = O.apply_dense(a, c, ub)
            err = np.linalg.norm(y[b] - ref) / (nrm * np.linalg.norm(ub))
        else:
            rows = _rows(shape, 40, b + 5)
            ref = O.apply_rows(a, c, ub, rows)
            got = y[b][tuple(rows.T)]
            err = np.linalg.norm(got - ref) / (nrm * np.linalg.norm(ub) * np.sqrt(len(rows) / ub.size))
        assert err <= tol, (b, err)
    op.close()


@pytest.mark.parametrize("d,n,p,alpha", [(1, 1001, 1, 1.3), (1, 2999, 2, 1.9), (2, 99, 2, 0.9), (2, (39, 23), 1, 1.5),
                                         (3, 23, 1, 0.5), (3, (19, 23, 11), 0, 1.2)])
def test_mixed_and_power_of_two_embeddings_agree(d, n, p, alpha):
    """Two circulant embeddings of the same Toeplitz matrix: the applies differ only by
    rounding (FP64: 1e-13 of ||A|| ||u||; FP32: 2e-6)."""
    op_m, op_p = _op(d, n, p, alpha), _op(d, n, p, alpha, fft="pow2")
    assert any(not _is_pow2(m) for m in op_m.info()["fft_lens"])
    assert np.array_equal(op_m.generator(), op_p.generator())
    nrm = op_p.info()["norm_bound"]
    rng = np.random.default_rng(11)
    u = rng.standard_normal((3,) + op_p.shape)
    for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
        ud = torch.tensor(u, dtype=dt, device="cuda")
        ym, yp = op_m.apply(ud).double(), op_p.apply(ud).double()
        err = float((ym - yp).norm() / (nrm * ud.double().norm()))
        assert err <= tol, (dt, err)
    assert abs(op_m.info()["norm_bound"] - nrm) <= 0.2 * nrm  # both sample the same symbol
    op_m.close()
    op_p.close()


PRECOND_CASES = [(1, 23, 1, 1.2, 0.0, 2), (1, 99, 2, 0.4, 0.0, 1), (1, 1001, 0, 1.5, 1.0, 2),
                 (2, 23, 1, 1.0, 0.0, 1), (2, 39, 2, 1.6, 0.3, 2), (2, (39, 23), 1, 0.8, 0.0, 1),
                 (3, 19, 1, 0.7, 0.0, 1), (3, (19, 23, 11), 1, 1.3, 0.0, 1)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,n,p,alpha,lam,batch", PRECOND_CASES)
def test_mixed_precond_matches_oracle(d, n, p, alpha, lam, batch, dtype):
    ns = tuple(n) if isinstance(n, tuple) else (n,) * d
    shape = tuple(reversed(ns))
    op = _op(d, n, p, alpha, lam)
    info = op.info()
    assert info["precond_ok"] == 1
    m = tuple(reversed([M // 2 - 1 for M in info["fft_lens"]]))  # per array axis
    a, c = _oracle(d, ns, p, alpha, lam)
    pnorm = 1.0 / np.min(O.tau_symbol(a, c, shape, m))
    R = _fields(shape, batch, 7 * sum(ns) + d)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    z = op.precond(torch.tensor(R, dtype=tdt, device="cuda")).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(batch):
        rr = R[b] if dtype == "f64" else R[b].astype(np.float32).astype(np.float64)
        ref = O.tau_precond(a, c, rr, m)
        err = np.linalg.norm(z[b] - ref) / (pnorm * np.linalg.norm(rr))
        assert err <= tol, (b, err)
    op.close()


def test_smooth_lengths_give_the_preconditioner_to_power_of_two_sizes():
    """n a power of two has no tau system on its power-of-two embedding (M/2 - 1 < n);
    the smooth length is >= 2 n + 2, so the preconditioner applies."""
    for d, n in ((1, 16), (1, 512), (2, 64), (3, 16)):
        op_p, op_m = _op(d, n, 1, 1.1, fft="pow2"), _op(d, n, 1, 1.1)
        assert op_p.info()["precond_ok"] == 0 and op_m.info()["precond_ok"] == 1
        f = torch.ones((n,) * d, dtype=torch.float64, device="cuda")
        u, info = op_m.solve(f, rtol=1e-10)
        assert info["status"] == 0 and info["precond"] == 1
        op_p.close()
        op_m.close()


SOLVE_CASES = [(1, 99, 1, 1.5, 0.0), (1, 1001, 2, 1.9, 1.2), (1, 2999, 1, 0.6, 0.0), (2, 39, 1, 1.2, 0.0),
               (2, 45, 2, 0.5, 0.7), (2, (39, 23), 0, 1.8, 0.0), (3, 19, 2, 1.6, 0.3), (3, 23, 1, 0.4, 0.0)]


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("d,n,p,alpha,lam", SOLVE_CASES)
def test_mixed_solve_residual_recomputed_by_oracle(d, n, p, alpha, lam, precision):
    ns = tuple(n) if isinstance(n, tuple) else (n,) * d
    shape = tuple(reversed(ns))
    a, c = _oracle(d, ns, p, alpha, lam)
    rng = np.random.default_rng(2103 + sum(ns))
    f = rng.standard_normal(shape) * 0.1 + 0.5
    op = _op(d, n, p, alpha, lam)
    assert any(not _is_pow2(m) for m in op.info()["fft_lens"])
    fd = torch.tensor(f, device="cuda")
    u, info = op.solve(fd, rtol=1e-10, precision=precision)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10 and info["precond"] == 1
    uh = u.cpu().numpy()
    if np.prod(shape) <= 16000:
        A = O.operator_matrix(a, c, shape)
        res = np.linalg.norm(f.reshape(-1) - A @ uh.reshape(-1)) / np.linalg.norm(f)
    else:
        rows = _rows(shape, 60, 3)
        r = f[tuple(rows.T)] - O.apply_rows(a, c, uh, rows)
        res = np.linalg.norm(r) / (np.linalg.norm(f) * np.sqrt(len(rows) / f.size))
    da = np.abs(op.generator() - a)
    K = np.indices(da.shape)
    slack = c * float(np.sum(2.0 ** np.sum(K > 0, axis=0) * da)) * np.linalg.norm(uh) / np.linalg.norm(f)
    assert res <= 1e-10 * 1.05 + 2 * slack + (0 if np.prod(shape) <= 16000 else 2e-10), (res, slack)
    # the same solution as on the power-of-two embedding
    op_p = _op(d, n, p, alpha, lam, fft="pow2")
    u_p, info_p = op_p.solve(fd, rtol=1e-10, precision=precision, precond="none")
    kappa = op.info()["norm_bound"] * float(u.norm()) / float(fd.norm())
    assert float((u - u_p).norm() / u_p.norm()) <= 4e-10 * max(kappa, 1.0)
    op.close()
    op_p.close()


def test_mixed_batch_and_engine_match_single_solves():
    """A batch mixing power-of-two and mixed lengths: 1D problems of both kinds in the
    captured graph (one whole-solve launch per length), square 2D power-of-two problems in
    the persistent launch, the mixed 2D and the 3D ones through the engine.  Every result
    equals the single solve of the same problem to the solve tolerance, and the oracle
    recomputes three residuals."""
    import paper_2103_03658_gb300 as fg
    probs = [(1, 99, 1, 0.7, "smooth"), (1, 127, 1, 0.7, "pow2"), (1, 1001, 2, 1.3, "smooth"),
             (1, 23, 0, 1.1, "smooth"), (2, 39, 1, 1.2, "smooth"), (2, 63, 1, 1.2, "pow2"),
             (2, 45, 2, 0.5, "smooth"), (3, 19, 1, 1.6, "smooth"), (1, 99, 1, 0.7, "smooth")]
    ops = [_op(d, n, p, al, fft=ff) for d, n, p, al, ff in probs]
    rng = np.random.default_rng(5)
    fs = [torch.tensor(rng.standard_normal((n,) * d) * 0.1 + 0.5, device="cuda") for d, n, _, _, _ in probs]
    us = [torch.empty_like(f) for f in fs]
    infos = fg.solve_batch(ops, fs, us, rtol=1e-10)
    for i, (op, f, u, inf) in enumerate(zip(ops, fs, us, infos)):
        assert inf["status"] == 0 and inf["rel_resid"] <= 1e-10, (i, inf)
        u1, _ = op.solve(f, rtol=1e-10)
        kappa = op.info()["norm_bound"] * float(u1.norm()) / float(f.norm())
        assert float((u - u1).norm() / u1.norm()) <= 4e-10 * max(kappa, 1.0), i
    for i in (0, 4, 7):
        d, n, p, al, _ = probs[i]
        a, c = _oracle(d, (n,) * d, p, al, 0.0)
        A = O.operator_matrix(a, c, (n,) * d)
        fh, uh = fs[i].cpu().numpy(), us[i].cpu().numpy()
        res = np.linalg.norm(fh.reshape(-1) - A @ uh.reshape(-1)) / np.linalg.norm(fh)
        assert res <= 2e-10, (i, res)
    for op in ops:
        op.close()


def test_mixed_apply_is_deterministic_and_host_buffers_match():
    op = _op(2, 99, 1, 1.1)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((5, 99, 99)).astype(np.float32)
    ud = torch.tensor(u, device="cuda")
    y1, y2 = op.apply(ud), op.apply(ud)
    assert torch.equal(y1, y2)
    yh = op.apply(torch.tensor(u))  # host buffers through the C ABI
    assert torch.equal(yh, y1.cpu())
    op.close()


def test_batch_slots_hold_the_largest_spectrum_not_the_largest_n():
    """With per-operator FFT lengths the largest n of a queue need not have the largest
    spectrum (n = 310 on 640 points against n = 300 on 1024): the persistent batch sizes
    each worker's scratch by the largest spectrum and the largest n separately.  Every
    result equals its single solve."""
    import paper_2103_03658_gb300 as fg
    probs = [(310, "smooth"), (300, "pow2"), (305, "pow2"), (200, "smooth"), (250, "pow2"), (311, "smooth")]
    ops = [_op(2, n, 1, 1.2, fft=ff) for n, ff in probs]
    lens = [op.info()["fft_len"] for op in ops]
    assert lens[0] == 640 and lens[1] == 1024
    rng = np.random.default_rng(8)
    fs = [torch.tensor(rng.standard_normal((n, n)) * 0.1 + 0.5, device="cuda") for n, _ in probs]
    us = [torch.empty_like(f) for f in fs]
    for size in (0, 1):  # the autotuner's choice, then every problem on a CTA of its own
        fg.batch_pin_plan(size)
        infos = fg.solve_batch(ops, fs, us, rtol=1e-10)
        fg.batch_pin_plan(0)
        for i, (op, f, u, inf) in enumerate(zip(ops, fs, us, infos)):
            assert inf["status"] == 0 and inf["rel_resid"] <= 1e-10, (size, i, inf)
            u1, _ = op.solve(f, rtol=1e-10)
            kappa = op.info()["norm_bound"] * float(u1.norm()) / float(f.norm())
            assert float((u - u1).norm() / u1.norm()) <= 4e-10 * max(kappa, 1.0), (size, i)
    for op in ops:
        op.close()


def test_boundary_vector_does_not_depend_on_the_fft_length():
    """frac_boundary convolves the exterior samples on a circulant of its own (power-of-two)
    side, so the boundary vector of an operator on mixed lengths is the one on powers of two."""
    for d, n in ((1, 99), (2, 39)):
        op_m, op_p = _op(d, n, 1, 1.3), _op(d, n, 1, 1.3, fft="pow2")
        rng = np.random.default_rng(d)
        g = torch.tensor(rng.standard_normal(op_p.ext_shape), device="cuda")
        assert torch.equal(op_m.boundary(g), op_p.boundary(g))
        op_m.close()
        op_p.close()
