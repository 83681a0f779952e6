"""GPU parity, coefficients and apply: the sm_103a library (through the C ABI)
against the FP64 oracle on the same seeded inputs.

Tolerances.  Generator a_k: 1e-13 relative to max |a| (both sides integrate
to ~1e-15; the centre coefficient is a sum of (N+1)^d terms).  Apply: the
normwise error ||y - y_ref||_2 / (||A||_2 ||u||_2), ||A||_2 bounded by the
oracle's row-sum bound, at most 1e-12 for FP64 and 1e-5 for FP32 (an FFT of
length M^d has relative error ~ eps log2(M^d): 3e-15 and 1.6e-6 here).
"""
import itertools

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
    import paper_2103_03658_gb300 as fg
    fg.load()


def _op(d, n, p, alpha, lam):
    import paper_2103_03658_gb300 as fg
    return fg.FracOp(d, n, alpha, degree=p, lam=lam)


_GEN_CACHE = {}


def oracle_operator(d, n, p, alpha, lam):
    key = (d, n, p, alpha, lam)
    if key not in _GEN_CACHE:
        N = n + 1
        a = O.stencil(d, N, 2.0 / N, alpha, p, lam, q=20 if d < 3 else 12)
        _GEN_CACHE[key] = (a, O.c_dalpha(d, alpha))
    return _GEN_CACHE[key]


GEN_CASES = [
    (1, 1, 1, 1.2, 0.0), (1, 2, 0, 0.5, 0.0), (1, 7, 2, 0.3, 0.8), (1, 31, 1, 1.5, 0.0), (1, 1023, 1, 0.5, 0.0),
    (1, 1023, 1, 1.0, 0.0), (1, 1023, 1, 1.5, 0.0), (1, 4095, 2, 1.9, 1.7),
    (2, 1, 2, 1.2, 0.0), (2, 3, 0, 1.9, 0.0), (2, 15, 1, 0.7, 0.0), (2, 31, 2, 1.2, 0.5), (2, 20, 0, 0.1, 2.0),
    (3, 1, 0, 1.0, 0.0), (3, 5, 0, 1.0, 1.3), (3, 7, 1, 0.4, 0.0), (3, 9, 2, 1.6, 0.0), (3, 16, 1, 1.6, 0.4),
]


@pytest.mark.parametrize("d,n,p,alpha,lam", GEN_CASES)
def test_generator_matches_oracle(d, n, p, alpha, lam):
    op = _op(d, n, p, alpha, lam)
    a_gpu = op.generator()
    a_ref, c = oracle_operator(d, n, p, alpha, lam)
    scale = np.max(np.abs(a_ref))
    assert np.max(np.abs(a_gpu - a_ref)) <= 1e-13 * scale
    info = op.info()
    assert abs(info["c_dalpha"] - c) <= 1e-14 * c
    F = O.far_field(d, alpha, 2.0, lam)
    assert abs(info["far_field"] - F) <= 1e-12 * F
    assert info["norm_bound"] <= O.norm_bound(a_ref, c, n) * (1 + 1e-12)
    op.close()


def test_generator_2d_full_size_quadratic():
    """1023^2 grid (N = 1024), alpha = 1.2, p = 2: the whole generator."""
    test_generator_matches_oracle(2, 1023, 2, 1.2, 0.0)


@pytest.mark.parametrize("alpha", [0.4, 1.6])
def test_generator_3d_full_size_sampled(alpha):
    """255^3 grid (N = 256), p = 1: sampled weights computed one by one by the
    oracle; a_k = 2^{z(k)} omega_k / |xi_k|^2 (+ origin rule on the axes)."""
    d, n, p = 3, 255, 1
    N = n + 1
    h = 2.0 / N
    op = _op(d, n, p, alpha, 0.0)
    a_gpu = op.generator()
    rng = np.random.default_rng(2103)
    nodes = [(0, 0, 0), (1, 0, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1), (2, 0, 0), (N, N, N), (N, 0, 0), (0, N, 3),
             (5, 7, 11), (128, 128, 128), (200, 3, 100)]
    nodes += [tuple(int(v) for v in rng.integers(0, N + 1, size=3)) for _ in range(40)]
    w = O.weights_at(d, N, h, alpha, p, 0.0, nodes + [(0, 0, 0)])
    w0 = w[-1]
    for k, wk in zip(nodes, w[:-1]):
        if k == (0, 0, 0):
            continue
        z = sum(1 for t in k if t == 0)
        ak = 2.0 ** z * wk / (h * h * sum(t * t for t in k))
        if z == d - 1 and max(k) == 1:
            ak += 2.0 ** (d - 1) * w0 / (d * h * h)
        # generator stored with k_1 fastest: a_gpu[k3, k2, k1]
        assert abs(a_gpu[k[2], k[1], k[0]] - ak) <= 1e-13 * abs(ak), k
    op.close()


@pytest.mark.parametrize("n,p,alpha,lam", [(127, 2, 0.9, 1.5), (255, 0, 1.7, 0.6)])
def test_generator_3d_tempered_sampled(n, p, alpha, lam):
    """Tempered 3D generators, sampled far and near nodes (the far elements' kernel comes from
    a per-element Taylor series on the device): a_k from the oracle's weights at those nodes,
    origin rule e = (1) (p <= 1) or (4/3, -1/3) (p = 2) on the axes."""
    d = 3
    N = n + 1
    h = 2.0 / N
    op = _op(d, n, p, alpha, lam)
    a_gpu = op.generator()
    rng = np.random.default_rng(31)
    nodes = [(1, 0, 0), (2, 0, 0), (0, 2, 0), (1, 1, 1), (N, N, N), (N, 1, 0), (N // 2, 3, N - 2), (40, 41, 42)]
    nodes += [tuple(int(v) for v in rng.integers(0, N + 1, size=3)) for _ in range(24)]
    w = O.weights_at(d, N, h, alpha, p, lam, nodes + [(0, 0, 0)])
    w0 = w[-1]
    e = (1.0,) if p <= 1 else (4.0 / 3.0, -1.0 / 3.0)
    for k, wk in zip(nodes, w[:-1]):
        z = sum(1 for t in k if t == 0)
        ak = 2.0 ** z * wk / (h * h * sum(t * t for t in k))
        if z == d - 1 and max(k) <= len(e):
            j = max(k)
            ak += 2.0 ** (d - 1) * e[j - 1] * w0 / (d * (j * h) ** 2)
        assert abs(a_gpu[k[2], k[1], k[0]] - ak) <= 1e-13 * abs(ak) + 1e-16 * abs(a_gpu).max(), k
    op.close()


# ---------------------------------------------------------------------------
# apply
# ---------------------------------------------------------------------------

def _fields(d, n, batch, seed):
    rng = np.random.default_rng(seed)
    out = [synth.smooth_field(d, n, seed + j) + 0.1 * rng.standard_normal((n,) * d) for j in range(batch)]
    return np.stack(out)


def _reference(a, c, u):
    """Oracle apply: all rows when n^d <= 5000, else seeded sampled rows."""
    d = u.ndim
    n = u.shape[0]
    if n ** d <= 5000:
        return O.apply_dense(a, c, u), None
    rng = np.random.default_rng(7)
    rows = [tuple([0] * d), tuple([n - 1] * d), tuple([n // 2] * d)]
    rows += [tuple(int(v) for v in rng.integers(0, n, size=d)) for _ in range(29)]
    rows = np.array(rows)
    return O.apply_rows(a, c, u, rows), rows


APPLY_CASES = [
    (1, 1, 1, 1.2, 0.0, 1), (1, 2, 0, 0.5, 0.0, 2), (1, 5, 1, 1.5, 0.0, 3), (1, 63, 2, 0.3, 0.8, 3),
    (1, 100, 1, 1.0, 0.0, 5), (1, 1023, 1, 1.5, 0.0, 3), (1, 4095, 2, 1.9, 1.7, 2),
    (2, 1, 2, 1.2, 0.0, 1), (2, 3, 0, 1.9, 0.0, 2), (2, 17, 1, 0.7, 0.0, 3), (2, 63, 2, 1.2, 0.5, 2),
    (2, 100, 0, 0.1, 2.0, 1), (2, 129, 1, 1.6, 0.0, 2),
    (3, 1, 0, 1.0, 0.0, 1), (3, 3, 1, 0.4, 0.0, 3), (3, 9, 2, 1.6, 0.0, 2), (3, 17, 1, 1.6, 0.4, 1),
    (3, 31, 1, 0.4, 0.0, 1),
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("d,n,p,alpha,lam,batch", APPLY_CASES)
def test_apply_matches_oracle(d, n, p, alpha, lam, batch, dtype):
    a, c = oracle_operator(d, n, p, alpha, lam)
    nrm = O.norm_bound(a, c, n)
    U = _fields(d, n, batch, 100 * n + d)
    op = _op(d, n, p, alpha, lam)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u_dev = torch.tensor(U, dtype=tdt, device="cuda")
    y = op.apply(u_dev).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(batch):
        ref, rows = _reference(a, c, U[b])
        got = y[b] if rows is None else y[b][tuple(rows.T)]
        uu = U[b] if dtype == "f64" else U[b].astype(np.float32).astype(np.float64)
        if dtype == "f32" and rows is None:
            ref = O.apply_dense(a, c, uu)
        elif dtype == "f32":
            ref = O.apply_rows(a, c, uu, rows)
        err = np.linalg.norm(got - ref) / (nrm * np.linalg.norm(uu) * (1 if rows is None else np.sqrt(len(rows) / uu.size)))
        assert err <= tol, (b, err)
    op.close()


def test_apply_batch_equals_single_and_host_buffers():
    d, n, p, alpha = 2, 33, 1, 0.9
    op = _op(d, n, p, alpha, 0.0)
    U = _fields(d, n, 3, 11)
    u_dev = torch.tensor(U, dtype=torch.float64, device="cuda")
    yb = op.apply(u_dev).cpu().numpy()
    for b in range(3):
        ys = op.apply(u_dev[b].contiguous()).cpu().numpy()
        assert np.array_equal(ys, yb[b]) or np.max(np.abs(ys - yb[b])) <= 1e-15 * np.max(np.abs(yb))
    yh = op.apply(U.copy())          # numpy host buffers: staged through the device by the library
    assert np.max(np.abs(yh - yb)) <= 1e-15 * np.max(np.abs(yb))
    op.close()


@pytest.mark.parametrize("dtype,batch", [("f32", 29), ("f64", 13)])
def test_apply_host_buffers_pipelined_equals_device(dtype, batch):
    """Large host batches (twice the 28 MB chunk or more; here >= 96 MB) go through the chunked
    copy/apply/copy pipeline of the library (three streams, a ring of device buffers); every field must match the device-buffer
    apply of the whole batch, from pageable and from pinned host memory.  Rows are
    paired two per complex FFT across the batch, so a chunk boundary changes which rows
    share a transform: equal up to the FFT's rounding (normwise 1e-6 FP32, 1e-14 FP64)."""
    op = _op(2, 1023, 2, 1.2, 0.0)
    U = np.random.default_rng(5).standard_normal((batch, 1023, 1023)).astype(np.float32 if dtype == "f32" else np.float64)
    assert U.nbytes >= 96 << 20
    y_dev = op.apply(torch.from_numpy(U).cuda()).cpu().numpy()
    tol = 1e-6 if dtype == "f32" else 1e-14
    y_host = op.apply(U)                                   # pageable numpy buffers
    hu = torch.from_numpy(U).pin_memory()
    hy = torch.empty_like(hu).pin_memory()
    op.apply(hu, out=hy)
    for y in (y_host, hy.numpy()):
        for b in range(batch):
            assert np.linalg.norm(y[b] - y_dev[b]) <= tol * np.linalg.norm(y_dev[b]), b
    op.close()


def _check_sampled(got, ref, uu, nrm, rho, tol, nrows, what):
    """Sampled-row checks of one field: the normwise error (the row error scaled by
    sqrt(rows / points) to a whole-vector estimate) against tol ||A|| ||u|| with the
    row-sum bound, and the plain relative error ||y - y_ref|| / ||y_ref|| over the rows
    against tol kappa_y, kappa_y = rho ||u|| / ||A u|| with rho the circulant bound of
    ||A||_2 (the tighter of the two).  Returns (relative error, kappa_y)."""
    scale = np.sqrt(nrows / uu.size)
    e = np.linalg.norm(got - ref)
    assert e <= tol * nrm * np.linalg.norm(uu) * scale, (what, e / (nrm * np.linalg.norm(uu) * scale))
    rel = e / np.linalg.norm(ref)
    kappa_y = rho * np.linalg.norm(uu) * scale / np.linalg.norm(ref)
    assert rel <= tol * kappa_y, (what, rel, kappa_y)
    return rel, kappa_y


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_apply_2d_full_size_sampled_rows(dtype):
    """The bench workload: 1023^2 grid, alpha = 1.2, p = 2, 65 fields (u_exact and 64
    smooth random fields) in one call, FP32 (the bench's precision) and FP64; sampled
    rows of four fields against the oracle, normwise and plain relative errors."""
    d, n, p, alpha = 2, 1023, 2, 1.2
    a, c = oracle_operator(d, n, p, alpha, 0.0)
    nrm = O.norm_bound(a, c, n)
    rho = O.spectral_bound(a, c, n)
    op = _op(d, n, p, alpha, 0.0)
    fields = np.concatenate([synth.ball_power(d, n, 1 + alpha / 2)[None], synth.smooth_fields(d, n, 64)])
    tdt = torch.float32 if dtype == "f32" else torch.float64
    u_dev = torch.tensor(fields, dtype=tdt, device="cuda")
    y = op.apply(u_dev).double().cpu().numpy()
    tol = 1e-5 if dtype == "f32" else 1e-12
    rng = np.random.default_rng(3)
    for b in (0, 1, 31, 64):
        rows = np.array([[0, 0], [n - 1, n - 1], [511, 511], [0, n - 1]] + [list(rng.integers(0, n, 2)) for _ in range(28)])
        uu = fields[b].astype(np.float32).astype(np.float64) if dtype == "f32" else fields[b]
        ref = O.apply_rows(a, c, uu, rows)
        got = y[b][tuple(rows.T)]
        rel, kap = _check_sampled(got, ref, uu, nrm, rho, tol, len(rows), (dtype, b))
        print(f"2D 1023^2 {dtype} field {b}: rel {rel:.2e}, kappa_y {kap:.1f}")
    op.close()


_GEN3D = {}


def _oracle_generator_3d(n, p, alpha):
    """The oracle's whole 3D generator for the 255^3 grid (N = 256), its weights summed
    by a pool of host processes (about a minute on 16 cores)."""
    import _oracle_pool as P
    key = (n, p, alpha)
    if key not in _GEN3D:
        a, c = P.stencil(3, n + 1, alpha, p, 0.0, q=12)
        _GEN3D[key] = (a, c, O.norm_bound(a, c, n), O.spectral_bound(a, c, n))
    return _GEN3D[key]


_ROWS3D = {}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_apply_3d_full_size_sampled_rows(dtype):
    """The 3D configuration at full size: 255^3 grid on a 512^3 FFT grid, alpha = 1.6,
    p = 1, one seeded smooth-plus-noise field (rounded to FP32, so that both precisions
    apply the same vector); 256 seeded rows (corners, faces, centre and random points)
    against the oracle's dense rows built from its own whole generator."""
    import _oracle_pool as P
    d, n, p, alpha = 3, 255, 1, 1.6
    a, c, nrm, rho = _oracle_generator_3d(n, p, alpha)
    rng = np.random.default_rng(255)
    U = (synth.smooth_field(d, n, 4242) + 0.1 * rng.standard_normal((n,) * d)).astype(np.float32).astype(np.float64)
    corners = [[i, j, k] for i in (0, n - 1) for j in (0, n - 1) for k in (0, n - 1)]
    rows = np.array(corners + [[n // 2] * 3, [0, n // 2, n // 2], [n - 1, 1, 128]] +
                    [list(rng.integers(0, n, 3)) for _ in range(256 - 11)])
    op = _op(d, n, p, alpha, 0.0)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    y = op.apply(torch.tensor(U, dtype=tdt, device="cuda")).double().cpu().numpy()
    op.close()
    if "ref" not in _ROWS3D:
        _ROWS3D["ref"] = P.apply_rows(a, c, U, rows)
    ref = _ROWS3D["ref"]
    got = y[tuple(rows.T)]
    tol = 1e-5 if dtype == "f32" else 1e-12
    rel, kap = _check_sampled(got, ref, U, nrm, rho, tol, len(rows), dtype)
    print(f"3D 255^3 {dtype}: rel {rel:.2e}, kappa_y {kap:.1f}")


def test_apply_3d_full_size_properties():
    """255^3 grid on a 512^3 FFT grid: the oracle cannot form the whole
    generator here, so check properties that hold at any size: symmetry
    <v, A u> = <A v, u>, FP32 against FP64, and the discretization error of
    A u against the closed form (-Delta)^{alpha/2} (1-|x|^2)_+^{1+alpha/2}."""
    d, n, p, alpha = 3, 255, 1, 1.6
    op = _op(d, n, p, alpha, 0.0)
    rng = np.random.default_rng(5)
    u = torch.tensor(rng.standard_normal((n,) * d), dtype=torch.float64, device="cuda")
    v = torch.tensor(rng.standard_normal((n,) * d), dtype=torch.float64, device="cuda")
    Au, Av = op.apply(u), op.apply(v)
    lhs, rhs = float((v * Au).sum()), float((Av * u).sum())
    nrm = op.info()["norm_bound"]
    assert abs(lhs - rhs) <= 1e-12 * nrm * float(u.norm()) * float(v.norm())
    Au32 = op.apply(u.float()).double()
    assert float((Au32 - Au).norm()) <= 1e-5 * nrm * float(u.norm())
    ue = torch.tensor(synth.ball_power(d, n, 1 + alpha / 2), device="cuda")
    f = torch.tensor(synth.ball_power_rhs(d, n, alpha), device="cuda")
    r2 = torch.tensor(synth.radius2(d, n), device="cuda")
    inner = r2 < 0.25
    err = float((op.apply(ue) - f)[inner].abs().max())
    assert err < 1e-2 * float(f.abs().max())
    op.close()
