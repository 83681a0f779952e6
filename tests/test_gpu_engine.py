"""GPU: the solve engine and the serving loop give, for every problem, the
solution that a solve alone gives (continuous batching changes scheduling,
not results), within the solve tolerance: ||u_mix - u_alone|| <= 1e-8 ||u_alone||
for rtol = 1e-10 solves of systems with kappa <= 1e3 scale."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


MIX = [(1, 255, 1, 0.7, 0.0, "mixed"), (1, 1023, 2, 1.5, 0.3, "f64"), (2, 63, 1, 1.2, 0.0, "mixed"),
       (2, 127, 2, 0.6, 1.1, "f64"), (3, 31, 1, 1.6, 0.0, "mixed"), (2, 255, 0, 1.9, 0.0, "mixed"),
       (1, 4095, 0, 0.3, 0.0, "mixed"), (3, 63, 2, 0.9, 0.5, "mixed")]


def test_engine_mix_equals_alone():
    import paper_2103_03658_gb300 as fg
    ops, fs = [], []
    for i, (d, n, p, a, lam, prec) in enumerate(MIX):
        ops.append(fg.FracOp(d, n, a, degree=p, lam=lam))
        fs.append(torch.tensor(synth.smooth_field(d, n, 50 + i) + 0.3, device="cuda"))
    eng = fg.Engine(nstreams=4)
    jobs = {}
    for i, (op, f, m) in enumerate(zip(ops, fs, MIX)):
        j, u = eng.submit(op, f, precision=m[5])
        jobs[j] = (i, u)
    got = {}
    while len(got) < len(MIX):
        for j, info, ms, u in eng.poll(block=True):
            got[jobs[j][0]] = (info, u)
    eng.close()
    for i, (op, f, m) in enumerate(zip(ops, fs, MIX)):
        info, u_mix = got[i]
        assert info["status"] == 0 and info["rel_resid"] <= 1e-10, (m, info)
        u_alone, info1 = op.solve(f, rtol=1e-10, precision=m[5])
        rel = float((u_mix - u_alone).norm() / u_alone.norm())
        assert rel <= 1e-8, (m, rel)
        op.close()


def test_engine_host_buffers():
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(2, 95, 1.1, degree=1)
    f = synth.smooth_field(2, 95, 9) + 1.0
    u = np.empty_like(f)
    eng = fg.Engine(nstreams=2)
    j, u_out = eng.submit(op, f, u)
    res = []
    while not res:
        res = eng.poll(block=True)
    eng.close()
    assert res[0][1]["status"] == 0
    u_dev, _ = op.solve(torch.tensor(f, device="cuda"), rtol=1e-10)
    assert np.linalg.norm(u - u_dev.cpu().numpy()) <= 1e-8 * np.linalg.norm(u)
    op.close()


def test_served_stream_each_result_same_as_alone():
    """A short Poisson-arrival stream of mixed requests through the serving loop;
    every result matches the solve of the same request alone."""
    import paper_2103_03658_gb300 as fg
    from paper_2103_03658_gb300 import serve
    probs = synth.served_problems(24, seed=11, sides3d=(15, 31))
    arr = synth.arrival_times(rate=200.0, duration=1.0, seed=11)[:24]
    reqs = []
    for i, (pb, t) in enumerate(zip(probs, arr)):
        n = min(pb.n, 255) if pb.d == 2 else pb.n
        if pb.degree == 2 and n % 2 == 0:
            n += 1
        reqs.append(serve.Request(i, pb.d, n, pb.alpha, pb.degree, pb.lam,
                                  synth.smooth_field(pb.d, n, pb.seed) + 0.2, float(t)))
    srv = serve.Server(hbm_budget=20e9, nstreams=8)
    res = srv.run(reqs, realtime=True)
    srv.close()
    assert len(res) == len(reqs)
    for r, q in zip(res, reqs):
        assert r.info["status"] == 0 and r.info["rel_resid"] <= 1e-10
        assert r.latency_s >= r.queue_s >= 0.0
        op = fg.FracOp(q.d, q.n, q.alpha, degree=q.degree, lam=q.lam)
        u1, _ = op.solve(torch.tensor(q.f, device="cuda"), rtol=1e-10)
        u1 = u1.cpu().numpy()
        assert np.linalg.norm(np.asarray(r.u) - u1) <= 1e-8 * np.linalg.norm(u1)
        op.close()


def test_served_results_checked_by_oracle():
    """Served results against the oracle: a stream of mixed requests (1D up to n = 4095,
    2D sides up to 255, 3D sides 15 and 31) through the serving loop, and for every other
    request the oracle's relative residual ||f - A u|| / ||f|| with its own generator (all
    rows in 1D and for n^d <= 4096, 64 seeded rows otherwise) within the solve tolerance
    plus the oracle's own FP64 rounding of A u."""
    import math

    from paper_2103_03658_gb300 import serve
    from oracle import frac_oracle as O
    probs = synth.served_problems(20, seed=29, sides3d=(15, 31))
    reqs = []
    for i, pb in enumerate(probs):
        n = min(pb.n, 255) if pb.d == 2 else pb.n
        if pb.degree == 2 and n % 2 == 0:
            n += 1
        reqs.append(serve.Request(i, pb.d, n, pb.alpha, pb.degree, pb.lam,
                                  synth.smooth_field(pb.d, n, pb.seed) + 0.2, 0.0))
    srv = serve.Server(hbm_budget=20e9, nstreams=8)
    res = srv.run(reqs, realtime=False)
    srv.close()
    rng = np.random.default_rng(3)
    for r, q in list(zip(res, reqs))[::2]:
        assert r.info["status"] == 0 and r.info["rel_resid"] <= 1e-10
        N = q.n + 1
        a = O.stencil(q.d, N, 2.0 / N, q.alpha, q.degree, q.lam, q=20 if q.d < 3 else 12)
        c = O.c_dalpha(q.d, q.alpha)
        u = np.asarray(r.u, dtype=np.float64)
        f = q.f
        if q.d == 1 or q.n ** q.d <= 4096:
            rel = np.linalg.norm(f - O.apply_dense(a, c, u)) / np.linalg.norm(f)
        else:
            rows = rng.integers(0, q.n, size=(64, q.d))
            fr = f[tuple(rows.T)]
            rel = np.linalg.norm(fr - O.apply_rows(a, c, u, rows)) / np.linalg.norm(fr)
        floor = 1e-15 * math.log2(4 * q.n) * O.norm_bound(a, c, q.n) * np.linalg.norm(u) / np.linalg.norm(f)
        assert rel <= 3e-10 + 10 * floor, (q.d, q.n, q.alpha, q.degree, q.lam, rel, floor)
