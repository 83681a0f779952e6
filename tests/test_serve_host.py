"""Host logic of the serving loop (no GPU): admission under the memory
budget, operator cache eviction, per-request latency bookkeeping.  The solve
engine and the operators are replaced by fakes; a fake job finishes after a
fixed number of polls."""
import numpy as np
import pytest

import paper_2103_03658_gb300.serve as serve


class FakeOp:
    built = 0

    ffts = []

    def __init__(self, d, n, alpha, degree=1, lam=0.0, fft="pow2"):
        FakeOp.built += 1
        FakeOp.ffts.append(fft)
        self.key = (d, n, alpha, degree, lam)
        self.closed = False

    def info(self):
        return {"device_bytes": 1000}

    def close(self):
        self.closed = True


class FakeEngine:
    def __init__(self, nstreams=16):
        self.jobs = {}
        self.next = 1
        self.max_active = 0

    def submit(self, op, f, u, rtol=1e-10, precision="mixed"):
        j = self.next
        self.next += 1
        self.jobs[j] = [3, f]          # finishes after three polls
        self.max_active = max(self.max_active, len(self.jobs))
        return j, np.zeros_like(np.asarray(f))

    def poll(self, block=False):
        out = []
        for j in list(self.jobs):
            self.jobs[j][0] -= 1
            if self.jobs[j][0] <= 0:
                out.append((j, {"status": 0, "iters": 1, "outer": 1, "rel_resid": 0.0}, 0.1,
                            np.asarray(self.jobs.pop(j)[1])))
        return out

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(serve, "Engine", FakeEngine)
    monkeypatch.setattr(serve, "FracOp", FakeOp)
    FakeOp.built = 0


def _reqs(count, d=2, n=63, distinct=4):
    rng = np.random.default_rng(0)
    # requests come in pairs with the same operator key
    return [serve.Request(i, d, n, 0.5 + 0.1 * ((i // 2) % distinct), 1, 0.0, rng.standard_normal((n,) * d), 0.0)
            for i in range(count)]


def test_admission_respects_budget(fakes):
    per = serve.job_bytes(2, 63)
    srv = serve.Server(hbm_budget=3 * per + 10_000, nstreams=4, op_cache_bytes=10_000, build_workers=0)
    res = srv.run(_reqs(12), realtime=False, device_inputs=True)
    assert [r.rid for r in res] == list(range(12))
    assert srv.engine.max_active <= 3
    assert all(r.info["status"] == 0 for r in res)


def test_op_cache_hits_and_eviction(fakes):
    per = serve.job_bytes(2, 63)
    srv = serve.Server(hbm_budget=per + 3000, nstreams=4, op_cache_bytes=2500, build_workers=0)   # one job, two ops
    srv.run(_reqs(20, distinct=4), realtime=False, device_inputs=True)
    assert srv.cache.misses >= 4 and srv.cache.hits >= 1
    assert srv.cache.bytes <= 2500 + 1000 and len(srv.cache.ops) <= 3


def test_latency_includes_queueing(fakes):
    per = serve.job_bytes(1, 255)
    srv = serve.Server(hbm_budget=per + 10, nstreams=1, op_cache_bytes=1e9, build_workers=0)
    reqs = _reqs(5, d=1, n=255, distinct=1)
    res = srv.run(reqs, realtime=True, device_inputs=True)
    assert all(r.latency_s >= r.queue_s >= 0.0 for r in res)
    # one job at a time: later requests wait for earlier ones
    assert res[-1].queue_s >= res[0].queue_s


def test_job_bytes_match_layout():
    # 2D: 4 FP64 vectors + FP64 and FP32 spectra + 4 FP32 vectors
    n = 1023
    nd = n * n
    K = 1025
    b = serve.job_bytes(2, n, "mixed")
    assert b == 4 * nd * 8 + (-(-K // 2) * n * 2) * 16 + (1 << 16) + 4 * nd * 4 + (-(-K // 4) * n * 4) * 8
    assert serve.job_bytes(3, 255) > 1.9e9
    assert serve.percentile([3, 1, 2], 50) == 2


def test_background_operator_builds(fakes, monkeypatch):
    """Misses are built by worker threads; requests behind a pending build are
    admitted once it finishes, and every request is served once."""
    import time as _t

    class SlowOp(FakeOp):
        def __init__(self, *a, **k):
            _t.sleep(0.01)
            super().__init__(*a, **k)
    monkeypatch.setattr(serve, "FracOp", SlowOp)
    srv = serve.Server(hbm_budget=1e12, nstreams=4, op_cache_bytes=1e9, build_workers=2)
    res = srv.run(_reqs(16, distinct=3), realtime=True, device_inputs=True)
    srv.close()
    assert [r.rid for r in res] == list(range(16))
    assert srv.cache.misses == 3 and srv.cache.hits == 13


def test_operators_built_ahead_are_bounded(fakes, monkeypatch):
    """A backlog of requests with distinct operators must not build all of them ahead of
    admission (each built operator holds device memory outside the cache): at most
    max_builds are pending or finished-but-unadmitted at any time, and every request is
    still served once."""
    import threading
    import time as _t
    live = {"now": 0, "peak": 0}
    lock = threading.Lock()

    class CountingOp(FakeOp):
        def __init__(self, *a, **k):
            _t.sleep(0.002)
            super().__init__(*a, **k)

    orig_build = serve.Server._build

    def counting_build(self, key):
        with lock:
            live["now"] = len(self.building)
            live["peak"] = max(live["peak"], live["now"])
        return orig_build(self, key)

    monkeypatch.setattr(serve, "FracOp", CountingOp)
    monkeypatch.setattr(serve.Server, "_build", counting_build)
    srv = serve.Server(hbm_budget=1e12, nstreams=4, op_cache_bytes=1e9, build_workers=2, max_builds=3)
    reqs = _reqs(40, distinct=20)
    res = srv.run(reqs, realtime=False, device_inputs=True)
    srv.close()
    assert [r.rid for r in res] == list(range(40))
    assert live["peak"] <= 3


def test_fft_policy_reaches_the_operators_and_the_admission_estimate(fakes):
    """Server(fft=...) builds its operators with that FFT-length policy, and sizes each job
    by the length the policy gives (a power of two n gets a longer smooth length: 2 n + 2)."""
    import paper_2103_03658_gb300 as fg
    FakeOp.ffts = []
    srv = serve.Server(hbm_budget=1e12, nstreams=4, op_cache_bytes=1e9, build_workers=0, fft="smooth")
    srv.run(_reqs(4, distinct=2), realtime=False, device_inputs=True)
    assert FakeOp.ffts and set(FakeOp.ffts) == {"smooth"}
    m = fg.fft_length(64, 2, "smooth")
    assert m == 144 and srv._fft_len(2, 64) == 144
    assert serve.job_bytes(2, 64, "mixed", m) > serve.job_bytes(2, 64, "mixed")
    assert serve.Server(build_workers=0)._fft_len(2, 64) is None

