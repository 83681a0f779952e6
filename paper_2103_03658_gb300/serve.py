"""Serving loop for fractional Poisson solves on one GPU (continuous batching).

Requests (d, n, alpha, degree, lambda, f) arrive over time.  Each is admitted
as soon as its device footprint fits the memory budget; its operator comes
from a cache keyed by (d, n, alpha, h, degree, lambda) (coefficients and
symbols are built on the GPU on a miss); it is submitted to the solve engine,
whose jobs progress together on a pool of streams.  A finished solve is copied
to the host, and its latency runs from arrival to the result being on the
host.  The host side here is bookkeeping only: every solve step runs in the
sm_103a library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from ._native import Engine, FracOp


@dataclass
class Request:
    rid: int
    d: int
    n: int
    alpha: float
    degree: int
    lam: float
    f: object            # host array of shape (n,)*d (float64)
    arrival: float = 0.0  # seconds after the start of the stream


@dataclass
class Result:
    rid: int
    u: object
    info: dict
    latency_s: float
    queue_s: float
    admitted_at: float
    op_cache_hit: bool


def job_bytes(d: int, n: int, precision: str = "mixed", M: int | None = None) -> int:
    """Device bytes of one solve job (vectors, FFT scratch, partial sums), as the
    library allocates them; d = 1 jobs hold only a few small records.  M: the
    operator's FFT length (default: the power of two)."""
    nd = n ** d
    if d == 1:
        return 4096 + 16 * nd
    if M is None:
        M = 2
        while M < 2 * n - 1:
            M *= 2
    K = M // 2 + 1

    def ws(cs, B):
        KB = -(-K // B)
        return (KB * n * B if d == 2 else n * KB * n * B + M * KB * n * B) * cs

    b = 4 * nd * 8 + ws(16, 2) + (1 << 16)
    if precision == "mixed":
        b += 4 * nd * 4 + ws(8, 4)
    else:
        b += 2 * nd * 8
    return b


@dataclass
class OpCache:
    """Operators keyed by (d, n, alpha, h, degree, lambda), least recently used
    evicted first when the cache's device bytes exceed `capacity`."""
    capacity: int
    fft: str = "pow2"   # FFT-length policy of the operators it builds
    ops: "collections.OrderedDict" = field(default_factory=collections.OrderedDict)
    bytes: int = 0
    hits: int = 0
    misses: int = 0

    def put(self, key, op, in_use=()):
        """Insert an operator built elsewhere (counted as a miss) and evict as in get()."""
        self.misses += 1
        self.ops[key] = op
        self.bytes += op.info()["device_bytes"]
        self._evict(key, in_use)
        return op

    def _evict(self, key, in_use):
        for k0 in list(self.ops.keys()):          # least recently used first
            if self.bytes <= self.capacity:
                break
            op0 = self.ops[k0]
            if k0 == key or any(op0 is x for x in in_use):
                continue                           # still needed by a job in flight
            del self.ops[k0]
            self.bytes -= op0.info()["device_bytes"]
            op0.close()

    def get(self, d, n, alpha, degree, lam, in_use=()) -> tuple:
        key = (d, n, float(alpha), 2.0 / (n + 1), degree, float(lam))
        if key in self.ops:
            self.ops.move_to_end(key)
            self.hits += 1
            return self.ops[key], True
        op = FracOp(d, n, alpha, degree=degree, lam=lam, fft=self.fft)
        self.misses += 1
        self.ops[key] = op
        self.bytes += op.info()["device_bytes"]
        self._evict(key, in_use)
        return op, False


class PinnedPool:
    """Reusable page-locked host buffers, one free list per shape (float64)."""

    def __init__(self):
        self.free = collections.defaultdict(list)

    def get(self, shape):
        import torch
        lst = self.free[tuple(shape)]
        return lst.pop() if lst else torch.empty(tuple(shape), dtype=torch.float64).pin_memory()

    def put(self, buf):
        self.free[tuple(buf.shape)].append(buf)


class Server:
    """Continuous-batching server on the current CUDA device.  Operators for
    cache misses are built by a background worker on its own stream, so the
    loop keeps admitting and polling while coefficients are computed."""

    def __init__(self, hbm_budget: float = 150e9, nstreams: int = 16, precision: str = "mixed",
                 rtol: float = 1e-10, op_cache_bytes: float = 8e9, build_workers: int = 2,
                 max_builds: int = 8, fft: str = "pow2"):
        from concurrent.futures import ThreadPoolExecutor
        self.engine = Engine(nstreams)
        self.fft = fft  # FFT-length policy of the operators (FracOp's fft)
        self.cache = OpCache(int(op_cache_bytes), fft)
        self.budget = int(hbm_budget)
        self.precision = precision
        self.rtol = rtol
        self.pool = PinnedPool()
        self.builder = ThreadPoolExecutor(max_workers=build_workers) if build_workers else None
        self.building = {}
        # operators built ahead of admission hold device memory outside the cache: at most
        # max_builds of them (queued, running or finished) at a time
        self.max_builds = max_builds

    def close(self):
        if self.builder:
            self.builder.shutdown(wait=True)
        self.engine.close()
        for op in self.cache.ops.values():
            op.close()
        self.cache.ops.clear()

    def _build(self, key):
        import torch
        d, n, alpha, h, degree, lam = key
        if not torch.cuda.is_available():
            return FracOp(d, n, alpha, degree=degree, lam=lam, fft=self.fft)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            op = FracOp(d, n, alpha, degree=degree, lam=lam, stream=st.cuda_stream, fft=self.fft)
        st.synchronize()
        return op

    def _fft_len(self, d, n):
        """The FFT length of the server's operators for (d, n); None: the power of two."""
        if self.fft == "pow2":
            return None
        from ._native import fft_length
        return fft_length(n, d, self.fft)

    def _op_ready(self, r, in_use):
        """The request's operator if it is available now (cache hit or finished build), else None."""
        key = (r.d, r.n, float(r.alpha), 2.0 / (r.n + 1), r.degree, float(r.lam))
        if key in self.cache.ops or self.builder is None:
            return self.cache.get(r.d, r.n, r.alpha, r.degree, r.lam, in_use)
        fut = self.building.get(key)
        if fut is None:
            if len(self.building) < self.max_builds:
                self.building[key] = self.builder.submit(self._build, key)
            return None
        if not fut.done():
            return None
        op = fut.result()
        del self.building[key]
        return self.cache.put(key, op, in_use), False

    def run(self, requests: list, realtime: bool = True, device_inputs: bool = False) -> list:
        """Serve `requests` (sorted by arrival); returns a Result per request."""
        import torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = {}
        results = []
        held = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else None
        while pending or waiting or active:
            now = clock() if realtime else float("inf")
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            blocked = []
            while waiting:
                r = waiting[0]
                need = job_bytes(r.d, r.n, self.precision, self._fft_len(r.d, r.n))
                if active and held + need + self.cache.bytes > self.budget:
                    break
                in_use = [a[1] for a in active.values()]
                got = self._op_ready(r, in_use)
                if got is None:                       # operator still being built: let others pass
                    blocked.append(waiting.popleft())
                    continue
                waiting.popleft()
                op, hit = got
                if device_inputs:
                    f, u = r.f, None
                else:
                    f = self.pool.get(np.shape(r.f))
                    f.numpy()[...] = r.f
                    u = self.pool.get(np.shape(r.f))
                job, u = self.engine.submit(op, f, u, rtol=self.rtol, precision=self.precision)
                t_adm = clock() if realtime else 0.0
                active[job] = (r, op, need, t_adm, hit, None if device_inputs else f)
                held += need
            waiting.extendleft(reversed(blocked))
            done = self.engine.poll(block=not waiting and not pending and not self.building)
            for job, info, _ms, u in done:
                r, op, need, t_adm, hit, fbuf = active.pop(job)
                held -= need
                if device_inputs:
                    u_host = u.cpu() if hasattr(u, "cpu") else u
                else:
                    u_host = np.array(u.numpy() if hasattr(u, "numpy") else u, copy=True)
                    self.pool.put(u)
                    self.pool.put(fbuf)
                t_done = clock() if realtime else 0.0
                results.append(Result(r.rid, u_host, info, t_done - r.arrival, t_adm - r.arrival, t_adm, hit))
            if not done and realtime and (pending or waiting):
                gap = pending[0].arrival - clock() if (pending and not waiting) else 0.0
                time.sleep(min(max(gap, 0.0), 2e-4) if gap > 0 else 5e-5)
        return sorted(results, key=lambda x: x.rid)


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]
