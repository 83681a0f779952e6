"""Process-pool drivers of the FP64 oracle for the largest grids (test
infrastructure only).  The arithmetic is the oracle's own: the 3D generator is
``oracle.weights`` summed over ranges of the first element index, one range per
worker, then ``oracle.stencil`` on the assembled weights; the sampled rows are
``oracle.apply_rows``, a slice of the rows per worker.  Workers start with the
``spawn`` method (the parent may already hold a CUDA context) and read the large
arrays from memory-mapped files instead of pickles."""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np


def workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _weights_part(args):
    from oracle import frac_oracle as O
    d, N, h, alpha, p, lam, q, lo, hi = args
    w = O.weights(d, N, h, alpha, p, lam, q=q, first=range(lo, hi))
    els = O.axis_elements(N, h, p)
    nlo = min(nd for e in range(lo, hi) for nd, _, _ in els[e][2])
    nhi = max(nd for e in range(lo, hi) for nd, _, _ in els[e][2])
    return nlo, np.ascontiguousarray(w[nlo:nhi + 1])


def stencil(d: int, N: int, alpha: float, p: int, lam: float = 0.0, q: int = 20):
    """The oracle's generator a (and c_{d,alpha}) on [0, 2]^d with N intervals, the
    weights computed by a pool of workers (d >= 2)."""
    from oracle import frac_oracle as O
    h = 2.0 / N
    ne = len(O.axis_elements(N, h, p))
    nw = workers()
    chunk = max(1, -(-ne // (4 * nw)))
    tasks = [(d, N, h, alpha, p, lam, q, lo, min(lo + chunk, ne)) for lo in range(0, ne, chunk)]
    omega = np.zeros((N + 1,) * d)
    with mp.get_context("spawn").Pool(nw) as pool:
        for nlo, slab in pool.imap_unordered(_weights_part, tasks):
            omega[nlo:nlo + len(slab)] += slab
    a = O.stencil(d, N, h, alpha, p, lam, omega=omega, q=q)
    return a, O.c_dalpha(d, alpha)


def _rows_part(args):
    from oracle import frac_oracle as O
    apath, upath, c, rows = args
    a = np.load(apath, mmap_mode="r")
    u = np.load(upath, mmap_mode="r")
    return O.apply_rows(np.asarray(a), c, np.asarray(u), rows)


def apply_rows(a: np.ndarray, c: float, u: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """oracle.apply_rows(a, c, u, rows), the rows spread over a pool of workers."""
    rows = np.asarray(rows)
    nw = workers()
    with tempfile.TemporaryDirectory() as tmp:
        apath, upath = os.path.join(tmp, "a.npy"), os.path.join(tmp, "u.npy")
        np.save(apath, a)
        np.save(upath, np.asarray(u, dtype=np.float64))
        parts = np.array_split(np.arange(len(rows)), min(nw, len(rows)))
        with mp.get_context("spawn").Pool(len(parts)) as pool:
            res = pool.map(_rows_part, [(apath, upath, c, rows[ix]) for ix in parts])
    return np.concatenate(res)
