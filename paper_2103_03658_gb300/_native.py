"""ctypes binding of the C ABI declared in include/frac.h.

Argument marshalling only: every step of the computation runs in the sm_103a
library.  There is no CPU fallback: if the library is missing or fails to
load, constructing an operator raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

F32, F64 = 0, 1
PLAIN_F64, MIXED_IR = 0, 1
STATUS = {0: "FRAC_OK", 1: "FRAC_EINVAL", 2: "FRAC_ENOMEM", 3: "FRAC_ENOTSUP", 4: "FRAC_ENOCONV",
          5: "FRAC_EBREAKDOWN", 6: "FRAC_ETIMEOUT", 7: "FRAC_ECUDA"}


class FracError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = _detail() if status in (2, 7) else ""
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_strerror(status)})"
                         + (f" [{detail}]" if detail else ""))


class Problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("degree", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("h", ctypes.c_double), ("n", ctypes.c_int64 * 3), ("lam", ctypes.c_double),
                ("gamma", ctypes.c_double), ("fft_lengths", ctypes.c_int32)]


FFT_LENGTHS = {"pow2": 0, "smooth": 1, "auto": 2}


class OpInfo(ctypes.Structure):
    _fields_ = [("c_dalpha", ctypes.c_double), ("a0", ctypes.c_double), ("far_field", ctypes.c_double),
                ("norm_bound", ctypes.c_double), ("fft_len", ctypes.c_int64), ("n_gen", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("precond_ok", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("fft_lens", ctypes.c_int64 * 3)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("use_x0", ctypes.c_int32), ("precond", ctypes.c_int32), ("inner_tol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("rel_resid", ctypes.c_double)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int32), ("clusters", ctypes.c_int32),
                ("first_cluster_logm", ctypes.c_int32), ("cluster_problems", ctypes.c_int32),
                ("local_problems", ctypes.c_int32), ("predicted_ms", ctypes.c_double)]


class JobResult(ctypes.Structure):
    _fields_ = [("job", ctypes.c_int64), ("info", SolveInfo), ("submit_to_done_ms", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libfrac.so (raising if it is absent and ``build_if_missing`` is False)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing: build it with paper_2103_03658_gb300.build.build() "
                               "(the library has no CPU fallback)")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.frac_coeffs.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(vp), vp]
    lib.frac_coeffs.restype = i32
    lib.frac_op_free.argtypes = [vp]
    lib.frac_op_free.restype = None
    lib.frac_op_info.argtypes = [vp, ctypes.POINTER(OpInfo)]
    lib.frac_op_info.restype = i32
    lib.frac_op_generator.argtypes = [vp, dp, ctypes.c_size_t]
    lib.frac_op_generator.restype = i32
    lib.frac_apply.argtypes = [vp, vp, vp, i32, i64, vp]
    lib.frac_apply.restype = i32
    lib.frac_apply_static.argtypes = [vp, vp, vp, i32, i64, vp]
    lib.frac_apply_static.restype = i32
    lib.frac_precond.argtypes = [vp, vp, vp, i32, i64, vp]
    lib.frac_precond.restype = i32
    lib.frac_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.frac_solve.restype = i32
    lib.frac_boundary.argtypes = [vp, vp, vp, vp, vp]
    lib.frac_boundary.restype = i32
    lib.frac_solve_batch.argtypes = [i64, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.frac_solve_batch.restype = i32
    lib.frac_batch_last_plan.argtypes = [ctypes.POINTER(BatchPlan)]
    lib.frac_batch_last_plan.restype = i32
    lib.frac_batch_pin_plan.argtypes = [i32, i32]
    lib.frac_batch_pin_plan.restype = i32
    lib.frac_engine_create.argtypes = [i32, ctypes.POINTER(vp)]
    lib.frac_engine_create.restype = i32
    lib.frac_engine_submit.argtypes = [vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(ctypes.c_int64)]
    lib.frac_engine_submit.restype = i32
    lib.frac_engine_poll.argtypes = [vp, i32, ctypes.POINTER(JobResult), i32, ctypes.POINTER(ctypes.c_int)]
    lib.frac_engine_poll.restype = i32
    lib.frac_engine_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t)]
    lib.frac_engine_stats.restype = i32
    lib.frac_engine_destroy.argtypes = [vp]
    lib.frac_engine_destroy.restype = None
    lib.frac_strerror.argtypes = [i32]
    lib.frac_strerror.restype = ctypes.c_char_p
    lib.frac_error_detail.argtypes = []
    lib.frac_error_detail.restype = ctypes.c_char_p
    lib.frac_profile_enable.argtypes = [i32]
    lib.frac_profile_enable.restype = i32
    lib.frac_profile_read.argtypes = [ctypes.c_void_p, i32, ctypes.POINTER(ctypes.c_int), i32]
    lib.frac_profile_read.restype = i32
    lib.frac_profile_alu_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.frac_profile_alu_peak.restype = i32
    lib.frac_far_nodes.argtypes = [i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, i32, vp, vp,
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.frac_far_nodes.restype = i32
    lib.frac_far_points.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp]
    lib.frac_far_points.restype = i32
    lib.frac_far_sum.argtypes = [vp, vp, i64, vp, i64, vp, vp]
    lib.frac_apply_3d_passes.restype = i32
    lib.frac_apply_3d_passes.argtypes = [i32]
    lib.frac_fft_length.restype = i32
    lib.frac_fft_length.argtypes = [i64, i32, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.frac_far_sum.restype = i32
    _lib = lib
    return lib


def _strerror(status: int) -> str:
    try:
        return load().frac_strerror(status).decode()
    except Exception:  # library not loadable: the status name is still shown
        return "?"


def _detail() -> str:
    try:
        return load().frac_error_detail().decode()
    except Exception:
        return ""


def far_nodes(d: int, alpha: float, lam: float, L: float, nr: int = 96, ns: int = 48):
    """The library's far-field rule (frac_far_nodes, host only): nodes xi (Q, d), column k
    along axis x^(k+1), and weights w (Q,)."""
    lib = load()
    cnt = ctypes.c_int64()
    s = lib.frac_far_nodes(d, alpha, lam, L, nr, ns, None, None, ctypes.byref(cnt))
    if s != 0:
        raise FracError(s, "frac_far_nodes")
    xi = np.empty((cnt.value, d))
    w = np.empty(cnt.value)
    s = lib.frac_far_nodes(d, alpha, lam, L, nr, ns, xi.ctypes.data, w.ctypes.data, ctypes.byref(cnt))
    if s != 0:
        raise FracError(s, "frac_far_nodes")
    return xi, w


def apply_3d_passes(fused: bool) -> None:
    """Schedule of the 3D FP32 apply (frac_apply_3d_passes): fused xy passes on thread-block
    clusters (True) or five pencil passes (False, the default, faster on GB300); the results
    agree to FP32 rounding."""
    load().frac_apply_3d_passes(1 if fused else 0)


def fft_length(n: int, d: int, fft: str = "pow2") -> int:
    """The circulant embedding length frac_coeffs gives an axis of n points (frac_fft_length,
    host only): fft "pow2" or "smooth" as in FracOp."""
    m = ctypes.c_int64()
    s = load().frac_fft_length(int(n), int(d), FFT_LENGTHS[fft], ctypes.byref(m))
    if s != 0:
        raise FracError(s, "frac_fft_length")
    return m.value


def alu_peak_tflops(kind: str, stream=None) -> float:
    """Measured arithmetic rate of the current GPU (frac_profile_alu_peak): kind "f32"
    (fma.rn.f32), "f64" (fma.rn.f64) or "f32x2" (paired FP32 FMAs), in TFLOP/s."""
    code = {"f32": 0, "f64": 1, "f32x2": 2}[kind]
    v = ctypes.c_double()
    s = load().frac_profile_alu_peak(code, ctypes.byref(v), _stream(stream))
    if s != 0:
        raise FracError(s, "frac_profile_alu_peak")
    return v.value


def declared_entry_points() -> list[str]:
    """Names of the functions declared in include/frac.h."""
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "frac.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(frac_\w+)\s*\(", text, re.M)))


# ---------------------------------------------------------------------------
# buffers: torch tensors (device or host) and numpy arrays (host)
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _ptr(x) -> int:
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return x.data_ptr()


def _dtype_code(x) -> int:
    if isinstance(x, np.ndarray):
        dt = x.dtype
        if dt == np.float64:
            return F64
        if dt == np.float32:
            return F32
    else:
        torch = _torch()
        if x.dtype == torch.float64:
            return F64
        if x.dtype == torch.float32:
            return F32
    raise TypeError("only float32 and float64 are supported")


def _stream(stream) -> int | None:
    if stream is not None:
        return int(stream)
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _empty_like(x):
    if isinstance(x, np.ndarray):
        return np.empty_like(x)
    return _torch().empty_like(x)


class FracOp:
    """Discretized (-Delta)^{alpha/2} (tempered when lam > 0) on a box with n interior points
    per axis: n an int (the cube (-1, 1)^d) or a sequence (n_1, .., n_d) of per-axis counts,
    axis 1 = x^(1) the fastest-varying (arrays have shape (n_d, .., n_1)).  h = 2 / (max n_i + 1)
    unless given (the longest axis spans (-1, 1)); gamma the splitting parameter in (alpha, 2]
    (Eq. (eq0)); fft the circulant embedding lengths: "pow2" (the next power of two) or
    "smooth" (the smallest 2^a 3^b 5^c 7^d >= 2 n_i + 2, a >= 4, on mixed-radix FFTs) or "auto"
    (the cheaper of the two by frac_fft_length's pass-count model);
    built on the current CUDA device."""

    def __init__(self, d: int, n, alpha: float, degree: int = 1, lam: float = 0.0,
                 h: float | None = None, stream=None, gamma: float = 2.0, fft: str = "pow2"):
        if fft not in FFT_LENGTHS:
            raise ValueError(f"fft must be one of {sorted(FFT_LENGTHS)}, not {fft!r}")
        lib = load()
        self._lib = lib
        ns = tuple(int(v) for v in n) if isinstance(n, (tuple, list)) else (int(n),) * d
        if len(ns) != d:
            raise ValueError(f"n has {len(ns)} entries for d = {d}")
        self.d, self.alpha, self.degree, self.lam, self.gamma, self.fft = d, alpha, degree, lam, gamma, fft
        self.n = ns[0] if len(set(ns)) == 1 else ns
        self.ns = ns
        self.nd = int(np.prod(ns))
        self.h = 2.0 / (max(ns) + 1) if h is None else h
        self._prob = Problem(d, degree, alpha, self.h, (ctypes.c_int64 * 3)(*(ns + (1,) * (3 - d))), lam, gamma,
                             FFT_LENGTHS[fft])
        handle = ctypes.c_void_p()
        s = lib.frac_coeffs(ctypes.byref(self._prob), ctypes.byref(handle), _stream(stream))
        if s != 0:
            raise FracError(s, "frac_coeffs")
        self._h = handle

    # -- lifecycle --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.frac_op_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.ns))

    def info(self) -> dict:
        inf = OpInfo()
        s = self._lib.frac_op_info(self._h, ctypes.byref(inf))
        if s != 0:
            raise FracError(s, "frac_op_info")
        out = {k: getattr(inf, k) for k, _ in OpInfo._fields_}
        out["n"] = tuple(out["n"])[: self.d]
        out["fft_lens"] = tuple(out["fft_lens"])[: self.d]
        return out

    def generator(self) -> np.ndarray:
        N1 = max(self.ns) + 2
        a = np.empty((N1,) * self.d, dtype=np.float64)
        s = self._lib.frac_op_generator(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size)
        if s != 0:
            raise FracError(s, "frac_op_generator")
        return a

    # -- apply --
    def apply(self, u, out=None, stream=None):
        """y = A u for u of shape (batch,) + shape or shape; float32 or float64."""
        code = _dtype_code(u)
        nd = self.nd
        numel = u.size if isinstance(u, np.ndarray) else u.numel()
        if numel % nd:
            raise ValueError(f"size {numel} is not a multiple of prod(n_i) = {nd}")
        y = _empty_like(u) if out is None else out
        s = self._lib.frac_apply(self._h, _ptr(u), _ptr(y), code, numel // nd, _stream(stream))
        if s != 0:
            raise FracError(s, "frac_apply")
        return y

    def precond(self, r, out=None, stream=None):
        """z = P r with the tau preconditioner (frac_precond); shapes and dtypes as apply."""
        code = _dtype_code(r)
        nd = self.nd
        numel = r.size if isinstance(r, np.ndarray) else r.numel()
        if numel % nd:
            raise ValueError(f"size {numel} is not a multiple of prod(n_i) = {nd}")
        z = _empty_like(r) if out is None else out
        s = self._lib.frac_precond(self._h, _ptr(r), _ptr(z), code, numel // nd, _stream(stream))
        if s != 0:
            raise FracError(s, "frac_precond")
        return z

    # -- boundary vector of exterior data --
    @property
    def ext_shape(self) -> tuple:
        """Array shape of the extended samples of ``boundary``: n_i + 2N per axis, N = max n_i + 1."""
        N = max(self.ns) + 1
        return tuple(m + 2 * N for m in self.shape)

    def far_field(self, g, lo=-1.0, nr: int = 96, ns: int = 48, max_values: int = 1 << 25, stream=None):
        """The far part of the boundary vector for exterior data g (frac_far_points and
        frac_far_sum): g is called on float64 device tensors of shape (P, d) whose column k
        is the coordinate along array axis k (the last array axis is x^(1)) and returns P
        values; lo is the domain's lower corner (a number or one value per array axis).
        Grid points are taken in chunks of at most max_values evaluation points.  Returns
        a float64 device tensor of the grid's shape."""
        import torch
        d = self.d
        los = [float(lo)] * d if np.isscalar(lo) else [float(v) for v in lo]
        L = (max(self.ns) + 1) * self.h
        xi_h, w_h = far_nodes(d, self.alpha, self.lam, L, nr, ns)
        nq = len(w_h)
        dev = torch.device("cuda", torch.cuda.current_device())
        xi = torch.tensor(xi_h, device=dev)
        w = torch.tensor(w_h, device=dev)
        far = torch.empty(self.shape, dtype=torch.float64, device=dev)
        per = (1 << d) * nq
        chunk = max(1, max_values // per)
        lo_c = (ctypes.c_double * 3)(*(list(reversed(los)) + [0.0] * (3 - d)))  # per axis x^(k+1)
        st = _stream(stream)
        flat = far.view(-1)
        for first in range(0, self.nd, chunk):
            cnt = min(chunk, self.nd - first)
            pts = torch.empty((cnt * per, d), dtype=torch.float64, device=dev)
            s = self._lib.frac_far_points(self._h, lo_c, xi.data_ptr(), nq, first, cnt, pts.data_ptr(), st)
            if s != 0:
                raise FracError(s, "frac_far_points")
            gv = g(pts.flip(1)).to(torch.float64).contiguous()  # columns in array-axis order
            s = self._lib.frac_far_sum(self._h, w.data_ptr(), nq, gv.data_ptr(), cnt, flat[first:].data_ptr(), st)
            if s != 0:
                raise FracError(s, "frac_far_sum")
            del pts, gv
        return far

    def boundary(self, g_ext, far=None, out=None, stream=None):
        """b = -c (near + far) (frac_boundary): g_ext holds g at the grid points e in
        [1-N, n_i+N] per axis (shape ``ext_shape``, float64; interior values unread),
        far the caller's far-field integrals (shape of u) or None."""
        if _dtype_code(g_ext) != F64 or (far is not None and _dtype_code(far) != F64):
            raise TypeError("boundary takes float64 data")
        want = int(np.prod(self.ext_shape))
        numel = g_ext.size if isinstance(g_ext, np.ndarray) else g_ext.numel()
        if numel != want:
            raise ValueError(f"g_ext has {numel} values, expected prod(n_i + 2N) = {want}")
        if out is None:
            if isinstance(g_ext, np.ndarray):
                out = np.empty(self.shape, dtype=np.float64)
            else:
                import torch
                out = torch.empty(self.shape, dtype=torch.float64, device=g_ext.device)
        s = self._lib.frac_boundary(self._h, _ptr(g_ext), None if far is None else _ptr(far), _ptr(out),
                                    _stream(stream))
        if s != 0:
            raise FracError(s, "frac_boundary")
        return out

    # -- solve --
    def solve(self, f, u=None, rtol: float = 1e-10, max_iter: int = 200000, precision: str = "mixed",
              inner_tol: float = 0.0, stream=None, precond: str = "tau", g=None):
        """Solve A u = f - g (g: None, or the boundary vector of ``boundary``); returns
        (u, info dict).  f, u, g float64."""
        if _dtype_code(f) != F64 or (g is not None and _dtype_code(g) != F64):
            raise TypeError("solve takes float64 data")
        use_x0 = u is not None
        if u is None:
            u = _empty_like(f)
        opts = _opts(rtol, max_iter, precision, use_x0, inner_tol, precond)
        info = SolveInfo()
        s = self._lib.frac_solve(self._h, _ptr(f), None if g is None else _ptr(g), _ptr(u), ctypes.byref(opts),
                                 ctypes.byref(info), _stream(stream))
        out = {k: getattr(info, k) for k, _ in SolveInfo._fields_}
        if s not in (0, 4):
            raise FracError(s, "frac_solve")
        return u, out


PRECOND_TAU, PRECOND_NONE = 0, 1


def _opts(rtol, max_iter, precision, use_x0, inner_tol, precond) -> "SolveOpts":
    if precision not in ("mixed", "f64"):
        raise ValueError("precision is 'mixed' or 'f64'")
    if precond not in ("tau", "none"):
        raise ValueError("precond is 'tau' or 'none'")
    return SolveOpts(rtol, max_iter, MIXED_IR if precision == "mixed" else PLAIN_F64, int(use_x0),
                     PRECOND_TAU if precond == "tau" else PRECOND_NONE, inner_tol)


def solve_batch(ops, fs, us, rtol: float = 1e-10, max_iter: int = 200000, precision: str = "mixed",
                inner_tol: float = 0.0, stream=None, precond: str = "tau"):
    """Solve ops[i] u[i] = f[i] for all i (device tensors); returns a list of info dicts."""
    lib = load()
    cnt = len(ops)
    H = (ctypes.c_void_p * cnt)(*[op.handle.value for op in ops])
    F = (ctypes.c_void_p * cnt)(*[_ptr(f) for f in fs])
    U = (ctypes.c_void_p * cnt)(*[_ptr(u) for u in us])
    opts = _opts(rtol, max_iter, precision, False, inner_tol, precond)
    infos = (SolveInfo * cnt)()
    s = lib.frac_solve_batch(cnt, H, F, U, ctypes.byref(opts), infos, _stream(stream))
    out = [{k: getattr(i, k) for k, _ in SolveInfo._fields_} for i in infos]
    if s not in (0, 4):
        raise FracError(s, "frac_solve_batch")
    return out


def batch_last_plan() -> dict:
    """Plan of this thread's last frac_solve_batch call with a persistent 2D launch."""
    p = BatchPlan()
    s = load().frac_batch_last_plan(ctypes.byref(p))
    if s != 0:
        raise FracError(s, "frac_batch_last_plan")
    return {k: getattr(p, k) for k, _ in BatchPlan._fields_}


def batch_pin_plan(cluster_size: int, first_cluster_logm: int = 11) -> None:
    """Pin the persistent 2D launch of this thread's later batches (cluster_size 0: autotune)."""
    s = load().frac_batch_pin_plan(cluster_size, first_cluster_logm)
    if s != 0:
        raise FracError(s, "frac_batch_pin_plan")


def _info(si: SolveInfo) -> dict:
    return {k: getattr(si, k) for k, _ in SolveInfo._fields_}


class Engine:
    """Many solves in flight at once (frac_engine_* of include/frac.h): jobs
    advance on a pool of `nstreams` streams; poll() advances them and returns
    the finished ones.  The buffers of a job are kept alive until it finishes."""

    def __init__(self, nstreams: int = 16):
        self._lib = load()
        h = ctypes.c_void_p()
        s = self._lib.frac_engine_create(nstreams, ctypes.byref(h))
        if s != 0:
            raise FracError(s, "frac_engine_create")
        self._h = h
        self._keep = {}

    def submit(self, op: "FracOp", f, u=None, rtol: float = 1e-10, max_iter: int = 200000,
               precision: str = "mixed", inner_tol: float = 0.0, use_x0: bool = False,
               precond: str = "tau") -> tuple:
        """Queue op u = f; the solution goes to `u` (a new buffer if None), whose
        contents are the initial guess only when use_x0 is set.  Returns (job id, u)."""
        if _dtype_code(f) != F64:
            raise TypeError("solve takes float64 data")
        if u is None:
            u = _empty_like(f)
            use_x0 = False
        opts = _opts(rtol, max_iter, precision, use_x0, inner_tol, precond)
        job = ctypes.c_int64()
        s = self._lib.frac_engine_submit(self._h, op.handle, _ptr(f), _ptr(u), ctypes.byref(opts), ctypes.byref(job))
        if s != 0:
            raise FracError(s, "frac_engine_submit")
        self._keep[job.value] = (op, f, u)
        return job.value, u

    def poll(self, block: bool = False, cap: int = 256) -> list:
        """Advance all jobs; list of (job, info dict, submit-to-done ms, u) for the finished ones."""
        arr = (JobResult * cap)()
        cnt = ctypes.c_int()
        s = self._lib.frac_engine_poll(self._h, int(block), arr, cap, ctypes.byref(cnt))
        out = []
        for i in range(cnt.value):
            r = arr[i]
            op, f, u = self._keep.pop(r.job, (None, None, None))
            out.append((r.job, _info(r.info), r.submit_to_done_ms, u))
        if s != 0 and not out:
            raise FracError(s, "frac_engine_poll")
        return out

    def stats(self) -> tuple:
        a = ctypes.c_int64()
        b = ctypes.c_size_t()
        self._lib.frac_engine_stats(self._h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.frac_engine_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
