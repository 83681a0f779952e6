"""frac_apply_static: the apply for callers that cannot allocate device memory
when they apply the operator (code under a fixed memory budget reserved up
front, a framework that forbids device allocations after start-up, or a
latency-critical loop that cannot let an allocation stall or fail mid-step).

It runs the same kernels as frac_apply on the same inputs, only with its
scratch in the library's fixed device array, so its output must equal
frac_apply's bit for bit, on two calls in a row (the second finds the first
call's data still in the array).  It is also checked once against the FP64
oracle, shown to allocate nothing (the default memory pool's high-water mark
and the device's free memory are unchanged across a call), and shown to
refuse a batch whose scratch clearly exceeds the array and host buffers.
Collected last, so that a first failure here comes after every other test
has run."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import frac_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATIC_BYTES = 64 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_03658_gb300 import _native as nat
    return nat.load()


def _static(lib, op, u, y, dtype):
    code = 1 if dtype == torch.float64 else 0
    stream = torch.cuda.current_stream().cuda_stream
    return lib.frac_apply_static(op.handle, u.data_ptr(), y.data_ptr(), code, u.shape[0], stream)


@pytest.mark.parametrize("d,n,p,alpha,batch,dtype,fft", [
    (2, 1023, 2, 1.2, 3, torch.float32, "pow2"),
    (3, 63, 1, 0.6, 2, torch.float64, "pow2"),
    (1, 1023, 1, 1.5, 5, torch.float32, "pow2"),
    (2, 599, 1, 1.1, 3, torch.float32, "smooth"),  # mixed-radix length 1200
    (3, 39, 2, 0.8, 2, torch.float64, "smooth"),  # 80
])
def test_static_scratch_apply_equals_frac_apply_twice(lib, d, n, p, alpha, batch, dtype, fft):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(d, n, alpha, degree=p, fft=fft)
    for call in range(2):
        u = torch.tensor(synth.smooth_fields(d, n, batch, 300 + 10 * call), dtype=dtype, device="cuda")
        y_static = torch.full_like(u, float("nan"))
        assert _static(lib, op, u, y_static, dtype) == 0
        y_ref = op.apply(u)
        torch.cuda.synchronize()
        assert torch.equal(y_static, y_ref), (call, float((y_static - y_ref).abs().max()))
    op.close()


def test_static_scratch_apply_matches_oracle(lib):
    """One small 2D case against the oracle's dense apply (normwise 1e-12 in FP64)."""
    import paper_2103_03658_gb300 as fg
    d, n, p, alpha = 2, 47, 2, 0.9
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, p)
    c = O.c_dalpha(d, alpha)
    U = synth.smooth_fields(d, n, 2, 77)
    op = fg.FracOp(d, n, alpha, degree=p)
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    y = torch.empty_like(u)
    assert _static(lib, op, u, y, torch.float64) == 0
    torch.cuda.synchronize()
    nrm = O.norm_bound(a, c, n)
    for b in range(2):
        err = np.linalg.norm(y[b].cpu().numpy() - O.apply_dense(a, c, U[b])) / (nrm * np.linalg.norm(U[b]))
        assert err <= 1e-12, (b, err)
    op.close()


class _Pool:
    """The current device's default memory pool through the driver API (the pool
    that stream-ordered allocations draw from)."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_static_scratch_apply_allocates_nothing(lib):
    """After a warm-up call, one call changes neither the default pool's high-water
    mark of used memory nor the device's free memory; frac_apply, which does
    allocate its scratch from that pool, moves the mark (so the probe sees it)."""
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(2, 1023, 1.2, degree=2)
    u = torch.tensor(synth.smooth_fields(2, 1023, 4, 5), dtype=torch.float32, device="cuda")
    y = torch.empty_like(u)
    assert _static(lib, op, u, y, torch.float32) == 0
    torch.cuda.synchronize()
    pool = _Pool()
    used = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    free0, _ = torch.cuda.mem_get_info()
    assert _static(lib, op, u, y, torch.float32) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert pool.get(pool.USED_MEM_HIGH) == used
    assert free1 == free0
    op.apply(u, out=y)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > used
    op.close()


def test_static_scratch_rejects_oversized_batch_and_host_buffers(lib):
    import paper_2103_03658_gb300 as fg
    from paper_2103_03658_gb300 import _native as nat
    n, batch = 1023, 16
    op = fg.FracOp(2, n, 1.2, degree=2)
    # FP32 scratch of the 2D apply: batch x ceil(K / 4) column blocks x n rows x 4 columns
    # of 8-byte complex values, K = 1025: 16 fields need 134.6 MB, twice the array
    need = batch * ((1025 + 3) // 4) * n * 4 * 8
    assert need > 2 * STATIC_BYTES
    u = torch.zeros(batch, n, n, device="cuda")
    y = torch.empty_like(u)
    assert _static(lib, op, u, y, torch.float32) == 1
    assert nat._detail() == (f"frac_apply_static: this call needs {need} bytes of scratch, more than the static "
                             f"{STATIC_BYTES} bytes; split the batch or use frac_apply")
    hu = np.zeros((1, n, n), dtype=np.float32)
    hy = np.zeros_like(hu)
    assert lib.frac_apply_static(op.handle, hu.ctypes.data, hy.ctypes.data, 0, 1, None) == 1
    assert "device buffers" in nat._detail()
    op.close()
