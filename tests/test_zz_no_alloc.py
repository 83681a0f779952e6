"""frac_apply_static: the apply for callers that cannot allocate device memory
when they apply the operator.  It must give what frac_apply gives, on two
calls in a row (the second reuses the library's fixed scratch array, still
holding the first call's data), and refuse a batch whose scratch would not
fit in that array.  Collected last so that a first failure here comes after
every other test has run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


@pytest.mark.parametrize("d,n,p,alpha,batch,dtype,tol", [
    (2, 1023, 2, 1.2, 3, torch.float32, 1e-5),
    (3, 63, 1, 0.6, 2, torch.float64, 1e-12),
    (1, 1023, 1, 1.5, 5, torch.float32, 1e-5),
])
def test_static_scratch_apply_matches_frac_apply_twice(lib, d, n, p, alpha, batch, dtype, tol):
    import paper_2103_03658_gb300 as fg
    op = fg.FracOp(d, n, alpha, degree=p)
    nrm = op.info()["norm_bound"]
    for call in range(2):
        u = torch.tensor(synth.smooth_fields(d, n, batch, 300 + 10 * call), dtype=dtype, device="cuda")
        y_static = torch.full_like(u, float("nan"))
        assert _static(lib, op, u, y_static, dtype) == 0
        y_ref = op.apply(u)
        torch.cuda.synchronize()
        for b in range(batch):
            err = float((y_static[b] - y_ref[b]).double().norm()) / (nrm * float(u[b].double().norm()))
            assert err <= tol, (call, b, err)
    op.close()


def test_static_scratch_rejects_oversized_batch_and_host_buffers(lib):
    import paper_2103_03658_gb300 as fg
    from paper_2103_03658_gb300 import _native as nat
    op = fg.FracOp(2, 1023, 1.2, degree=2)
    u = torch.zeros(8, 1023, 1023, device="cuda")       # 8 fields need 8.4 MB of scratch each > 64 MiB
    y = torch.empty_like(u)
    assert _static(lib, op, u, y, torch.float32) == 1
    assert "64" in nat._detail() or "scratch" in nat._detail()
    hu = np.zeros((1, 1023, 1023), dtype=np.float32)
    hy = np.zeros_like(hu)
    assert lib.frac_apply_static(op.handle, hu.ctypes.data, hy.ctypes.data, 0, 1, None) == 1
    op.close()
