"""CPU check of the algebra behind the tau preconditioner's packed column passes: two
real columns carried by one complex transform on the odd extension separate again into
the real and imaginary parts, for each of the four pass forms the kernels use (the 2D
symbol pass on imaginary columns, the 3D z pass on real ones, the forward y pass from
imaginary to real columns and the inverse y pass back).  numpy's FFT stands in for the
device transforms; the device passes themselves are compared with the oracle in
test_gpu_precond and test_gpu_rect."""
import numpy as np
import pytest


def odd_ext(x, M):
    """Odd extension of the columns x[0..n) to length M: x_j at j + 1, -x_j at M - 1 - j."""
    n = x.shape[0]
    e = np.zeros((M,) + x.shape[1:], dtype=complex)
    e[1:n + 1] = x
    e[M - n:] = -x[::-1]
    return e


def keep(y, n):
    return y[1:n + 1]


@pytest.fixture
def case():
    rng = np.random.default_rng(3)
    M, n = 64, 29
    lam_a = rng.uniform(0.5, 2.0, M // 2 + 1)
    lam_b = rng.uniform(0.5, 2.0, M // 2 + 1)
    k = np.arange(M)
    kr = np.minimum(k, M - k)  # even symbol
    return rng, M, n, lam_a[kr], lam_b[kr]


def test_symbol_pass_on_imaginary_columns(case):
    rng, M, n, la, lb = case
    sa, sb = rng.standard_normal(n), rng.standard_normal(n)
    full = lambda s, lam: keep(np.fft.ifft(np.fft.fft(odd_ext(1j * s, M)) * lam), n)
    F = np.fft.fft(odd_ext(sa + 1j * sb, M))
    z = keep(np.fft.ifft(F.real * lb + 1j * F.imag * la), n)
    ya, yb = full(sa, la), full(sb, lb)
    assert np.allclose(ya.real, 0, atol=1e-13) and np.allclose(yb.real, 0, atol=1e-13)
    assert np.allclose(1j * z.real, ya, atol=1e-13) and np.allclose(1j * z.imag, yb, atol=1e-13)


def test_z_pass_on_real_columns(case):
    rng, M, n, la, lb = case
    ra, rb = rng.standard_normal(n), rng.standard_normal(n)
    full = lambda r, lam: keep(np.fft.ifft(np.fft.fft(odd_ext(r, M)) * lam), n)
    F = np.fft.fft(odd_ext(ra + 1j * rb, M))
    z = keep(np.fft.ifft(F.real * lb + 1j * F.imag * la), n)
    assert np.allclose(z.real, full(ra, la), atol=1e-13) and np.allclose(z.imag, full(rb, lb), atol=1e-13)


def test_forward_y_pass_imaginary_to_real(case):
    rng, M, n, _, _ = case
    sa, sb = rng.standard_normal(n), rng.standard_normal(n)
    full = lambda s: np.fft.fft(odd_ext(1j * s, M))  # all M outputs, real
    F = np.fft.fft(odd_ext(sa + 1j * sb, M))
    Ra, Rb = full(sa), full(sb)
    assert np.allclose(Ra.imag, 0, atol=1e-12) and np.allclose(Rb.imag, 0, atol=1e-12)
    assert np.allclose(-F.imag, Ra.real, atol=1e-12) and np.allclose(F.real, Rb.real, atol=1e-12)


def test_inverse_y_pass_real_to_imaginary(case):
    rng, M, n, _, _ = case
    # real odd-symmetric spectra, as the forward y pass produces them
    Ra = np.fft.fft(odd_ext(1j * rng.standard_normal(n), M)).real
    Rb = np.fft.fft(odd_ext(1j * rng.standard_normal(n), M)).real
    full = lambda R: keep(np.fft.ifft(R), n)  # purely imaginary
    w = keep(np.fft.ifft(Ra + 1j * Rb), n)
    assert np.allclose(full(Ra).real, 0, atol=1e-13) and np.allclose(full(Rb).real, 0, atol=1e-13)
    assert np.allclose(1j * w.imag, full(Ra), atol=1e-13) and np.allclose(-1j * w.real, full(Rb), atol=1e-13)
