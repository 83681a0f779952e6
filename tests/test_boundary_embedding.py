"""The near field of the boundary vector as a circulant convolution (the reading
the GPU path is built on): with the extended samples G on [0, 3N-2]^d (shifted
index p = e + N - 1) zero-padded to side M' = nextpow2(3N - 1) and the generator
placed at o mod M' for o in [-N, N]^d, the cyclic convolution equals the oracle's
near field on the interior window p in [N, 2N-2]^d: no wrap-around reaches it,
even when 3N - 1 = M' exactly.  Also with only the M'/2 + 1 frequencies of the
first axis carried (the real input's other half rebuilt by conjugate symmetry).
numpy FFTs, no CUDA."""
import numpy as np
import pytest

from oracle import frac_oracle as O


def _embedded_kernel(a, M):
    d = a.ndim
    N = a.shape[0] - 1
    k = np.zeros((M,) * d)
    for o in np.ndindex(*((2 * N + 1,) * d)):
        off = tuple(t - N for t in o)
        k[tuple(t % M for t in off)] = a[tuple(abs(t) for t in off)]
    return k


def _random_samples(d, N, seed):
    G = np.random.default_rng(seed).standard_normal((3 * N - 1,) * d)
    ext = np.arange(1 - N, 2 * N)
    inside = np.ones(G.shape, dtype=bool)
    for i in range(d):
        shape = [1] * d
        shape[i] = len(ext)
        inside = inside & ((ext >= 1) & (ext <= N - 1)).reshape(shape)
    G[inside] = 0.0
    return G


@pytest.mark.parametrize("d,N", [(1, 2), (1, 3), (1, 11), (2, 2), (2, 3), (2, 6), (2, 11), (3, 3), (3, 4)])
def test_cyclic_convolution_on_side_nextpow2_of_3N_minus_1(d, N):
    a = O.stencil(d, N, 2.0 / N, 1.3, 1, q=12)
    G = _random_samples(d, N, 5 * N + d)
    M = 1 << int(np.ceil(np.log2(3 * N - 1)))
    X = np.zeros((M,) * d)
    X[tuple(slice(0, 3 * N - 1) for _ in range(d))] = G
    S = np.fft.fftn(_embedded_kernel(a, M))
    assert np.max(np.abs(S.imag)) <= 1e-12 * np.abs(a).sum()        # real even kernel: real symbol
    Y = np.fft.ifftn(np.fft.fftn(X) * S.real).real
    win = tuple(slice(N, 2 * N - 1) for _ in range(d))
    ref = O.boundary_near(a, G)
    scale = np.abs(a).sum() * 2 ** d * np.abs(G).max()
    assert np.max(np.abs(Y[win] - ref)) <= 1e-13 * scale
    # half spectrum along the fastest axis (the GPU's axis 0): rfftn / irfftn give the same window
    Yh = np.fft.irfftn(np.fft.rfftn(X) * S.real[..., : M // 2 + 1], s=(M,) * d, axes=tuple(range(d)))
    assert np.max(np.abs(Yh[win] - ref)) <= 1e-13 * scale


def test_smaller_side_wraps_around():
    """The bound is tight in the sense that matters: a side below 3N - 1 cannot hold
    the samples, and at side 2N + 2 (enough for the kernel alone) offsets wrap into
    the window."""
    d, N = 1, 8
    a = O.stencil(d, N, 2.0 / N, 1.3, 1)
    G = _random_samples(d, N, 1)
    ref = O.boundary_near(a, G)
    M = 2 * N + 2
    X = np.zeros(M)
    X[: M] = G[:M]                      # what fits; the rest of G is lost or would alias
    Y = np.fft.ifft(np.fft.fft(X) * np.fft.fft(_embedded_kernel(a, M)).real).real
    assert np.max(np.abs(Y[N:2 * N - 1] - ref)) > 1e-6 * np.abs(ref).max()
