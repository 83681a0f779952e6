"""Circulant embedding lengths (frac_fft_length, host only; Sec. 2.1 needs M_i >= 2 n_i - 1):
the power-of-two policy gives the next power of two, the smooth policy the smallest
2^a 3^b 5^c 7^d >= 2 n + 2 with a >= 4 (so M/2 - 1 >= n keeps the tau system), both
against a brute-force search written here, and the per-dimension limits."""
import pytest

import paper_2103_03658_gb300 as fg
from paper_2103_03658_gb300 import _native as nat

CAP = {1: 8192, 2: 2048, 3: 512}


def _smooth_ok(m):
    if m % 16:
        return False
    for q in (2, 3, 5, 7):
        while m % q == 0:
            m //= q
    return m == 1


def _brute(n, d, fft):
    m = 2
    while m < 2 * n - 1:
        m *= 2
    if fft == "smooth":
        s = 2 * n + 2
        while not _smooth_ok(s):
            s += 1
        if s <= CAP[d]:
            m = s
    return m


def test_lengths_match_brute_force():
    fg.load()
    for d in (1, 2, 3):
        for n in list(range(1, 300)) + [511, 512, 513, 700, 1000, 1023, 1024, 1500, 3000, 4000, 4095, 4096]:
            for fft in ("pow2", "smooth"):
                want = _brute(n, d, fft)
                if want > CAP[d]:
                    with pytest.raises(fg.FracError) as e:
                        fg.fft_length(n, d, fft)
                    assert e.value.status == 3  # FRAC_ENOTSUP
                    continue
                got = fg.fft_length(n, d, fft)
                assert got == want, (n, d, fft, got, want)
                assert got >= 2 * n - 1


def test_smooth_lengths_are_shorter_and_keep_the_tau_system():
    fg.load()
    assert fg.fft_length(1023, 2, "smooth") == 2048  # a power of two already
    assert fg.fft_length(99, 1, "smooth") == 224      # 2^5 7
    assert fg.fft_length(39, 2, "smooth") == 80       # 2^4 5
    assert fg.fft_length(1024, 2, "smooth") == 2048   # 2160 is beyond the 2D limit: the power of two
    for n in range(8, 1000, 7):
        m = fg.fft_length(n, 1, "smooth")
        assert m // 2 - 1 >= n and m <= fg.fft_length(n, 1, "pow2") * 2


def test_huge_sizes_are_refused_at_once():
    """Sizes far beyond every limit return FRAC_ENOTSUP without searching for a length."""
    import time
    fg.load()
    t0 = time.perf_counter()
    for fft in ("pow2", "smooth", "auto"):
        for n in (10 ** 6, 10 ** 9, 2 ** 40):
            with pytest.raises(fg.FracError) as e:
                fg.fft_length(n, 1, fft)
            assert e.value.status == 3
    assert time.perf_counter() - t0 < 1.0


def test_invalid_arguments():
    lib = nat.load()
    import ctypes
    m = ctypes.c_int64()
    assert lib.frac_fft_length(0, 1, 0, ctypes.byref(m)) == 1
    assert lib.frac_fft_length(5, 4, 0, ctypes.byref(m)) == 1
    assert lib.frac_fft_length(5, 1, 3, ctypes.byref(m)) == 1
    assert lib.frac_fft_length(5, 1, 0, None) == 1


def _np_plan(m):
    a = 0
    while m % 2 == 0:
        m //= 2
        a += 1
    odd = 0
    for q in (3, 5, 7):
        while m % q == 0:
            m //= q
            odd += 1
    return (a + 3) // 4 + odd


def _auto(n, d):
    p2 = 2
    while p2 < 2 * n - 1:
        p2 *= 2
    cap = CAP[d]

    def cost(m):
        if m & (m - 1) == 0:
            return m * ((m.bit_length() - 1 + 3) // 4)
        return m * (_np_plan(m) + (2 if d == 1 else 1))
    tau = p2 // 2 - 1 >= n
    best, pick = (cost(p2) if tau else float("inf")), p2
    c = (2 * n + 2 + 15) // 16 * 16
    while c <= min(cap, p2 if tau else 2 * p2):
        if _smooth_ok(c) and cost(c) < best:
            best, pick = cost(c), c
        c += 16
    return pick


def test_auto_policy_follows_the_pass_count_model():
    """FRAC_FFT_AUTO: the power of two or a 7-smooth length, whichever makes fewer
    shared-memory passes per point by the model of frac_fft_length; the measured cases
    that calibrate it pick what measured faster."""
    fg.load()
    for d in (1, 2, 3):
        for n in list(range(1, 260, 3)) + [300, 600, 700, 1000, 1100, 3000]:
            want = _auto(n, d)
            if want > CAP[d]:
                continue
            assert fg.fft_length(n, d, "auto") == want, (n, d)
    assert fg.fft_length(600, 2, "auto") == 1280 and fg.fft_length(300, 2, "auto") == 640
    assert fg.fft_length(700, 2, "auto") == 2048 and fg.fft_length(1000, 2, "auto") == 2048
    assert fg.fft_length(200, 3, "auto") == 512 and fg.fft_length(100, 3, "auto") == 256
    assert fg.fft_length(3000, 1, "auto") == 8192 and fg.fft_length(1100, 1, "auto") == 4096
    for d, n in ((1, 64), (2, 64), (3, 16)):  # the power of two lacks the tau system
        m = fg.fft_length(n, d, "auto")
        assert m // 2 - 1 >= n
