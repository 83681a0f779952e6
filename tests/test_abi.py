"""The C-ABI library loads and exports every entry point of include/frac.h;
argument validation that needs no GPU (no compute calls here)."""
import ctypes

import pytest

import paper_2103_03658_gb300 as fg
from paper_2103_03658_gb300 import _native as nat


@pytest.fixture(scope="module")
def lib():
    return nat.load(build_if_missing=True)


def test_exports_every_declared_symbol(lib):
    names = nat.declared_entry_points()
    assert {"frac_coeffs", "frac_apply", "frac_solve", "frac_solve_batch", "frac_op_free",
            "frac_op_info", "frac_op_generator", "frac_strerror"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_strerror(lib):
    for s in range(8):
        assert lib.frac_strerror(s)
    assert lib.frac_strerror(99) == b"unknown status"


def test_invalid_problems_rejected_before_any_device_work(lib):
    bad = [dict(d=4), dict(alpha=0.0), dict(alpha=2.0), dict(degree=5), dict(degree=-1), dict(h=-1.0),
           dict(lam=-0.1), dict(n=0), dict(degree=2, n=8), dict(degree=3, n=7), dict(degree=4, n=9),
           dict(degree=3, n=9, d=2), dict(degree=4, n=6, d=3), dict(lam=float("nan")), dict(gamma=1.0),
           dict(gamma=0.5), dict(gamma=2.5), dict(gamma=-1.0)]
    for b in bad:
        kw = dict(d=1, degree=1, alpha=1.0, h=0.25, n=7, lam=0.0, gamma=0.0)
        kw.update(b)
        prob = nat.Problem(kw["d"], kw["degree"], kw["alpha"], kw["h"], (ctypes.c_int64 * 3)(kw["n"], kw["n"], kw["n"]),
                           kw["lam"], kw["gamma"])
        out = ctypes.c_void_p()
        assert lib.frac_coeffs(ctypes.byref(prob), ctypes.byref(out), None) == 1, b
        assert not out.value
    # rectangular grids (unequal extents) are valid; a bad extent on any axis is not: an
    # empty second axis, and an odd N_2 with the quadratic basis
    for n3, degree in (((7, 0, 1), 1), ((7, 6, 1), 2), ((5, 5, 0), 0)):
        prob = nat.Problem(2 if n3[2] == 1 else 3, degree, 1.0, 0.25, (ctypes.c_int64 * 3)(*n3), 0.0)
        out = ctypes.c_void_p()
        assert lib.frac_coeffs(ctypes.byref(prob), ctypes.byref(out), None) == 1, n3
        assert not out.value


def test_null_arguments(lib):
    assert lib.frac_coeffs(None, None, None) == 1
    assert lib.frac_apply(None, None, None, 0, 1, None) == 1
    assert lib.frac_op_info(None, None) == 1
    lib.frac_op_free(None)
    opts = nat.SolveOpts(1e-10, 10, 0, 0, 0, 1e-4)
    info = nat.SolveInfo()
    assert lib.frac_solve(None, None, None, None, ctypes.byref(opts), ctypes.byref(info), None) == 1
    assert lib.frac_boundary(None, None, None, None, None) == 1
    assert lib.frac_solve_batch(-1, None, None, None, None, None, None) == 1
    assert lib.frac_solve_batch(0, None, None, None, None, None, None) == 0


def test_package_exports():
    assert fg.FracOp and fg.solve_batch and fg.library_path().endswith("libfrac.so")
