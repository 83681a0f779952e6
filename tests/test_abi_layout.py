"""The ctypes mirrors of the C ABI's structs (the Python binding, the bench's kernel
statistics) have the sizes and field offsets that a C compiler gives the structs of
include/frac.h.  A probe program compiled with gcc against the header prints them."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2103_03658_gb300 import _native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class KernelStat(ctypes.Structure):  # as bench.py reads frac_profile_read
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


# C struct name -> (ctypes class, [(C field, ctypes field)])
STRUCTS = {
    "frac_problem": (nat.Problem, [("d", "d"), ("degree", "degree"), ("alpha", "alpha"), ("h", "h"), ("n", "n"),
                                   ("lambda", "lam"), ("gamma", "gamma"),
                                   ("fft_lengths", "fft_lengths")]),
    "frac_op_info_t": (nat.OpInfo, [(f, f) for f, _ in nat.OpInfo._fields_]),
    "frac_solve_opts": (nat.SolveOpts, [(f, f) for f, _ in nat.SolveOpts._fields_]),
    "frac_solve_info": (nat.SolveInfo, [(f, f) for f, _ in nat.SolveInfo._fields_]),
    "frac_batch_plan": (nat.BatchPlan, [(f, f) for f, _ in nat.BatchPlan._fields_]),
    "frac_job_result": (nat.JobResult, [(f, f) for f, _ in nat.JobResult._fields_]),
    "frac_kernel_stat": (KernelStat, [(f, f) for f, _ in KernelStat._fields_]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "frac.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for cf, _ in fields:
            lines.append(f'  printf("{cname} {cf} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = d / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_ctypes_mirror_matches_c_layout(c_layout, cname):
    cls, fields = STRUCTS[cname]
    assert ctypes.sizeof(cls) == c_layout[(cname, "size")], cname
    for cf, pf in fields:
        assert getattr(cls, pf).offset == c_layout[(cname, cf)], (cname, cf)
