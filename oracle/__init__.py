"""FP64 CPU oracle for the operator-factorization discretization of the
integral fractional Laplacian (Wu & Zhang, arXiv 2103.03658).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.

Every function is a plain, slow restatement of one passage of the paper,
written in numpy/scipy double precision with no blocking or fusion, and no
FFT in the method's arithmetic: the Toeplitz apply is the dense sum of the
scheme, the solve is a dense Cholesky factorisation (or plain CG with the
dense apply).  The one FFT (numpy's) is in ``spectral_bound``, the scale of
the tests' tolerances, which is not a step of the method.
"""
from .frac_oracle import *  # noqa: F401,F403
