"""GB300 (sm_103a) library for the operator-factorization discretization of
the integral fractional Laplacian and its tempered form (Wu & Zhang,
arXiv 2103.03658): coefficients, FFT Toeplitz apply and CG / mixed-precision
iterative-refinement solves, behind the C ABI of include/frac.h.
"""
from ._native import (F32, F64, MIXED_IR, PLAIN_F64, Engine, FracError, FracOp, apply_3d_passes,  # noqa: F401
                      batch_last_plan,
                      batch_pin_plan, declared_entry_points, far_nodes, fft_length, library_path, load,
                      solve_batch)
