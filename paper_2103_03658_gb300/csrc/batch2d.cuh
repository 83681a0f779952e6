// Persistent batched 2D solver (batch2d.cu).
#pragma once

#include "apply.cuh"

namespace frac {

// FFT lengths handled by the persistent kernel: 2^5 .. 2^10 (n = 9 .. 511) and the
// mixed (7-smooth) lengths between.
constexpr int kBatch2dMinLog = 5, kBatch2dMaxLog = 10;

// True when a problem can go to the persistent kernel (square d = 2, mixed precision,
// FFT length in range); f and u must also be device pointers.
bool batch2d_eligible(const frac_op* op, const frac_solve_opts* opts);

// Everything of a solve_batch_2d call that must not run inside a stream capture:
// the kernel attributes, the twiddle tables and the autotuner's timings of every
// FFT length among idx[0..count) not yet timed on this device (kernels that run,
// and are waited for, on st).
int batch2d_prepare(int64_t count, const frac_op* const* ops, const double* const* f, const int64_t* idx,
                    cudaStream_t st);

// Launches the problems idx[0..count) of (ops, f, u) in one persistent launch
// on st (the autotuner's first timings of a new FFT length run, and wait,
// before it); the results arrive through pend->collect().  Fills the plan used
// when plan is not null.  pin_size > 0 fixes the cluster size (and pin_cut the
// first cluster-wide log2 FFT length) instead of the autotuner's choice.
int solve_batch_2d(int64_t count, const frac_op* const* ops, const double* const* f, double* const* u,
                   const frac_solve_opts* opts, const int64_t* idx, cudaStream_t st, frac_batch_plan* plan,
                   int pin_size, int pin_cut, BatchPending* pend);

}  // namespace frac
