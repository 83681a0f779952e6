// Whole-solve kernel for 1D problems (one thread block per problem).
#pragma once

#include "common.cuh"

namespace frac {

struct Solve1dTask {
  const double* f;        // device, n values
  double* u;              // device, n values (initial guess if use_x0)
  const float* lam32;     // scaled symbols of the problem's op
  const double* lam64;
  frac_solve_info* info;  // device, one record
  double rtol, inner_tol;
  int n, max_iter, use_x0;
};

// Launch one block per task; all tasks share FFT length 2^logm (<= 8192).
int solve1d_launch(int logm, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st);

}  // namespace frac
