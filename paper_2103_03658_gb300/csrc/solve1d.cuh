// Whole-solve kernel for 1D problems (one thread block per problem).
#pragma once

#include "common.cuh"

namespace frac {

struct Solve1dTask {
  const double* f;        // device, n values
  double* u;              // device, n values (initial guess if use_x0)
  const float* lam32;     // scaled symbols of the problem's op
  const double* lam64;
  const float* pinv32;    // tau preconditioner symbols (used when pcg)
  const double* pinv64;
  frac_solve_info* info;  // device, one record
  double rtol, inner_tol;
  int n, max_iter, use_x0, pcg;
};

// The task record of one 1D solve.
inline Solve1dTask make_task1d(const frac_op* op, const double* f, double* u, frac_solve_info* info,
                               const frac_solve_opts* o) {
  return Solve1dTask{f, u, op->lam32, op->lam64, op->pinv32, op->pinv64, info, o->rtol,
                     o->inner_tol > 0.0 ? o->inner_tol : auto_inner_tol(op, o->rtol), (int)op->n, o->max_iter, o->use_x0 ? 1 : 0,
                     (o->precond == FRAC_PRECOND_TAU && op->precond_ok) ? 1 : 0};
}

// Launch one block per task; all tasks share FFT length M (a power of two or a
// 7-smooth mixed length, <= 8192).
int solve1d_launch(int64_t M, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st);
// The same for a mixed length (solve1d_mx.cu).
int solve1d_launch_mx(int64_t M, bool mixed, const Solve1dTask* d_tasks, int ntasks, cudaStream_t st);

}  // namespace frac
