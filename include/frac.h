/*
 * frac.h -- C ABI of the GB300 (sm_103a) library for the operator-factorization
 * discretization of the integral fractional Laplacian (-Delta)^{alpha/2} and its
 * tempered generalization (Wu & Zhang, arXiv 2103.03658).
 *
 * Discrete operator (Sec. 2, Eq. (1D-scheme), Eq. (2D-scheme), Remark 2.2):
 *   (-Delta)^{alpha/2}_h u = A u + b,   A = -c_{d,alpha} T(a),
 * T(a) the symmetric multilevel Toeplitz matrix with generator a_k,
 * k in {0..N}^d, built from the weight integrals omega_k^p of Lagrange
 * bases of degree p (Eq. (wi-1D), Eq. (2D-scheme0)), splitting parameter
 * gamma in (alpha, 2] (default 2).
 *
 * Conventions for every entry point:
 *   - Grid vectors are C-ordered arrays of shape [n3][n2][n1] (d = 3),
 *     [n2][n1] (d = 2) or [n1] (d = 1): x^{(1)} is the fastest axis.  A batch
 *     of vectors is contiguous, vector after vector.
 *   - Pointers may be device or host memory; host buffers are staged through
 *     device memory on the given stream (the call then synchronises that
 *     stream before returning).  Device buffers must be aligned to their
 *     element size.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Calls on device buffers are stream-ordered and do not synchronise the
 *     host, except where stated.
 *   - Ownership: callers own every vector; the library owns frac_op objects
 *     and the scratch it allocates (stream-ordered, cudaMallocAsync).
 *   - Return value: FRAC_OK or one of the error codes below; frac_strerror()
 *     names it.  On error no output is written unless stated.
 *   - Devices: an operator's tables live on the device that was current when
 *     frac_coeffs built it.  frac_apply, frac_apply_static, frac_precond,
 *     frac_boundary and frac_solve return FRAC_EINVAL (frac_error_detail says
 *     why) when that device is not the current one, or when a buffer is device
 *     memory of another device.
 */
#ifndef FRAC_H
#define FRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum frac_status {
  FRAC_OK = 0,
  FRAC_EINVAL = 1,      /* invalid argument (see each entry point)              */
  FRAC_ENOMEM = 2,      /* device allocation failed                             */
  FRAC_ENOTSUP = 3,     /* valid but not supported by this build                */
  FRAC_ENOCONV = 4,     /* solver hit max_iter; u holds the last iterate        */
  FRAC_EBREAKDOWN = 5,  /* CG breakdown: p^T A p <= 0 or non-finite             */
  FRAC_ETIMEOUT = 6,    /* a bounded device wait ran out                        */
  FRAC_ECUDA = 7        /* a CUDA runtime call failed                           */
};

enum frac_dtype { FRAC_F32 = 0, FRAC_F64 = 1 };

enum frac_precision {
  FRAC_PLAIN_F64 = 0,   /* CG with the FP64 apply throughout                    */
  FRAC_MIXED_IR = 1     /* FP32 CG inside FP64 iterative refinement             */
};

/* One discretized problem on Omega = prod_i (lo_i, lo_i + (n_i + 1) h). */
typedef struct frac_problem {
  int32_t d;        /* dimension, 1..3                                             */
  int32_t degree;   /* Lagrange basis degree p: 0 (constant), 1 (linear), 2 (quadratic),
                       3 and 4 (higher degrees: origin rules of order 6, 8), any d;
                       p >= 2 needs N_i = n_i + 1 divisible by p                     */
  double alpha;     /* fractional power, 0 < alpha < 2                             */
  double h;         /* mesh size, > 0                                              */
  int64_t n[3];     /* interior points per axis (N_i - 1); entries i >= d ignored.
                       Unequal extents (a rectangular domain, Sec. 2.2) are allowed:
                       the generator covers [0, L]^d with L = max_i N_i h        */
  double lambda;    /* tempering: kernel e^{-lambda |xi|} (Remark 2.2); 0 = (-Delta)^{alpha/2} */
  double gamma;     /* splitting parameter of Eq. (eq0) in (alpha, 2]; 0 means 2 (the default and
                       the most accurate, Sec. 3.1); below 2 the origin term drops (zeta = 0) */
  int32_t fft_lengths; /* circulant embedding lengths M_i (Sec. 2.1 needs M_i >= 2 n_i - 1):
                       FRAC_FFT_POW2 (0, the default): the next power of two >= 2 n_i - 1;
                       FRAC_FFT_SMOOTH (1): the smallest 2^a 3^b 5^c 7^d >= 2 n_i + 2 with a >= 4
                       (mixed-radix FFTs; less padding, and M_i/2 - 1 >= n_i keeps the tau
                       preconditioner for every n_i); FRAC_FFT_AUTO (2): the cheaper of the
                       two by a pass-count model (frac_fft_length).  Axes whose M_i is a power of two run
                       the power-of-two kernels either way; the others the mixed-radix
                       kernels, whose passes all go through shared memory.  Limits as for
                       powers of two: M_i <= 8192 (d = 1), 2048 (d = 2), 512 (d = 3).  The
                       persistent 2D batch launch of frac_solve_batch takes power-of-two
                       problems only; mixed-length ones run through the solve engine. */
} frac_problem;

enum frac_fft_lengths { FRAC_FFT_POW2 = 0, FRAC_FFT_SMOOTH = 1, FRAC_FFT_AUTO = 2 };

typedef struct frac_op frac_op;  /* opaque, immutable after frac_coeffs, shareable across streams */

typedef struct frac_op_info_t {
  double c_dalpha;        /* c_{d,alpha} (definition after Eq. (fL-nD))           */
  double a0;              /* centre coefficient a_0 (Eq. (1D-scheme), a_00 of Eq. (2D-scheme)) */
  double far_field;       /* F_d = int over R_+^d \ [0,L]^d of |xi|^{-d-alpha} e^{-lambda|xi|} */
  double norm_bound;      /* max_k |Lambda_k| = ||A||_2 (from the FP64 symbol)    */
  int64_t fft_len;        /* M_1: circulant embedding length of axis 1 (see frac_problem.fft_lengths) */
  int64_t n_gen;          /* N + 1: generator entries per axis, N = the largest N_i */
  size_t device_bytes;    /* device memory owned by the op                         */
  int32_t precond_ok;     /* 1: the tau preconditioner applies (n_i <= M_i/2 - 1, positive symbol) */
  int64_t n[3];           /* interior points per axis (1 for axes >= d)            */
  int64_t fft_lens[3];    /* M_i per axis (1 for axes >= d)                        */
} frac_op_info_t;

/*
 * frac_coeffs -- build the operator of `prob` on the device.
 * Computes, in FP64 on the GPU: the weight integrals omega_k^p for
 * k in {0..N}^d (Eq. (wi-1D); Eq. (2D-scheme0); its 3D analogue), the
 * stencil a_k = 2^{z(k)} omega_k / |xi_k|^2 with the origin rule, the centre
 * coefficient a_0 = -sum_{k!=0} 2^{d-z(k)} a_k - 2^d F_d, and the symbol
 * Lambda = -c_{d,alpha} DFT_M(circulant embedding of a) (real, even), kept in
 * FP64 and FP32.  *out receives a new op (release with frac_op_free).
 * Errors: FRAC_EINVAL (d not in 1..3, alpha not in (0,2), degree not in 0..4, n_i < 1, N_i not divisible by a degree >= 2, h <= 0 or
 * non-finite, gamma not 0 and not in (alpha, 2], fft_lengths not a frac_fft_lengths value,
 * lambda < 0 or non-finite, out == NULL), FRAC_ENOTSUP (M beyond the FFT
 * sizes of this build, per axis: M_i <= 8192 for d = 1, <= 2048 for d = 2,
 * <= 512 for d = 3), FRAC_ENOMEM, FRAC_ECUDA.  Synchronises `stream` before returning.
 */
int frac_coeffs(const frac_problem* prob, frac_op** out, void* stream);

/*
 * frac_fft_length -- the circulant embedding length M that frac_coeffs gives an
 * axis of n interior points in dimension d under the policy fft_lengths (see
 * frac_problem.fft_lengths), written to *M.  Host only (no device work).
 * FRAC_FFT_AUTO compares M times the transform's passes through shared memory:
 * ceil(log2 M / 4) for a power of two (register-interface radix-16 passes), the
 * plan's passes plus one for a mixed length (plus two for d = 1), over the power
 * of two (if M/2 - 1 >= n) and every mixed length from 2 n + 2 up to it (up to
 * twice it when it does not hold the tau system); ties keep the power of two.
 * Errors: FRAC_EINVAL (n < 1, d not in 1..3, unknown policy, M == NULL),
 * FRAC_ENOTSUP (the length is beyond this build's limit for d).
 */
int frac_fft_length(int64_t n, int32_t d, int32_t fft_lengths, int64_t* M);

/*
 * frac_apply_3d_passes -- schedule of the 3D FP32 apply (frac_apply, frac_precond and
 * the FP32 CG of the solvers) for this process: fused != 0 runs the x and y transforms
 * of each z-plane fused on a thread-block cluster of 8 CTAs, the plane's x spectra kept
 * in distributed shared memory (three passes over device memory: xy forward, z with the
 * symbol, xy inverse); 0 (the default) runs five pencil passes (x, y, z, y, x), which
 * measured faster on GB300 (255^3: 0.49 against 0.82 ms).  Both run the same device
 * functions and agree to FP32 rounding.  The fused schedule applies to operators with
 * equal power-of-two x and y FFT lengths 32..512 on a device that can hold a cluster of
 * 8 CTAs of the pass's shared memory; others always take the five passes.  Host only,
 * returns FRAC_OK.
 */
int frac_apply_3d_passes(int32_t fused);

/* Release an op (NULL is ignored).  The caller must ensure no work using it is in flight. */
void frac_op_free(frac_op* op);

/* Fill *info (host pointer).  Errors: FRAC_EINVAL for NULL arguments. */
int frac_op_info(const frac_op* op, frac_op_info_t* info);

/*
 * Copy the FP64 generator a_k (k in {0..N}^d, C order, k_1 fastest, a[0] = a_0)
 * to the host buffer `a` of `count` doubles.  Errors: FRAC_EINVAL if count
 * differs from (N+1)^d or a pointer is NULL; FRAC_ECUDA.  Synchronous.
 */
int frac_op_generator(const frac_op* op, double* a, size_t count);

/*
 * frac_apply -- y = A u for `batch` grid vectors (Eq. (1D-scheme) and
 * Eq. (2D-scheme) with b = 0, i.e. g = 0), by circulant embedding and FFT
 * (Sec. 2.1 notes that the Toeplitz structure allows an O(N log N) FFT product).  u and y hold
 * batch * prod(n_i) values of `dtype` (FRAC_F32: float, FP32 FFT and symbol;
 * FRAC_F64: double, FP64 FFT and symbol).  u and y must not overlap.
 * Errors: FRAC_EINVAL (NULL op/pointers with batch > 0, batch < 0, unknown
 * dtype, misaligned device pointer), FRAC_ENOMEM, FRAC_ECUDA.
 * batch == 0 is a no-op.
 */
int frac_apply(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, void* stream);

/*
 * frac_apply_static -- the same y = A u as frac_apply, for callers that cannot
 * allocate device memory when they apply the operator (a fixed memory budget
 * reserved up front, a host framework that forbids device allocations after
 * start-up, or a latency-critical loop that cannot let an allocation stall or
 * fail mid-step).  This entry point has no counterpart in the paper.
 * Its spectral scratch is one fixed 64 MiB device array inside the library,
 * reserved on every GPU that loads the library and held until the process
 * exits; it calls no cudaMalloc, cudaFree or other allocating routine.  The
 * first call on a device looks up that array's device address (with the
 * device current), so make that first call before any stream capture.
 * u and y must be device buffers (host buffers would need staging memory).
 * Every call shares the one array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on it and must be
 * serialised by the caller; nothing needs clearing between calls, because
 * every scratch entry an apply reads is written earlier in the same apply.
 * Errors: as frac_apply, plus FRAC_EINVAL for host buffers or for a batch
 * whose scratch exceeds 64 MiB (frac_error_detail() gives the sizes; split
 * the batch or call frac_apply).  d = 1 applies need no scratch at all.
 */
int frac_apply_static(const frac_op* op, const void* u, void* y, int dtype, int64_t batch, void* stream);

/*
 * frac_precond -- z = P r, the tau preconditioner of the CG solves (the paper
 * names no solver; this is the library's).  With m = M/2 - 1 >= n per axis,
 * P = R tau(T_m)^{-1} R^T: T_m is the Toeplitz matrix of the generator a
 * zero-extended to size m (T_n is its leading block, R the restriction to it)
 * and tau(T_m) = T_m - H_m (H_m the Hankel correction, levelwise in d >= 2) is
 * diagonalised by the sine transform of size m with the circulant-embedding
 * eigenvalues of A as its eigenvalues; P is symmetric positive definite.
 * Computed as the FFT pipeline of frac_apply on the odd extension of r with the
 * reciprocal symbol.  Layout, dtype, batch, buffers (device or host) and
 * stream as frac_apply; r and z must not overlap.
 * Errors: as frac_apply, plus FRAC_ENOTSUP when the preconditioner does not
 * apply to op (n a power of two, so that M/2 - 1 < n, or a symbol that is not
 * positive; frac_op_info reports precond_ok).
 */
int frac_precond(const frac_op* op, const void* r, void* z, int dtype, int64_t batch, void* stream);

/* Preconditioner of the CG iterations (frac_solve_opts.precond). */
enum {
  FRAC_PRECOND_TAU = 0,   /* the tau preconditioner (see frac_precond); plain CG where it does not apply */
  FRAC_PRECOND_NONE = 1   /* plain CG */
};

typedef struct frac_solve_opts {
  double rtol;          /* target ||f - A u||_2 / ||f||_2 (true residual, FP64); e.g. 1e-10 */
  int32_t max_iter;     /* cap on CG iterations (all inner iterations summed for MIXED_IR) */
  int32_t precision;    /* FRAC_PLAIN_F64 or FRAC_MIXED_IR                                  */
  int32_t use_x0;       /* nonzero: u holds the initial guess on entry                      */
  int32_t precond;      /* FRAC_PRECOND_TAU (0, the default) or FRAC_PRECOND_NONE           */
  double inner_tol;     /* MIXED_IR: relative residual reduction of each FP32 inner solve;
                           0 = automatic: max(1e-6, sqrt(rtol)/10) when the symbol's max/min
                           ratio is below 50, else 1e-4                                      */
} frac_solve_opts;

typedef struct frac_solve_info {
  int32_t status;       /* FRAC_OK, FRAC_ENOCONV or FRAC_EBREAKDOWN                    */
  int32_t iters;        /* CG iterations (inner iterations summed for MIXED_IR)        */
  int32_t outer;        /* refinement steps (MIXED_IR), 0 for PLAIN_F64                */
  int32_t precond;      /* 1: the tau preconditioner was used, 0: plain CG               */
  double rel_resid;     /* final ||f - A u||_2 / ||f||_2, recomputed with the FP64 apply */
} frac_solve_info;

/*
 * frac_boundary -- boundary vector of nonhomogeneous exterior data g (Eq. (L2),
 * the b of the schemes' matrix forms in 1D and 2D):
 *   b_i = -c (near_i + far_i),  near_i = sum over o in [-N, N]^d of
 *   a_{|o|} g(x_i + o h) over the points x_i + o h outside the domain,
 * far_i the integrals of g over the far region (the sum over the 2^d
 * reflections of int over Upsilon_+^c of g(x_i + s xi) |xi|^{-d-alpha}
 * e^{-lambda |xi|} dxi), which depend on g beyond every grid point and are the
 * caller's.  Then A u = f - b is the discrete problem with u = g outside
 * (frac_solve takes b as its g argument).
 *   g_ext: prod_i (n_i + 2N) doubles, N = max_i n_i + 1 (the generator's cube
 *          spans the longest axis, so its reach is N points on every axis): g at
 *          the grid points x_0 + e h (x_0 the domain's lower corner), e in
 *          [1 - N, n_i + N] on axis i, axis 0 fastest as in u; the interior
 *          points are e in [1, n_i] on every axis and their values are not read.
 *   far:   prod(n_i) doubles, or NULL for zero (g of compact support within
 *          reach of the grid).
 *   b:     prod(n_i) doubles, written.
 * Device or host pointers (host buffers are staged).  The near field is a
 * convolution on a circulant of sides M'_i = nextpow2(n_i + 2N) in FP64 (d = 2, 3:
 * a transient complex array of (M'_0/2 + 1) prod_{i>0} M'_i entries, 8.6 GB at 3D
 * n = 256) or a direct sum (d = 1).  Synchronises `stream`.  Errors: FRAC_EINVAL
 * (NULL op/g_ext/b), FRAC_ENOTSUP (M'_i beyond 4096), FRAC_ENOMEM, FRAC_ECUDA
 * (including a failed device bounds check, named by frac_error_detail).
 */
int frac_boundary(const frac_op* op, const double* g_ext, const double* far, double* b, void* stream);

/*
 * Far field of exterior data g (the far_i of frac_boundary: the second integral of
 * Eq. (L2), over Upsilon_+^c, summed over the 2^d reflections), on the device.  The
 * C ABI cannot carry the function g, so the caller evaluates it between two calls
 * (reverse communication): frac_far_points lists the points at which g is needed,
 * the caller writes g there into a device buffer, frac_far_sum forms the weighted
 * sums.  The rule is the same for every grid point: Q nodes xi_q in R_+^d outside
 * [0, L]^d and weights w_q with
 *     far_i ~ sum_{m in {0,1}^d} sum_q w_q g(x_i + s(m) o xi_q),  s(m)_k = -1 if bit k of m is set,
 * from the split of the region into the d pyramids where coordinate k is the largest,
 * xi = rho (1, s) (coordinate k first), rho = L / t with t by an nr-point Gauss-Jacobi
 * rule for the weight t^{alpha-1} and each s_j by an ns-point Gauss-Legendre rule on
 * [0, 1]; w_q carries L^{-alpha}, |(1, s)|^{-d-alpha} and e^{-lambda rho |(1, s)|}.
 * Q = d ns^{d-1} nr.  The error falls quickly with nr and ns for g smooth and bounded
 * outside the domain (96 and 48 give about 1e-14 for the paper's exterior data).
 *
 * frac_far_nodes (host only, no device work): the rule for dimension d, power alpha,
 * tempering lambda and cube side L = N h (N = max_i n_i + 1, the side of the
 * generator's cube): *count = Q; xi (Q*d doubles, node-major, coordinate k along
 * axis x^(k+1)) and w (Q doubles) are filled when not NULL.  Errors: FRAC_EINVAL (d
 * not in 1..3, alpha not in (0,2), lambda < 0 or not finite, L <= 0, nr or ns not in
 * 1..512, NULL count), FRAC_ECUDA (an eigenvalue iteration that did not converge).
 *
 * frac_far_points: for the `count` grid points first..first+count-1 (flat index,
 * axis x^(1) fastest as in u), writes the points x_i + s(m) o xi_q to pts (device,
 * count * 2^d * nq * d doubles, ordered (point, m, q, coordinate)); x_i has coordinate
 * lo[k] + (j_k + 1) h along axis x^(k+1), lo (host, d doubles) the domain's lower
 * corner.  xi: the nq nodes of frac_far_nodes in a device buffer.
 * frac_far_sum: far[p] = sum_m sum_q w[q] g[(p 2^d + m) nq + q] for p < count
 * (device buffers; far receives count doubles, in the order of the points).
 * Both are stream-ordered on `stream`.  Errors: FRAC_EINVAL (NULL pointers, nq < 1,
 * points outside the grid, host buffers or buffers of another device).
 */
int frac_far_nodes(int32_t d, double alpha, double lambda, double L, int32_t nr, int32_t ns, double* xi,
                   double* w, int64_t* count);
int frac_far_points(const frac_op* op, const double* lo, const double* xi, int64_t nq, int64_t first,
                    int64_t count, double* pts, void* stream);
int frac_far_sum(const frac_op* op, const double* w, int64_t nq, const double* g, int64_t count, double* far,
                 void* stream);

/*
 * frac_solve -- solve A u = f - g for one right-hand side (the fractional
 * Poisson problem Eq. (Poisson)-(BC); Example 3.2.3 asks for an FFT-based
 * fast solver without naming one).  A is symmetric positive
 * definite, so the solver is conjugate gradients with the FFT apply, either in
 * FP64 or as FP32 CG inside FP64 iterative refinement.  f and u hold prod(n_i)
 * doubles (device or host).  g is NULL (homogeneous exterior data) or the
 * boundary vector b of frac_boundary (prod(n_i) doubles, device or host); the
 * residual of info->rel_resid is then relative to ||f - g||.  `info` is a host
 * pointer filled before return (the call synchronises `stream`).  Errors:
 * FRAC_EINVAL (NULL op/f/u/opts/info, rtol <= 0, max_iter < 1, unknown
 * precision, non-finite host f or g), FRAC_ENOCONV / FRAC_EBREAKDOWN (u holds
 * the last iterate, info filled), FRAC_ENOMEM, FRAC_ECUDA.
 */
int frac_solve(const frac_op* op, const double* f, const double* g, double* u,
               const frac_solve_opts* opts, frac_solve_info* info, void* stream);

/*
 * frac_solve_batch -- solve `count` independent problems (ops[i], f[i], u[i],
 * all device pointers) with the same options; info[i] filled per problem
 * (host array).  Problems run concurrently on the device:
 *   - 1D problems of M <= 8192: solved whole inside one thread block each,
 *     one launch per FFT length;
 *   - 2D problems of M in [32, 1024] with FRAC_MIXED_IR: one persistent launch
 *     of thread-block clusters takes them from work queues, largest first; the
 *     larger FFT lengths are solved by a whole cluster each, the smaller by one
 *     block each, as chosen by an autotuner that times each FFT length once
 *     per device (the first batch with a new length pays for that timing);
 *   - the others share a solve engine (frac_engine_*) on several streams.
 * The 1D and 2D launches (with their uploads) are captured into one CUDA graph
 * and launched once on `stream`; the autotuner's first timings run before the
 * capture.  `stream` must not be capturing when this is called.
 * Errors as frac_solve, per problem in info[i].status; the return value is the
 * first nonzero status or FRAC_OK.  Synchronizes `stream` before returning.
 */
int frac_solve_batch(int64_t count, const frac_op* const* ops, const double* const* f,
                     double* const* u, const frac_solve_opts* opts, frac_solve_info* info,
                     void* stream);

/*
 * frac_batch_last_plan -- the plan of the calling thread's last
 * frac_solve_batch call that used the persistent 2D launch: cluster size,
 * resident clusters launched, the smallest FFT length (log2) solved
 * cluster-wide (11 = none), problems in each queue and the autotuner's
 * predicted makespan in ms (from timed probe solves of each FFT length and
 * estimated iteration and refinement counts; on a 117-problem 2D mix it came
 * within 20 % of the measured time, below it).  Errors: FRAC_EINVAL (NULL
 * out, or no such call on this thread).
 */
typedef struct frac_batch_plan {
  int32_t cluster_size;
  int32_t clusters;
  int32_t first_cluster_logm;
  int32_t cluster_problems;
  int32_t local_problems;
  double predicted_ms;
} frac_batch_plan;
int frac_batch_last_plan(frac_batch_plan* out);

/*
 * frac_batch_pin_plan -- pin the persistent 2D launch of the calling thread's
 * later frac_solve_batch calls: clusters of `cluster_size` CTAs (1, 2, 4, 8 or
 * 16), with FFT lengths >= 2^first_cluster_logm solved cluster-wide (11: none,
 * every problem on one block); cluster_size 0 returns to the autotuner.  The
 * solutions do not depend on the plan beyond rounding.  Errors: FRAC_EINVAL
 * (another size, or first_cluster_logm outside [5, 11]); a pinned size that the
 * device cannot launch makes frac_solve_batch return FRAC_ENOTSUP.
 */
int frac_batch_pin_plan(int32_t cluster_size, int32_t first_cluster_logm);

/*
 * Kernel timing (tracing aid, off by default; not part of the paper's method).
 * frac_profile_enable(1) makes every library kernel launch record a pair of
 * CUDA events on its own stream; frac_profile_read() waits for the recorded
 * events, folds them into per-kernel totals (launch count, summed device time
 * in ms), copies up to `cap` of them to `out` (host array), stores the number
 * of kernels in *count and, if `reset`, clears the totals.  Names identify the
 * kernel, precision and FFT length (e.g. "cols_sym_f32_M2048").
 * Errors: FRAC_EINVAL (NULL count, cap < 0), FRAC_ECUDA.
 */
typedef struct frac_kernel_stat {
  char name[48];
  int64_t launches;
  double total_ms;
} frac_kernel_stat;

int frac_profile_enable(int on);
int frac_profile_read(frac_kernel_stat* out, int cap, int* count, int reset);

/*
 * frac_profile_alu_peak -- measures the arithmetic rate of the current GPU for
 * the rooflines of the library's ALU-bound kernels (a measurement aid, not
 * part of the paper's method): a grid of 8 blocks of 256 threads per SM runs 8
 * independent fused multiply-add chains per thread; `kind` 0 = FP32 (fma.rn.f32),
 * 1 = FP64 (fma.rn.f64), 2 = FP32 in pairs (fma.rn.f32x2, two FMAs per
 * instruction).  *tflops receives 2 flops per FMA over the best of three timed
 * launches (CUDA events on `stream`); the call synchronises `stream` and
 * allocates (and frees) a small result buffer.  Errors: FRAC_EINVAL (kind
 * unknown, NULL tflops), FRAC_ENOMEM, FRAC_ECUDA.
 */
int frac_profile_alu_peak(int kind, double* tflops, void* stream);

/*
 * Solve engine: many solves in flight at once (continuous batching).  Each
 * submitted job advances through its own stream from a fixed pool: d = 1 as
 * one whole-solve block, d >= 2 as FP32 CG chunks (replayed CUDA graphs) and
 * FP64 refinement steps (or FP64 CG chunks for FRAC_PLAIN_F64), exactly the
 * computation of frac_solve.  Jobs submitted while others run start at once;
 * their kernels overlap on the device.  Not thread safe: one host thread
 * drives an engine.
 *
 * frac_engine_create: `nstreams` >= 1 streams (non-blocking, created on the
 *   current device).  Errors: FRAC_EINVAL (nstreams < 1, out NULL), FRAC_ECUDA.
 * frac_engine_submit: queue A u = f with `opts`; f and u are device or host
 *   buffers of prod(n_i) doubles that must stay valid until the job is
 *   returned by frac_engine_poll (host buffers are staged on the job's
 *   stream).  *job receives an id > 0.  Errors: as frac_solve's argument checks,
 *   FRAC_ENOMEM.  The op must outlive the job.
 * frac_engine_poll: advance every job whose pending device work finished;
 *   copy up to `cap` finished jobs to out (host array), *count = how many.
 *   With block != 0 it waits until at least one job finishes (returns at once
 *   when none is in flight).
 * frac_engine_stats: jobs in flight and device bytes they hold (host pointers).
 * frac_engine_destroy: waits for all work, releases every job and stream.
 */
typedef struct frac_engine frac_engine;
typedef struct frac_job_result {
  int64_t job;
  frac_solve_info info;
  double submit_to_done_ms;  /* host wall time from submit to completion seen by poll */
} frac_job_result;

int frac_engine_create(int nstreams, frac_engine** out);
int frac_engine_submit(frac_engine* e, const frac_op* op, const double* f, double* u, const frac_solve_opts* opts,
                       int64_t* job);
int frac_engine_poll(frac_engine* e, int block, frac_job_result* out, int cap, int* count);
int frac_engine_stats(const frac_engine* e, int64_t* active, size_t* device_bytes);
void frac_engine_destroy(frac_engine* e);

/* Static string naming a status code. */
const char* frac_strerror(int status);

/* Text of the last failed CUDA runtime call made by the library in the calling
 * thread ("file:line call -> error"), or "" if none; valid until the next failure. */
const char* frac_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* FRAC_H */
