/*
 * sphere_poisson.h -- C ABI of the GB300 (sm_103a) spherical Poisson solver.
 *
 * Solves Poisson's equation on the unit sphere,  Delta u = f  with
 * int_S u = 0, by the double-Fourier-sphere (DFS) Fourier spectral method of
 * Townsend, Wilber & Wright, "Computing with functions in spherical and polar
 * geometries I. The sphere", Section 5:
 *   - sin^2(theta)-multiplied Laplacian, eq. SphericalLaplacian, doubled up
 *     to [-pi, pi]^2 by the glide reflection of eq. BMCsphere (eq. BMCPoisson);
 *   - 2D Fourier coefficients F of sin^2(theta) f~ (eq. 2DFourierExpansion);
 *   - one banded system per longitudinal wavenumber k, eq. linearSystems,
 *     with the k = 0 zeroth row replaced by the zero-mean constraint w^T X_0 = 0
 *     (eq. pentdiagonalPlusRankOne, weights w of eq. integrationCoeffs);
 *   - inverse 2D expansion back to grid values (eq. tildeuFourierExpansion).
 *
 * Grid.  f and u are row-major arrays [n_theta][n_lambda] of doubles,
 *   row i    = colatitude theta_i  = (i + 1/2) pi / n_theta   (no pole samples),
 *   column q = longitude  lambda_q = -pi + 2 pi q / n_lambda.
 * The DFS grid then has m = 2 n_theta colatitudes and n = n_lambda longitudes.
 * Truncation: coefficients X_{j,k} with |j| <= m/2 - 1 and -n/2 <= k <= n/2 - 1;
 * the theta-Nyquist mode j = -m/2 is set to zero (the symmetric window keeps
 * the BMC symmetry X_{-j,k} = (-1)^k X_{j,k} exact).
 *
 * Memory.  All array arguments of the solve calls are DEVICE pointers unless a
 * name says _host.  The caller owns f, u and the workspace; the library owns
 * the plan and the device tables inside it (twiddle factors and the factorised
 * per-k systems).  f, u and workspace must be 16-byte aligned and must not
 * overlap.  Calls are asynchronous on the given stream (a cudaStream_t passed
 * as void*, or NULL for the legacy default stream) except where stated.
 *
 * Errors.  Every call returns an int status: 0 = success, > 0 = success with a
 * warning, < 0 = error (nothing was launched).  sphere_poisson_status_string()
 * gives a message.  No call aborts the process.
 */
#ifndef SPHERE_POISSON_H
#define SPHERE_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SP_OK                0
#define SP_WARN_NONZERO_MEAN 1   /* success; |mean of f| > 1e3 eps max|f| (sphere_poisson_solve_host) */
#define SP_ERR_BAD_SIZE     -1   /* n_theta < 1, n_lambda < 2 or odd, too large, or a prime factor > 31 */
#define SP_ERR_NULL         -2   /* a required pointer is NULL */
#define SP_ERR_MISALIGNED   -3   /* a device pointer is not 16-byte aligned */
#define SP_ERR_WORKSPACE    -4   /* workspace smaller than the plan requires */
#define SP_ERR_CUDA         -5   /* a CUDA runtime call failed (message via status_string) */
#define SP_ERR_UNSUPPORTED  -6   /* precision / flag combination not built */
#define SP_ERR_BAD_PLAN     -7   /* NULL or destroyed plan handle */
#define SP_ERR_BAD_ARG      -8   /* other invalid argument */
#define SP_ERR_SCRATCH_LIMIT -9  /* grid too large for the fixed scratch of sphere_poisson_solve_noalloc */
#define SP_ERR_TIMEOUT      -10  /* a kernel's bounded wait for its asynchronous copies gave up (see
                                    sphere_poisson_device_status) */

/* precision of the arithmetic inside the solve (inputs and outputs are always double) */
#define SP_FP64         0   /* IEEE double throughout */
#define SP_FP32         1   /* single precision transforms and eliminations */
#define SP_FP32_REFINE  2   /* FP32 eliminations + FP64 residual refinement, FP64-accurate transforms */

typedef struct sp_plan_s* sp_plan_t;

/* plan flag: tune the transform tiles at plan time (see the plan calls) */
#define SP_FLAG_AUTOTUNE 1u
/*
 * plan flag: the grid with both poles.  f and u are [n_theta + 1][n_lambda],
 * row i = colatitude theta_i = i pi / n_theta, i = 0..n_theta (row 0 the north
 * pole, row n_theta the south pole; the DFS grid of Section 2 sampled on
 * theta in [0, pi]).  Doubled, the colatitudes are theta_p = -pi + 2 pi p / m,
 * m = 2 n_theta; the coefficients, their truncation and the per-k systems are
 * those of the pole-free grid.  The samples of f on the pole rows are
 * multiplied by sin^2 theta = 0 and do not enter; u is written on every row,
 * the poles included.  SP_FP64 single plans only (other precisions return
 * SP_ERR_UNSUPPORTED), 2 n_theta <= 12288 with 2 n_theta factoring into primes
 * <= 31 (else SP_ERR_BAD_SIZE).  Such a plan supports sphere_poisson_solve
 * (f_mean_out included: the same quadrature on this grid, each pole row
 * weighted once), _solve_adjoint (the transpose of that solve, on the same
 * [n_theta + 1][n_lambda] arrays), _solve_host, _solve_noalloc, the profiling
 * and size queries; every other call on it returns SP_ERR_UNSUPPORTED (the
 * transforms alone, sum2, the derivatives and the low-rank calls).
 */
#define SP_FLAG_POLES 2u

/*
 * Create a plan for grids of n_theta colatitudes x n_lambda longitudes.
 *   n_theta >= 1, n_lambda >= 2 and even (the glide reflection lambda -> lambda+pi
 *   of eq. BMCsphere must map the grid to itself); n_theta and n_lambda/2 must
 *   factor into primes <= 31 and be at most 12288.
 *   precision     SP_FP64; SP_FP32 (FP32 transforms and eliminations, the ill-
 *                 conditioned k = 0 column in FP64); or SP_FP32_REFINE (double-
 *                 float transforms, FP32 eliminations refined by residual sweeps
 *                 computed to FP64 accuracy, the k = 0 column in FP64).  Other
 *                 values return SP_ERR_UNSUPPORTED.
 *   refine_sweeps 0..16 residual sweeps for SP_FP32_REFINE (ignored otherwise;
 *                 outside 0..16 SP_ERR_BAD_ARG).
 *   flags         0, SP_FLAG_POLES (above: the grid with both poles), and/or
 *                 SP_FLAG_AUTOTUNE (below): time the transform tiles
 *                 (rows / columns per CTA and threads per CTA of the longitude
 *                 and colatitude kernels) as whole solves on zero input at plan
 *                 time and keep the fastest; cached like the batched tuner's.
 *                 Tuning allocates an input, an output and a workspace for the
 *                 duration of the call.
 *   workspace_bytes (out, optional) device workspace the solve calls need.
 * Synchronous: allocates the plan's device tables and fills them on the
 * current device; the plan may only be used with that device.
 */
int sphere_poisson_plan(sp_plan_t* plan, int n_theta, int n_lambda, int precision,
                        int refine_sweeps, unsigned flags, size_t* workspace_bytes);

/*
 * Batched plan: `count` independent spheres of uneven resolution, problem b on
 * an n_theta[b] x n_lambda[b] grid (each size obeying the rules above), solved
 * together by persistent kernels: every CTA repeatedly claims the next problem
 * (largest first) from an atomic counter and runs all stages of that problem
 * itself, with the spectrum in its own scratch slot.  Sizes whose transforms
 * use radices <= 8 only and sizes that need the large-prime passes go to two
 * launches (one per group, each with its own counter): the first kernel needs
 * half the registers and runs two CTAs per SM.  Problem sizes share tables.  f and u of the solve calls are then the problems'
 * [n_theta][n_lambda] arrays packed back to back in problem order, problem b
 * starting at offsets[b] doubles (sphere_poisson_batch_offsets).
 *   precision   SP_FP64, or SP_FP32_REFINE (the arithmetic of the single-plan
 *               form, refine_sweeps 0..16 as there; SP_FP32 returns
 *               SP_ERR_UNSUPPORTED).
 *   flags       0, or SP_FLAG_AUTOTUNE: time the transform tiles (rows / columns
 *               per CTA pass) of every problem size at plan time and keep the
 *               fastest; results are cached in the file named by the
 *               environment variable SPHERE_POISSON_TUNE_CACHE if it is set.
 * count = 0 gives a plan whose solve does nothing.  The batched plan supports
 * sphere_poisson_solve (and _solve_host); the adjoint returns SP_ERR_UNSUPPORTED.
 * The solve issues one cudaMemsetAsync (the two work counters) and one kernel
 * per non-empty group (sphere_poisson_launch_count), and can be captured in a
 * CUDA graph as a whole.
 */
int sphere_poisson_plan_batched(sp_plan_t* plan, int count, const int* n_theta, const int* n_lambda,
                                int precision, int refine_sweeps, unsigned flags, size_t* workspace_bytes);

/* offsets[0..count]: start of problem b in the packed arrays (doubles); offsets[count] = total. */
int sphere_poisson_batch_offsets(sp_plan_t plan, size_t* offsets);

/* Device workspace size of a plan (bytes). */
int sphere_poisson_workspace_size(sp_plan_t plan, size_t* workspace_bytes);

/*
 * u = S f: the zero-mean solution of Delta u = f on the plan's grid.
 *   f          device, [n_theta][n_lambda] doubles, read only.  The paper assumes
 *              int_S f = 0 (Section 5, the problem statement of eq.
 *              SphericalLaplacian and eq. integralConstraint2); for other f the
 *              k = 0, j = 0 equation is dropped as in eq. pentdiagonalPlusRankOne
 *              and u solves the remaining equations.
 *   u          device, [n_theta][n_lambda] doubles, written.
 *   workspace  device, >= workspace_bytes; contents are scratch.
 *   stream     cudaStream_t (as void*) or NULL.
 *   f_mean_out optional DEVICE pointer (8-byte aligned) or NULL: receives the
 *              mean of f over the sphere, (1/4 pi) int_S f, by the quadrature of
 *              eq. integrationCoeffs on the grid (the w-weights applied to the
 *              colatitude coefficients of the lambda mean of f, theta-Nyquist
 *              mode dropped; the value sphere_poisson_sum2 gives, divided by 4 pi).
 *              Written asynchronously on `stream` by two extra kernels that read
 *              f once before the solve; nothing is synchronised, so the call stays
 *              capturable in a CUDA graph.  A caller compares it with its own
 *              scale of f (sphere_poisson_solve_host does that check itself).
 *              Single plans only (batched plans: SP_ERR_UNSUPPORTED).
 * Errors: SP_ERR_BAD_ARG when the current device is not the plan's device.
 */
int sphere_poisson_solve(sp_plan_t plan, const double* f, double* u, void* workspace,
                         size_t workspace_bytes, void* stream, double* f_mean_out);

/*
 * fbar = S^T ubar: the transpose of the linear map f -> u of sphere_poisson_solve
 * with respect to the plain Euclidean inner product on [n_theta][n_lambda]
 * arrays (the vector-Jacobian product of the solve).  Same layouts and rules.
 */
int sphere_poisson_solve_adjoint(sp_plan_t plan, const double* ubar, double* fbar,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Host-buffer convenience form of sphere_poisson_solve: copies f_host to the
 * device, solves, copies u back to u_host and synchronises before returning.
 * device_buffer must hold host_buffer_bytes (from sphere_poisson_host_buffer_size):
 * room for f, u and the workspace.  For single plans with n_theta >= 32 the grid
 * moves in 16 row chunks on a plan-owned copy stream, overlapped with the
 * longitude transforms (the forward transform of a chunk starts when its rows
 * have arrived; the rows of u return as the inverse transform finishes them),
 * and consecutive chunks' transforms alternate between `stream` and a second
 * plan-owned stream; calls on one plan from several host threads must be
 * serialised.  Pinned host memory gives the fastest copies; pageable memory
 * also works.
 *   f_mean_out optional HOST pointer or NULL: receives the mean of f over the
 *              sphere as in sphere_poisson_solve (computed on the device after
 *              the solve, with max |f| in the same pass), and the call then
 *              returns SP_WARN_NONZERO_MEAN (> 0: u is still written) when
 *              |mean| > 1e3 eps max |f|, eps = 2^-52: f is not mean-zero to
 *              rounding, so the dropped k = 0, j = 0 equation was not redundant.
 *              Single plans only (batched plans: SP_ERR_UNSUPPORTED).
 */
int sphere_poisson_host_buffer_size(sp_plan_t plan, size_t* device_buffer_bytes);
int sphere_poisson_solve_host(sp_plan_t plan, const double* f_host, double* u_host,
                              void* device_buffer, size_t device_buffer_bytes, void* stream,
                              double* f_mean_out);

/*
 * Allocation-free solve.  The paper has no counterpart; this is a service for
 * callers that cannot obtain device memory at the moment they need a solve:
 * code running where a cudaMalloc is not allowed or would stall the device
 * (a real-time loop, a host callback, a section holding a runtime lock),
 * programs whose device memory belongs to a framework allocator that forbids
 * raw allocations, or plug-ins that are handed only the input and output
 * buffers by their host application.  It computes exactly what
 * sphere_poisson_solve computes but takes no workspace and allocates nothing:
 * its scratch is one fixed device array inside the library of
 * SP_NOALLOC_SCRATCH_BYTES (32 MiB), which every GPU that loads the library
 * holds until the process exits.
 *   plan    an existing plan (creating the plan allocates its tables; do it at
 *           start-up), single or batched, of any precision.  Its workspace size
 *           (sphere_poisson_workspace_size) must not exceed SP_NOALLOC_SCRATCH_BYTES;
 *           larger plans get SP_ERR_SCRATCH_LIMIT and nothing runs.  For example
 *           an SP_FP64 plan needs n_theta * Kp * 16 bytes (Kp = n_lambda/2 + 1
 *           rounded up to even), so 1024 x 2048 fits and 2048 x 4096 does not; an
 *           SP_FP32_REFINE plan needs about 2.5 times that (two double-float
 *           spectra and an FP32 one), so 512 x 1024 fits and 1024 x 2048 does not.
 *   f, u    device arrays as for sphere_poisson_solve.
 *   stream  cudaStream_t (as void*) or NULL.
 * The current device must be the plan's device (else SP_ERR_BAD_ARG).  The first
 * call on each device looks up the device address of the scratch array
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call uses the same scratch array: calls that can overlap on the GPU
 * (different streams, or from several threads) race and corrupt each other's
 * results, so serialise them.  The scratch needs no clearing: the first kernel
 * of a solve overwrites the whole region before any kernel reads it.
 */
#define SP_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int sphere_poisson_solve_noalloc(sp_plan_t plan, const double* f, double* u, void* stream);

/*
 * The transforms on their own (Section 4, "Computation of Fourier coefficients",
 * eq. 2DFourierExpansion, and "Integration", eq. integrationCoeffs), on an
 * SP_FP64 single-grid plan.
 *
 * sphere_poisson_coeffs2: coefficients X_{j,k} of f~ (the DFS doubling of f) in
 *   f~(lambda, theta) = sum_{j,k} X_{j,k} e^{i j theta} e^{i k lambda},
 *   written to coeffs as [n_theta][Kp] complex doubles (re, im interleaved),
 *   Kp = n_lambda/2 + 1 rounded up to even: row j = 0..n_theta-1, column
 *   k = 0..n_lambda/2, the last one holding k = -n_lambda/2; the pad column is
 *   unspecified.  The other coefficients follow from the BMC symmetry
 *   X_{-j,k} = (-1)^k X_{j,k} and from f being real, X_{j,-k} = (-1)^k conj X_{j,k};
 *   the theta-Nyquist mode j = -n_theta is not represented.  Uses the workspace.
 * sphere_poisson_sample: the inverse, values of the expansion on the grid
 *   from coefficients in that layout (which must have the BMC symmetry a
 *   function on the sphere has: k odd columns with X_{0,k} = 0).
 * sphere_poisson_sum2: the surface integral of f over the unit sphere,
 *   2 pi sum_j w_j X_{j,0}, written as one double to device memory `result`.
 * All three are asynchronous on `stream`; coeffs and result are device pointers.
 */
int sphere_poisson_coeffs2(sp_plan_t plan, const double* f, void* coeffs, void* workspace,
                           size_t workspace_bytes, void* stream);
int sphere_poisson_sample(sp_plan_t plan, const void* coeffs, double* f, void* workspace,
                          size_t workspace_bytes, void* stream);
int sphere_poisson_sum2(sp_plan_t plan, const double* f, double* result, void* workspace,
                        size_t workspace_bytes, void* stream);

/*
 * Tangential derivatives (Section 4, Differentiation; eqs. diff_x, diff_y,
 * diff_z, dfdx, Msin): the Cartesian components of the surface gradient of f,
 *   gx = d^t f/dx = -(sin lambda / sin theta) df/dlambda + cos lambda cos theta df/dtheta,
 *   gy = d^t f/dy =  (cos lambda / sin theta) df/dlambda + sin lambda cos theta df/dtheta,
 *   gz = d^t f/dz = -sin theta df/dtheta,
 * computed on the coefficients of coeffs2 (the maps of Section 4: multiplication
 * by cos / sin of either angle shifts the index by one, d/dtheta and d/dlambda
 * multiply by ij and ik) with the division by sin theta done as M_sin^{-1}
 * (eq. Msin) on the m-point coefficient window j in [-m/2, m/2-1].  Only the
 * folded half j >= 0 of the quotient is formed, whose symmetry a quotient by
 * sin theta of a function on the sphere has: odd-k columns by the recurrence of
 * M_sin x = a run down from the top of the window, even-k columns (x_0 = 0) run
 * up from row 0.  That is the part of the window solve with this symmetry, and
 * the rest of the window solve does not reach the samples on theta > 0, so the
 * results are those of the dense solve for every f.  The sign of gz is the
 * chain rule's for the colatitude theta of eq. sphericalCoordinates (the paper
 * prints +sin theta d/dtheta).  The theta- and lambda-Nyquist modes are dropped
 * from f and from the results.  Exact (to rounding) for f band-limited within
 * the grid's window; for other f the results carry the window's truncation.
 *   f, gx, gy, gz  device, [n_theta][n_lambda] doubles, 16-byte aligned.
 *   workspace      device, >= sphere_poisson_gradient_workspace_size bytes
 *                  (five half spectra of n_theta Kp 16 bytes, Kp = n_lambda/2 + 1
 *                  rounded up to even, plus 2 ceil(n_theta/64) Kp 16 bytes of
 *                  chunk sums for the division and 256 bytes).
 * FP64 single plans only (others: SP_ERR_UNSUPPORTED).  Asynchronous on stream;
 * 12 kernel launches: the two of coeffs2, three for the division, one forming the
 * three components' coefficients, then per component the two inverse transforms
 * (two more with the chop of sphere_poisson_set_chop).
 */
int sphere_poisson_gradient_workspace_size(sp_plan_t plan, size_t* workspace_bytes);
int sphere_poisson_tangential_gradient(sp_plan_t plan, const double* f, double* gx, double* gy, double* gz,
                                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * Vector calculus (Section 4, vector-valued functions), built on the tangential
 * derivatives above; a vector field is three Cartesian components on the grid.
 *   sphere_poisson_divergence:  div = d^t f1/dx + d^t f2/dy + d^t f3/dz.
 *   sphere_poisson_curl:        (c1, c2, c3) = (d^t f3/dy - d^t f2/dz,
 *                               d^t f1/dz - d^t f3/dx, d^t f2/dx - d^t f1/dy).
 *                               For a tangent field the normal part n . c is the
 *                               vorticity, so c is tangent only where that is zero
 *                               (the solid rotation (-y, x, 0) has c = (xz, yz, 1 + z^2)).
 *   sphere_poisson_scalar_curl: the curl of a scalar function f (eq. CurlScalarF),
 *                               n x grad f = (y gz - z gy, z gx - x gz, x gy - y gx)
 *                               with n = (x, y, z) of eq. sphericalCoordinates.
 *   sphere_poisson_vorticity:   zeta = (curl f) . n.
 * The sums of derivative terms are formed in coefficient space (one inverse
 * transform per output); the products with n are taken pointwise on the grid.
 * The formulas are applied as printed whether or not the field is tangent.
 *   f1, f2, f3, f, outputs  device, [n_theta][n_lambda] doubles, 16-byte aligned;
 *                           outputs must not overlap the inputs.
 *   workspace  >= sphere_poisson_curl_workspace_size bytes, the same size as the
 *              gradient's (five half spectra plus the division's scratch); the
 *              divergence uses the first three spectra and accepts a workspace
 *              two spectra (2 n_theta Kp 16 bytes) smaller.
 * FP64 single plans only (others: SP_ERR_UNSUPPORTED); asynchronous on stream.
 * Accuracy as for the gradient: exact to rounding for band-limited inputs, with
 * the rounding of the x and y derivative terms amplified up to ~k_max m/pi by
 * the division by sin theta.
 */
int sphere_poisson_curl_workspace_size(sp_plan_t plan, size_t* workspace_bytes);
/*
 * Optional truncation of the derivative operators' inputs (tangential_gradient,
 * divergence, curl, scalar_curl, vorticity): after each input's forward
 * transform, the coefficients with |X_jk| <= rtol max |X| are set to zero, the
 * grid counterpart of building a function to machine precision relative to its
 * maximum (Section 3) and discarding the rest.  Without it the rounding noise in
 * modes a band-limited input does not have is amplified by the division by
 * sin theta, which matters when derivatives are chained (the vorticity of the
 * curl of a degree-5 function at 5000 x 10000: 3e-3 off, 4e-15 with rtol = 1e-14).  rtol in [0, 1); 0 (the
 * default) is off.  A plain field of the plan: set it before enqueuing calls.
 * Errors: SP_ERR_BAD_PLAN, SP_ERR_BAD_ARG (rtol negative, >= 1 or NaN).
 */
int sphere_poisson_set_chop(sp_plan_t plan, double rtol);
int sphere_poisson_divergence(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* div,
                              void* workspace, size_t workspace_bytes, void* stream);
int sphere_poisson_curl(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* c1,
                        double* c2, double* c3, void* workspace, size_t workspace_bytes, void* stream);
int sphere_poisson_scalar_curl(sp_plan_t plan, const double* f, double* c1, double* c2, double* c3,
                               void* workspace, size_t workspace_bytes, void* stream);
int sphere_poisson_vorticity(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* zeta,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * Low-rank form (Section 3, Figure GaussianElimination; Section 4, low-rank
 * form of eq. 2DFourierExpansion).  A term t is
 *   [c_t(theta) c_t(-theta)] [[P00, P01], [P01, P00]] [r_t(lambda); r_t(lambda + pi)]
 * with c_t sampled on the full DFS colatitude grid theta_p = -pi + (p + 1/2) pi / n_theta,
 * p < m = 2 n_theta (cols[t][p]), r_t on the longitudes (rows[t][q], q < n_lambda) and
 * the centrosymmetric pivot pseudoinverse in piv[t][0..1]; such terms are BMC
 * (eq. BMCsphere), so their sum is a function on the sphere.
 *
 * sphere_poisson_lowrank_ge: the structure-preserving GE of f (device [n_theta][n_lambda]):
 *   step k takes the grid point (lambda*, theta*) in [0, pi) x (0, pi) whose pivot
 *   matrix [[e(lambda* - pi, theta*), e(lambda*, theta*)], [e(lambda*, theta*), e(lambda* - pi, theta*)]]
 *   has the largest sigma_1 (eq. SingularValues; the smallest grid index among
 *   ties), its epsilon-pseudoinverse with eps = alpha sigma_1 (Definition
 *   pseudoinverse; the paper uses alpha = 1/100), and subtracts the term
 *   (eq. GEstructurePreservingStepPseudoinverse).  Stops when max |e| <= rtol max |f|,
 *   when the residual, below 1e-9 max |f|, has not decreased for three steps, or
 *   after max_terms (0..n_theta) steps; *terms receives the count.  cols, rows,
 *   piv: device arrays of max_terms x m, max_terms x n_lambda, max_terms x 2 doubles.
 *   Synchronous: the host reads each step's pivot.
 * sphere_poisson_solve_lowrank: u = S f for f = the sum of `terms` terms, with the
 *   right-hand side F formed from the factors (one colatitude transform per term
 *   column, one longitude transform per term row, one outer-product kernel)
 *   instead of the 2D transform of f; then the eliminations and inverse
 *   transforms of sphere_poisson_solve.  u device [n_theta][n_lambda].
 * Workspace of either call: sphere_poisson_lowrank_workspace_size(plan, max_terms).
 * FP64 single plans only (others SP_ERR_UNSUPPORTED); terms and max_terms
 * at most min(n_theta, 1024) (SP_ERR_BAD_ARG).
 */
int sphere_poisson_lowrank_workspace_size(sp_plan_t plan, int max_terms, size_t* workspace_bytes);
int sphere_poisson_lowrank_ge(sp_plan_t plan, const double* f, int max_terms, double rtol, double alpha,
                              int* terms, double* cols, double* piv, double* rows, void* workspace,
                              size_t workspace_bytes, void* stream);
int sphere_poisson_solve_lowrank(sp_plan_t plan, int terms, const double* cols, const double* piv,
                                 const double* rows, double* u, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Number of kernel launches one solve (adjoint = 1) issues for this plan. */
int sphere_poisson_launch_count(sp_plan_t plan, int adjoint, int* launches);

/*
 * Stage timing.  After profile_begin, each solve / adjoint call on the plan (up
 * to max_solves of them) records a CUDA event before each of its kernel
 * launches and one after the last, on the call's stream.  profile_end waits for
 * those events, writes the summed milliseconds of stage s over the recorded
 * calls to stage_ms[s] (s < max_stages), the number of recorded calls to
 * *solves and the number of stages per call to *stages, and releases the events.
 * Stage names: sphere_poisson_stage_name.  Host-side bookkeeping only.
 */
int sphere_poisson_profile_begin(sp_plan_t plan, int max_solves);
int sphere_poisson_profile_end(sp_plan_t plan, double* stage_ms, int max_stages, int* solves, int* stages);
const char* sphere_poisson_stage_name(sp_plan_t plan, int stage);

/*
 * Diagnostic, not part of the solve: measured FMA issue rates of the current
 * GPU in G instructions/s (FP64 and FP32 pipes, register-only loops filling
 * every SM, about 50 ms).  Used as the denominator of the ALU roofline of the
 * transform kernels, which this GPU's FP64 rate bounds.  The paper has no
 * counterpart.  Synchronous.
 */
int sphere_poisson_pipe_rates(double* fp64_fma_gops, double* fp32_fma_gops);

/* Release the plan and its device tables.  Synchronous; NULL is accepted. */
int sphere_poisson_destroy(sp_plan_t plan);

/*
 * Status of a plan's kernels that wait on asynchronous copies.  The SP_FP32_REFINE
 * form's fused colatitude stage has the tensor memory accelerator (TMA) copy
 * the next column into shared memory and waits for the copy on an mbarrier;
 * that wait polls a bounded number of times, and if the copy never lands the
 * kernel stops and sets the plan's device status word instead of hanging (the
 * results of that solve are then not valid).  Synchronises `stream` (the
 * stream the solves ran on, as void*, or NULL), reads the status word and
 * clears it: SP_OK, or SP_ERR_TIMEOUT if a wait gave up since the last check.
 * sphere_poisson_solve_host makes the same check before it returns.  Not part
 * of the paper's method: the bookkeeping of this implementation's copies.
 */
int sphere_poisson_device_status(sp_plan_t plan, void* stream);

/*
 * Diagnostic of that mechanism: launches, on `stream`, one thread that waits
 * `polls` polls on an mbarrier nothing completes and then sets the plan's
 * status word as a timed-out copy wait would.  The next
 * sphere_poisson_device_status returns SP_ERR_TIMEOUT.  SP_ERR_UNSUPPORTED on a
 * batched plan.
 */
int sphere_poisson_wait_selftest(sp_plan_t plan, unsigned polls, void* stream);

/* Static message for a status code (the last CUDA error text for SP_ERR_CUDA). */
const char* sphere_poisson_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SPHERE_POISSON_H */
