/*
 * dse.h -- C ABI of the GB300 (sm_103a) solver for the Landau-gauge ghost-gluon
 * Dyson-Schwinger system of Hopfer, Alkofer and Haase, "Solving the Ghost-Gluon
 * System of Yang-Mills Theory on GPUs" (arXiv:1206.1779).
 *
 * The ghost and gluon dressing functions G(x), Z(x) are expanded as
 *   ln G(x) = b_0/2 + sum_{j>=1} b_j T_j(s(x)),   ln Z(x) = a_0/2 + sum_{j>=1} a_j T_j(s(x))
 * in the mapped variable s(x) = log(x/(Lambda eps)) / log(Lambda/eps)  (Sec. 3),
 * with N_Z coefficients a_j and N_G coefficients b_j (N_G = N_Z unless
 * n_cheb_G says otherwise).  The unknown vector is
 * c = (a_0 .. a_{N_Z-1}, b_0 .. b_{N_G-1})  (n = N_Z + N_G doubles).
 * The residual F has the rows  z(x_0..x_{N_Z-1})  at the N_Z mapped Chebyshev
 * roots of T_{N_Z}, then  g(x_0..x_{N_G-1})  at the roots of T_{N_G} (Sec. 3,
 * residual equations; one shared set of points when N_Z = N_G), with
 *   z(x) = Z(x)^{-1} - Z(x_Z)^{-1} - Pi_Z(x) + Pi_Z(x_Z)
 *   g(x) = G(x)^{-1} - G(x_G)^{-1} - Pi_G(x) + Pi_G(x_G)
 * and the self-energies of the ghost and gluon equations of Sec. 2 (bare
 * ghost-gluon vertex, three-gluon vertex model with a = b = 3 delta, kernels M and
 * Q including the +15/4 term, O(4) reduction with a sharp cutoff).  Every
 * integral is a radial Gauss-Legendre rule in ln y over [eps2, lambda2] (or the
 * paper's split of the radial range at x, radial_mode 1) times an angular rule in
 * theta over [0, pi] (Gauss-Legendre, or the paper's tanh-sinh rule in cos theta,
 * angular_mode 1); outside [eps2, lambda2] the dressing functions follow the IR
 * power laws and UV logarithms of Sec. 2.
 *
 * Conventions for every entry point
 *  - Pointers prefixed d_ are CUDA device pointers (FP64, contiguous), owned by
 *    the caller, that must stay valid until the work queued on the plan's stream
 *    has finished.  Pointers prefixed h_ are host pointers.
 *  - All work is queued on the plan's CUDA stream.  dse_residual,
 *    dse_newton_matrix, dse_dressing, dse_quadrature and dse_schwinger return
 *    without waiting; dse_newton_step, dse_solve and dse_plan_status wait for the
 *    stream.
 *  - Every call returns DSE_OK (0) or a negative status (below); nothing is
 *    printed and no C++ exception crosses the ABI.  Argument errors are detected
 *    before any work is queued.  A non-finite value produced on the device sets a
 *    sticky flag that the next synchronising call reports (DSE_ERR_NONFINITE).
 *  - The plan owns its device workspace (allocated once in dse_plan_create) and
 *    is not thread-safe: calls on one plan must not overlap.
 */
#ifndef DSE_H
#define DSE_H

#ifdef __cplusplus
extern "C" {
#endif

#define DSE_OK 0
#define DSE_ERR_ARG (-1)           /* bad size, null pointer or parameter       */
#define DSE_ERR_NONFINITE (-2)     /* NaN/Inf in F, J or the Newton update      */
#define DSE_ERR_SINGULAR (-3)      /* LU pivot below 1e-300 or not finite       */
#define DSE_ERR_CUDA (-4)          /* a CUDA runtime call failed                */
#define DSE_ERR_UNSUPPORTED (-5)   /* mode not implemented in this library      */
#define DSE_ERR_NOT_CONVERGED (-6) /* dse_solve reached max_iter                */

/* Limits of this build. */
#define DSE_MAX_CHEB 256           /* N_Z, N_G per dressing function            */
#define DSE_MAX_NODES 65536        /* n_radial, n_angular                       */
#define DSE_MAX_SCHWINGER_NODES (1 << 20)

/* Problem definition (Sec. 2.1 and Sec. 3 of the paper give the values used
 * there: g2nc = 12 pi (alpha(mu^2) = 1, N_c = 3), x_Z = lambda2, Z(x_Z) = 0.256,
 * x_G = 0, ginv_G = 0 for the scaling solution, delta = -9/44, kappa ~ 0.595353). */
typedef struct {
    int n_cheb;       /* N_Z Chebyshev coefficients of ln Z, 1..DSE_MAX_CHEB              */
    int n_radial;     /* radial Gauss-Legendre nodes in ln y (per piece in radial_mode 1) */
    int n_angular;    /* angular nodes                                                   */
    double eps2;      /* IR matching point epsilon^2 (> 0)                               */
    double lambda2;   /* UV cutoff Lambda^2 (> eps2)                                     */
    double g2nc;      /* g^2 N_c; the equations carry K = g2nc/(2 pi)^3                  */
    double x_G;       /* ghost subtraction point (>= 0)                                  */
    double ginv_G;    /* G(x_G)^{-1}                                                     */
    double x_Z;       /* gluon subtraction point (> 0)                                   */
    double zinv_Z;    /* Z(x_Z)^{-1}                                                     */
    double kappa;     /* IR exponent: Z ~ x^{2 kappa}, G ~ x^{-kappa} below eps2         */
    double delta;     /* ghost anomalous dimension; gamma = -1 - 2 delta                 */
    int radial_mode;  /* 0: one Gauss-Legendre rule in ln y over [eps2, lambda2];        *
                       * 1: the paper's split [0,eps2] + [eps2,x] + [x,lambda2] (Sec. 3), *
                       *    n_radial nodes in ln y per piece, the first piece over        *
                       *    [1e-6 eps2, eps2]; every external momentum has its own rule   */
    int extrap_mode;  /* 0: IR power laws and UV logarithms; 1: constant continuation    */
    int precision;    /* 0: FP64 throughout; 1: mixed (FP32 integrands for J, FP64 F)   */
    int n_cheb_G;     /* N_G Chebyshev coefficients of ln G, 0..DSE_MAX_CHEB (0: N_Z)    */
    int angular_mode; /* 0: Gauss-Legendre in theta; 1: the paper's tanh-sinh rule in    *
                       *    xi = cos theta (Sec. 2): xi = tanh((pi/2) sinh t), trapezoidal *
                       *    in t with n_angular points over |t| <= 4                       */
} dse_problem;

typedef struct dse_plan dse_plan;

/* Create a plan: validates the problem, allocates the device workspace and runs
 * the set-up kernels (Gauss-Legendre nodes and weights by Newton iteration on the
 * Legendre recurrence, mapped radial/angular rules, collocation points; Sec. 2,
 * Sec. 3, Sec. 4.2).  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  Waits for the set-up kernels.  On failure *out is NULL. */
int dse_plan_create(const dse_problem* problem, void* cuda_stream, dse_plan** out);

/* Release the plan and its workspace (waits for its stream).  NULL is accepted. */
int dse_plan_destroy(dse_plan* plan);

/* Queue later calls on another stream. */
int dse_plan_set_stream(dse_plan* plan, void* cuda_stream);

/* Wait for the plan's stream and report the sticky device status
 * (DSE_OK, DSE_ERR_NONFINITE or DSE_ERR_SINGULAR); the flag is cleared. */
int dse_plan_status(dse_plan* plan);

/* Copy the plan's rules: d_y, d_W (n_radial; int_{eps2}^{lambda2} dy f ~ sum W_k f(y_k);
 * radial_mode 1: the 3 n_radial nodes of the x_Z row),
 * d_theta, d_wt (n_angular; int_0^pi dtheta g ~ sum w_l g(theta_l)), d_x
 * (the collocation points: N_Z ascending points shared by both equations when
 * N_Z = N_G, otherwise the N_Z gluon points followed by the N_G ghost points).
 * Any pointer may be NULL. */
int dse_quadrature(dse_plan* plan, double* d_y, double* d_W, double* d_theta, double* d_wt,
                   double* d_x);

/* ln G(x_m), ln Z(x_m) for m < n (Sec. 3 expansion; Sec. 2 IR/UV forms outside
 * [eps2, lambda2]).  d_coeffs: N_Z + N_G; d_x: n positive momenta; outputs n each. */
int dse_dressing(dse_plan* plan, const double* d_coeffs, int n, const double* d_x,
                 double* d_lnG, double* d_lnZ);

/* Residual F (N_Z + N_G): z at the N_Z gluon points, then g at the N_G ghost
 * points (Sec. 3, residual equations). */
int dse_residual(dse_plan* plan, const double* d_coeffs, double* d_F);

/* Newton matrix J (n x n with n = N_Z + N_G, row-major; rows z then g, columns a then b, the
 * layout of Sec. 3) with every entry dF_i/dc_j an analytic radial x angular
 * quadrature, and the residual F (d_F may be NULL). */
int dse_newton_matrix(dse_plan* plan, const double* d_coeffs, double* d_J, double* d_F);

/* The paper's Newton matrix (Sec. 4.2, central differences of the residual):
 *   J[:, j] = (F(c + h_j e_j) - F(c - h_j e_j)) / ((c_j + h_j) - (c_j - h_j)),
 *   h_j = rel_step * max(|c_j|, 1e-3)   (the paper uses about 1e-5 a_j),
 * with the 2n perturbed residuals evaluated together as a batch (one persistent
 * quadrature launch).  For comparisons with the analytic dse_newton_matrix, which
 * the Newton steps use.  d_F (nullable) receives F(c).  The first call allocates
 * the batch (2n copies of the plan's workspace) and the plan keeps it until
 * dse_plan_destroy or dse_plan_set_couplings.  Queued without waiting. */
int dse_newton_matrix_fd(dse_plan* plan, const double* d_coeffs, double rel_step, double* d_J, double* d_F);

/* One Newton-Raphson step (Sec. 3): J Delta = F solved on the device, then
 * c <- c - rho Delta in place.  For n <= 160 the rows of J are scaled by powers
 * of two, inverted in FP32 and the solution refined in FP64 to a backward-stable
 * residual; otherwise (or if refinement stalls) LU with partial pivoting in FP64.
 * h_stats (host, 4 doubles, nullable): ||F||_inf, ||diag(Z(x_i), G(x_i)) F||_inf
 * (the dimensionless residual used as the stopping test), ||Delta||_inf, all for
 * the coefficients on entry, and the number of FP64 refinement sweeps (-1 when
 * the FP64 LU solved the system).  For n <= 128 the FP32 inverse of the last
 * eliminated step is kept and tried first (a few refinement sweeps; the
 * elimination runs only if they do not converge): dse_plan_solver_counters.
 * Waits for the stream.  On DSE_ERR_SINGULAR / DSE_ERR_NONFINITE the
 * coefficients are left unchanged. */
int dse_newton_step(dse_plan* plan, double* d_coeffs, double rho, double* h_stats);

/* Newton iteration from d_coeffs until the dimensionless residual (h_stats[1]
 * of dse_newton_step) drops below tol: the first n_relax steps use rho_relax,
 * the rest rho = 1 (under-relaxation of Sec. 3).  *h_iters receives the number
 * of steps taken, h_stats (nullable, 3 doubles) the first three stats of the
 * last step.  Returns
 * DSE_ERR_NOT_CONVERGED after max_iter steps. */
int dse_solve(dse_plan* plan, double* d_coeffs, double tol, int max_iter, double rho_relax,
              int n_relax, int* h_iters, double* h_stats);

/* Gluon Schwinger function (Sec. 2.2):
 *   Delta(t_m) = (1/pi) int_0^inf d|p| cos(t_m |p|) Z(p^2)/p^2,
 * with n_nodes Gauss-Legendre nodes in u = ln p^2 over [ln eps2, ln lambda2]
 * (tails outside the range are left out).  The nodes for a given n_nodes are
 * generated on the device on first use and kept in the plan.  cos(t p) is taken
 * at the FP64 product t p to a few units in the last place for any finite t p;
 * weights Z/(pi p^2) of any FP64 magnitude.  A non-finite Delta sets the
 * sticky DSE_ERR_NONFINITE flag (dse_plan_status). */
int dse_schwinger(dse_plan* plan, const double* d_coeffs, const double* d_t, int n_t,
                  int n_nodes, double* d_delta);

/* ---- Differentiation --------------------------------------------------------
 * The residual F(c; g2nc, ginv_G, zinv_Z) of Sec. 3 as a function of the
 * coefficients and of the coupling g^2 Nc and the two renormalisation
 * (boundary) values G(x_G)^{-1}, Z(x_Z)^{-1} of Sec. 2.2.  All derivatives are
 * FP64 whatever the plan's precision.  All calls are queued on the plan's
 * stream without waiting, except dse_adjoint_solve. */

/* Replace g2nc, ginv_G and zinv_Z of the plan's problem (the quadrature rules
 * and workspace are kept).  Same argument checks as dse_plan_create. */
int dse_plan_set_couplings(dse_plan* plan, double g2nc, double ginv_G, double zinv_Z);

/* Vector-Jacobian product out_j = sum_i v_i dF_i/dc_j (n each).  The products
 * are contracted from the per-external-momentum derivative sums of Sec. 3
 * without forming the n x n Newton matrix; d_F (nullable) receives F(c). */
int dse_vjp(dse_plan* plan, const double* d_coeffs, const double* d_v, double* d_out, double* d_F);

/* Parameter derivatives of F.  d_dF (nullable): n x 3 row-major, columns
 * dF/d g2nc, dF/d ginv_G, dF/d zinv_Z.  g2nc enters through the prefactor
 * g^2 Nc/(2 pi)^3 of both self-energies and through omega = 11 g^2 Nc/(48 pi^2)
 * of the UV forms of G(z), Z(z) for z > lambda2 (Sec. 2); the boundary values
 * enter the subtracted rows with coefficient -1.  d_v (nullable, n) with d_vdF
 * (3): v^T dF.  At least one of d_dF, d_v.  DSE_ERR_ARG if g2nc = 0. */
int dse_param_derivatives(dse_plan* plan, const double* d_coeffs, double* d_dF, const double* d_v,
                          double* d_vdF);

/* Adjoint of the Newton system at c: solves J(c)^T lambda = g (n each; J the
 * FP64 Newton matrix of dse_newton_matrix).  The rows of J are first scaled by
 * exact powers of two (S), and (S J)^T mu = g is solved with the dense solver of
 * dse_newton_step; lambda = S mu.  For the implicit function c*(theta) defined
 * by F(c*, theta) = 0, dL/dtheta = -lambda^T dF/dtheta with g = dL/dc*.
 * h_stats (nullable, 4): ||g||_inf, unused, ||lambda||_inf, refinement sweeps
 * (-1: FP64 LU).  Waits for the stream. */
int dse_adjoint_solve(dse_plan* plan, const double* d_coeffs, const double* d_g, double* d_lambda,
                      double* h_stats);

/* Vector-Jacobian product of dse_dressing at n points x (positive):
 *   d_out[j] = sum_m gZ_m d ln Z(x_m)/d a_j (j < N_Z),  d_out[N_Z + j] = sum_m gG_m d ln G(x_m)/d b_j,
 * i.e. sums of the basis phi_j(x_m) (s clamped to [-1, 1] outside [eps2, lambda2]);
 * d_out_g2nc (nullable, 1 double): sum_m gG_m d ln G/d g2nc + gZ_m d ln Z/d g2nc,
 * non-zero only through the UV form for x_m > lambda2.  Non-positive x flag
 * DSE_ERR_NONFINITE in the plan status. */
int dse_dressing_vjp(dse_plan* plan, int n, const double* d_x, const double* d_gG, const double* d_gZ,
                     double* d_out, double* d_out_g2nc);

/* ---- Batches of independent problems ------------------------------------------
 * A parameter sweep: n_problems problems, each with its own orders N_Z, N_G,
 * quadrature sizes and parameters (precision 0, N_Z + N_G <= 128 each).  Their
 * coefficient vectors are concatenated in problem order; dse_batch_offsets
 * gives the offsets (n_problems + 1 entries; problem b owns
 * [off[b], off[b+1]) = N_Z + N_G doubles, the same for F) and the offsets of
 * the concatenated Newton matrices (n_b^2 each).  One Newton step of the whole
 * batch is a CUDA graph of seven launches, the quadrature of all problems in one
 * persistent kernel that takes (problem, external momentum, radial block) work
 * items longest first from a device counter; the radial nodes per work item
 * come from dse_batch_tune.  The paper solves one problem at a time; the batch
 * is its Newton method (Sec. 3) applied to many problems at once. */
typedef struct dse_batch dse_batch;

/* Create the batch (workspace for every problem, rules and collocation points
 * set up on the device; waits for the set-up).  DSE_ERR_UNSUPPORTED for
 * N_Z + N_G > 128, precision != 0 or an unsupported mode.  Both quadrature
 * variants (radial_mode, angular_mode) are supported. */
int dse_batch_create(const dse_problem* problems, int n_problems, void* cuda_stream, dse_batch** out);
int dse_batch_destroy(dse_batch* batch);
int dse_batch_set_stream(dse_batch* batch, void* cuda_stream);

/* h_offsets (nullable): n_problems + 1 coefficient offsets; h_matrix_offsets
 * (nullable): n_problems + 1 offsets of the concatenated Newton matrices. */
int dse_batch_offsets(const dse_batch* batch, long long* h_offsets, long long* h_matrix_offsets);

/* Time the quadrature pass for 8, 16, 32, 64 and 128 radial nodes per work
 * item at d_coeffs and keep the fastest.  h_units (nullable): the choice;
 * h_ms (nullable, 5 doubles): the time of each candidate.  Waits. */
int dse_batch_tune(dse_batch* batch, const double* d_coeffs, int* h_units, double* h_ms);

/* Residuals of every problem at d_coeffs into the concatenated d_F (coefficient
 * offsets).  Queued without waiting. */
int dse_batch_residual(dse_batch* batch, const double* d_coeffs, double* d_F);

/* Newton matrices and residuals of every problem at d_coeffs into the
 * concatenated d_J (matrix offsets) and d_F (coefficient offsets; nullable).
 * Queued without waiting. */
int dse_batch_newton_matrix(dse_batch* batch, const double* d_coeffs, double* d_J, double* d_F);

/* Newton iteration of every problem from d_coeffs (in place), as dse_solve:
 * rho_relax for the first n_relax steps, stop when the dimensionless residual
 * drops below tol.  Converged problems leave the iteration (their work items
 * are skipped); the loop ends when none is left or after max_iter steps.
 * Per problem (nullable): h_iters steps taken, h_status DSE_OK /
 * DSE_ERR_NOT_CONVERGED / DSE_ERR_SINGULAR / DSE_ERR_NONFINITE, h_stats three
 * doubles of the last step (as dse_solve).  Returns DSE_OK when every problem
 * converged, else DSE_ERR_NOT_CONVERGED.  Waits. */
int dse_batch_solve(dse_batch* batch, double* d_coeffs, double tol, int max_iter, double rho_relax,
                    int n_relax, int* h_iters, int* h_status, double* h_stats);

/* Kernels launched by the batch since creation, graph launches, and the radial
 * nodes per work item in use; any pointer may be NULL. */
int dse_batch_counters(dse_batch* batch, long long* h_launches, long long* h_graph_launches, int* h_units);

/* Allocation-free residual.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code that runs where device
 * memory is owned by another allocator (a framework's caching pool, a fixed
 * memory budget) or where the implicit device synchronisation of cudaMalloc /
 * cudaFree is not acceptable.  For radial_mode 0 and precision 0 it computes the
 * same F as dse_residual (Gauss-Legendre rules, dressing tables, quadrature
 * kernel, contraction, assembly; the dressing series summed per triple, without
 * the plan's series table), but needs no plan: every intermediate buffer is carved
 * out of one static device array of DSE_STATIC_SCRATCH_BYTES compiled into the
 * library, which every GPU that loads the library holds until the process exits.
 *  - d_coeffs (n) and d_F (n) are caller-owned device buffers; cuda_stream is
 *    a cudaStream_t (NULL = legacy default stream).  Queued without waiting.
 *  - Returns DSE_ERR_UNSUPPORTED for radial_mode != 0 or precision != 0,
 *    DSE_ERR_ARG for bad arguments and when the problem needs more than
 *    DSE_STATIC_SCRATCH_BYTES of scratch; nothing is queued then.  The largest
 *    part is the angular sums, (R_c + 2) x n_radial x ceil(n_angular/32) x 3
 *    doubles with R_c = N for N_Z = N_G and R_c = N_Z + N_G otherwise (about
 *    12 MB for N = 128 with 512 x 256 nodes; N_Z = 128, N_G = 96 at that size
 *    needs about 22 MB and is rejected).  Non-finite values are not reported:
 *    they appear in d_F.
 *  - It calls no cudaMalloc, cudaFree or other allocating routine.  Every call
 *    looks up the array's device address on the current device (a host-side
 *    lookup); the first call on a device also loads the library's device code
 *    there, so make that first call before any stream capture.
 *  - All calls share the one array and it keeps the previous call's contents:
 *    calls that overlap on the GPU (different streams, or different host
 *    threads on the same device) race on it and must be serialised by the
 *    caller. */
#define DSE_STATIC_SCRATCH_BYTES (16u << 20)
int dse_residual_static(const dse_problem* problem, const double* d_coeffs, double* d_F,
                        void* cuda_stream);

/* Instrumentation.  dse_plan_profile(plan, 1) makes every later assembly record
 * CUDA events around its quadrature kernel (the hot kernel) on the plan's
 * stream; dse_plan_counters waits for the stream and reports the number of
 * kernels this plan has launched since creation (h_launches), the number of
 * timed quadrature-kernel launches and their summed device time in ms since
 * profiling was enabled.  At most 4096 launches are timed per enable; any
 * pointer may be NULL. */
int dse_plan_profile(dse_plan* plan, int enable);
int dse_plan_counters(dse_plan* plan, long long* h_launches, int* h_timed, double* h_timed_ms);

/* How the plan's Newton steps with n <= 128 solved J Delta = F since creation:
 * h_eliminations counts steps that inverted their own row-scaled matrix
 * (Gauss-Jordan in FP32), h_reused the steps whose FP64 refinement converged
 * with the inverse kept from an earlier step of the same dse_solve (or of the
 * preceding dse_newton_step calls), so that no elimination ran.  Both solve to
 * the same backward-error bound.  Waits for the stream; either pointer may be NULL. */
int dse_plan_solver_counters(dse_plan* plan, int* h_eliminations, int* h_reused);

/* Human-readable name of a status code (static storage). */
const char* dse_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* DSE_H */
