/*
 * dse_oracle.h -- FP64 CPU oracle for the ghost-gluon Dyson-Schwinger system
 * (Hopfer, Alkofer, Haase, "Solving the Ghost-Gluon System of Yang-Mills Theory
 * on GPUs", arXiv:1206.1779).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links, includes or calls anything here, and this file shares no header,
 * table or helper with it.
 *
 * Every routine computes in IEEE double precision with plain loops, in the order
 * the paper states the method (Sec. 2 and Sec. 3), with Neumaier-compensated
 * sums for the quadratures.  All pointers are host pointers owned by the caller.
 * Every routine returns DSE_REF_OK (0) or a negative status; nothing is printed.
 *
 * Parity status of each routine: all routines are pinned by the tests under
 * tests/ (Gauss-Legendre exactness, Chebyshev identities, closed-form angular and
 * radial integrals, the paper's printed kernels in 60-digit arithmetic, the
 * Jacobian against central differences, Newton convergence and the infrared
 * exponents of the converged solution, the Schwinger transform of 1/(p^2+m^2)).
 */
#ifndef DSE_ORACLE_H
#define DSE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define DSE_REF_OK 0
#define DSE_REF_ERR_ARG (-1)
#define DSE_REF_ERR_NONFINITE (-2)
#define DSE_REF_ERR_SINGULAR (-3)
#define DSE_REF_ERR_UNSUPPORTED (-5)

/* Problem definition (same field order as the product's dse_problem, defined
 * independently here).  n_cheb = N_Z Chebyshev coefficients of ln Z, n_cheb_G =
 * N_G coefficients of ln G (0: N_G = N_Z); the unknown vector is
 * c = (a_0..a_{N_Z-1}, b_0..b_{N_G-1}) with a for ln Z (gluon) and b for ln G
 * (ghost), Sec. 3.  The gluon residual rows sit at the N_Z mapped roots of
 * T_{N_Z}, the ghost rows at the N_G roots of T_{N_G}. */
typedef struct {
    int n_cheb;
    int n_radial;
    int n_angular;
    double eps2;      /* IR matching point epsilon^2 (lower end of the expansion) */
    double lambda2;   /* UV cutoff Lambda^2 */
    double g2nc;      /* g^2 * N_c */
    double x_G;       /* ghost subtraction point */
    double ginv_G;    /* G(x_G)^{-1} */
    double x_Z;       /* gluon subtraction point */
    double zinv_Z;    /* Z(x_Z)^{-1} */
    double kappa;     /* IR exponent */
    double delta;     /* ghost anomalous dimension; gamma = -1 - 2 delta */
    int radial_mode;  /* 0: one Gauss-Legendre rule in ln y over [eps2, lambda2];
                         1: split at x with an infrared piece (3 n_radial nodes) */
    int extrap_mode;  /* 0: IR power laws / UV logarithms; 1: constant continuation */
    int precision;    /* 0: FP64 */
    int n_cheb_G;     /* N_G (0: equal to n_cheb) */
    int angular_mode; /* 0: Gauss-Legendre in theta; 1: tanh-sinh in xi = cos theta */
} dse_ref_problem;

/* n-point Gauss-Legendre rule on [-1,1], nodes ascending (Newton iteration on
 * the three-term Legendre recurrence). */
int dse_ref_gauss_legendre(int n, double* x, double* w);

/* Radial nodes y_k and weights W_k with  int dy f(y) ~ sum_k W_k f(y_k)
 * (Gauss-Legendre in t = ln y, Jacobian y included in W_k), and angular nodes
 * theta_l, weights w_l with int_0^pi dtheta g ~ sum_l w_l g(theta_l) (Gauss-Legendre
 * in theta, or the paper's tanh-sinh rule in xi = cos theta for angular_mode 1).
 * radial_mode 0: [eps2, lambda2], n_radial nodes; radial_mode 1: the rule of
 * dse_ref_radial_rule at x = lambda2 (3 n_radial nodes). */
int dse_ref_quadrature(const dse_ref_problem* p, double* y, double* W, double* theta, double* wt);

/* The radial rule used for external momentum x: radial_mode 0 as above; radial_mode
 * 1 the paper's split [0, eps2] + [eps2, x] + [x, lambda2] (Sec. 3), n_radial nodes
 * in ln y per piece, the first piece over [1e-6 eps2, eps2].  3 n_radial nodes. */
int dse_ref_radial_rule(const dse_ref_problem* p, double x, double* y, double* W);

/* Collocation points x_i, i < N_Z: the mapped roots of T_{N_Z}, ascending (Sec. 3);
 * the gluon rows of the residual.  _ghost: the N_G roots of T_{N_G} (ghost rows). */
int dse_ref_collocation(const dse_ref_problem* p, double* x);
int dse_ref_collocation_ghost(const dse_ref_problem* p, double* x);

/* Mapping s(x) = log(x/(Lambda eps)) / log(Lambda/eps) of Sec. 3 (unclamped). */
double dse_ref_map(const dse_ref_problem* p, double x);

/* phi_j(x) = d ln G(x) / d b_j = d ln Z(x) / d a_j for j < max(N_Z, N_G) (1/2 for
 * j = 0, T_j(s(x)) otherwise, x clamped into [eps2, lambda2]). */
int dse_ref_basis(const dse_ref_problem* p, double x, double* phi);

/* ln G(x_m), ln Z(x_m) for m < n from coefficients c (N_Z + N_G): Chebyshev series
 * inside [eps2, lambda2], the paper's IR/UV forms outside (Sec. 2, Sec. 3). */
int dse_ref_dressing(const dse_ref_problem* p, const double* c, int n, const double* x,
                     double* lnG, double* lnZ);

/* Kernels M(x,y,z), Q(x,y,z) of the gluon equation at z = x + y - 2 sqrt(xy) cos theta,
 * evaluated in cancellation-free forms algebraically equal to the printed ones. */
int dse_ref_kernels(double x, double y, double theta, double* M, double* Q, double* z);

/* Self-energies Pi_G(x), Pi_Z(x) (Pi_Z only for x > 0) and, if d_PiG / d_PiZ are
 * non-NULL, their gradients (N_Z + N_G each) with respect to c = (a, b). */
int dse_ref_self_energy(const dse_ref_problem* p, const double* c, double x,
                        double* PiG, double* PiZ, double* d_PiG, double* d_PiZ);

/* Residual F (n = N_Z + N_G): rows z at the N_Z gluon points, then g at the N_G ghost points, Sec. 3. */
int dse_ref_residual(const dse_ref_problem* p, const double* c, double* F);

/* Newton matrix J (n x n row-major, columns a then b) and residual F (nullable). */
int dse_ref_newton_matrix(const dse_ref_problem* p, const double* c, double* J, double* F);

/* Magnitude sums that bound the rounding of each entry: A_ij is the sum of the
 * absolute values of every summand that forms J_ij (the -Z^{-1} phi_j term, each
 * quadrature summand of the row and of the subtraction row), AF_i the same for
 * F_i (AF nullable).  Same layout as dse_ref_newton_matrix. */
int dse_ref_newton_matrix_magnitudes(const dse_ref_problem* p, const double* c, double* A, double* AF);

/* Derivatives of F (n rows) with respect to the parameters (g2nc, ginv_G, zinv_Z),
 * n x 3 row-major.  g2nc enters through K and through omega in the UV forms. */
int dse_ref_param_derivatives(const dse_ref_problem* p, const double* c, double* dF);

/* Solve A x = b (n x n row-major) by LU with partial pivoting. */
int dse_ref_lu_solve(int n, const double* A, const double* b, double* x);

/* One Newton-Raphson step c <- c - rho * J^{-1} F.  stats (nullable, 3 doubles):
 * ||F||_inf, ||diag(Z(x_i), G(x_i)) F||_inf, ||Delta||_inf, all before the update. */
int dse_ref_newton_step(const dse_ref_problem* p, double* c, double rho, double* stats);

/* Schwinger-function quadrature: n nodes p_n, weights w_n for int_0^inf d|p|,
 * Gauss-Legendre in u = ln p^2 over [ln eps2, ln lambda2]. */
int dse_ref_schwinger_nodes(const dse_ref_problem* p, int n, double* pn, double* wn);

/* Delta(t_m) = (1/pi) sum_n w_n cos(t_m p_n) Z(p_n^2)/p_n^2 for m < n_t (Sec. 2.2). */
int dse_ref_schwinger(const dse_ref_problem* p, const double* c, const double* t, int n_t,
                      int n_nodes, double* delta);

/* Number of OpenMP threads the row loops use. */
int dse_ref_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
