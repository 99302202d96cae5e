/*
 * dse_oracle.c -- FP64 CPU oracle for the ghost-gluon Dyson-Schwinger system of
 * arXiv:1206.1779.  TEST INFRASTRUCTURE ONLY (see dse_oracle.h): the product
 * library never links or calls this code.
 *
 * The code follows the paper's order:
 *   Sec. 2  O(4) reduction, radial/angular quadratures, ghost and gluon equations,
 *           kernels M and Q (with the +15/4 term), IR/UV asymptotic forms,
 *           MOM subtraction;
 *   Sec. 3  Chebyshev expansion of ln G, ln Z in the mapped variable s(x),
 *           collocation at the mapped Chebyshev roots, residuals g and z,
 *           Newton matrix (rows z then g, columns a then b) and the relaxed update;
 *   Sec. 2.2 Schwinger function.
 * Quadrature sums use Neumaier compensation; the order of every sum is fixed,
 * so results do not depend on the number of OpenMP threads.
 */
#include "dse_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- sums ---- */

typedef struct { double s, c; } nsum;

static void ns_add(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double ns_val(const nsum* a) { return a->s + a->c; }

/* -------------------------------------------------------- parameters ---- */

/* Derived constants of Sec. 2:  K = g^2 Nc/(2 pi)^3 (prefactor of both
 * equations), gamma = -1 - 2 delta, vertex exponents p = -2 - 6 delta on G and
 * q = -3 delta on Z (three-gluon vertex model with a = b = 3 delta),
 * omega = 11 Nc alpha / (12 pi) with alpha = g^2/(4 pi). */
typedef struct {
    int NZ, NG, N;            /* orders of ln Z and ln G; N = max(NZ, NG) */
    double K, gam, pG, qZ, omega;
    double L0, L1;            /* ln x = L0 + L1 s */
    double ln_eps2, ln_lam2;
} consts;

static int check_problem(const dse_ref_problem* p) {
    if (!p) return DSE_REF_ERR_ARG;
    if (p->n_cheb < 1 || p->n_cheb_G < 0 || p->n_radial < 1 || p->n_angular < 1) return DSE_REF_ERR_ARG;
    if (p->n_cheb > 1024 || p->n_cheb_G > 1024) return DSE_REF_ERR_ARG;
    if (!(p->eps2 > 0.0) || !(p->lambda2 > p->eps2)) return DSE_REF_ERR_ARG;
    if (!(p->x_Z > 0.0) || !(p->x_G >= 0.0)) return DSE_REF_ERR_ARG;
    if (!isfinite(p->g2nc) || !isfinite(p->kappa) || !isfinite(p->delta)) return DSE_REF_ERR_ARG;
    if ((p->radial_mode != 0 && p->radial_mode != 1) || p->precision != 0) return DSE_REF_ERR_UNSUPPORTED;
    if (p->angular_mode != 0 && p->angular_mode != 1) return DSE_REF_ERR_UNSUPPORTED;
    if (p->extrap_mode != 0 && p->extrap_mode != 1) return DSE_REF_ERR_UNSUPPORTED;
    return DSE_REF_OK;
}

static consts make_consts(const dse_ref_problem* p) {
    consts k;
    k.NZ = p->n_cheb;
    k.NG = p->n_cheb_G > 0 ? p->n_cheb_G : p->n_cheb;
    k.N = k.NZ > k.NG ? k.NZ : k.NG;
    k.K = p->g2nc / (8.0 * PI_D * PI_D * PI_D);
    k.gam = -1.0 - 2.0 * p->delta;
    k.pG = -2.0 - 6.0 * p->delta;
    k.qZ = -3.0 * p->delta;
    k.omega = 11.0 * p->g2nc / (48.0 * PI_D * PI_D);
    k.ln_eps2 = log(p->eps2);
    k.ln_lam2 = log(p->lambda2);
    k.L0 = 0.5 * (k.ln_eps2 + k.ln_lam2);
    k.L1 = 0.5 * (k.ln_lam2 - k.ln_eps2);
    return k;
}

/* ------------------------------------------------------- quadrature ---- */

int dse_ref_gauss_legendre(int n, double* x, double* w) {
    if (n < 1 || !x || !w) return DSE_REF_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        /* i-th largest root; start from the classic cosine estimate */
        double r = cos(PI_D * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = r;  /* P_0, P_1 */
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * r * p1 - k * p0) / (k + 1.0);
                p0 = p1; p1 = p2;
            }
            /* p1 = P_n(r), p0 = P_{n-1}(r) */
            dp = n * (r * p1 - p0) / (r * r - 1.0);
            double dr = p1 / dp;
            r -= dr;
            if (fabs(dr) <= 1e-16 * (1.0 + fabs(r))) {
                /* one more evaluation of P_n' at the final root for the weight */
                p0 = 1.0; p1 = r;
                for (int k = 1; k < n; ++k) {
                    double p2 = ((2.0 * k + 1.0) * r * p1 - k * p0) / (k + 1.0);
                    p0 = p1; p1 = p2;
                }
                dp = n * (r * p1 - p0) / (r * r - 1.0);
                break;
            }
        }
        x[n - 1 - i] = r;
        w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
    return DSE_REF_OK;
}

/* Gauss-Legendre in t = ln y over [lo, hi] (ln y bounds), n nodes; dy = y dt.
 * A zero-width interval gives zero weights. */
static void log_gl(const double* tx, const double* tw, int n, double lo, double hi, double* y, double* W) {
    double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    for (int i = 0; i < n; ++i) {
        double t = c + h * tx[i];
        double yy = exp(t);
        y[i] = yy;
        W[i] = h * tw[i] * yy;
    }
}

/* Radial rule at external momentum x (Sec. 2 radial integral, Sec. 3 interval split):
 *  radial_mode 0: one Gauss-Legendre rule in ln y over [eps2, lambda2] (n_radial nodes);
 *  radial_mode 1: the paper's split int_0^lambda2 = int_0^eps2 + int_eps2^x + int_x^lambda2
 *    with n_radial Gauss-Legendre nodes in ln y per piece (3 n_radial nodes); the
 *    piece [0, eps2] is taken over [1e-6 eps2, eps2] (the paper gives no mapping for
 *    it; the dropped [0, 1e-6 eps2] is O(1e-12 eps2^2) for the ghost and O(1e-6 eps2)
 *    for the gluon integrand relative to the first piece), x clamped into
 *    [eps2, lambda2]. */
int dse_ref_radial_rule(const dse_ref_problem* p, double x, double* y, double* W) {
    int st = check_problem(p);
    if (st) return st;
    if (!y || !W || !(x >= 0.0)) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    int nr = p->n_radial;
    double* tx = (double*)malloc(sizeof(double) * (size_t)nr);
    double* tw = (double*)malloc(sizeof(double) * (size_t)nr);
    if (!tx || !tw) { free(tx); free(tw); return DSE_REF_ERR_ARG; }
    dse_ref_gauss_legendre(nr, tx, tw);
    if (p->radial_mode == 0) {
        log_gl(tx, tw, nr, k.ln_eps2, k.ln_lam2, y, W);
    } else {
        double xs = x < p->eps2 ? p->eps2 : (x > p->lambda2 ? p->lambda2 : x);
        double lx = log(xs);
        log_gl(tx, tw, nr, k.ln_eps2 + log(1e-6), k.ln_eps2, y, W);
        log_gl(tx, tw, nr, k.ln_eps2, lx, y + nr, W + nr);
        log_gl(tx, tw, nr, lx, k.ln_lam2, y + 2 * nr, W + 2 * nr);
    }
    free(tx); free(tw);
    return DSE_REF_OK;
}

/* Nodes per external momentum of the radial rule. */
static int radial_count(const dse_ref_problem* p) { return p->radial_mode == 1 ? 3 * p->n_radial : p->n_radial; }

/* Angular rule with int_0^pi dtheta g(theta) ~ sum_l w_l g(theta_l):
 *  angular_mode 0: Gauss-Legendre in theta over [0, pi];
 *  angular_mode 1: the paper's tanh-sinh rule in xi = cos theta (Sec. 2): the
 *    trapezoidal rule in t for xi = tanh(u), u = (pi/2) sinh t, with n_angular
 *    points t_l = t_max - (l + 1/2) h, h = 2 t_max / n_angular, t_max = 4.  Then
 *    theta = arccos(xi) = 2 atan(e^{-u}) and dtheta = (pi/2) cosh t / cosh u dt. */
static void angular_rule(const dse_ref_problem* p, double* theta, double* wt) {
    int na = p->n_angular;
    if (p->angular_mode == 1) {
        const double tmax = 4.0;
        double h = 2.0 * tmax / na;
        for (int l = 0; l < na; ++l) {
            double t = tmax - (l + 0.5) * h;
            double u = 0.5 * PI_D * sinh(t);
            if (theta) theta[l] = 2.0 * atan(exp(-u));
            if (wt) wt[l] = h * 0.5 * PI_D * cosh(t) / cosh(u);
        }
        return;
    }
    double* tx = (double*)malloc(sizeof(double) * (size_t)na);
    double* tw = (double*)malloc(sizeof(double) * (size_t)na);
    if (!tx || !tw) { free(tx); free(tw); return; }
    dse_ref_gauss_legendre(na, tx, tw);
    for (int i = 0; i < na; ++i) {
        if (theta) theta[i] = 0.5 * PI_D * (1.0 + tx[i]);
        if (wt) wt[i] = 0.5 * PI_D * tw[i];
    }
    free(tx); free(tw);
}

int dse_ref_quadrature(const dse_ref_problem* p, double* y, double* W, double* theta, double* wt) {
    int st = check_problem(p);
    if (st) return st;
    if (y && W) {
        /* radial_mode 1: the rule of x = lambda2 (dse_ref_radial_rule for other x) */
        st = dse_ref_radial_rule(p, p->lambda2, y, W);
        if (st) return st;
    }
    angular_rule(p, theta, wt);
    return DSE_REF_OK;
}

/* ---------------------------------------------------- Chebyshev map ---- */

double dse_ref_map(const dse_ref_problem* p, double x) {
    consts k = make_consts(p);
    return (log(x) - k.L0) / k.L1;
}

/* the n mapped roots of T_n, ascending */
static void mapped_roots(const consts* k, int n, double* x) {
    for (int i = 0; i < n; ++i) {
        double s = -cos(PI_D * (2.0 * i + 1.0) / (2.0 * n));
        x[i] = exp(k->L0 + k->L1 * s);
    }
}

int dse_ref_collocation(const dse_ref_problem* p, double* x) {
    int st = check_problem(p);
    if (st) return st;
    if (!x) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    mapped_roots(&k, k.NZ, x);
    return DSE_REF_OK;
}

int dse_ref_collocation_ghost(const dse_ref_problem* p, double* x) {
    int st = check_problem(p);
    if (st) return st;
    if (!x) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    mapped_roots(&k, k.NG, x);
    return DSE_REF_OK;
}

/* phi_j(x) for the clamped mapped variable */
static void basis(const consts* k, double x, double* phi) {
    double s = (log(x) - k->L0) / k->L1;
    if (s < -1.0) s = -1.0;
    if (s > 1.0) s = 1.0;
    phi[0] = 0.5;
    if (k->N == 1) return;
    double tm = 1.0, tc = s;
    phi[1] = s;
    for (int j = 2; j < k->N; ++j) {
        double tn = 2.0 * s * tc - tm;
        tm = tc; tc = tn;
        phi[j] = tc;
    }
}

int dse_ref_basis(const dse_ref_problem* p, double x, double* phi) {
    int st = check_problem(p);
    if (st) return st;
    if (!phi || !(x > 0.0)) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    basis(&k, x, phi);
    return DSE_REF_OK;
}

/* ln G(x), ln Z(x) and (optionally) phi_j(x).  Inside [eps2, lambda2] the
 * Chebyshev series of Sec. 3; below eps2  Z = A x^{2 kappa},  G = B x^{-kappa};
 * above lambda2  G = G_UV [omega ln(x/lambda2) + 1]^delta,
 * Z = Z_UV [...]^gamma, with A, B, G_UV, Z_UV matched to the series at the
 * end points (Sec. 2).  extrap_mode 1 continues the end values as constants. */
static void dressing_w(const dse_ref_problem* p, const consts* k, const double* c, double x,
                       double* lnG, double* lnZ, double* phi_out, double* dG_dw, double* dZ_dw);

static void dressing(const dse_ref_problem* p, const consts* k, const double* c, double x,
                     double* lnG, double* lnZ, double* phi_out) {
    dressing_w(p, k, c, x, lnG, lnZ, phi_out, NULL, NULL);
}

/* ... and the derivatives of ln G(x), ln Z(x) with respect to omega, which
 * enters only the UV form: d/d omega of ln(1 + omega ln(x/lambda2)). */
static void dressing_w(const dse_ref_problem* p, const consts* k, const double* c, double x,
                       double* lnG, double* lnZ, double* phi_out, double* dG_dw, double* dZ_dw) {
    double phi_local[1024];
    double* phi = phi_out ? phi_out : phi_local;
    basis(k, x, phi);
    double lg = 0.0, lz = 0.0;
    for (int j = 0; j < k->NZ; ++j) lz += c[j] * phi[j];
    for (int j = 0; j < k->NG; ++j) lg += c[k->NZ + j] * phi[j];
    if (p->extrap_mode == 0) {
        if (x < p->eps2) {
            double r = log(x) - k->ln_eps2;
            lg += -p->kappa * r;
            lz += 2.0 * p->kappa * r;
        } else if (x > p->lambda2) {
            double lu = log(x) - k->ln_lam2;
            double L = log1p(k->omega * lu);
            lg += p->delta * L;
            lz += k->gam * L;
            if (dG_dw) *dG_dw = p->delta * lu / (1.0 + k->omega * lu);
            if (dZ_dw) *dZ_dw = k->gam * lu / (1.0 + k->omega * lu);
            *lnG = lg;
            *lnZ = lz;
            return;
        }
    }
    if (dG_dw) *dG_dw = 0.0;
    if (dZ_dw) *dZ_dw = 0.0;
    *lnG = lg;
    *lnZ = lz;
}

int dse_ref_dressing(const dse_ref_problem* p, const double* c, int n, const double* x,
                     double* lnG, double* lnZ) {
    int st = check_problem(p);
    if (st) return st;
    if (!c || !x || !lnG || !lnZ || n < 0) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    for (int m = 0; m < n; ++m) {
        if (!(x[m] > 0.0)) return DSE_REF_ERR_ARG;
        dressing(p, &k, c, x[m], &lnG[m], &lnZ[m], NULL);
    }
    return DSE_REF_OK;
}

/* ---------------------------------------------------------- kernels ---- */

/* z = x + y - 2 sqrt(xy) cos(theta) written as d + 2 b sigma with
 * d = (sqrt x - sqrt y)^2, b = 2 sqrt(xy), sigma = sin^2(theta/2).
 * M: the printed M equals [2x + 2y - z - (x-y)^2/z]/(4x) = y sin^2(theta)/z.
 * Q: multiplying the printed Q by 8 x y z^2 gives a quartic in z; written in
 * (d, b, sigma) it is 2 b^2 (n0 + n1 sigma + ... + n4 sigma^4) with the
 * coefficients below, so Q = (n0 + ... + n4 sigma^4) / (2 z^2).  Neither form
 * cancels large terms, unlike the printed one at x << y. */
static void kernels(double x, double y, double sig, double s2, double* M, double* Q, double* zout) {
    double sx = sqrt(x), sy = sqrt(y);
    double d = (sx - sy) * (sx - sy);
    double b = 2.0 * sx * sy;
    double z = d + 2.0 * b * sig;
    double n0 = 7.5 * d * d;
    double n1 = -(48.0 * d * d + 18.0 * d * b + 12.0 * b * b);
    double n2 = 48.0 * d * d - 48.0 * d * b - 38.0 * b * b;
    double n3 = 96.0 * d * b + 64.0 * b * b;
    double n4 = 16.0 * b * b;
    double num = n0 + sig * (n1 + sig * (n2 + sig * (n3 + sig * n4)));
    *Q = num / (2.0 * z * z);
    *M = y * s2 / z;
    *zout = z;
}

int dse_ref_kernels(double x, double y, double theta, double* M, double* Q, double* z) {
    if (!(x > 0.0) || !(y > 0.0) || !M || !Q || !z) return DSE_REF_ERR_ARG;
    double sh = sin(0.5 * theta);
    double st = sin(theta);
    kernels(x, y, sh * sh, st * st, M, Q, z);
    return DSE_REF_OK;
}

/* ---------------------------------------------------- self-energies ---- */

/* Pi_G(x) = -K int dy y G(y) int dtheta sin^4(theta) Z(z)/z^2
 *   (ghost equation of Sec. 2 with xi = cos theta: (1 - xi^2)^{3/2} dxi -> sin^4 dtheta)
 * Pi_Z(x) = K/(3x) int dy int dtheta sin^2(theta) [Q W + M G(y) G(z)],
 *   W = (G(y) G(z))^{-2-6 delta} (Z(y) Z(z))^{-3 delta}.
 * Gradients: d ln G(u)/d b_j = d ln Z(u)/d a_j = phi_j(u) for u in {y, z}. */
static int self_energy_impl(const dse_ref_problem* p, const double* c, double x, int magnitudes,
                            double* PiG, double* PiZ, double* d_PiG, double* d_PiZ) {
    int st = check_problem(p);
    if (st) return st;
    if (!c || !(x >= 0.0)) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    int N = k.N, NZ = k.NZ, NG = k.NG, nr = p->n_radial, na = p->n_angular;
    int want_d = (d_PiG != NULL) || (d_PiZ != NULL);
    int gluon = x > 0.0;

    nr = radial_count(p);
    double* y = (double*)malloc(sizeof(double) * nr);
    double* W = (double*)malloc(sizeof(double) * nr);
    double* th = (double*)malloc(sizeof(double) * na);
    double* wt = (double*)malloc(sizeof(double) * na);
    double* phiy = (double*)malloc(sizeof(double) * N);
    double* phiz = (double*)malloc(sizeof(double) * N);
    nsum* acc = (nsum*)calloc((size_t)(2 + 2 * (NZ + NG)), sizeof(nsum));
    if (!y || !W || !th || !wt || !phiy || !phiz || !acc) {
        free(y); free(W); free(th); free(wt); free(phiy); free(phiz); free(acc);
        return DSE_REF_ERR_ARG;
    }
    dse_ref_radial_rule(p, x, y, W);
    angular_rule(p, th, wt);
    nsum* sG = &acc[0];
    nsum* sZ = &acc[1];
    nsum* gZa = &acc[2];                 /* d Pi_Z / d a_j (without prefactor), j < NZ */
    nsum* gZb = &acc[2 + NZ];            /* d Pi_Z / d b_j, j < NG */
    nsum* gGa = &acc[2 + NZ + NG];       /* d Pi_G / d a_j */
    nsum* gGb = &acc[2 + 2 * NZ + NG];   /* d Pi_G / d b_j */

    for (int kk = 0; kk < nr; ++kk) {
        double lGy, lZy;
        dressing(p, &k, c, y[kk], &lGy, &lZy, phiy);
        double Gy = exp(lGy);
        for (int l = 0; l < na; ++l) {
            double sh = sin(0.5 * th[l]);
            double sn = sin(th[l]);
            double sig = sh * sh, s2 = sn * sn;
            double M = 0.0, Q = 0.0, z;
            if (gluon) {
                kernels(x, y[kk], sig, s2, &M, &Q, &z);
            } else {
                /* x = 0: z = y, only the ghost integrand exists */
                double sy = sqrt(y[kk]);
                z = sy * sy;
            }
            double lGz, lZz;
            dressing(p, &k, c, z, &lGz, &lZz, want_d ? phiz : NULL);
            double Gz = exp(lGz), Zz = exp(lZz);
            double wgt = W[kk] * wt[l];
            /* ghost integrand y G(y) sin^4 Z(z)/z^2 */
            double fG = wgt * y[kk] * Gy * s2 * s2 * Zz / (z * z);
            double hQ = 0.0, hM = 0.0;
            if (gluon) {
                double Wv = exp(k.pG * (lGy + lGz) + k.qZ * (lZy + lZz));
                hQ = wgt * s2 * Q * Wv;
                hM = wgt * s2 * M * Gy * Gz;
            }
            if (!magnitudes) {
                ns_add(sG, fG);
                if (gluon) ns_add(sZ, hQ + hM);
                if (want_d) {
                    for (int j = 0; j < NZ; ++j) {
                        if (gluon) ns_add(&gZa[j], k.qZ * hQ * (phiy[j] + phiz[j]));
                        ns_add(&gGa[j], fG * phiz[j]);
                    }
                    for (int j = 0; j < NG; ++j) {
                        if (gluon) ns_add(&gZb[j], (k.pG * hQ + hM) * (phiy[j] + phiz[j]));
                        ns_add(&gGb[j], fG * phiy[j]);
                    }
                }
            } else {
                /* sums of the magnitudes of every summand, term by term */
                ns_add(sG, fabs(fG));
                if (gluon) ns_add(sZ, fabs(hQ) + fabs(hM));
                if (want_d) {
                    for (int j = 0; j < NZ; ++j) {
                        if (gluon) ns_add(&gZa[j], fabs(k.qZ * hQ) * (fabs(phiy[j]) + fabs(phiz[j])));
                        ns_add(&gGa[j], fabs(fG * phiz[j]));
                    }
                    for (int j = 0; j < NG; ++j) {
                        if (gluon) ns_add(&gZb[j], (fabs(k.pG * hQ) + fabs(hM)) * (fabs(phiy[j]) + fabs(phiz[j])));
                        ns_add(&gGb[j], fabs(fG * phiy[j]));
                    }
                }
            }
        }
    }
    double preZ = gluon ? k.K / (3.0 * x) : 0.0;
    double preG = -k.K;
    if (magnitudes) {
        preZ = fabs(preZ);
        preG = fabs(preG);
    }
    if (PiG) *PiG = preG * ns_val(sG);
    if (PiZ) *PiZ = gluon ? preZ * ns_val(sZ) : 0.0;
    for (int j = 0; j < NZ; ++j) {
        if (d_PiZ) d_PiZ[j] = preZ * ns_val(&gZa[j]);
        if (d_PiG) d_PiG[j] = preG * ns_val(&gGa[j]);
    }
    for (int j = 0; j < NG; ++j) {
        if (d_PiZ) d_PiZ[NZ + j] = preZ * ns_val(&gZb[j]);
        if (d_PiG) d_PiG[NZ + j] = preG * ns_val(&gGb[j]);
    }
    free(y); free(W); free(th); free(wt); free(phiy); free(phiz); free(acc);
    return DSE_REF_OK;
}

int dse_ref_self_energy(const dse_ref_problem* p, const double* c, double x,
                        double* PiG, double* PiZ, double* d_PiG, double* d_PiZ) {
    return self_energy_impl(p, c, x, 0, PiG, PiZ, d_PiG, d_PiZ);
}

/* Derivatives of Pi_G(x), Pi_Z(x) with respect to g^2 Nc.  The coupling enters
 * through the prefactor K = g^2 Nc/(2 pi)^3 (so Pi/g2nc) and through
 * omega = 11 g^2 Nc/(48 pi^2) in the UV forms of G(z), Z(z) for z > lambda2:
 *   d Pi/d g2nc = Pi/g2nc + (d omega/d g2nc) sum h * d ln h/d omega,
 * with d ln W/d omega = p dlnG/dw + q dlnZ/dw, d ln G(z)/d omega for the M term
 * and d ln Z(z)/d omega for the ghost term (y <= lambda2 carries no omega). */
static int self_energy_dg2(const dse_ref_problem* p, const double* c, double x, double* dPiG, double* dPiZ) {
    consts k = make_consts(p);
    int N = p->n_cheb, nr = radial_count(p), na = p->n_angular;
    int gluon = x > 0.0;
    double* y = (double*)malloc(sizeof(double) * nr);
    double* W = (double*)malloc(sizeof(double) * nr);
    double* th = (double*)malloc(sizeof(double) * na);
    double* wt = (double*)malloc(sizeof(double) * na);
    if (!y || !W || !th || !wt) { free(y); free(W); free(th); free(wt); return DSE_REF_ERR_ARG; }
    (void)N;
    dse_ref_radial_rule(p, x, y, W);
    angular_rule(p, th, wt);
    nsum sG = {0, 0}, sZ = {0, 0}, wG = {0, 0}, wZ = {0, 0};
    for (int kk = 0; kk < nr; ++kk) {
        double lGy, lZy;
        dressing(p, &k, c, y[kk], &lGy, &lZy, NULL);
        double Gy = exp(lGy);
        for (int l = 0; l < na; ++l) {
            double sh = sin(0.5 * th[l]);
            double sn = sin(th[l]);
            double sig = sh * sh, s2 = sn * sn;
            double M = 0.0, Q = 0.0, z;
            if (gluon) kernels(x, y[kk], sig, s2, &M, &Q, &z);
            else { double sy = sqrt(y[kk]); z = sy * sy; }
            double lGz, lZz, gw, zw;
            dressing_w(p, &k, c, z, &lGz, &lZz, NULL, &gw, &zw);
            double wgt = W[kk] * wt[l];
            double fG = wgt * y[kk] * Gy * s2 * s2 * exp(lZz) / (z * z);
            ns_add(&sG, fG);
            ns_add(&wG, fG * zw);
            if (gluon) {
                double Wv = exp(k.pG * (lGy + lGz) + k.qZ * (lZy + lZz));
                double hQ = wgt * s2 * Q * Wv;
                double hM = wgt * s2 * M * Gy * exp(lGz);
                ns_add(&sZ, hQ + hM);
                ns_add(&wZ, hQ * (k.pG * gw + k.qZ * zw) + hM * gw);
            }
        }
    }
    double dw = 11.0 / (48.0 * PI_D * PI_D);
    double preZ = gluon ? k.K / (3.0 * x) : 0.0;
    /* Pi_G = -K S_G, Pi_Z = preZ S_Z; K and preZ are proportional to g2nc */
    *dPiG = -k.K * (ns_val(&sG) / p->g2nc + dw * ns_val(&wG));
    *dPiZ = gluon ? preZ * (ns_val(&sZ) / p->g2nc + dw * ns_val(&wZ)) : 0.0;
    free(y); free(W); free(th); free(wt);
    return DSE_REF_OK;
}

/* External momenta at which the self-energies are evaluated: the collocation
 * points (shared by both equations when N_Z = N_G; otherwise the N_Z gluon points
 * followed by the N_G ghost points), then x_Z and x_G.  xr holds N_Z + N_G + 2
 * doubles.  Returns the number Rc of collocation rows; *gofs is the row of the
 * first ghost point. */
static int row_points(const dse_ref_problem* p, const consts* k, double* xr, int* gofs) {
    int Rc;
    mapped_roots(k, k->NZ, xr);
    if (k->NZ == k->NG) {
        Rc = k->NZ;
        *gofs = 0;
    } else {
        mapped_roots(k, k->NG, xr + k->NZ);
        Rc = k->NZ + k->NG;
        *gofs = k->NZ;
    }
    xr[Rc] = p->x_Z;
    xr[Rc + 1] = p->x_G;
    return Rc;
}

int dse_ref_param_derivatives(const dse_ref_problem* p, const double* c, double* dF) {
    int st = check_problem(p);
    if (st) return st;
    if (!c || !dF) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    int NZ = k.NZ, NG = k.NG, gofs;
    double* xr = (double*)malloc(sizeof(double) * (NZ + NG + 2));
    double* dG = (double*)malloc(sizeof(double) * (NZ + NG + 2));
    double* dZ = (double*)malloc(sizeof(double) * (NZ + NG + 2));
    int* rst = (int*)calloc((size_t)(NZ + NG + 2), sizeof(int));
    if (!xr || !dG || !dZ || !rst) { free(xr); free(dG); free(dZ); free(rst); return DSE_REF_ERR_ARG; }
    int Rc = row_points(p, &k, xr, &gofs);
    int R = Rc + 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < R; ++r) rst[r] = self_energy_dg2(p, c, xr[r], &dG[r], &dZ[r]);
    for (int r = 0; r < R; ++r)
        if (rst[r]) { st = rst[r]; break; }
    if (!st) {
        /* columns: g2nc, ginv_G, zinv_Z */
        for (int i = 0; i < NZ; ++i) {
            dF[(size_t)i * 3 + 0] = -dZ[i] + dZ[Rc];
            dF[(size_t)i * 3 + 1] = 0.0;
            dF[(size_t)i * 3 + 2] = -1.0;
        }
        for (int i = 0; i < NG; ++i) {
            dF[(size_t)(NZ + i) * 3 + 0] = -dG[gofs + i] + dG[Rc + 1];
            dF[(size_t)(NZ + i) * 3 + 1] = -1.0;
            dF[(size_t)(NZ + i) * 3 + 2] = 0.0;
        }
    }
    free(xr); free(dG); free(dZ); free(rst);
    return st;
}

/* ------------------------------------------------ residual and matrix ---- */

/* Residuals at the collocation points (Sec. 3, MOM scheme of Sec. 2):
 *   z(x_i) = Z(x_i)^{-1} - Z(x_Z)^{-1} - Pi_Z(x_i) + Pi_Z(x_Z)   (N_Z gluon points)
 *   g(x_i) = G(x_i)^{-1} - G(x_G)^{-1} - Pi_G(x_i) + Pi_G(x_G)   (N_G ghost points)
 * and the Newton matrix of their derivatives; rows (z; g), columns (a; b). */
static int assemble(const dse_ref_problem* p, const double* c, int magnitudes, double* J, double* F) {
    int st = check_problem(p);
    if (st) return st;
    if (!c) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    int NZ = k.NZ, NG = k.NG, n = NZ + NG, gofs;
    int want_d = J != NULL;
    double* xr = (double*)malloc(sizeof(double) * (n + 2));
    double* PiGr = (double*)malloc(sizeof(double) * (n + 2));
    double* PiZr = (double*)malloc(sizeof(double) * (n + 2));
    double* dG = want_d ? (double*)malloc(sizeof(double) * (size_t)(n + 2) * n) : NULL;
    double* dZ = want_d ? (double*)malloc(sizeof(double) * (size_t)(n + 2) * n) : NULL;
    int* rst = (int*)calloc((size_t)(n + 2), sizeof(int));
    double* phi = (double*)malloc(sizeof(double) * k.N);
    if (!xr || !PiGr || !PiZr || !rst || !phi || (want_d && (!dG || !dZ))) {
        free(xr); free(PiGr); free(PiZr); free(dG); free(dZ); free(rst); free(phi);
        return DSE_REF_ERR_ARG;
    }
    int Rc = row_points(p, &k, xr, &gofs);
    int R = Rc + 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < R; ++r) {
        rst[r] = self_energy_impl(p, c, xr[r], magnitudes, &PiGr[r], &PiZr[r],
                                  want_d ? &dG[(size_t)r * n] : NULL,
                                  want_d ? &dZ[(size_t)r * n] : NULL);
    }
    for (int r = 0; r < R; ++r)
        if (rst[r]) { st = rst[r]; break; }
    if (!st) {
        const double* dZref = want_d ? &dZ[(size_t)Rc * n] : NULL;
        const double* dGref = want_d ? &dG[(size_t)(Rc + 1) * n] : NULL;
        /* gluon rows */
        for (int i = 0; i < NZ; ++i) {
            double lG, lZ;
            dressing(p, &k, c, xr[i], &lG, &lZ, phi);
            double Zinv = exp(-lZ);
            if (F) F[i] = magnitudes ? Zinv + fabs(p->zinv_Z) + PiZr[i] + PiZr[Rc]
                                     : Zinv - p->zinv_Z - PiZr[i] + PiZr[Rc];
            if (want_d) {
                const double* dZi = &dZ[(size_t)i * n];
                double* Jz = &J[(size_t)i * n];
                for (int j = 0; j < n; ++j) {
                    /* d Z(x)^{-1}/d a_j = -Z(x)^{-1} phi_j(x) */
                    double diagZ = j < NZ ? -Zinv * phi[j] : 0.0;
                    Jz[j] = magnitudes ? fabs(diagZ) + dZi[j] + dZref[j] : diagZ - dZi[j] + dZref[j];
                }
            }
        }
        /* ghost rows */
        for (int i = 0; i < NG; ++i) {
            int r = gofs + i;
            double lG, lZ;
            dressing(p, &k, c, xr[r], &lG, &lZ, phi);
            double Ginv = exp(-lG);
            if (F) F[NZ + i] = magnitudes ? Ginv + fabs(p->ginv_G) + PiGr[r] + PiGr[Rc + 1]
                                          : Ginv - p->ginv_G - PiGr[r] + PiGr[Rc + 1];
            if (want_d) {
                const double* dGi = &dG[(size_t)r * n];
                double* Jg = &J[(size_t)(NZ + i) * n];
                for (int j = 0; j < n; ++j) {
                    /* d G(x)^{-1}/d b_j = -G(x)^{-1} phi_j(x) */
                    double diagG = j >= NZ ? -Ginv * phi[j - NZ] : 0.0;
                    Jg[j] = magnitudes ? fabs(diagG) + dGi[j] + dGref[j] : diagG - dGi[j] + dGref[j];
                }
            }
        }
        if (F) {
            for (int i = 0; i < n; ++i)
                if (!isfinite(F[i])) { st = DSE_REF_ERR_NONFINITE; break; }
        }
        if (!st && want_d) {
            for (size_t e = 0; e < (size_t)n * n; ++e)
                if (!isfinite(J[e])) { st = DSE_REF_ERR_NONFINITE; break; }
        }
    }
    free(xr); free(PiGr); free(PiZr); free(dG); free(dZ); free(rst); free(phi);
    return st;
}

int dse_ref_residual(const dse_ref_problem* p, const double* c, double* F) {
    if (!F) return DSE_REF_ERR_ARG;
    return assemble(p, c, 0, NULL, F);
}

int dse_ref_newton_matrix(const dse_ref_problem* p, const double* c, double* J, double* F) {
    if (!J) return DSE_REF_ERR_ARG;
    return assemble(p, c, 0, J, F);
}

int dse_ref_newton_matrix_magnitudes(const dse_ref_problem* p, const double* c, double* A, double* AF) {
    if (!A) return DSE_REF_ERR_ARG;
    return assemble(p, c, 1, A, AF);
}

/* --------------------------------------------------------------- LU ---- */

int dse_ref_lu_solve(int n, const double* A, const double* b, double* x) {
    if (n < 1 || !A || !b || !x) return DSE_REF_ERR_ARG;
    double* LU = (double*)malloc(sizeof(double) * (size_t)n * n);
    int* piv = (int*)malloc(sizeof(int) * n);
    if (!LU || !piv) { free(LU); free(piv); return DSE_REF_ERR_ARG; }
    memcpy(LU, A, sizeof(double) * (size_t)n * n);
    int st = DSE_REF_OK;
    for (int kk = 0; kk < n; ++kk) {
        int pr = kk;
        double best = fabs(LU[(size_t)kk * n + kk]);
        for (int i = kk + 1; i < n; ++i) {
            double v = fabs(LU[(size_t)i * n + kk]);
            if (v > best) { best = v; pr = i; }
        }
        if (!(best > 1e-300)) { st = DSE_REF_ERR_SINGULAR; break; }
        piv[kk] = pr;
        if (pr != kk) {
            for (int j = 0; j < n; ++j) {
                double t = LU[(size_t)kk * n + j];
                LU[(size_t)kk * n + j] = LU[(size_t)pr * n + j];
                LU[(size_t)pr * n + j] = t;
            }
        }
        double d = LU[(size_t)kk * n + kk];
        for (int i = kk + 1; i < n; ++i) {
            double l = LU[(size_t)i * n + kk] / d;
            LU[(size_t)i * n + kk] = l;
            for (int j = kk + 1; j < n; ++j) LU[(size_t)i * n + j] -= l * LU[(size_t)kk * n + j];
        }
    }
    if (!st) {
        for (int i = 0; i < n; ++i) x[i] = b[i];
        for (int kk = 0; kk < n; ++kk) {
            if (piv[kk] != kk) { double t = x[kk]; x[kk] = x[piv[kk]]; x[piv[kk]] = t; }
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) x[i] -= LU[(size_t)i * n + j] * x[j];
        for (int i = n - 1; i >= 0; --i) {
            for (int j = i + 1; j < n; ++j) x[i] -= LU[(size_t)i * n + j] * x[j];
            x[i] /= LU[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i)
            if (!isfinite(x[i])) { st = DSE_REF_ERR_NONFINITE; break; }
    }
    free(LU); free(piv);
    return st;
}

/* --------------------------------------------------------- Newton ---- */

/* a^{n+1} = a^n - rho Delta a,  b^{n+1} = b^n - rho Delta b  with J Delta = F (Sec. 3) */
int dse_ref_newton_step(const dse_ref_problem* p, double* c, double rho, double* stats) {
    int st = check_problem(p);
    if (st) return st;
    if (!c || !isfinite(rho)) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    int NZ = k.NZ, NG = k.NG, n = NZ + NG;
    double* J = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* F = (double*)malloc(sizeof(double) * n);
    double* D = (double*)malloc(sizeof(double) * n);
    double* xz = (double*)malloc(sizeof(double) * NZ);
    double* xg = (double*)malloc(sizeof(double) * NG);
    double* lG = (double*)malloc(sizeof(double) * n);
    double* lZ = (double*)malloc(sizeof(double) * n);
    if (!J || !F || !D || !xz || !xg || !lG || !lZ) {
        free(J); free(F); free(D); free(xz); free(xg); free(lG); free(lZ);
        return DSE_REF_ERR_ARG;
    }
    st = assemble(p, c, 0, J, F);
    if (!st) st = dse_ref_lu_solve(n, J, F, D);
    if (!st) {
        /* dimensionless residual: Z(x_i) z_i at the gluon points, G(x_i) g_i at the ghost points */
        dse_ref_collocation(p, xz);
        dse_ref_collocation_ghost(p, xg);
        dse_ref_dressing(p, c, NZ, xz, lG, lZ);
        dse_ref_dressing(p, c, NG, xg, lG + NZ, lZ + NZ);
        double nF = 0.0, nS = 0.0, nD = 0.0;
        for (int i = 0; i < n; ++i) {
            nF = fmax(nF, fabs(F[i]));
            double scale = i < NZ ? exp(lZ[i]) : exp(lG[i]);
            nS = fmax(nS, fabs(F[i]) * scale);
            nD = fmax(nD, fabs(D[i]));
        }
        for (int i = 0; i < n; ++i) c[i] -= rho * D[i];
        if (stats) { stats[0] = nF; stats[1] = nS; stats[2] = nD; }
    }
    free(J); free(F); free(D); free(xz); free(xg); free(lG); free(lZ);
    return st;
}

/* -------------------------------------------------------- Schwinger ---- */

/* Nodes for int_0^inf d|p| f(p): Gauss-Legendre in u = ln p^2 over
 * [ln eps2, ln lambda2]; p = exp(u/2), d|p| = (p/2) du.  The tails below eps
 * and above Lambda are left out. */
int dse_ref_schwinger_nodes(const dse_ref_problem* p, int n, double* pn, double* wn) {
    int st = check_problem(p);
    if (st) return st;
    if (n < 1 || !pn || !wn) return DSE_REF_ERR_ARG;
    consts k = make_consts(p);
    double* tx = (double*)malloc(sizeof(double) * n);
    double* tw = (double*)malloc(sizeof(double) * n);
    if (!tx || !tw) { free(tx); free(tw); return DSE_REF_ERR_ARG; }
    dse_ref_gauss_legendre(n, tx, tw);
    for (int i = 0; i < n; ++i) {
        double u = k.L0 + k.L1 * tx[i];
        double pp = exp(0.5 * u);
        pn[i] = pp;
        wn[i] = k.L1 * tw[i] * 0.5 * pp;
    }
    free(tx); free(tw);
    return DSE_REF_OK;
}

/* Delta(t) = (1/pi) int_0^inf d|p| cos(t |p|) sigma(p^2),  sigma = Z(p^2)/p^2 (Sec. 2.2) */
int dse_ref_schwinger(const dse_ref_problem* p, const double* c, const double* t, int n_t,
                      int n_nodes, double* delta) {
    int st = check_problem(p);
    if (st) return st;
    if (!c || !t || !delta || n_t < 0 || n_nodes < 1) return DSE_REF_ERR_ARG;
    double* pn = (double*)malloc(sizeof(double) * n_nodes);
    double* wn = (double*)malloc(sizeof(double) * n_nodes);
    double* sg = (double*)malloc(sizeof(double) * n_nodes);
    double* lG = (double*)malloc(sizeof(double) * n_nodes);
    double* lZ = (double*)malloc(sizeof(double) * n_nodes);
    double* x2 = (double*)malloc(sizeof(double) * n_nodes);
    if (!pn || !wn || !sg || !lG || !lZ || !x2) {
        free(pn); free(wn); free(sg); free(lG); free(lZ); free(x2);
        return DSE_REF_ERR_ARG;
    }
    dse_ref_schwinger_nodes(p, n_nodes, pn, wn);
    for (int i = 0; i < n_nodes; ++i) x2[i] = pn[i] * pn[i];
    st = dse_ref_dressing(p, c, n_nodes, x2, lG, lZ);
    if (!st) {
        for (int i = 0; i < n_nodes; ++i) sg[i] = exp(lZ[i]) / x2[i];
#pragma omp parallel for schedule(static)
        for (int m = 0; m < n_t; ++m) {
            nsum acc = {0.0, 0.0};
            for (int i = 0; i < n_nodes; ++i) ns_add(&acc, wn[i] * cos(t[m] * pn[i]) * sg[i]);
            delta[m] = ns_val(&acc) / PI_D;
        }
        for (int m = 0; m < n_t; ++m)
            if (!isfinite(delta[m])) { st = DSE_REF_ERR_NONFINITE; break; }
    }
    free(pn); free(wn); free(sg); free(lG); free(lZ); free(x2);
    return st;
}

int dse_ref_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
