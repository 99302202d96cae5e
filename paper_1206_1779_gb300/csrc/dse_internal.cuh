// dse_internal.cuh -- internal types and launchers of the sm_103a solver for the
// ghost-gluon Dyson-Schwinger system (arXiv:1206.1779).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dse.h"

namespace dse {

// Device status bits (sticky until read by a synchronising call).
enum : int { kStatusNonfinite = 1, kStatusSingular = 2 };

// Derived constants of Sec. 2 / Sec. 3, passed by value to every kernel.
// Orders: NZ coefficients a_j of ln Z, NG coefficients b_j of ln G, N = max(NZ, NG)
// (length of the T_j recurrence and of every phi table row), n = NZ + NG unknowns
// c = (a; b).  Collocation rows: Rc = N shared points when NZ = NG, otherwise the
// NZ gluon points followed by the NG ghost points (gofs = index of the first
// ghost point, 0 when shared).  Per-row derivative vectors D[r] (ldD() doubles):
// dPi_Z/dc_j at j, dPi_G/dc_j at n + j (j < n), Pi_Z at 2n, Pi_G at 2n + 1, for
// r < Rc (collocation), Rc (x_Z) and Rc + 1 (x_G).
// Radial rule: nr nodes per external momentum; radmode 0 shares one rule of
// nrule = nr nodes between all rows, radmode 1 (the paper's split at x with an
// infrared piece) gives every D row r its own nr = 3 nrule nodes, stored from
// r * nr on (rowrad() = 1).  angmode 0: Gauss-Legendre in theta; 1: tanh-sinh in
// xi = cos theta.
struct Consts {
    int N, nr, na, extrap;
    int NZ, NG, n, Rc, gofs;
    int nrule, radmode, angmode, sM;  // sM: series-table intervals (0: no table)
    double eps2, lam2, ln_eps2, ln_lam2;
    double L0, L1, invL1;          // ln x = L0 + L1 s
    double sL0;                    // -L0 / L1 (s = fma(ln x, invL1, sL0))
    double K;                      // g^2 Nc / (2 pi)^3
    double kappa, delta, gam;      // IR exponent, anomalous dimensions
    double pG, qZ;                 // vertex-model exponents on G and Z
    double omega;                  // UV log coefficient 11 g^2 Nc / (48 pi^2)
    double x_G, x_Z, ginv_G, zinv_Z;
};

__host__ __device__ inline size_t ldD(const Consts& c) { return 2 * (size_t)c.n + 2; }
// offset of row r's radial tables (Rad, YTab, and phi_y in units of N)
__host__ __device__ inline size_t rad_offset(const Consts& c, int r) {
    return c.radmode == 1 ? (size_t)r * c.nr : 0;
}
// number of radial table entries: nr, or nr per D row (Rc + 2 rows)
__host__ __device__ inline size_t rad_entries(const Consts& c) {
    return c.radmode == 1 ? (size_t)(c.Rc + 2) * c.nr : (size_t)c.nr;
}

// Per radial node: y_k, quadrature weight W_k (Jacobian y_k included), sqrt(y_k).
struct Rad { double y, W, sy, pad; };
// Per angular node: weight w_l, sigma_l = sin^2(theta_l/2), sin^2 theta_l, sin^4 theta_l,
// and the products w_l sin^2 theta_l, w_l sin^4 theta_l.
struct Ang { double w, sig, s2, s4, ws2, ws4; };
// Per triple-kernel row (external momentum): x, sqrt(x), K/(3x), flags.
struct Row { double x, sx, pre; int flags, pad; };
enum : int { kRowGluon = 1, kRowGhost = 2 };
// Per radial node, per coefficient vector: ln G(y), ln Z(y), G(y), Z(y),
// p ln G(y) + q ln Z(y), y G(y), exp(p ln G(y) + q ln Z(y)).
struct YTab { double lG, lZ, G, Z, pq, yG, Wy, pad1; };
// Per collocation point: ln G, ln Z, G, Z, 1/G, 1/Z.
struct XTab { double lG, lZ, G, Z, Ginv, Zinv, pad0, pad1; };

// Piecewise-polynomial table of the dressing functions on s in [-1, 1] (inside
// [eps2, lambda2]): M = series_intervals(N) = kSeriesM intervals uniform in
// theta = arccos s, on each a polynomial of degree kSeriesP in u = (s - mid) * invhalf
// in [-1, 1] (monomial coefficients) for Z(s), G(s) (pairs e[k]) and W(s) = G^p Z^q
// (w[k]), fitted at kSeriesP + 1 Chebyshev points where ln Z, ln G come from a
// compensated Clenshaw recurrence.  With interval width h = pi/M the interpolation
// error of a mode T_j is at most 4 (j h/4)^(P+1)/(P+1)! (modes j <= P exactly), so
// for ln Z = sum a_j T_j the relative error of the table's Z is below
// 4 (N h/4)^16/16! sum_{j>=16} |a_j|: 3.8e-15 times that sum at N = 256, 1e-24 at
// N = 64.  The FP64 quadrature kernel therefore reads the table for
// kSeriesMinN <= N <= kSeriesMaxN in place of the per-triple series sums and
// exponentials.  Every coefficient is a double-float pair (hi, lo) of the
// coefficient times 2^-E, E the record's exponent of that function (ex[F]: the
// largest coefficient lands in [1, 2), so no value leaves the FP32 range); the
// polynomials are summed on the FP32 pipe and widened with E folded in.
constexpr int kSeriesM = 256;
constexpr int kSeriesP = 15;
constexpr int kSeriesQ = kSeriesP + 1;
constexpr int kSeriesMinN = 24;
constexpr int kSeriesMaxN = 256;  // DSE_MAX_CHEB: every N >= kSeriesMinN
struct SeriesRec {
    double mid, invhalf;
    int ex[4];                  // biased FP64 exponents E of Z, G, W; ex[3]: the degree kf from
                                // which on the coefficients (hi parts) are summed in FP32 alone
    float4 e[kSeriesQ];         // (Z hi, G hi, Z lo, G lo) 2^-E, coefficients 0 .. kSeriesP
    float2 w[kSeriesQ];         // (W hi, W lo) 2^-E
};
// A table is kSeriesRecords records: the kSeriesM intervals, then one record whose
// first four doubles are the series at the end points, ln Z(s=1), ln G(s=1),
// ln Z(s=-1), ln G(s=-1) (summed in the order of the per-triple recurrence).
constexpr int kSeriesRecords = kSeriesM + 1;
__host__ __device__ inline bool use_series_table(int N) { return N >= kSeriesMinN && N <= kSeriesMaxN; }
// Intervals of a problem's table (the end-point record stays at index kSeriesM).
// Fewer intervals would not shorten the build, whose time is the length of one
// lane's compensated Clenshaw chain (N steps), and at N = 64 the hot kernel ran
// 4 % slower with 128 intervals than with 256.
__host__ __device__ inline int series_intervals(int N) { return use_series_table(N) ? kSeriesM : 0; }

struct TripleArgs {
    Consts c;
    int Rt;         // rows handled by the triple kernel
    int KB;         // radial nodes per block
    int KS;         // radial splits (gridDim.x)
    int nch;        // angular chunks of 32 per radial node
    const Rad* rad;
    const Ang* ang;
    const Row* rows;
    const YTab* ytab;
    const double* coef;   // n: a (NZ) then b (NG)
    double* Upart;        // [Rt][nr][nch][3]   angular sums per radial node
    double* Vpart;        // [Rt][KS][3][N]     z-derivative sums per split
    const SeriesRec* stab;  // series table (nullptr: sum the series per triple)
};

// One problem of a batch: its constants, its slice of the batch workspace and its
// Newton-iteration state (iter, active, result), read and written on the device.
struct BatchProblem {
    TripleArgs t;          // t.coef is unused: coefficients come from coef_base + coef_off
    YTab* ytab;            // = t.ytab, writable
    SeriesRec* stab;       // = t.stab, writable (nullptr when N < kSeriesMinN)
    double* xcol;
    double* phiy;
    XTab* xtab;
    double* phix;
    double* D;
    double* J;
    double* F;
    double* work;
    float* As;
    double2* rowinfo;
    float* Xinv;           // FP32 inverse kept from the last eliminated Newton step (n <= 128)
    double* Sinv;          // its row scales
    double* stats;         // 4 doubles of the last Newton step
    int* status;
    long long coef_off;    // offset of the problem's c (and F) in the concatenated vectors
    long long J_off;       // offset of its J in a concatenated matrix output
    int iter;              // Newton steps taken
    int active;            // 1 while the problem still iterates
    int result;            // 0 running, 1 converged, -1 non-finite, -2 singular
    int xstate;            // 1 while Xinv holds a usable inverse
};
// One work item of the persistent quadrature kernel.
struct BatchItem { int b, rt, ks, pad; };

// Argument checks of a dse_problem (DSE_OK, DSE_ERR_ARG or DSE_ERR_UNSUPPORTED) and
// its derived constants (dse_plan.cu).
int check_problem(const dse_problem* p);
Consts make_consts(const dse_problem* p);

// launchers (return cudaError_t of the launch)
cudaError_t launch_gauss_legendre(int n, double* inv, double* x, double* w, cudaStream_t s);
cudaError_t launch_setup_rules(const Consts& c, const double* gl_r, const double* gw_r,
                               const double* gl_a, const double* gw_a, Rad* rad, Ang* ang, double* theta,
                               double* xcol, Row* rows, int Rt, cudaStream_t s);
cudaError_t launch_tables(const Consts& c, const double* coef, const Rad* rad, const double* xcol,
                          YTab* ytab, double* phiy, XTab* xtab, double* phix, cudaStream_t s);
cudaError_t launch_triple(bool full, const TripleArgs& a, cudaStream_t s);
// Series table for the coefficients coef (n: a then b), kSeriesM records.
// The node values of a problem's series table depend on the table's geometry alone:
// tq (sM x kSeriesQ x N double2) holds T_j(s_q) as double-doubles, cst (2 kSeriesQ^2
// doubles) the interpolation and monomial tables; both written once by launch_series_init,
// which also writes the records' interval geometry.
constexpr size_t series_node_values(int N) { return (size_t)kSeriesM * kSeriesQ * (size_t)N; }
constexpr int kSeriesConsts = 2 * kSeriesQ * kSeriesQ;
cudaError_t launch_series_init(const Consts& c, double2* tq, double* cst, SeriesRec* tab, cudaStream_t s);
cudaError_t launch_series_table(const Consts& c, const double* coef, const double2* tq, const double* cst,
                                SeriesRec* tab, cudaStream_t s);
cudaError_t launch_series_table_batched(const BatchProblem* P, int nb, const double* coef_base, cudaStream_t s);
// FP32-integrand variant (mixed precision), same outputs and layouts.
cudaError_t launch_triple32(bool full, const TripleArgs& a, cudaStream_t s);
size_t triple_smem_bytes(bool full, int N, int KB);
int triple_block_threads(int N);
int triple_max_blocks_per_sm(bool full, int N);
cudaError_t launch_rowreduce(bool full, const Consts& c, int Rt, int KS, int nch, const Rad* rad,
                             const Ang* ang, const Row* rows, const YTab* ytab, const double* phiy,
                             const double* Upart, const double* Vpart, double* D, cudaStream_t s);
cudaError_t launch_assemble(bool full, const Consts& c, const XTab* xtab, const double* phix,
                            const double* D, double* J, double* F, int* status, cudaStream_t s);
// Newton step: J Delta = F, c <- c - rho Delta (n = NZ + NG).  For n > 160 with
// done given (an int on the device): the FP32 LU + FP64 refinement of dse_lu32.cu,
// and the FP64 LU only where that one did not converge (*done = 0).  As (n*n floats)
// and rowinfo (n double2) are scratch for the row-scaled FP32 copy of J.  For
// n <= 128, Xinv (n*n floats), Sinv (n doubles) and *xstate keep the inverse of
// an eliminated step for the next one (all three nullptr: no reuse).
cudaError_t launch_lu_newton(const Consts& c, double* J, const double* F, const XTab* xtab,
                             double* coef, double rho, double* work, float* As, double2* rowinfo,
                             double* stats, int* status, cudaStream_t s, float* Xinv = nullptr,
                             double* Sinv = nullptr, int* xstate = nullptr, int* done = nullptr,
                             bool prescaled = false);
// The Newton-step kernel's set-up for n unknowns ahead of its first launch (its
// shared-memory limit, and whether its thread-block cluster can be placed), so
// that a graph capture of the step makes no such query.
cudaError_t prepare_newton_step(int n);
// Whether launch_lu_newton scales the rows of J (n <= 128, or the FP32 LU path
// when lu32 is set); prescaled = the rows were scaled by launch_assemble_scale.
bool lu_scales_rows(int n, bool lu32);
// The assembly of J and F fused with the row scaling that launch_lu_newton
// would otherwise launch (one block per row; J, F, As, rowinfo as there).
cudaError_t launch_assemble_scale(const Consts& c, const XTab* xtab, const double* phix, const double* D, double* J,
                                  double* F, float* As, double2* rowinfo, int* status, cudaStream_t s);
// Control block of a Newton iteration run as one CUDA graph (a while node whose
// body is one Newton step followed by the decision kernel).
struct SolveCtl {
    double tol;       // stop when the dimensionless residual of a step is below it
    int max_steps;    // at most this many steps
    int steps;        // steps taken
    int status;       // the status word when the iteration stopped
    int converged;    // 1 when it stopped on tol
    double stats[4];  // the last step's stats (max|F|, dimensionless residual, max|Delta|, sweeps)
};
// begin: ctl <- (tol, max_steps), dst[0..n) <- src; decide: after a step, counts it
// and sets the while node's condition (0: stop on a status, on tol or at max_steps);
// end: dst[0..n) <- src.
cudaError_t launch_solve_begin(SolveCtl* ctl, double tol, int max_steps, const double* src, double* dst, int n,
                               cudaStream_t s);
cudaError_t launch_solve_decide(SolveCtl* ctl, const double* stats, const int* status,
                                cudaGraphConditionalHandle cond, cudaStream_t s);
cudaError_t launch_solve_end(const double* src, double* dst, int n, cudaStream_t s);
size_t newton_lu32_smem_bytes(int n);
cudaError_t launch_newton_lu32(const Consts& c, const double* J, float* As, const double2* rowinfo, const double* F,
                               const XTab* xtab, double* coef, double rho, double* stats, int* status, int* done,
                               cudaStream_t s);
cudaError_t launch_dressing(const Consts& c, const double* coef, int n, const double* x, double* lG,
                            double* lZ, int* status, cudaStream_t s);
cudaError_t launch_schwinger_map(const Consts& c, int n, const double* gx, const double* gw, double* pn,
                                 double* wn, cudaStream_t s);
cudaError_t launch_schwinger(const Consts& c, const double* coef, int n_nodes, const double* pn,
                             const double* wn, double* sigw, const double* t, int n_t, double* partial,
                             int nsplit, double* delta, int* status, cudaStream_t s);
int schwinger_splits(int n_t, int n_nodes);

// Batched forms (dse_batch.cu drives them): one launch covers every problem of
// the batch; problems with active == 0 are skipped.
cudaError_t launch_triple_batched(bool full, const BatchProblem* P, const BatchItem* items, int n_items,
                                  int* counter, const double* coef_base, int maxN, int grid, cudaStream_t s);
int triple_batched_blocks_per_sm(bool full, int maxN);
cudaError_t launch_tables_batched(const BatchProblem* P, int nb, int max_units, const double* coef_base,
                                  cudaStream_t s);
cudaError_t launch_rowreduce_batched(bool full, const BatchProblem* P, int nb, int max_rows, int maxN,
                                     cudaStream_t s);
// J_base/F_base: NULL = each problem's own J, F; else outputs at J_off / coef_off.
cudaError_t launch_assemble_batched(bool full, const BatchProblem* P, int nb, double* J_base, double* F_base,
                                    cudaStream_t s);
// Newton step of every active problem (n <= 128): rho = rho_relax for the first
// n_relax steps, 1 after; a problem whose dimensionless residual on entry is
// below tol is marked converged (after its update, as dse_solve does).
cudaError_t prepare_newton_batched(int max_n);  // sets the kernel's shared-memory limit (outside capture)
cudaError_t launch_newton_batched(const BatchProblem* P, int nb, int max_n, double* coef_base, double tol,
                                  double rho_relax, int n_relax, int* n_active, cudaStream_t s);

// Differentiation (dse_adjoint.cu).
constexpr int kDressingVjpMaxSplits = 64;
// dPi: 2 (Rc + 2) scratch; dF (n x 3) and/or vdF = v^T dF (3) are outputs.
cudaError_t launch_param_derivatives(const Consts& c, const Rad* rad, const Ang* ang, const Row* rows,
                                     const YTab* ytab, const double* coef, const double* D, double g2nc,
                                     double* dPi, double* dF, const double* v, double* vdF, cudaStream_t s);
cudaError_t launch_vjp(const Consts& c, const XTab* xtab, const double* phix, const double* D, const double* v,
                       double* out, int* status, cudaStream_t s);
// A <- (S A)^T with S the power-of-two row equilibration (scale: n doubles out);
// then lambda <- S lambda and stats[2] = ||lambda||_inf after the solve.
cudaError_t launch_equilibrate_transpose(int n, double* A, double* scale, cudaStream_t s);
cudaError_t launch_adjoint_finish(int n, const double* scale, double* lam, double* stats, cudaStream_t s);
int dressing_vjp_splits(int n);
// part: dressing_vjp_splits(m) * (n + 1) scratch for m points
cudaError_t launch_dressing_vjp(const Consts& c, int n, const double* x, const double* gG, const double* gZ,
                                double* part, int nsplit, double* out, double* out_g2nc, int* status,
                                cudaStream_t s);
cudaError_t launch_row_prefactors(const Consts& c, Row* rows, int Rt, cudaStream_t s);
// Finite-difference Newton matrix: out (2n x n) = the perturbed vectors c +- h_j e_j;
// J from the 2n residuals Fall (2n x n, same order).
cudaError_t launch_fd_perturb(int n, const double* coef, double rel, double* out, cudaStream_t s);
cudaError_t launch_fd_columns(int n, const double* pert, const double* Fall, double* J, int* status, cudaStream_t s);

}  // namespace dse

// Batch construction without the n <= 128 limit of the batched Newton step (for
// batches that only evaluate residuals, as the finite-difference Newton matrix).
int batch_create_impl(const dse_problem* problems, int n_problems, void* cuda_stream, bool newton,
                      dse_batch** out);
