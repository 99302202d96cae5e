// dse_plan.cu -- plan object and the C ABI entry points declared in include/dse.h.
// Host code only orchestrates: every step of the computation runs in the
// kernels of dse_triple.cu and dse_kernels.cu on the plan's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "dse_internal.cuh"

using namespace dse;

struct dse_plan {
    dse_problem prob;
    Consts c;
    cudaStream_t stream;
    // the series table is built on side while the tables kernel runs on stream
    cudaStream_t side;
    cudaEvent_t fork, join;
    int Rt, KB, KS, nch;
    int KB32, KS32;  // the radial split of the FP32-integrand kernel (mixed precision)
    // fixed workspace (one allocation)
    void* ws;
    Rad* rad;
    Ang* ang;
    double* theta;
    Row* rows;
    double* xcol;
    YTab* ytab;
    double* phiy;
    XTab* xtab;
    double* phix;
    double* Upart;
    double* Vpart;
    double* D;
    double* J;
    double* F;
    double* work;
    SeriesRec* stab;    // series table (read by the FP64 quadrature kernel when use_series_table(N))
    double2* stq;       // the table's node values T_j(s_q) as double-doubles (set-up)
    double* scst;       // the table's interpolation and monomial tables (set-up)
    float* As;          // row-scaled FP32 copy of J (Newton step)
    double2* rowinfo;   // row scales and row sums (Newton step)
    float* Xinv;        // FP32 inverse of the last eliminated Newton step, reused while it suffices
    double* Sinv;       // its row scales
    int* xstate;        // 1 while Xinv is usable, then 2 counters: eliminations, reuses (after the status word);
                        // [4], [5]: the reuse gate's max |Delta| of the last step and before the last failed try
    int* lu_done;       // 1 when the FP32 LU path took the Newton step (n > 160)
    double* aux;        // derivative scratch: dPi rows, dressing-VJP partial sums
    // finite-difference Newton matrix: a batch of 2n copies of the problem
    dse_batch* fd_batch;
    double* fd_buf;     // perturbed vectors (2n x n), then their residuals (2n x n)
    double* stats;  // 4 doubles, followed by the int status word
    int* status;
    // Schwinger-function rule (allocated on first use, per node count)
    int sch_n;
    double* sch;  // gx, gw, inv, pn, wn, sigw
    double* sch_partial;
    size_t sch_partial_cap;
    // pinned host mirror of stats + status
    double* h_misc;
    // the Newton iteration as one CUDA graph: a while node whose body is one
    // Newton step with rho = 1 and FP64 residual, then the decision kernel
    // (captured on cap at the first dse_solve that can use it)
    cudaStream_t cap;
    cudaGraphExec_t sgx;
    int sg_state;            // 0 not built, 1 built, -1 unavailable (host-driven loop)
    long long sg_launches;   // kernels per iteration of the body
    double* coef_g;          // the coefficient vector the body's kernels update
    SolveCtl* ctl;           // device control block
    SolveCtl* h_ctl;         // pinned host copy
    // instrumentation
    long long launches;
    int profiling;
    int n_ev;
    cudaEvent_t ev[2 * 4096];
};

namespace dse {

// Argument checks shared by every entry point that takes a dse_problem.
int check_problem(const dse_problem* p) {
    if (!p) return DSE_ERR_ARG;
    if (p->n_cheb < 1 || p->n_cheb > DSE_MAX_CHEB) return DSE_ERR_ARG;
    if (p->n_cheb_G < 0 || p->n_cheb_G > DSE_MAX_CHEB) return DSE_ERR_ARG;
    if (p->n_radial < 1 || p->n_radial > DSE_MAX_NODES) return DSE_ERR_ARG;
    if (p->n_angular < 1 || p->n_angular > DSE_MAX_NODES) return DSE_ERR_ARG;
    if (!(p->eps2 > 0.0) || !(p->lambda2 > p->eps2) || !isfinite(p->lambda2)) return DSE_ERR_ARG;
    if (!(p->x_Z > 0.0) || !isfinite(p->x_Z) || !(p->x_G >= 0.0) || !isfinite(p->x_G)) return DSE_ERR_ARG;
    if (!isfinite(p->g2nc) || !isfinite(p->kappa) || !isfinite(p->delta) || !isfinite(p->ginv_G) ||
        !isfinite(p->zinv_Z))
        return DSE_ERR_ARG;
    if ((p->radial_mode != 0 && p->radial_mode != 1) || (p->precision != 0 && p->precision != 1))
        return DSE_ERR_UNSUPPORTED;
    if (p->angular_mode != 0 && p->angular_mode != 1) return DSE_ERR_UNSUPPORTED;
    if (p->extrap_mode != 0 && p->extrap_mode != 1) return DSE_ERR_UNSUPPORTED;
    return DSE_OK;
}

// Derived constants of Sec. 2 / Sec. 3 (the series table's interval count from N).
Consts make_consts(const dse_problem* p) {
    constexpr double kPi = 3.14159265358979323846264338327950288;
    Consts c;
    c.NZ = p->n_cheb;
    c.NG = p->n_cheb_G > 0 ? p->n_cheb_G : p->n_cheb;
    c.N = c.NZ > c.NG ? c.NZ : c.NG;
    c.n = c.NZ + c.NG;
    c.Rc = c.NZ == c.NG ? c.N : c.n;
    c.gofs = c.NZ == c.NG ? 0 : c.NZ;
    c.nrule = p->n_radial;
    c.radmode = p->radial_mode;
    c.angmode = p->angular_mode;
    c.sM = series_intervals(c.N);
    c.nr = p->radial_mode == 1 ? 3 * p->n_radial : p->n_radial;
    c.na = p->n_angular;
    c.extrap = p->extrap_mode;
    c.eps2 = p->eps2;
    c.lam2 = p->lambda2;
    c.ln_eps2 = log(p->eps2);
    c.ln_lam2 = log(p->lambda2);
    c.L0 = 0.5 * (c.ln_eps2 + c.ln_lam2);
    c.L1 = 0.5 * (c.ln_lam2 - c.ln_eps2);
    c.invL1 = 1.0 / c.L1;
    c.sL0 = -c.L0 * c.invL1;
    c.K = p->g2nc / (8.0 * kPi * kPi * kPi);
    c.kappa = p->kappa;
    c.delta = p->delta;
    c.gam = -1.0 - 2.0 * p->delta;
    c.pG = -2.0 - 6.0 * p->delta;
    c.qZ = -3.0 * p->delta;
    c.omega = 11.0 * p->g2nc / (48.0 * kPi * kPi);
    c.x_G = p->x_G;
    c.x_Z = p->x_Z;
    c.ginv_G = p->ginv_G;
    c.zinv_Z = p->zinv_Z;
    return c;
}

}  // namespace dse

namespace {


int cuda_status(cudaError_t e) { return e == cudaSuccess ? DSE_OK : DSE_ERR_CUDA; }


size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Radial nodes per block: several waves of Rt * KS blocks over the resident slots,
// so that the block scheduler evens out rows of unequal cost (rows near Lambda^2
// evaluate the UV forms with exponentials for many triples); at least two radial
// nodes per block and at most 128 splits.  Measured at N = 64 with 256 x 128 nodes
// on an earlier version of the kernel: one wave (KS = 11) 0.84 ms per launch,
// KS = 23 / 35 / 47 / 64: 0.81 / 0.78 / 0.76 / 0.74 ms.
#ifndef DSE_SPLIT_WAVES
#define DSE_SPLIT_WAVES 8
#endif
constexpr int kSplitWaves = DSE_SPLIT_WAVES;
// With 128-thread blocks (N <= 96) fewer, longer blocks pay: at N = 64 with 256 x 128
// nodes one Newton matrix took 0.480 / 0.472 / 0.470 / 0.513 ms for 8 / 6 / 4 / 2 waves,
// while at N = 128 (64-thread blocks, 512 x 256 nodes) 5.50 / 5.61 / 5.84 / 6.81 ms.
#ifndef DSE_SPLIT_WAVES_WIDE
#define DSE_SPLIT_WAVES_WIDE 6
#endif
constexpr int kSplitWavesWide = DSE_SPLIT_WAVES_WIDE;
// The FP32-integrand kernel's blocks hold at least this many radial nodes: its
// per-block set-up and final group sums weigh more against its cheaper tiles
// (one Newton matrix at N = 64 with 256 x 128 nodes: 0.529 ms at two nodes per
// block, 0.486 ms at four; eight and sixteen were slower).
#ifndef DSE_MIXED_SPLIT_NODES
#define DSE_MIXED_SPLIT_NODES 4
#endif
constexpr int kMixedSplitNodes = DSE_MIXED_SPLIT_NODES;

void choose_split(dse_plan* pl) {
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int occ = triple_max_blocks_per_sm(true, pl->c.N);
    if (occ < 1) occ = 1;
    const long long slots = (long long)nsm * occ;
    const int nr = pl->c.nr;
    const int waves = triple_block_threads(pl->c.N) == 128 ? kSplitWavesWide : kSplitWaves;
    long long kb = ((long long)nr * pl->Rt) / (waves * slots);
    if (kb < 2) kb = 2;
    if (kb > nr) kb = nr;
    while ((nr + kb - 1) / kb > 128) ++kb;
    pl->KB = (int)kb;
    pl->KS = (int)((nr + kb - 1) / kb);
    const long long kb32 = kb > kMixedSplitNodes ? kb : (kMixedSplitNodes < nr ? kMixedSplitNodes : nr);
    pl->KB32 = (int)kb32;
    pl->KS32 = (int)((nr + kb32 - 1) / kb32);  // <= KS: the split sums fit the same buffer
}

void release_events(dse_plan* pl) {
    for (int i = 0; i < 2 * pl->n_ev; ++i) cudaEventDestroy(pl->ev[i]);
    pl->n_ev = 0;
}

void free_fd(dse_plan* pl) {
    if (pl->fd_batch) dse_batch_destroy(pl->fd_batch);
    if (pl->fd_buf) cudaFree(pl->fd_buf);
    pl->fd_batch = nullptr;
    pl->fd_buf = nullptr;
}

void free_solve_graph(dse_plan* pl) {
    if (pl->sg_state == 1) cudaGraphExecDestroy(pl->sgx);
    pl->sg_state = 0;
}

void free_plan(dse_plan* pl) {
    if (!pl) return;
    free_fd(pl);
    free_solve_graph(pl);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->coef_g) cudaFree(pl->coef_g);
    if (pl->ctl) cudaFree(pl->ctl);
    if (pl->h_ctl) cudaFreeHost(pl->h_ctl);
    release_events(pl);
    if (pl->fork) cudaEventDestroy(pl->fork);
    if (pl->join) cudaEventDestroy(pl->join);
    if (pl->side) cudaStreamDestroy(pl->side);
    if (pl->ws) cudaFree(pl->ws);
    if (pl->sch) cudaFree(pl->sch);
    if (pl->sch_partial) cudaFree(pl->sch_partial);
    if (pl->h_misc) cudaFreeHost(pl->h_misc);
    delete pl;
}

TripleArgs triple_args(const dse_plan* pl, const double* coef) {
    TripleArgs a;
    a.c = pl->c;
    a.Rt = pl->Rt;
    a.KB = pl->KB;
    a.KS = pl->KS;
    a.nch = pl->nch;
    a.rad = pl->rad;
    a.ang = pl->ang;
    a.rows = pl->rows;
    a.ytab = pl->ytab;
    a.coef = coef;
    a.Upart = pl->Upart;
    a.Vpart = pl->Vpart;
    a.stab = use_series_table(pl->c.N) ? pl->stab : nullptr;
    return a;
}

// tables -> quadrature kernel -> per-row contraction (the D vectors).  fp32: the
// FP32-integrand kernel (mixed precision) instead of the FP64 one.
cudaError_t build_rows(dse_plan* pl, const double* coef, bool full, bool fp32) {
    cudaError_t e = cudaSuccess;
    const bool table = use_series_table(pl->c.N);
    if (table) {
        // the series table (independent of the tables kernel) on the side stream
        e = cudaEventRecord(pl->fork, pl->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->side, pl->fork, 0);
        if (e == cudaSuccess) e = launch_series_table(pl->c, coef, pl->stq, pl->scst, pl->stab, pl->side);
        if (e == cudaSuccess) e = cudaEventRecord(pl->join, pl->side);
        pl->launches += 1;
    }
    if (e == cudaSuccess)
        e = launch_tables(pl->c, coef, pl->rad, pl->xcol, pl->ytab, pl->phiy, pl->xtab, pl->phix, pl->stream);
    if (e == cudaSuccess && table) e = cudaStreamWaitEvent(pl->stream, pl->join, 0);
    const bool timed = pl->profiling && pl->n_ev < 4096 && !fp32;
    if (timed && e == cudaSuccess) {
        e = cudaEventCreate(&pl->ev[2 * pl->n_ev]);
        if (e == cudaSuccess) {
            e = cudaEventCreate(&pl->ev[2 * pl->n_ev + 1]);
            if (e != cudaSuccess) cudaEventDestroy(pl->ev[2 * pl->n_ev]);
        }
        if (e == cudaSuccess) e = cudaEventRecord(pl->ev[2 * pl->n_ev], pl->stream);
    }
    TripleArgs a = triple_args(pl, coef);
    if (fp32) {
        a.KB = pl->KB32;
        a.KS = pl->KS32;
    }
    if (e == cudaSuccess) e = fp32 ? launch_triple32(full, a, pl->stream) : launch_triple(full, a, pl->stream);
    if (timed && e == cudaSuccess) {
        e = cudaEventRecord(pl->ev[2 * pl->n_ev + 1], pl->stream);
        ++pl->n_ev;
    }
    pl->launches += 4;
    if (e == cudaSuccess)
        e = launch_rowreduce(full, pl->c, pl->Rt, a.KS, pl->nch, pl->rad, pl->ang, pl->rows, pl->ytab, pl->phiy,
                             pl->Upart, pl->Vpart, pl->D, pl->stream);
    return e;
}

// ... followed by the assembly of J (full) and F; scale: fused with the row
// scaling of the Newton step (plan->As, plan->rowinfo).
int build_system(dse_plan* pl, const double* coef, double* J, double* F, bool full, bool fp32 = false,
                 bool scale = false) {
    cudaError_t e = build_rows(pl, coef, full, fp32);
    if (e == cudaSuccess)
        e = full && scale ? launch_assemble_scale(pl->c, pl->xtab, pl->phix, pl->D, J, F, pl->As, pl->rowinfo,
                                                  pl->status, pl->stream)
                          : launch_assemble(full, pl->c, pl->xtab, pl->phix, pl->D, J, F, pl->status, pl->stream);
    return cuda_status(e);
}

// Newton matrix of the plan's precision: FP64 throughout, or (mixed) J from FP32
// integrands followed by an FP64 residual pass that overwrites F (f64_residual).
int build_newton(dse_plan* pl, const double* coef, double* J, double* F, bool f64_residual, bool scale = false) {
    if (pl->prob.precision == 0) return build_system(pl, coef, J, F, true, false, scale);
    int st = build_system(pl, coef, J, F, true, true, scale);
    if (st || !f64_residual || !F) return st;
    // the FP64 residual pass reuses the tables, writes Upart and the Pi entries of D only
    cudaError_t e = launch_triple(false, triple_args(pl, coef), pl->stream);
    if (e == cudaSuccess)
        e = launch_rowreduce(false, pl->c, pl->Rt, pl->KS, pl->nch, pl->rad, pl->ang, pl->rows, pl->ytab, pl->phiy,
                             pl->Upart, pl->Vpart, pl->D, pl->stream);
    if (e == cudaSuccess) e = launch_assemble(false, pl->c, pl->xtab, pl->phix, pl->D, nullptr, F, pl->status, pl->stream);
    pl->launches += 3;
    return cuda_status(e);
}

int read_status(dse_plan* pl, double* h_stats) {
    cudaError_t e = cudaMemcpyAsync(pl->h_misc, pl->stats, 4 * sizeof(double) + sizeof(int), cudaMemcpyDeviceToHost,
                                    pl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    int st = 0;
    memcpy(&st, pl->h_misc + 4, sizeof(int));
    if (h_stats) memcpy(h_stats, pl->h_misc, 4 * sizeof(double));
    if (st) {
        e = cudaMemsetAsync(pl->status, 0, sizeof(int), pl->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
        if (e != cudaSuccess) return DSE_ERR_CUDA;
    }
    if (st & kStatusSingular) return DSE_ERR_SINGULAR;
    if (st & kStatusNonfinite) return DSE_ERR_NONFINITE;
    return DSE_OK;
}

}  // namespace

extern "C" {

int dse_plan_create(const dse_problem* problem, void* cuda_stream, dse_plan** out) {
    if (!out) return DSE_ERR_ARG;
    *out = nullptr;
    int st = check_problem(problem);
    if (st) return st;
    dse_plan* pl = new (std::nothrow) dse_plan();
    if (!pl) return DSE_ERR_CUDA;
    memset(pl, 0, sizeof(*pl));
    pl->prob = *problem;
    pl->c = make_consts(problem);
    pl->stream = (cudaStream_t)cuda_stream;
    const int N = pl->c.N, nr = pl->c.nr, na = pl->c.na, Rc = pl->c.Rc;
    pl->Rt = Rc + 1 + (problem->x_G > 0.0 ? 1 : 0);
    pl->nch = (na + 31) / 32;
    if (cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->join, cudaEventDisableTiming) != cudaSuccess) {
        free_plan(pl);
        return DSE_ERR_CUDA;
    }
    choose_split(pl);
    const int n = pl->c.n;
    const int nrule = pl->c.nrule;
    const int gmax = nrule > na ? nrule : na;
    const size_t nrad = rad_entries(pl->c);

    size_t off = 0;
    size_t o_rad = off; off = align_up(off + sizeof(Rad) * nrad);
    size_t o_ang = off; off = align_up(off + sizeof(Ang) * na);
    size_t o_th = off; off = align_up(off + sizeof(double) * na);
    size_t o_rows = off; off = align_up(off + sizeof(Row) * pl->Rt);
    size_t o_xcol = off; off = align_up(off + sizeof(double) * Rc);
    size_t o_ytab = off; off = align_up(off + sizeof(YTab) * nrad);
    size_t o_phiy = off; off = align_up(off + sizeof(double) * nrad * N);
    size_t o_xtab = off; off = align_up(off + sizeof(XTab) * Rc);
    size_t o_phix = off; off = align_up(off + sizeof(double) * (size_t)Rc * N);
    size_t o_U = off; off = align_up(off + sizeof(double) * (size_t)pl->Rt * nr * pl->nch * 3);
    size_t o_V = off; off = align_up(off + sizeof(double) * (size_t)pl->Rt * pl->KS * 3 * N);
    size_t o_D = off; off = align_up(off + sizeof(double) * (size_t)(Rc + 2) * ldD(pl->c));
    size_t o_J = off; off = align_up(off + sizeof(double) * (size_t)n * n);
    size_t o_F = off; off = align_up(off + sizeof(double) * n);
    size_t o_work = off; off = align_up(off + sizeof(double) * 2 * n);
    size_t o_stab = off; off = align_up(off + sizeof(SeriesRec) * kSeriesRecords);
    const bool table = use_series_table(N);
    size_t o_stq = off; off = align_up(off + (table ? sizeof(double2) * series_node_values(N) : 0));
    size_t o_scst = off; off = align_up(off + (table ? sizeof(double) * kSeriesConsts : 0));
    size_t o_As = off; off = align_up(off + sizeof(float) * (size_t)n * n);
    size_t o_ri = off; off = align_up(off + sizeof(double2) * n);
    size_t o_X = off; off = align_up(off + (n <= 128 ? sizeof(float) * (size_t)n * n : 0));
    size_t o_S = off; off = align_up(off + sizeof(double) * n);
    const size_t n_aux_a = 2 * (size_t)(Rc + 2) + (size_t)n + 3;
    const size_t n_aux_b = (size_t)kDressingVjpMaxSplits * ((size_t)n + 1);
    size_t o_aux = off; off = align_up(off + sizeof(double) * (n_aux_a > n_aux_b ? n_aux_a : n_aux_b));
    size_t o_misc = off; off = align_up(off + 4 * sizeof(double) + 8 * sizeof(int));
    // Gauss-Legendre scratch (set-up only): nodes/weights for both rules and 1/k
    size_t o_gl = off; off = align_up(off + sizeof(double) * (2 * (size_t)nrule + 2 * (size_t)na + gmax + 2));

    cudaError_t e = cudaMalloc(&pl->ws, off);
    if (e != cudaSuccess) {
        free_plan(pl);
        return DSE_ERR_CUDA;
    }
    char* base = (char*)pl->ws;
    pl->rad = (Rad*)(base + o_rad);
    pl->ang = (Ang*)(base + o_ang);
    pl->theta = (double*)(base + o_th);
    pl->rows = (Row*)(base + o_rows);
    pl->xcol = (double*)(base + o_xcol);
    pl->ytab = (YTab*)(base + o_ytab);
    pl->phiy = (double*)(base + o_phiy);
    pl->xtab = (XTab*)(base + o_xtab);
    pl->phix = (double*)(base + o_phix);
    pl->Upart = (double*)(base + o_U);
    pl->Vpart = (double*)(base + o_V);
    pl->D = (double*)(base + o_D);
    pl->J = (double*)(base + o_J);
    pl->F = (double*)(base + o_F);
    pl->work = (double*)(base + o_work);
    pl->stab = (SeriesRec*)(base + o_stab);
    pl->stq = table ? (double2*)(base + o_stq) : nullptr;
    pl->scst = table ? (double*)(base + o_scst) : nullptr;
    pl->As = (float*)(base + o_As);
    pl->rowinfo = (double2*)(base + o_ri);
    pl->Xinv = n <= 128 ? (float*)(base + o_X) : nullptr;
    pl->Sinv = (double*)(base + o_S);
    pl->aux = (double*)(base + o_aux);
    pl->stats = (double*)(base + o_misc);
    pl->status = (int*)(base + o_misc + 4 * sizeof(double));
    pl->xstate = pl->status + 1;
    pl->lu_done = pl->status + 4;
    double* gl = (double*)(base + o_gl);
    double* glr = gl;
    double* gwr = glr + nrule;
    double* gla = gwr + nrule;
    double* gwa = gla + na;
    double* inv = gwa + na;

    e = cudaMallocHost(&pl->h_misc, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ws, 0, off, pl->stream);
    if (e == cudaSuccess) e = launch_gauss_legendre(nrule, inv, glr, gwr, pl->stream);
    if (e == cudaSuccess) e = launch_gauss_legendre(na, inv, gla, gwa, pl->stream);
    if (e == cudaSuccess)
        e = launch_setup_rules(pl->c, glr, gwr, gla, gwa, pl->rad, pl->ang, pl->theta, pl->xcol, pl->rows, pl->Rt,
                               pl->stream);
    if (e == cudaSuccess && table) e = launch_series_init(pl->c, pl->stq, pl->scst, pl->stab, pl->stream);
    if (e == cudaSuccess) e = prepare_newton_step(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) {
        free_plan(pl);
        return DSE_ERR_CUDA;
    }
    pl->launches = table ? 6 : 5;
    *out = pl;
    return DSE_OK;
}

int dse_plan_destroy(dse_plan* plan) {
    if (!plan) return DSE_OK;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return cuda_status(e);
}

int dse_plan_set_stream(dse_plan* plan, void* cuda_stream) {
    if (!plan) return DSE_ERR_ARG;
    plan->stream = (cudaStream_t)cuda_stream;
    return DSE_OK;
}

int dse_plan_status(dse_plan* plan) {
    if (!plan) return DSE_ERR_ARG;
    return read_status(plan, nullptr);
}

int dse_quadrature(dse_plan* plan, double* d_y, double* d_W, double* d_theta, double* d_wt, double* d_x) {
    if (!plan) return DSE_ERR_ARG;
    const int nr = plan->c.nr, na = plan->c.na, Rc = plan->c.Rc;
    cudaError_t e = cudaSuccess;
    cudaStream_t s = plan->stream;
    // radial_mode 1: the rule of the x_Z row
    const Rad* r0 = plan->rad + rad_offset(plan->c, Rc);
    if (d_y && e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_y, sizeof(double), &r0->y, sizeof(Rad), sizeof(double), nr,
                              cudaMemcpyDeviceToDevice, s);
    if (d_W && e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_W, sizeof(double), &r0->W, sizeof(Rad), sizeof(double), nr,
                              cudaMemcpyDeviceToDevice, s);
    if (d_wt && e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_wt, sizeof(double), &plan->ang->w, sizeof(Ang), sizeof(double), na,
                              cudaMemcpyDeviceToDevice, s);
    if (d_theta && e == cudaSuccess)
        e = cudaMemcpyAsync(d_theta, plan->theta, sizeof(double) * na, cudaMemcpyDeviceToDevice, s);
    if (d_x && e == cudaSuccess) e = cudaMemcpyAsync(d_x, plan->xcol, sizeof(double) * Rc, cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
}

int dse_dressing(dse_plan* plan, const double* d_coeffs, int n, const double* d_x, double* d_lnG, double* d_lnZ) {
    if (!plan || n < 0) return DSE_ERR_ARG;
    if (n == 0) return DSE_OK;
    if (!d_coeffs || !d_x || !d_lnG || !d_lnZ) return DSE_ERR_ARG;
    plan->launches += 1;
    return cuda_status(launch_dressing(plan->c, d_coeffs, n, d_x, d_lnG, d_lnZ, plan->status, plan->stream));
}

int dse_residual(dse_plan* plan, const double* d_coeffs, double* d_F) {
    if (!plan || !d_coeffs || !d_F) return DSE_ERR_ARG;
    return build_system(plan, d_coeffs, nullptr, d_F, false);
}

int dse_newton_matrix(dse_plan* plan, const double* d_coeffs, double* d_J, double* d_F) {
    if (!plan || !d_coeffs || !d_J) return DSE_ERR_ARG;
    return build_newton(plan, d_coeffs, d_J, d_F, true);
}

namespace {
// One Newton step; in mixed precision f64_residual selects the FP64 residual
// (otherwise F comes from the FP32 integrands as well).
int newton_step_impl(dse_plan* plan, double* d_coeffs, double rho, double* h_stats, bool f64_residual) {
    const bool pre = lu_scales_rows(plan->c.n, plan->lu_done != nullptr);
    int st = build_newton(plan, d_coeffs, plan->J, plan->F, f64_residual, pre);
    if (st) return st;
    cudaError_t e = launch_lu_newton(plan->c, plan->J, plan->F, plan->xtab, d_coeffs, rho, plan->work, plan->As,
                                     plan->rowinfo, plan->stats, plan->status, plan->stream, plan->Xinv, plan->Sinv,
                                     plan->xstate, plan->lu_done, pre);
    plan->launches += (plan->c.n <= 128 ? 2 : plan->c.n <= 160 ? 1 : 3) - (pre ? 1 : 0);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    return read_status(plan, h_stats);
}

// Captures the Newton step (rho = 1, FP64 residual) and the decision kernel into
// the body of a while node.  The capture runs on the plan's private stream, so
// that the graph can be launched on any stream, the legacy default one included.
// On any failure the plan keeps the host-driven loop (sg_state = -1).
void build_solve_graph(dse_plan* pl) {
    pl->sg_state = -1;
    const int n = pl->c.n;
    if (!pl->cap && cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) {
        pl->cap = nullptr;
        return;
    }
    if (!pl->coef_g && cudaMalloc(&pl->coef_g, sizeof(double) * n) != cudaSuccess) {
        pl->coef_g = nullptr;
        return;
    }
    if (!pl->ctl && cudaMalloc(&pl->ctl, sizeof(SolveCtl)) != cudaSuccess) {
        pl->ctl = nullptr;
        return;
    }
    if (!pl->h_ctl && cudaMallocHost(&pl->h_ctl, sizeof(SolveCtl)) != cudaSuccess) {
        pl->h_ctl = nullptr;
        return;
    }
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return;
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    cudaGraphNode_t node;
    bool ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const cudaStream_t user = pl->stream;
        const long long l0 = pl->launches;
        pl->stream = pl->cap;
        ok = cudaStreamBeginCaptureToGraph(pl->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            const bool pre = lu_scales_rows(n, pl->lu_done != nullptr);
            int st = build_newton(pl, pl->coef_g, pl->J, pl->F, true, pre);
            cudaError_t e = st ? cudaErrorUnknown
                               : launch_lu_newton(pl->c, pl->J, pl->F, pl->xtab, pl->coef_g, 1.0, pl->work, pl->As,
                                                  pl->rowinfo, pl->stats, pl->status, pl->cap, pl->Xinv, pl->Sinv,
                                                  pl->xstate, pl->lu_done, pre);
            pl->launches += (n <= 128 ? 2 : n <= 160 ? 1 : 3) - (pre ? 1 : 0);
            if (e == cudaSuccess) e = launch_solve_decide(pl->ctl, pl->stats, pl->status, cond, pl->cap);
            cudaGraph_t out = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(pl->cap, &out);
            ok = e == cudaSuccess && ec == cudaSuccess;
        }
        pl->sg_launches = pl->launches - l0 + 1;
        pl->launches = l0;
        pl->stream = user;
    }
    if (ok) ok = cudaGraphInstantiate(&pl->sgx, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
    if (ok) pl->sg_state = 1;
}

// Runs at most max_steps Newton steps through the graph: copies the coefficients
// in, launches the while node, copies them back and reads the control block.
// Returns DSE_OK (converged), DSE_ERR_NOT_CONVERGED (step limit) or the status
// of the step that stopped it; *taken = the steps run, st4 = their last stats.
int run_solve_graph(dse_plan* pl, double* d_coeffs, double tol, int max_steps, int* taken, double* st4) {
    const cudaStream_t s = pl->stream;
    const int n = pl->c.n;
    *taken = 0;
    cudaError_t e = launch_solve_begin(pl->ctl, tol, max_steps, d_coeffs, pl->coef_g, n, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(pl->sgx, s);
    if (e == cudaSuccess) e = launch_solve_end(pl->coef_g, d_coeffs, n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl->h_ctl, pl->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    const SolveCtl& h = *pl->h_ctl;
    *taken = h.steps;
    memcpy(st4, h.stats, 4 * sizeof(double));
    pl->launches += 2 + (long long)h.steps * pl->sg_launches;
    if (h.status) {
        e = cudaMemsetAsync(pl->status, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return DSE_ERR_CUDA;
        if (h.status & kStatusSingular) return DSE_ERR_SINGULAR;
        if (h.status & kStatusNonfinite) return DSE_ERR_NONFINITE;
    }
    return h.converged ? DSE_OK : DSE_ERR_NOT_CONVERGED;
}
}  // namespace

int dse_newton_step(dse_plan* plan, double* d_coeffs, double rho, double* h_stats) {
    if (!plan || !d_coeffs || !isfinite(rho)) return DSE_ERR_ARG;
    return newton_step_impl(plan, d_coeffs, rho, h_stats, true);
}

int dse_solve(dse_plan* plan, double* d_coeffs, double tol, int max_iter, double rho_relax, int n_relax,
              int* h_iters, double* h_stats) {
    if (!plan || !d_coeffs || !(tol > 0.0) || max_iter < 1 || !isfinite(rho_relax) || n_relax < 0) return DSE_ERR_ARG;
    double st3[4] = {0.0, 0.0, 0.0, 0.0};
    int it = 0;
    int st = DSE_ERR_NOT_CONVERGED;
    // mixed precision: FP32 residual while the dimensionless residual is above
    // kSwitch and still falling by at least a half per step (FP32 rounding has
    // not become the floor), FP64 residual after
    const double kSwitch = 1e-5;
    bool f64_res = plan->prob.precision == 0;
    double prev = INFINITY;
    // every solve starts without a kept inverse (and without the record of the last
    // failed attempt to reuse one), so its steps depend on its input alone
    if (cudaMemsetAsync(plan->xstate, 0, sizeof(int), plan->stream) != cudaSuccess ||
        cudaMemsetAsync(plan->xstate + 4, 0, 2 * sizeof(int), plan->stream) != cudaSuccess)
        return DSE_ERR_CUDA;
    for (; it < max_iter; ++it) {
        // past the relaxed steps and the FP32 residuals, the remaining steps run as
        // one CUDA graph with the stopping test on the device (no host round trip per
        // step); the host loop serves instrumented plans, whose events a graph body
        // cannot hold
        if (f64_res && it >= n_relax && !plan->profiling) {
            if (plan->sg_state == 0) build_solve_graph(plan);
            if (plan->sg_state == 1) {
                int taken = 0;
                st = run_solve_graph(plan, d_coeffs, tol, max_iter - it, &taken, st3);
                it += taken;
                break;
            }
        }
        const double rho = it < n_relax ? rho_relax : 1.0;
        const int s = newton_step_impl(plan, d_coeffs, rho, st3, f64_res);
        if (!s && !f64_res && (st3[1] < kSwitch || (it >= n_relax && st3[1] > 0.5 * prev))) {
            // this step's residual was FP32: continue from here with FP64 residuals
            f64_res = true;
            continue;
        }
        prev = st3[1];
        if (s) {
            st = s;
            ++it;
            break;
        }
        if (st3[1] < tol) {
            st = DSE_OK;
            ++it;
            break;
        }
    }
    if (h_iters) *h_iters = it;
    if (h_stats) memcpy(h_stats, st3, 3 * sizeof(double));
    return st;
}

int dse_schwinger(dse_plan* plan, const double* d_coeffs, const double* d_t, int n_t, int n_nodes, double* d_delta) {
    if (!plan || !d_coeffs || n_t < 0 || n_nodes < 1 || n_nodes > DSE_MAX_SCHWINGER_NODES) return DSE_ERR_ARG;
    if (n_t > 0 && (!d_t || !d_delta)) return DSE_ERR_ARG;
    cudaError_t e = cudaSuccess;
    cudaStream_t s = plan->stream;
    if (plan->sch_n != n_nodes) {
        if (plan->sch) {
            e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaFree(plan->sch);
            plan->sch = nullptr;
            plan->sch_n = 0;
            if (e != cudaSuccess) return DSE_ERR_CUDA;
        }
        e = cudaMalloc(&plan->sch, sizeof(double) * (6 * (size_t)n_nodes + 2));
        if (e != cudaSuccess) {
            plan->sch = nullptr;
            return DSE_ERR_CUDA;
        }
        double* gx = plan->sch;
        double* gw = gx + n_nodes;
        double* pn = gw + n_nodes;
        double* wn = pn + n_nodes;
        double* inv = wn + 2 * (size_t)n_nodes;  // n + 2 doubles (overlaps nothing live)
        e = launch_gauss_legendre(n_nodes, inv, gx, gw, s);
        if (e == cudaSuccess) e = launch_schwinger_map(plan->c, n_nodes, gx, gw, pn, wn, s);
        plan->launches += 3;
        if (e != cudaSuccess) return DSE_ERR_CUDA;
        plan->sch_n = n_nodes;
    }
    const int nsplit = schwinger_splits(n_t, n_nodes);
    const size_t need = (size_t)nsplit * (size_t)(n_t > 0 ? n_t : 1);
    if (need > plan->sch_partial_cap) {
        if (plan->sch_partial) {
            e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaFree(plan->sch_partial);
            plan->sch_partial = nullptr;
            plan->sch_partial_cap = 0;
            if (e != cudaSuccess) return DSE_ERR_CUDA;
        }
        e = cudaMalloc(&plan->sch_partial, sizeof(double) * need);
        if (e != cudaSuccess) return DSE_ERR_CUDA;
        plan->sch_partial_cap = need;
    }
    double* pn = plan->sch + 2 * (size_t)n_nodes;
    double* wn = pn + n_nodes;
    double* sigw = wn + n_nodes;
    e = launch_schwinger(plan->c, d_coeffs, n_nodes, pn, wn, sigw, d_t, n_t, plan->sch_partial, nsplit, d_delta,
                         plan->status, s);
    plan->launches += n_t > 0 ? 3 : 1;
    return cuda_status(e);
}

int dse_plan_set_couplings(dse_plan* plan, double g2nc, double ginv_G, double zinv_Z) {
    if (!plan) return DSE_ERR_ARG;
    dse_problem p = plan->prob;
    p.g2nc = g2nc;
    p.ginv_G = ginv_G;
    p.zinv_Z = zinv_Z;
    const int st = check_problem(&p);
    if (st) return st;
    plan->prob = p;
    plan->c = make_consts(&p);
    free_solve_graph(plan);  // its kernels hold the old constants
    plan->launches += 1;
    if (plan->fd_batch) {
        cudaError_t e = cudaStreamSynchronize(plan->stream);
        free_fd(plan);
        if (e != cudaSuccess) return DSE_ERR_CUDA;
    }
    return cuda_status(launch_row_prefactors(plan->c, plan->rows, plan->Rt, plan->stream));
}

int dse_vjp(dse_plan* plan, const double* d_coeffs, const double* d_v, double* d_out, double* d_F) {
    if (!plan || !d_coeffs || !d_v || !d_out) return DSE_ERR_ARG;
    cudaError_t e = build_rows(plan, d_coeffs, true, false);
    if (e == cudaSuccess && d_F)
        e = launch_assemble(false, plan->c, plan->xtab, plan->phix, plan->D, nullptr, d_F, plan->status, plan->stream);
    if (e == cudaSuccess) e = launch_vjp(plan->c, plan->xtab, plan->phix, plan->D, d_v, d_out, plan->status, plan->stream);
    plan->launches += d_F ? 2 : 1;
    return cuda_status(e);
}

int dse_param_derivatives(dse_plan* plan, const double* d_coeffs, double* d_dF, const double* d_v, double* d_vdF) {
    if (!plan || !d_coeffs || (!d_dF && !d_v) || (!d_v != !d_vdF)) return DSE_ERR_ARG;
    if (!(plan->prob.g2nc != 0.0)) return DSE_ERR_ARG;
    cudaError_t e = build_rows(plan, d_coeffs, false, false);
    if (e == cudaSuccess)
        e = launch_param_derivatives(plan->c, plan->rad, plan->ang, plan->rows, plan->ytab, d_coeffs, plan->D,
                                     plan->prob.g2nc, plan->aux, d_dF, d_v, d_vdF, plan->stream);
    plan->launches += 2;
    return cuda_status(e);
}

int dse_adjoint_solve(dse_plan* plan, const double* d_coeffs, const double* d_g, double* d_lambda, double* h_stats) {
    if (!plan || !d_coeffs || !d_g || !d_lambda) return DSE_ERR_ARG;
    const int n = plan->c.n;
    int st = build_system(plan, d_coeffs, plan->J, plan->F, true, false);
    if (st) return st;
    // (S J)^T mu = g with S the power-of-two row equilibration of J, lambda = S mu
    cudaError_t e = launch_equilibrate_transpose(n, plan->J, plan->aux, plan->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_lambda, 0, sizeof(double) * n, plan->stream);
    // mu = 0 - (-1) Delta with (S J)^T Delta = g
    if (e == cudaSuccess)
        e = launch_lu_newton(plan->c, plan->J, d_g, plan->xtab, d_lambda, -1.0, plan->work, plan->As, plan->rowinfo,
                             plan->stats, plan->status, plan->stream);
    if (e == cudaSuccess) e = launch_adjoint_finish(n, plan->aux, d_lambda, plan->stats, plan->stream);
    plan->launches += n <= 128 ? 5 : 4;
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    return read_status(plan, h_stats);
}

int dse_newton_matrix_fd(dse_plan* plan, const double* d_coeffs, double rel_step, double* d_J, double* d_F) {
    if (!plan || !d_coeffs || !d_J || !(rel_step > 0.0) || !isfinite(rel_step)) return DSE_ERR_ARG;
    const int n = plan->c.n;
    if (!plan->fd_batch) {
        dse_problem q = plan->prob;
        q.precision = 0;
        dse_problem* probs = new (std::nothrow) dse_problem[2 * (size_t)n];
        if (!probs) return DSE_ERR_CUDA;
        for (int v = 0; v < 2 * n; ++v) probs[v] = q;
        int st = batch_create_impl(probs, 2 * n, plan->stream, false, &plan->fd_batch);
        delete[] probs;
        if (st) {
            plan->fd_batch = nullptr;
            return st;
        }
        if (cudaMalloc(&plan->fd_buf, sizeof(double) * 4 * (size_t)n * n) != cudaSuccess) {
            plan->fd_buf = nullptr;
            free_fd(plan);
            return DSE_ERR_CUDA;
        }
    }
    dse_batch_set_stream(plan->fd_batch, plan->stream);
    double* pert = plan->fd_buf;
    double* Fall = plan->fd_buf + 2 * (size_t)n * n;
    cudaError_t e = launch_fd_perturb(n, d_coeffs, rel_step, pert, plan->stream);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    int st = dse_batch_residual(plan->fd_batch, pert, Fall);
    if (st) return st;
    e = launch_fd_columns(n, pert, Fall, d_J, plan->status, plan->stream);
    plan->launches += 2;
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    if (d_F) return build_system(plan, d_coeffs, nullptr, d_F, false, false);
    return DSE_OK;
}

int dse_dressing_vjp(dse_plan* plan, int n, const double* d_x, const double* d_gG, const double* d_gZ, double* d_out,
                     double* d_out_g2nc) {
    if (!plan || n < 0 || !d_out) return DSE_ERR_ARG;
    if (n > 0 && (!d_x || !d_gG || !d_gZ)) return DSE_ERR_ARG;
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(d_out, 0, sizeof(double) * plan->c.n, plan->stream);
        if (e == cudaSuccess && d_out_g2nc) e = cudaMemsetAsync(d_out_g2nc, 0, sizeof(double), plan->stream);
        return cuda_status(e);
    }
    const int nsplit = dressing_vjp_splits(n);
    e = launch_dressing_vjp(plan->c, n, d_x, d_gG, d_gZ, plan->aux, nsplit, d_out, d_out_g2nc, plan->status,
                            plan->stream);
    plan->launches += 2;
    return cuda_status(e);
}

int dse_plan_profile(dse_plan* plan, int enable) {
    if (!plan) return DSE_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    release_events(plan);
    plan->profiling = enable != 0;
    return cuda_status(e);
}

int dse_plan_counters(dse_plan* plan, long long* h_launches, int* h_timed, double* h_timed_ms) {
    if (!plan) return DSE_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    double total = 0.0;
    for (int i = 0; i < plan->n_ev; ++i) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, plan->ev[2 * i], plan->ev[2 * i + 1]);
        if (e != cudaSuccess) return DSE_ERR_CUDA;
        total += ms;
    }
    long long fd_launches = 0;
    if (plan->fd_batch) dse_batch_counters(plan->fd_batch, &fd_launches, nullptr, nullptr);
    if (h_launches) *h_launches = plan->launches + fd_launches;
    if (h_timed) *h_timed = plan->n_ev;
    if (h_timed_ms) *h_timed_ms = total;
    return DSE_OK;
}

int dse_plan_solver_counters(dse_plan* plan, int* h_eliminations, int* h_reused) {
    if (!plan) return DSE_ERR_ARG;
    int v[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(v, plan->xstate + 1, sizeof(v), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    if (h_eliminations) *h_eliminations = v[0];
    if (h_reused) *h_reused = v[1];
    return DSE_OK;
}

const char* dse_status_string(int status) {
    switch (status) {
        case DSE_OK: return "ok";
        case DSE_ERR_ARG: return "invalid argument";
        case DSE_ERR_NONFINITE: return "non-finite value in residual, matrix or update";
        case DSE_ERR_SINGULAR: return "singular Newton matrix";
        case DSE_ERR_CUDA: return "CUDA runtime error";
        case DSE_ERR_UNSUPPORTED: return "unsupported mode";
        case DSE_ERR_NOT_CONVERGED: return "Newton iteration did not converge";
        default: return "unknown status";
    }
}

}  // extern "C"
