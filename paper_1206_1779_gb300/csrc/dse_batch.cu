// dse_batch.cu -- batches of independent problems (a parameter sweep): every
// problem keeps its own orders N_Z, N_G, quadrature sizes and boundary values;
// one Newton step of the whole batch is one CUDA graph of seven launches, with the
// quadrature over all problems in one persistent kernel (dse_triple.cu) that
// takes (problem, row, radial split) items from a global counter, longest first.
// The number of radial nodes per item is chosen by timing candidates
// (dse_batch_tune).  Host code only orchestrates.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dse_internal.cuh"

using namespace dse;

struct dse_batch {
    int nb;
    std::vector<dse_problem> probs;
    std::vector<BatchProblem> h_P;   // descriptors with the initial iteration state
    std::vector<long long> coef_off;  // nb + 1
    std::vector<long long> J_off;     // nb + 1
    cudaStream_t stream;              // the caller's stream
    cudaStream_t cap;                 // internal stream for graph capture
    void* ws;
    BatchProblem* d_P;
    BatchItem* d_items;
    int n_items;
    int items_cap;
    int* d_counter;
    int* d_nactive;
    double* d_stats_out;              // nb x 4 gathered stats
    int* h_nactive;                   // pinned
    int maxN, max_n, max_rows, max_units;
    int grid;                         // persistent quadrature grid
    int units;                        // radial nodes per work item
    int min_units;                    // smallest candidate (sizes Vpart)
    // captured Newton step
    cudaGraphExec_t exec;
    bool have_graph;
    double g_tol, g_rho;
    int g_nrelax;
    double* g_coef;
    long long launches;
    long long graph_launches;
};

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kTuneCandidates[] = {8, 16, 32, 64, 128};
constexpr int kDefaultUnits = 16;

int cuda_status(cudaError_t e) { return e == cudaSuccess ? DSE_OK : DSE_ERR_CUDA; }

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int check_batch_problem(const dse_problem* p, bool newton) {
    if (p->n_cheb < 1 || p->n_cheb > DSE_MAX_CHEB || p->n_cheb_G < 0 || p->n_cheb_G > DSE_MAX_CHEB) return DSE_ERR_ARG;
    if (p->n_radial < 1 || p->n_radial > DSE_MAX_NODES || p->n_angular < 1 || p->n_angular > DSE_MAX_NODES)
        return DSE_ERR_ARG;
    if (!(p->eps2 > 0.0) || !(p->lambda2 > p->eps2) || !isfinite(p->lambda2)) return DSE_ERR_ARG;
    if (!(p->x_Z > 0.0) || !isfinite(p->x_Z) || !(p->x_G >= 0.0) || !isfinite(p->x_G)) return DSE_ERR_ARG;
    if (!isfinite(p->g2nc) || !isfinite(p->kappa) || !isfinite(p->delta) || !isfinite(p->ginv_G) ||
        !isfinite(p->zinv_Z))
        return DSE_ERR_ARG;
    if ((p->radial_mode != 0 && p->radial_mode != 1) || p->precision != 0) return DSE_ERR_UNSUPPORTED;
    if (p->angular_mode != 0 && p->angular_mode != 1) return DSE_ERR_UNSUPPORTED;
    if (p->extrap_mode != 0 && p->extrap_mode != 1) return DSE_ERR_UNSUPPORTED;
    const int ng = p->n_cheb_G > 0 ? p->n_cheb_G : p->n_cheb;
    if (newton && p->n_cheb + ng > 128) return DSE_ERR_UNSUPPORTED;  // the batched Newton step holds n <= 128
    return DSE_OK;
}

Consts batch_consts(const dse_problem* p) {
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
    c.nr = p->radial_mode == 1 ? 3 * p->n_radial : p->n_radial;
    c.sM = series_intervals(c.N);
    c.na = p->n_angular;
    c.extrap = p->extrap_mode;
    c.eps2 = p->eps2;
    c.lam2 = p->lambda2;
    c.ln_eps2 = log(p->eps2);
    c.ln_lam2 = log(p->lambda2);
    c.L0 = 0.5 * (c.ln_eps2 + c.ln_lam2);
    c.L1 = 0.5 * (c.ln_lam2 - c.ln_eps2);
    c.invL1 = 1.0 / c.L1;
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

// Per-problem workspace layout; Vpart sized for ks_cap radial splits.
struct Slice {
    size_t rad, ang, theta, rows, xcol, ytab, phiy, xtab, phix, U, V, D, J, F, work, As, ri, X, S, stats, stab, gl,
        total;
};

Slice slice_layout(const Consts& c, int Rt, int nch, int ks_cap) {
    Slice L;
    size_t off = 0;
    const int N = c.N, n = c.n, nr = c.nr, na = c.na, Rc = c.Rc;
    const size_t nrad = rad_entries(c);
    L.rad = off; off = up256(off + sizeof(Rad) * nrad);
    L.ang = off; off = up256(off + sizeof(Ang) * (size_t)na);
    L.theta = off; off = up256(off + sizeof(double) * (size_t)na);
    L.rows = off; off = up256(off + sizeof(Row) * (size_t)Rt);
    L.xcol = off; off = up256(off + sizeof(double) * (size_t)Rc);
    L.ytab = off; off = up256(off + sizeof(YTab) * nrad);
    L.phiy = off; off = up256(off + sizeof(double) * nrad * N);
    L.xtab = off; off = up256(off + sizeof(XTab) * (size_t)Rc);
    L.phix = off; off = up256(off + sizeof(double) * (size_t)Rc * N);
    L.U = off; off = up256(off + sizeof(double) * (size_t)Rt * nr * nch * 3);
    L.V = off; off = up256(off + sizeof(double) * (size_t)Rt * ks_cap * 3 * N);
    L.D = off; off = up256(off + sizeof(double) * (size_t)(Rc + 2) * ldD(c));
    L.J = off; off = up256(off + sizeof(double) * (size_t)n * n);
    L.F = off; off = up256(off + sizeof(double) * (size_t)n);
    L.work = off; off = up256(off + sizeof(double) * 2 * (size_t)n);
    L.As = off; off = up256(off + sizeof(float) * (size_t)n * n);
    L.ri = off; off = up256(off + sizeof(double2) * (size_t)n);
    L.X = off; off = up256(off + (n <= 128 ? sizeof(float) * (size_t)n * n : 0));
    L.S = off; off = up256(off + sizeof(double) * (size_t)n);
    L.stats = off; off = up256(off + 4 * sizeof(double) + sizeof(int));
    L.stab = off; off = up256(off + (use_series_table(c.N) ? sizeof(SeriesRec) * kSeriesRecords : 0));
    const size_t nrule = c.nrule;
    const size_t gmax = nrule > (size_t)na ? nrule : (size_t)na;
    L.gl = off; off = up256(off + sizeof(double) * (2 * nrule + 2 * (size_t)na + gmax + 2));
    L.total = off;
    return L;
}

// Reset every problem's iteration state and status word.
__global__ void k_batch_reset(BatchProblem* __restrict__ P, int nb, int* __restrict__ n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) {
        P[b].iter = 0;
        P[b].active = 1;
        P[b].result = 0;
        P[b].xstate = 0;
        *P[b].status = 0;
    }
    if (b == 0) *n_active = nb;
}

__global__ void k_batch_gather(const BatchProblem* __restrict__ P, int nb, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int q = 0; q < 4; ++q) out[4 * b + q] = P[b].stats[q];
}

void free_batch(dse_batch* B) {
    if (!B) return;
    if (B->have_graph) cudaGraphExecDestroy(B->exec);
    if (B->ws) cudaFree(B->ws);
    if (B->h_nactive) cudaFreeHost(B->h_nactive);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
}

// Work items for the given radial nodes per item, longest first; descriptors
// get the matching KB, KS.  Items are ordered by (cost desc, problem, row,
// split), so the list is the same on every call.
void build_items(dse_batch* B, int units, std::vector<BatchItem>& items) {
    struct Keyed { double cost; BatchItem w; };
    std::vector<Keyed> v;
    for (int b = 0; b < B->nb; ++b) {
        BatchProblem& P = B->h_P[b];
        const int nr = P.t.c.nr;
        const int KB = units < nr ? units : nr;
        const int KS = (nr + KB - 1) / KB;
        P.t.KB = KB;
        P.t.KS = KS;
        for (int rt = 0; rt < P.t.Rt; ++rt)
            for (int ks = 0; ks < KS; ++ks) {
                const int k0 = ks * KB;
                const int kn = (k0 + KB < nr ? KB : nr - k0);
                Keyed e;
                e.cost = (double)kn * P.t.nch * (P.t.c.N + 8.0);
                e.w.b = b;
                e.w.rt = rt;
                e.w.ks = ks;
                e.w.pad = 0;
                v.push_back(e);
            }
    }
    std::stable_sort(v.begin(), v.end(), [](const Keyed& a, const Keyed& b) { return a.cost > b.cost; });
    items.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) items[i] = v[i].w;
}

int set_units(dse_batch* B, int units) {
    std::vector<BatchItem> items;
    build_items(B, units, items);
    if ((int)items.size() > B->items_cap) return DSE_ERR_ARG;
    B->n_items = (int)items.size();
    B->units = units;
    cudaError_t e = cudaMemcpyAsync(B->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                    cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_P, B->h_P.data(), sizeof(BatchProblem) * B->nb, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (B->have_graph) {
        cudaGraphExecDestroy(B->exec);
        B->have_graph = false;
    }
    return cuda_status(e);
}

// One Newton matrix of every active problem: tables, quadrature, contraction, assembly.
cudaError_t enqueue_matrix(dse_batch* B, const double* coef, double* J_base, double* F_base, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_tables_batched(B->d_P, B->nb, B->max_units, coef, s);
    if (e == cudaSuccess) e = launch_series_table_batched(B->d_P, B->nb, coef, s);
    if (e == cudaSuccess)
        e = launch_triple_batched(true, B->d_P, B->d_items, B->n_items, B->d_counter, coef, B->maxN, B->grid, s);
    if (e == cudaSuccess) e = launch_rowreduce_batched(true, B->d_P, B->nb, B->max_rows, B->maxN, s);
    if (e == cudaSuccess) e = launch_assemble_batched(true, B->d_P, B->nb, J_base, F_base, s);
    return e;
}

// Residuals only (no derivative sums, no Newton matrix).
cudaError_t enqueue_residual(dse_batch* B, const double* coef, double* F_base, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_tables_batched(B->d_P, B->nb, B->max_units, coef, s);
    if (e == cudaSuccess) e = launch_series_table_batched(B->d_P, B->nb, coef, s);
    if (e == cudaSuccess)
        e = launch_triple_batched(false, B->d_P, B->d_items, B->n_items, B->d_counter, coef, B->maxN, B->grid, s);
    if (e == cudaSuccess) e = launch_rowreduce_batched(false, B->d_P, B->nb, B->max_rows, B->maxN, s);
    if (e == cudaSuccess) e = launch_assemble_batched(false, B->d_P, B->nb, nullptr, F_base, s);
    return e;
}

cudaError_t enqueue_step(dse_batch* B, double* coef, double tol, double rho_relax, int n_relax, cudaStream_t s) {
    cudaError_t e = enqueue_matrix(B, coef, nullptr, nullptr, s);
    if (e == cudaSuccess)
        e = launch_newton_batched(B->d_P, B->nb, B->max_n, coef, tol, rho_relax, n_relax, B->d_nactive, s);
    return e;
}

int capture_step(dse_batch* B, double* coef, double tol, double rho_relax, int n_relax) {
    if (B->have_graph && B->g_coef == coef && B->g_tol == tol && B->g_rho == rho_relax && B->g_nrelax == n_relax)
        return DSE_OK;
    if (B->have_graph) {
        cudaGraphExecDestroy(B->exec);
        B->have_graph = false;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    cudaError_t e2 = enqueue_step(B, coef, tol, rho_relax, n_relax, B->cap);
    e = cudaStreamEndCapture(B->cap, &g);
    if (e2 != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return DSE_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    B->have_graph = true;
    B->g_coef = coef;
    B->g_tol = tol;
    B->g_rho = rho_relax;
    B->g_nrelax = n_relax;
    return DSE_OK;
}

}  // namespace

// Batch of problems for which only residuals and Newton matrices will be asked
// (newton = false lifts the n <= 128 limit of the batched Newton step).
int batch_create_impl(const dse_problem* problems, int n_problems, void* cuda_stream, bool newton,
                      dse_batch** out) {
    if (!out) return DSE_ERR_ARG;
    *out = nullptr;
    if (!problems || n_problems < 1 || n_problems > 65535) return DSE_ERR_ARG;
    for (int b = 0; b < n_problems; ++b) {
        const int st = check_batch_problem(&problems[b], newton);
        if (st) return st;
    }
    dse_batch* B = new (std::nothrow) dse_batch();
    if (!B) return DSE_ERR_CUDA;
    B->nb = n_problems;
    B->probs.assign(problems, problems + n_problems);
    B->stream = (cudaStream_t)cuda_stream;
    B->ws = nullptr;
    B->cap = nullptr;
    B->h_nactive = nullptr;
    B->have_graph = false;
    B->launches = 0;
    B->graph_launches = 0;
    B->min_units = kTuneCandidates[0];
    cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        B->cap = nullptr;
        free_batch(B);
        return DSE_ERR_CUDA;
    }

    // layout of every slice, then one allocation
    std::vector<Slice> L(n_problems);
    std::vector<size_t> base(n_problems);
    size_t off = 0;
    B->h_P.resize(n_problems);
    B->coef_off.assign(n_problems + 1, 0);
    B->J_off.assign(n_problems + 1, 0);
    B->maxN = B->max_n = B->max_rows = B->max_units = 0;
    int items_cap = 0;
    for (int b = 0; b < n_problems; ++b) {
        const Consts c = batch_consts(&problems[b]);
        const int Rt = c.Rc + 1 + (problems[b].x_G > 0.0 ? 1 : 0);
        const int nch = (c.na + 31) / 32;
        const int ks_cap = (c.nr + B->min_units - 1) / B->min_units;
        L[b] = slice_layout(c, Rt, nch, ks_cap);
        base[b] = off;
        off = up256(off + L[b].total);
        B->coef_off[b + 1] = B->coef_off[b] + c.n;
        B->J_off[b + 1] = B->J_off[b] + (long long)c.n * c.n;
        B->maxN = std::max(B->maxN, c.N);
        B->max_n = std::max(B->max_n, c.n);
        B->max_rows = std::max(B->max_rows, c.Rc + 2);
        B->max_units = std::max(B->max_units, (int)rad_entries(c) + c.Rc);
        items_cap += Rt * ks_cap;
        BatchProblem& P = B->h_P[b];
        memset(&P, 0, sizeof(P));
        P.t.c = c;
        P.t.Rt = Rt;
        P.t.nch = nch;
        P.coef_off = B->coef_off[b];
        P.J_off = B->J_off[b];
        P.iter = 0;
        P.active = 1;
        P.result = 0;
    }
    const size_t o_P = off;
    off = up256(off + sizeof(BatchProblem) * n_problems);
    const size_t o_items = off;
    off = up256(off + sizeof(BatchItem) * (size_t)items_cap);
    const size_t o_misc = off;
    off = up256(off + 2 * sizeof(int));
    const size_t o_stats = off;
    off = up256(off + 4 * sizeof(double) * n_problems);
    e = cudaMalloc(&B->ws, off);
    if (e != cudaSuccess) {
        B->ws = nullptr;
        free_batch(B);
        return DSE_ERR_CUDA;
    }
    e = cudaMallocHost(&B->h_nactive, sizeof(int));
    if (e != cudaSuccess) {
        B->h_nactive = nullptr;
        free_batch(B);
        return DSE_ERR_CUDA;
    }
    char* w = (char*)B->ws;
    B->d_P = (BatchProblem*)(w + o_P);
    B->d_items = (BatchItem*)(w + o_items);
    B->items_cap = items_cap;
    B->d_counter = (int*)(w + o_misc);
    B->d_nactive = B->d_counter + 1;
    B->d_stats_out = (double*)(w + o_stats);
    e = cudaMemsetAsync(B->ws, 0, off, B->stream);

    // set-up kernels of every problem (rules, collocation points, rows)
    for (int b = 0; b < n_problems && e == cudaSuccess; ++b) {
        BatchProblem& P = B->h_P[b];
        char* s = w + base[b];
        const Slice& S = L[b];
        P.t.rad = (Rad*)(s + S.rad);
        P.t.ang = (Ang*)(s + S.ang);
        P.t.rows = (Row*)(s + S.rows);
        P.ytab = (YTab*)(s + S.ytab);
        P.t.ytab = P.ytab;
        P.t.coef = nullptr;
        P.t.Upart = (double*)(s + S.U);
        P.t.Vpart = (double*)(s + S.V);
        P.xcol = (double*)(s + S.xcol);
        P.phiy = (double*)(s + S.phiy);
        P.xtab = (XTab*)(s + S.xtab);
        P.phix = (double*)(s + S.phix);
        P.D = (double*)(s + S.D);
        P.J = (double*)(s + S.J);
        P.F = (double*)(s + S.F);
        P.work = (double*)(s + S.work);
        P.As = (float*)(s + S.As);
        P.rowinfo = (double2*)(s + S.ri);
        P.Xinv = P.t.c.n <= 128 ? (float*)(s + S.X) : nullptr;
        P.Sinv = (double*)(s + S.S);
        P.stats = (double*)(s + S.stats);
        P.status = (int*)(s + S.stats + 4 * sizeof(double));
        P.stab = use_series_table(P.t.c.N) ? (SeriesRec*)(s + S.stab) : nullptr;
        P.t.stab = P.stab;
        const Consts& c = P.t.c;
        double* gl = (double*)(s + S.gl);
        double* glr = gl;
        double* gwr = glr + c.nrule;
        double* gla = gwr + c.nrule;
        double* gwa = gla + c.na;
        double* inv = gwa + c.na;
        e = launch_gauss_legendre(c.nrule, inv, glr, gwr, B->stream);
        if (e == cudaSuccess) e = launch_gauss_legendre(c.na, inv, gla, gwa, B->stream);
        if (e == cudaSuccess)
            e = launch_setup_rules(c, glr, gwr, gla, gwa, (Rad*)P.t.rad, (Ang*)P.t.ang, (double*)(s + S.theta), P.xcol,
                                   (Row*)P.t.rows, P.t.Rt, B->stream);
        B->launches += 5;
    }
    if (e != cudaSuccess) {
        free_batch(B);
        return DSE_ERR_CUDA;
    }
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // (the occupancy query also sets the kernels' shared-memory limits, so that
    // no attribute changes fall inside a graph capture)
    int occ = triple_batched_blocks_per_sm(true, B->maxN);
    if (occ < 1) occ = 1;
    B->grid = nsm * occ;
    if (B->max_n <= 128 && prepare_newton_batched(B->max_n) != cudaSuccess) {
        free_batch(B);
        return DSE_ERR_CUDA;
    }
    const int st = set_units(B, kDefaultUnits);
    if (st) {
        free_batch(B);
        return st;
    }
    *out = B;
    return DSE_OK;
}

extern "C" {

int dse_batch_create(const dse_problem* problems, int n_problems, void* cuda_stream, dse_batch** out) {
    return batch_create_impl(problems, n_problems, cuda_stream, true, out);
}

int dse_batch_destroy(dse_batch* batch) {
    if (!batch) return DSE_OK;
    cudaError_t e = cudaStreamSynchronize(batch->stream);
    free_batch(batch);
    return cuda_status(e);
}

int dse_batch_set_stream(dse_batch* batch, void* cuda_stream) {
    if (!batch) return DSE_ERR_ARG;
    batch->stream = (cudaStream_t)cuda_stream;
    return DSE_OK;
}

int dse_batch_offsets(const dse_batch* batch, long long* h_offsets, long long* h_matrix_offsets) {
    if (!batch) return DSE_ERR_ARG;
    for (int b = 0; b <= batch->nb; ++b) {
        if (h_offsets) h_offsets[b] = batch->coef_off[b];
        if (h_matrix_offsets) h_matrix_offsets[b] = batch->J_off[b];
    }
    return DSE_OK;
}

int dse_batch_newton_matrix(dse_batch* batch, const double* d_coeffs, double* d_J, double* d_F) {
    if (!batch || !d_coeffs || !d_J) return DSE_ERR_ARG;
    dse_batch* B = batch;
    cudaError_t e = cudaSuccess;
    k_batch_reset<<<(B->nb + 127) / 128, 128, 0, B->stream>>>(B->d_P, B->nb, B->d_nactive);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = enqueue_matrix(B, d_coeffs, d_J, d_F, B->stream);
    B->launches += 6;
    return cuda_status(e);
}

int dse_batch_residual(dse_batch* batch, const double* d_coeffs, double* d_F) {
    if (!batch || !d_coeffs || !d_F) return DSE_ERR_ARG;
    dse_batch* B = batch;
    k_batch_reset<<<(B->nb + 127) / 128, 128, 0, B->stream>>>(B->d_P, B->nb, B->d_nactive);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = enqueue_residual(B, d_coeffs, d_F, B->stream);
    B->launches += 6;
    return cuda_status(e);
}

int dse_batch_tune(dse_batch* batch, const double* d_coeffs, int* h_units, double* h_ms) {
    if (!batch || !d_coeffs) return DSE_ERR_ARG;
    dse_batch* B = batch;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DSE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DSE_ERR_CUDA;
    }
    int best = B->units;
    double best_ms = 1e300;
    int st = DSE_OK;
    int q = 0;
    for (int units : kTuneCandidates) {
        st = set_units(B, units);
        if (st) break;
        cudaError_t e = cudaSuccess;
        k_batch_reset<<<(B->nb + 127) / 128, 128, 0, B->stream>>>(B->d_P, B->nb, B->d_nactive);
        // one untimed pass, then three timed quadrature passes
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            if (rep == 1) e = cudaEventRecord(e0, B->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(B->d_counter, 0, sizeof(int), B->stream);
            if (e == cudaSuccess) e = launch_tables_batched(B->d_P, B->nb, B->max_units, d_coeffs, B->stream);
            if (e == cudaSuccess) e = launch_series_table_batched(B->d_P, B->nb, d_coeffs, B->stream);
            if (e == cudaSuccess)
                e = launch_triple_batched(true, B->d_P, B->d_items, B->n_items, B->d_counter, d_coeffs, B->maxN,
                                          B->grid, B->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        B->launches += 13;
        if (e != cudaSuccess) {
            st = DSE_ERR_CUDA;
            break;
        }
        if (h_ms) h_ms[q] = ms / 3.0;
        if (ms < best_ms) {
            best_ms = ms;
            best = units;
        }
        ++q;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!st) st = set_units(B, best);
    if (!st && h_units) *h_units = best;
    return st;
}

int dse_batch_solve(dse_batch* batch, double* d_coeffs, double tol, int max_iter, double rho_relax, int n_relax,
                    int* h_iters, int* h_status, double* h_stats) {
    if (!batch || !d_coeffs || !(tol > 0.0) || max_iter < 1 || !isfinite(rho_relax) || n_relax < 0)
        return DSE_ERR_ARG;
    dse_batch* B = batch;
    if (B->max_n > 128) return DSE_ERR_UNSUPPORTED;
    int st = capture_step(B, d_coeffs, tol, rho_relax, n_relax);
    if (st) return st;
    k_batch_reset<<<(B->nb + 127) / 128, 128, 0, B->stream>>>(B->d_P, B->nb, B->d_nactive);
    cudaError_t e = cudaGetLastError();
    B->launches += 1;
    for (int it = 0; it < max_iter && e == cudaSuccess; ++it) {
        e = cudaGraphLaunch(B->exec, B->stream);
        B->graph_launches += 1;
        B->launches += 7;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->h_nactive, B->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, B->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        if (e == cudaSuccess && *B->h_nactive <= 0) break;
    }
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    // per-problem results
    std::vector<BatchProblem> P(B->nb);
    std::vector<double> S(4 * (size_t)B->nb);
    k_batch_gather<<<(B->nb + 127) / 128, 128, 0, B->stream>>>(B->d_P, B->nb, B->d_stats_out);
    B->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.data(), B->d_P, sizeof(BatchProblem) * B->nb, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.data(), B->d_stats_out, sizeof(double) * 4 * B->nb, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    int all = DSE_OK;
    for (int b = 0; b < B->nb; ++b) {
        int code = DSE_ERR_NOT_CONVERGED;
        if (P[b].result == 1) code = DSE_OK;
        else if (P[b].result == -1) code = DSE_ERR_NONFINITE;
        else if (P[b].result == -2) code = DSE_ERR_SINGULAR;
        if (h_iters) h_iters[b] = P[b].iter;
        if (h_status) h_status[b] = code;
        if (h_stats)
            for (int q = 0; q < 3; ++q) h_stats[3 * b + q] = S[4 * b + q];
        if (code != DSE_OK) all = DSE_ERR_NOT_CONVERGED;
    }
    return all;
}

int dse_batch_counters(dse_batch* batch, long long* h_launches, long long* h_graph_launches, int* h_units) {
    if (!batch) return DSE_ERR_ARG;
    if (h_launches) *h_launches = batch->launches;
    if (h_graph_launches) *h_graph_launches = batch->graph_launches;
    if (h_units) *h_units = batch->units;
    return DSE_OK;
}

}  // extern "C"
