// dse_noalloc.cu -- dse_residual_static: the residual of dse_residual computed
// without any device allocation, for callers that cannot call cudaMalloc.
//
// All intermediate buffers (quadrature rules, dressing tables, the per-radial-
// node angular sums of the quadrature kernel, the per-row contractions) are
// carved out of one file-scope __device__ array of DSE_STATIC_SCRATCH_BYTES.
// The kernels are the same as those of dse_residual.
#include <math.h>

#include <mutex>

#include "dse_internal.cuh"

using namespace dse;

namespace {

// The scratch every call shares.  It is part of this file's device code, so
// every GPU that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_dse_static_scratch[DSE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The host-side
// name g_dse_static_scratch is only a stand-in, not a device address: it is
// resolved once per device with cudaGetSymbolAddress while that device is
// current.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dse_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    size_t rad, ang, theta, rows, xcol, ytab, phiy, xtab, phix, U, D, gl, status, total;
};

Layout layout(const Consts& c, int Rt, int nch) {
    const int N = c.N, nr = c.nr, na = c.na, Rc = c.Rc;
    Layout L;
    size_t off = 0;
    L.rad = off; off = up256(off + sizeof(Rad) * (size_t)nr);
    L.ang = off; off = up256(off + sizeof(Ang) * (size_t)na);
    L.theta = off; off = up256(off + sizeof(double) * (size_t)na);
    L.rows = off; off = up256(off + sizeof(Row) * (size_t)Rt);
    L.xcol = off; off = up256(off + sizeof(double) * (size_t)Rc);
    L.ytab = off; off = up256(off + sizeof(YTab) * (size_t)nr);
    L.phiy = off; off = up256(off + sizeof(double) * (size_t)nr * N);
    L.xtab = off; off = up256(off + sizeof(XTab) * (size_t)Rc);
    L.phix = off; off = up256(off + sizeof(double) * (size_t)Rc * N);
    L.U = off; off = up256(off + sizeof(double) * (size_t)Rt * nr * nch * 3);
    L.D = off; off = up256(off + sizeof(double) * (size_t)(Rc + 2) * ldD(c));
    const size_t gmax = nr > na ? nr : na;
    L.gl = off; off = up256(off + sizeof(double) * (2 * (size_t)nr + 2 * (size_t)na + gmax + 2));
    L.status = off; off = up256(off + sizeof(int));
    L.total = off;
    return L;
}

}  // namespace

extern "C" int dse_residual_static(const dse_problem* problem, const double* d_coeffs, double* d_F,
                                   void* cuda_stream) {
    if (!problem || !d_coeffs || !d_F) return DSE_ERR_ARG;
    const dse_problem* p = problem;
    if (p->n_cheb < 1 || p->n_cheb > DSE_MAX_CHEB || p->n_cheb_G < 0 || p->n_cheb_G > DSE_MAX_CHEB ||
        p->n_radial < 1 || p->n_radial > DSE_MAX_NODES ||
        p->n_angular < 1 || p->n_angular > DSE_MAX_NODES)
        return DSE_ERR_ARG;
    if (!(p->eps2 > 0.0) || !(p->lambda2 > p->eps2) || !isfinite(p->lambda2) || !(p->x_Z > 0.0) ||
        !isfinite(p->x_Z) || !(p->x_G >= 0.0) || !isfinite(p->x_G) || !isfinite(p->g2nc) || !isfinite(p->kappa) ||
        !isfinite(p->delta) || !isfinite(p->ginv_G) || !isfinite(p->zinv_Z))
        return DSE_ERR_ARG;
    if (p->radial_mode != 0 || p->precision != 0 || (p->extrap_mode != 0 && p->extrap_mode != 1) ||
        (p->angular_mode != 0 && p->angular_mode != 1))
        return DSE_ERR_UNSUPPORTED;

    const double kPi = 3.14159265358979323846264338327950288;
    Consts c;
    c.NZ = p->n_cheb;
    c.NG = p->n_cheb_G > 0 ? p->n_cheb_G : p->n_cheb;
    c.N = c.NZ > c.NG ? c.NZ : c.NG;
    c.n = c.NZ + c.NG;
    c.Rc = c.NZ == c.NG ? c.N : c.n;
    c.gofs = c.NZ == c.NG ? 0 : c.NZ;
    c.nr = p->n_radial;
    c.nrule = p->n_radial;
    c.radmode = 0;
    c.angmode = p->angular_mode;
    c.sM = 0;  // no series table here
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

    const int nr = c.nr, na = c.na;
    const int Rt = c.Rc + 1 + (p->x_G > 0.0 ? 1 : 0);
    const int nch = (na + 31) / 32;
    const Layout L = layout(c, Rt, nch);
    if (L.total > (size_t)DSE_STATIC_SCRATCH_BYTES) return DSE_ERR_ARG;  // does not fit the static scratch

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return DSE_ERR_CUDA;
    char* b = (char*)base;
    Rad* rad = (Rad*)(b + L.rad);
    Ang* ang = (Ang*)(b + L.ang);
    double* theta = (double*)(b + L.theta);
    Row* rows = (Row*)(b + L.rows);
    double* xcol = (double*)(b + L.xcol);
    YTab* ytab = (YTab*)(b + L.ytab);
    double* phiy = (double*)(b + L.phiy);
    XTab* xtab = (XTab*)(b + L.xtab);
    double* phix = (double*)(b + L.phix);
    double* U = (double*)(b + L.U);
    double* D = (double*)(b + L.D);
    double* glr = (double*)(b + L.gl);
    double* gwr = glr + nr;
    double* gla = gwr + nr;
    double* gwa = gla + na;
    double* inv = gwa + na;
    int* status = (int*)(b + L.status);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // radial splits: about three blocks per SM of 152
    int KS = (3 * 152 + Rt - 1) / Rt;
    if (KS > nr) KS = nr;
    if (KS < 1) KS = 1;
    const int KB = (nr + KS - 1) / KS;
    KS = (nr + KB - 1) / KB;

    // only the status word must start at zero; every other buffer is written
    // in full before it is read
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_gauss_legendre(nr, inv, glr, gwr, s);
    if (e == cudaSuccess) e = launch_gauss_legendre(na, inv, gla, gwa, s);
    if (e == cudaSuccess) e = launch_setup_rules(c, glr, gwr, gla, gwa, rad, ang, theta, xcol, rows, Rt, s);
    if (e == cudaSuccess) e = launch_tables(c, d_coeffs, rad, xcol, ytab, phiy, xtab, phix, s);
    if (e == cudaSuccess) {
        TripleArgs a;
        a.c = c;
        a.Rt = Rt;
        a.KB = KB;
        a.KS = KS;
        a.nch = nch;
        a.rad = rad;
        a.ang = ang;
        a.rows = rows;
        a.ytab = ytab;
        a.coef = d_coeffs;
        a.Upart = U;
        a.Vpart = nullptr;  // not used by the residual-only kernel
        a.stab = nullptr;   // series summed per triple (no table in the static scratch)
        e = launch_triple(false, a, s);
    }
    if (e == cudaSuccess) e = launch_rowreduce(false, c, Rt, KS, nch, rad, ang, rows, ytab, phiy, U, nullptr, D, s);
    if (e == cudaSuccess) e = launch_assemble(false, c, xtab, phix, D, nullptr, d_F, status, s);
    return e == cudaSuccess ? DSE_OK : DSE_ERR_CUDA;
}
