// dse_noalloc.cu -- dse_residual_static: the residual of dse_residual computed
// without any device allocation, for callers that cannot call cudaMalloc.
//
// All intermediate buffers (quadrature rules, dressing tables, the per-radial-
// node angular sums of the quadrature kernel, the per-row contractions) are
// carved out of one file-scope __device__ array of DSE_STATIC_SCRATCH_BYTES.
// The kernels are the same as those of dse_residual.
#include <math.h>

#include "dse_internal.cuh"

using namespace dse;

namespace {

// The scratch every call shares.  It is part of this file's device code, so
// every GPU that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_dse_static_scratch[DSE_STATIC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  The host-side name
// g_dse_static_scratch is only a stand-in, not a device address: it is looked up
// with cudaGetSymbolAddress, with the device current, on every call (a host-side
// lookup that allocates nothing), so that an address never outlives the context it
// belongs to.  The first call on a device also loads the library's device code there.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dse_static_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
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
    const int st = check_problem(problem);
    if (st != DSE_OK) return st;
    const dse_problem* p = problem;
    // the plan's single radial rule and the FP64 kernels only
    if (p->radial_mode != 0 || p->precision != 0) return DSE_ERR_UNSUPPORTED;
    Consts c = make_consts(p);
    c.sM = 0;  // no series table here: the dressing series are summed per triple

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

    // radial splits: about eight waves of blocks over the resident slots, at least
    // two radial nodes per block, at most 128 splits; the queries allocate nothing
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        return DSE_ERR_CUDA;
    int occ = triple_max_blocks_per_sm(false, c.N);
    if (occ < 1) occ = 1;
    long long kb = ((long long)nr * Rt) / (8LL * nsm * occ);
    if (kb < 2) kb = 2;
    if (kb > nr) kb = nr;
    while ((nr + kb - 1) / kb > 128) ++kb;
    const int KB = (int)kb;
    const int KS = (int)((nr + kb - 1) / kb);

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
