// extern "C" entry points of libsbq (declared in include/sbq.h): argument checks,
// handle management, dispatch to the engine.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>
#include <new>
#include <thread>

namespace sbq {
const char *last_error_cstr();
int gmres_solve_impl(Op *op, const double *b, double *x, const sbq_gmres_opts &o,
                     sbq_gmres_report &rep, cudaStream_t s);
int op_autotune(Op *op, int prec, cudaStream_t s);
}  // namespace sbq

using namespace sbq;

namespace {

bool prec_ok(int prec)
{
    return prec == SBQ_FP64 || prec == SBQ_FP32 || prec == SBQ_FP32_COMP || prec == SBQ_DF32;
}

int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

// Generic apply: u = alpha S[sigma] + beta D[sigma] at the targets.
int apply_generic(int64_t ns, const double *src, const double *nrm, const double *w,
                  const double *sigma, int64_t nt, const double *trg, double alpha, double beta,
                  double *u, int prec, void *stream, bool laplace = false)
{
    clear_error();
    if (ns < 0 || nt < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    if (!std::isfinite(alpha) || !std::isfinite(beta))
        return fail(SBQ_EINVAL, "non-finite prefactor");
    if (nt > 0 && (!trg || !u))
        return fail(SBQ_EINVAL, "null target or output pointer");
    if (ns > 0 && nt > 0 && (!src || !w || !sigma))
        return fail(SBQ_EINVAL, "null source, weight or density pointer");
    if (ns > 0 && nt > 0 && beta != 0.0 && !nrm)
        return fail(SBQ_EINVAL, "double layer needs normals");
    if (ns > (1LL << 31) || nt > (1LL << 31))
        return fail(SBQ_EINVAL, "size above 2^31");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nt == 0)
        return SBQ_OK;
    const size_t ncomp = laplace ? 1 : 3;
    if (ns == 0 || (alpha == 0.0 && beta == 0.0)) {
        SBQ_CUDA(cudaMemsetAsync(u, 0, ncomp * static_cast<size_t>(nt) * sizeof(double), s));
        return SBQ_OK;
    }
    int kind;
    double scale, kappa;
    if (laplace)
        laplace_kind_and_scale(alpha, beta, &kind, &scale, &kappa);
    else
        kind_and_scale(alpha, beta, &kind, &scale, &kappa);
    const int layout = (prec == SBQ_FP64 || prec == SBQ_DF32) ? prec : SBQ_FP32;
    AsyncAllocScope scope(s);
    SrcPack sp;
    TrgSet ts;
    std::vector<int64_t> soff = {0, ns}, toff = {0, nt};
    SBQ_TRY(build_src_pack(sp, layout, soff, src, kind_has_normals(kind) ? nrm : nullptr,
                           (kind == KIND_CF || kind == KIND_LCF) ? kappa : 1.0, ns, s));
    SBQ_TRY(build_trg_set(ts, kind, prec, default_tune(prec, nt), sp, toff, trg, nt, soff, s));
    SBQ_TRY(run_pairsum(kind, prec, sp, ts, w, sigma, ns, trg, nt, u, scale, kappa, 0.0, nullptr, s));
    return SBQ_OK;
}

// Recursive coordinate bisection of the nodes [b, e): split at the median of the longest
// bounding-box axis, at a multiple of 256 nodes (128 at the last level), so that every
// aligned block of 128 or 256 nodes is one subtree: a compact patch of the surface.  hx
// holds the coordinates component-major (x of all n nodes, then y, then z).  The two halves
// of a large range are ordered by two threads while `par` > 1 (the result does not depend
// on it: the halves are disjoint).
static void rcb_order(const double *hx, long long n, int *b, int *e, int par)
{
    const long long m = e - b;
    if (m <= 128)
        return;
    double mn[3], mx[3];
    for (int c = 0; c < 3; ++c) {
        mn[c] = INFINITY;
        mx[c] = -INFINITY;
    }
    for (int *p = b; p < e; ++p)
        for (int c = 0; c < 3; ++c) {
            mn[c] = std::min(mn[c], hx[c * n + *p]);
            mx[c] = std::max(mx[c], hx[c * n + *p]);
        }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
        if (mx[c] - mn[c] > mx[ax] - mn[ax])
            ax = c;
    const long long unit = m > 256 ? 256 : 128;
    long long half = std::llround(0.5 * static_cast<double>(m) / unit) * unit;
    half = std::max(half, unit);
    if (half >= m)
        half = m - unit;
    std::nth_element(b, b + half, e,
                     [&](int i, int j) { return hx[ax * n + i] < hx[ax * n + j]; });
    if (par > 1 && m >= 65536) {
        bool spawned = false;
        std::thread th;
        try {
            th = std::thread([=] { rcb_order(hx, n, b, b + half, par / 2); });
            spawned = true;
        } catch (...) {
        }
        if (!spawned)
            rcb_order(hx, n, b, b + half, 1);
        rcb_order(hx, n, b + half, e, par - par / 2);
        if (spawned)
            th.join();
        return;
    }
    rcb_order(hx, n, b, b + half, 1);
    rcb_order(hx, n, b + half, e, 1);
}

// Mean bounding radius (about the bounding-box midpoint) of the blocks of 256 consecutive
// nodes of order[a..b).
static double mean_tile_radius(const double *hx, long long n, const int *order, long long cnt)
{
    double sum = 0.0;
    long long tiles = 0;
    for (long long t = 0; t < cnt; t += 256) {
        const long long te = std::min(cnt, t + 256);
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (long long k = t; k < te; ++k)
            for (int c = 0; c < 3; ++c) {
                mn[c] = std::min(mn[c], hx[c * n + order[k]]);
                mx[c] = std::max(mx[c], hx[c * n + order[k]]);
            }
        double r2 = 0.0;
        for (long long k = t; k < te; ++k) {
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double d = hx[c * n + order[k]] - 0.5 * (mn[c] + mx[c]);
                d2 += d * d;
            }
            r2 = std::max(r2, d2);
        }
        sum += std::sqrt(r2);
        ++tiles;
    }
    return tiles ? sum / tiles : 0.0;
}

// out[c n + k] = in[c n + perm[k]] for the ncomp components of n nodes
__global__ void k_gather_nodes(const double *__restrict__ in, const int *__restrict__ perm, long long n,
                               int ncomp, double *__restrict__ out)
{
    const long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (k >= n)
        return;
    const long long u = perm[k];
    for (int c = 0; c < ncomp; ++c)
        out[c * n + k] = in[c * n + u];
}

// Internal node order of an operator: within each segment, either the caller's order or a
// recursive coordinate bisection of the nodes, whichever makes the smaller tiles (mean
// bounding radius of blocks of 256).  Consecutive caller nodes are often compact already
// (rings of a thin tube); on a fat tube a block of 256 nodes is a full ring as wide as the
// tube, and bisection turns it into a compact patch.  Small tiles have small bounding
// spheres: fewer tile pairs need the near-field treatment (coincidence test, high/low or
// exact differences).  The operator keeps its geometry in the internal order and
// perm[k] = the caller's index of internal node k; the density pack gathers through perm
// and the reductions scatter through it, so callers never see the internal order.
// host_geom: src, nrm, w are host arrays (else device arrays; only the coordinates are read
// back).  The order is computed on the host from the coordinates; the geometry is gathered
// into it on the device (host arrays are uploaded as they are, then gathered).
static int internal_order(Op *op, const double *src, const double *nrm, const double *w,
                          bool host_geom)
{
    const long long n = op->n;
    std::vector<double> hbuf;
    const double *hx = src;
    cudaError_t e = cudaSuccess;
    if (!host_geom) {
        hbuf.resize(3 * n);
        e = cudaMemcpy(hbuf.data(), src, 3 * n * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_status(e, "cudaMemcpy (operator geometry)");
        hx = hbuf.data();
    }
    for (long long k = 0; k < 3 * n; ++k)
        if (!std::isfinite(hx[k]))
            return fail(SBQ_EINVAL, "non-finite source coordinate");
    const int par = static_cast<int>(std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    std::vector<int> perm(n), alt;
    for (long long k = 0; k < n; ++k)
        perm[k] = static_cast<int>(k);
    for (int sgi = 0; sgi < op->plan.nseg; ++sgi) {
        const long long a = op->plan.src_off[sgi], b = op->plan.src_off[sgi + 1];
        if (b - a <= 256)
            continue;
        alt.assign(perm.begin() + a, perm.begin() + b);
        rcb_order(hx, n, alt.data(), alt.data() + alt.size(), par);
        if (mean_tile_radius(hx, n, alt.data(), b - a) <
            mean_tile_radius(hx, n, perm.data() + a, b - a))
            std::copy(alt.begin(), alt.end(), perm.begin() + a);
    }
    e = cudaMemcpy(op->perm.p, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_status(e, "cudaMemcpy (operator node order)");
    const unsigned grid = static_cast<unsigned>((n + 255) / 256);
    struct Arr {
        const double *in;
        int ncomp;
        DevBuf *out;
    };
    const Arr arrs[3] = {{src, 3, &op->src}, {nrm, 3, &op->nrm}, {w, 1, &op->w}};
    DevBuf tmp;
    if (host_geom)
        SBQ_TRY(tmp.alloc(3 * static_cast<size_t>(n) * sizeof(double)));
    for (const Arr &ar : arrs) {
        const double *in = ar.in;
        if (host_geom) {
            // the legacy stream orders this copy after the previous gather out of tmp
            e = cudaMemcpy(tmp.p, ar.in, ar.ncomp * n * sizeof(double), cudaMemcpyHostToDevice);
            if (e != cudaSuccess)
                return cuda_status(e, "cudaMemcpy (operator geometry)");
            in = tmp.as<double>();
        }
        k_gather_nodes<<<grid, 256>>>(in, op->perm.as<int>(), n, ar.ncomp, ar.out->as<double>());
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_status(e, "k_gather_nodes");
    }
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess)
        return cuda_status(e, "operator geometry gather");
    return SBQ_OK;
}

Op *as_op(const void *h)
{
    Op *op = static_cast<Op *>(const_cast<void *>(h));
    if (!op || op->magic != OP_MAGIC)
        return nullptr;
    return op;
}

}  // namespace

extern "C" {

SBQ_API int sbq_version(void) { return 300; }

SBQ_API const char *sbq_last_error(void) { return last_error_cstr(); }

SBQ_API int sbq_device_info(int *num_sms, int *fp32_lanes_per_sm, int *cc_major, int *cc_minor)
{
    clear_error();
    int dev = 0;
    SBQ_CUDA(cudaGetDevice(&dev));
    const DeviceProps &p = device_props();
    if (num_sms)
        *num_sms = p.sms;
    if (fp32_lanes_per_sm)
        *fp32_lanes_per_sm = 128;   // FP32 lanes per SM on sm_100-class parts
    if (cc_major)
        *cc_major = p.cc_major;
    if (cc_minor)
        *cc_minor = p.cc_minor;
    return SBQ_OK;
}

SBQ_API int stokes_sl_apply(int64_t ns, const double *src, const double *w, const double *sigma,
                            int64_t nt, const double *trg, double *u, int prec, void *stream)
{
    return apply_generic(ns, src, nullptr, w, sigma, nt, trg, 1.0, 0.0, u, prec, stream);
}

SBQ_API int stokes_dl_apply(int64_t ns, const double *src, const double *nrm, const double *w,
                            const double *sigma, int64_t nt, const double *trg, double *u,
                            int prec, void *stream)
{
    return apply_generic(ns, src, nrm, w, sigma, nt, trg, 0.0, 1.0, u, prec, stream);
}

SBQ_API int stokes_combined_apply(int64_t ns, const double *src, const double *nrm,
                                  const double *w, const double *sigma, int64_t nt,
                                  const double *trg, double alpha, double beta, double *u,
                                  int prec, void *stream)
{
    return apply_generic(ns, src, nrm, w, sigma, nt, trg, alpha, beta, u, prec, stream);
}

SBQ_API int laplace_sl_apply(int64_t ns, const double *src, const double *w, const double *sigma,
                             int64_t nt, const double *trg, double *u, int prec, void *stream)
{
    return apply_generic(ns, src, nullptr, w, sigma, nt, trg, 1.0, 0.0, u, prec, stream, true);
}

SBQ_API int laplace_dl_apply(int64_t ns, const double *src, const double *nrm, const double *w,
                             const double *sigma, int64_t nt, const double *trg, double *u,
                             int prec, void *stream)
{
    return apply_generic(ns, src, nrm, w, sigma, nt, trg, 0.0, 1.0, u, prec, stream, true);
}

SBQ_API int laplace_combined_apply(int64_t ns, const double *src, const double *nrm,
                                   const double *w, const double *sigma, int64_t nt,
                                   const double *trg, double alpha, double beta, double *u,
                                   int prec, void *stream)
{
    return apply_generic(ns, src, nrm, w, sigma, nt, trg, alpha, beta, u, prec, stream, true);
}

SBQ_API int batch_plan(int nseg, const int64_t *seg_src_off, const int64_t *seg_trg_off,
                       const sbq_tune *tune, void **plan_out)
{
    clear_error();
    if (!plan_out)
        return fail(SBQ_EINVAL, "null plan_out");
    *plan_out = nullptr;
    if (nseg < 1 || !seg_src_off || !seg_trg_off)
        return fail(SBQ_EINVAL, "nseg < 1 or null offsets");
    if (seg_src_off[0] != 0 || seg_trg_off[0] != 0)
        return fail(SBQ_EINVAL, "offsets must start at 0");
    for (int i = 0; i < nseg; ++i)
        if (seg_src_off[i + 1] < seg_src_off[i] || seg_trg_off[i + 1] < seg_trg_off[i])
            return fail(SBQ_EINVAL, "offsets must be non-decreasing");
    if (tune && tune->r != 0 && !pairsum_shape_supported(SBQ_FP32, tune->r, tune->warps) &&
        !pairsum_shape_supported(SBQ_FP64, tune->r, tune->warps) &&
        !pairsum_shape_supported(SBQ_DF32, tune->r, tune->warps))
        return fail(SBQ_EINVAL, "unsupported tile shape");
    if (tune && tune->chunk_tiles < 0)
        return fail(SBQ_EINVAL, "chunk_tiles must be >= 0");
    PlanH *p = new (std::nothrow) PlanH();
    if (!p)
        return fail(SBQ_ENOMEM, "out of host memory");
    p->nseg = nseg;
    p->src_off.assign(seg_src_off, seg_src_off + nseg + 1);
    p->trg_off.assign(seg_trg_off, seg_trg_off + nseg + 1);
    if (tune && tune->r != 0) {
        p->has_tune = true;
        p->tune = *tune;
    }
    *plan_out = p;
    return SBQ_OK;
}

static int op_create_impl(int64_t n, const double *src, const double *nrm, const double *w,
                          double eta, double diag, int64_t nnz, const int64_t *rowptr,
                          const int64_t *col, const double *val, const void *plan, void **op_out,
                          bool laplace, bool host_geom = false)
{
    clear_error();
    if (!op_out)
        return fail(SBQ_EINVAL, "null op_out");
    *op_out = nullptr;
    if (n < 0 || nnz < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (n > (1LL << 31) / 3)
        return fail(SBQ_EINVAL, "n above 2^31 / 3");
    if (n > 0 && (!src || !nrm || !w))
        return fail(SBQ_EINVAL, "null source, normal or weight pointer");
    if (nnz > 0 && (!rowptr || !col || !val))
        return fail(SBQ_EINVAL, "null CSR pointer");
    if (!std::isfinite(eta) || !std::isfinite(diag))
        return fail(SBQ_EINVAL, "non-finite eta or diag");
    const PlanH *pl = static_cast<const PlanH *>(plan);
    if (pl && pl->magic != PLAN_MAGIC)
        return fail(SBQ_EINVAL, "plan is not a batch_plan handle");
    if (pl) {
        if (pl->src_off.back() != n || pl->trg_off.back() != n)
            return fail(SBQ_EINVAL, "plan offsets do not cover the n nodes");
        for (int i = 0; i <= pl->nseg; ++i)
            if (pl->src_off[i] != pl->trg_off[i])
                return fail(SBQ_EINVAL, "operator plans need equal source and target offsets");
    }
    Op *op = new (std::nothrow) Op();
    if (!op)
        return fail(SBQ_ENOMEM, "out of host memory");
    auto bail = [&](int st) {
        delete op;
        return st;
    };
    cudaGetDevice(&op->device);
    op->n = n;
    op->eta = eta;
    op->diag = diag;
    op->nnz = nnz;
    op->laplace = laplace;
    op->ncomp = laplace ? 1 : 3;
    if (pl)
        op->plan = *pl;
    else {
        op->plan.nseg = 1;
        op->plan.src_off = {0, n};
        op->plan.trg_off = {0, n};
    }
    const size_t vb = 3 * static_cast<size_t>(n) * sizeof(double);
    int st = SBQ_OK;
    if ((st = op->src.alloc(vb)) != SBQ_OK) return bail(st);
    if ((st = op->nrm.alloc(vb)) != SBQ_OK) return bail(st);
    if ((st = op->w.alloc(static_cast<size_t>(n) * sizeof(double))) != SBQ_OK) return bail(st);
    if ((st = op->perm.alloc(static_cast<size_t>(n) * sizeof(int))) != SBQ_OK) return bail(st);
    if (n > 0 && (st = internal_order(op, src, nrm, w, host_geom)) != SBQ_OK)
        return bail(st);
    if (nnz > 0) {
        const size_t rows = static_cast<size_t>(op->ncomp) * n;
        if ((st = op->rowptr.alloc((rows + 1) * sizeof(int64_t))) != SBQ_OK)
            return bail(st);
        if ((st = op->col.alloc(static_cast<size_t>(nnz) * sizeof(int64_t))) != SBQ_OK) return bail(st);
        if ((st = op->val.alloc(static_cast<size_t>(nnz) * sizeof(double))) != SBQ_OK) return bail(st);
        cudaError_t e = cudaMemcpy(op->rowptr.p, rowptr, (rows + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(op->col.p, col, nnz * sizeof(int64_t), cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(op->val.p, val, nnz * sizeof(double), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return bail(cuda_status(e, "cudaMemcpy (correction)"));
    }
    cudaStream_t s = nullptr;
    int kind;
    double scale, kappa;
    if (laplace)
        laplace_kind_and_scale(eta, 1.0, &kind, &scale, &kappa);
    else
        kind_and_scale(eta, 1.0, &kind, &scale, &kappa);
    const double nscale = (kind == KIND_CF || kind == KIND_LCF) ? kappa : 1.0;
    if ((st = build_src_pack(op->sp32, SBQ_FP32, op->plan.src_off, op->src.as<double>(),
                             op->nrm.as<double>(), nscale, n, s)) != SBQ_OK)
        return bail(st);
    if ((st = build_src_pack(op->sp64, SBQ_FP64, op->plan.src_off, op->src.as<double>(),
                             op->nrm.as<double>(), nscale, n, s)) != SBQ_OK)
        return bail(st);
    if ((st = build_src_pack(op->spdf, SBQ_DF32, op->plan.src_off, op->src.as<double>(),
                             op->nrm.as<double>(), nscale, n, s)) != SBQ_OK)
        return bail(st);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_status(e, "stokes_op_create"));
    *op_out = op;
    return SBQ_OK;
}

SBQ_API int stokes_op_create(int64_t n, const double *src, const double *nrm, const double *w,
                             double eta, double diag, int64_t nnz, const int64_t *rowptr,
                             const int64_t *col, const double *val, const void *plan,
                             void **op_out)
{
    return op_create_impl(n, src, nrm, w, eta, diag, nnz, rowptr, col, val, plan, op_out, false);
}

SBQ_API int laplace_op_create(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, int64_t nnz, const int64_t *rowptr,
                              const int64_t *col, const double *val, const void *plan,
                              void **op_out)
{
    return op_create_impl(n, src, nrm, w, eta, diag, nnz, rowptr, col, val, plan, op_out, true);
}

SBQ_API int sbq_slender_eta(double eps, double *eta)
{
    clear_error();
    if (!eta)
        return fail(SBQ_EINVAL, "null output");
    if (!(eps > 0.0 && eps < 1.0))
        return fail(SBQ_EINVAL, "slenderness must lie in (0, 1)");
    // Sec. 4.1: eta = 1 / (2 eps log(1/eps)), natural logarithm
    *eta = 1.0 / (2.0 * eps * std::log(1.0 / eps));
    return SBQ_OK;
}

// Operator of the host-buffer entry points: geometry read from host arrays, no correction
// or the double-layer singularity subtraction over the bodies (built on the device).
namespace {

struct HostOpGuard {
    Op *op = nullptr;
    ~HostOpGuard() { delete op; }
};

int host_vec_ok(const double *p, long long cnt)
{
    for (long long i = 0; i < cnt; ++i)
        if (!std::isfinite(p[i]))
            return 0;
    return 1;
}

}  // namespace

SBQ_API int stokes_apply_host(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, const double *sigma, double *out, int prec,
                              const sbq_tune *tune, void *stream)
{
    clear_error();
    if (n < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    if (n > 0 && (!src || !nrm || !w || !sigma || !out))
        return fail(SBQ_EINVAL, "null host pointer");
    if (tune && tune->r != 0 && !pairsum_shape_supported(prec, tune->r, tune->warps))
        return fail(SBQ_EINVAL, "unsupported tile shape for this precision");
    if (n == 0)
        return SBQ_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HostOpGuard g;
    void *h = nullptr;
    SBQ_TRY(op_create_impl(n, src, nrm, w, eta, diag, 0, nullptr, nullptr, nullptr, nullptr, &h,
                           false, true));
    g.op = static_cast<Op *>(h);
    const size_t vb = 3 * static_cast<size_t>(n) * sizeof(double);
    DevBuf d_sig, d_out;
    SBQ_TRY(d_sig.alloc(vb));
    SBQ_TRY(d_out.alloc(vb));
    SBQ_CUDA(cudaMemcpyAsync(d_sig.p, sigma, vb, cudaMemcpyHostToDevice, s));
    SBQ_TRY(op_prepare_untimed(g.op, prec, tune, s));
    SBQ_TRY(op_matvec(g.op, d_sig.as<double>(), d_out.as<double>(), prec, s));
    SBQ_CUDA(cudaMemcpyAsync(out, d_out.p, vb, cudaMemcpyDeviceToHost, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

SBQ_API int stokes_solve_host(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, int nbody, const int64_t *body_off,
                              int corr_prec, const double *rhs, double *x,
                              const sbq_gmres_opts *o, sbq_gmres_report *rep, void *stream)
{
    clear_error();
    if (n < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (!o)
        return fail(SBQ_EINVAL, "null options");
    if (n > 0 && (!src || !nrm || !w || !rhs || !x))
        return fail(SBQ_EINVAL, "null host pointer");
    if (nbody < 0 || (nbody > 0 && !body_off))
        return fail(SBQ_EINVAL, "nbody < 0 or null body offsets");
    if (nbody > 0) {
        if (body_off[0] != 0 || body_off[nbody] != n)
            return fail(SBQ_EINVAL, "body offsets must run from 0 to n");
        for (int b = 0; b < nbody; ++b)
            if (body_off[b + 1] < body_off[b])
                return fail(SBQ_EINVAL, "body offsets must be non-decreasing");
        if (!prec_ok(corr_prec))
            return fail(SBQ_EINVAL, "unknown correction precision");
    }
    if (!(o->tol > 0.0) || o->restart < 1 || o->restart > 256 || o->max_iter < 1 ||
        !prec_ok(o->inner_prec))
        return fail(SBQ_EINVAL, "bad GMRES options (tol > 0, 1 <= restart <= 256, max_iter >= 1)");
    const bool mixed = (o->inner_prec == SBQ_FP32 || o->inner_prec == SBQ_FP32_COMP);
    if (mixed && (!(o->inner_tol > 0.0) || o->inner_tol >= 1.0 || o->max_outer < 1))
        return fail(SBQ_EINVAL, "bad refinement options (0 < inner_tol < 1, max_outer >= 1)");
    if (mixed && o->resid_prec != SBQ_FP64 && o->resid_prec != SBQ_DF32)
        return fail(SBQ_EINVAL, "resid_prec must be SBQ_FP64 or SBQ_DF32");
    sbq_gmres_report local{};
    sbq_gmres_report &r = rep ? *rep : local;
    r = sbq_gmres_report{};
    if (n == 0)
        return SBQ_OK;
    if (!host_vec_ok(rhs, 3 * n))
        return fail(SBQ_ENONFINITE, "non-finite right-hand side");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vb = 3 * static_cast<size_t>(n) * sizeof(double);
    DevBuf d_rowptr, d_col, d_val;
    int64_t nnz = 0;
    if (nbody > 0) {
        // the correction is built from device copies of the geometry
        DevBuf d_src, d_nrm, d_w;
        SBQ_TRY(d_src.alloc(vb));
        SBQ_TRY(d_nrm.alloc(vb));
        SBQ_TRY(d_w.alloc(static_cast<size_t>(n) * sizeof(double)));
        SBQ_CUDA(cudaMemcpyAsync(d_src.p, src, vb, cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_nrm.p, nrm, vb, cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_w.p, w, static_cast<size_t>(n) * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
        nnz = 9 * n;
        SBQ_TRY(d_rowptr.alloc((3 * static_cast<size_t>(n) + 1) * sizeof(int64_t)));
        SBQ_TRY(d_col.alloc(static_cast<size_t>(nnz) * sizeof(int64_t)));
        SBQ_TRY(d_val.alloc(static_cast<size_t>(nnz) * sizeof(double)));
        SBQ_TRY(dl_gauss_correction(nbody, body_off, d_src.as<double>(), d_nrm.as<double>(),
                                    d_w.as<double>(), corr_prec, d_rowptr.as<int64_t>(),
                                    d_col.as<int64_t>(), d_val.as<double>(), s));
        SBQ_CUDA(cudaStreamSynchronize(s));
    }
    HostOpGuard g;
    void *h = nullptr;
    SBQ_TRY(op_create_impl(n, src, nrm, w, eta, diag, nnz, d_rowptr.as<int64_t>(),
                           d_col.as<int64_t>(), d_val.as<double>(), nullptr, &h, false, true));
    g.op = static_cast<Op *>(h);
    DevBuf d_rhs, d_x;
    SBQ_TRY(d_rhs.alloc(vb));
    SBQ_TRY(d_x.alloc(vb));
    SBQ_CUDA(cudaMemcpyAsync(d_rhs.p, rhs, vb, cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(d_x.p, x, vb, cudaMemcpyHostToDevice, s));
    // every precision the solve applies K in: shapes from the tuning cache, nothing timed
    SBQ_TRY(op_prepare_untimed(g.op, o->inner_prec, nullptr, s));
    if (mixed) {
        SBQ_TRY(op_prepare_untimed(g.op, o->resid_prec, nullptr, s));
        if (o->resid_prec == SBQ_DF32)
            SBQ_TRY(op_prepare_untimed(g.op, SBQ_FP64, nullptr, s));
    }
    const int st = gmres_solve_impl(g.op, d_rhs.as<double>(), d_x.as<double>(), *o, r, s);
    r.status = st;
    if (st != SBQ_OK && st != SBQ_ENOCONV)
        return st;
    SBQ_CUDA(cudaMemcpyAsync(x, d_x.p, vb, cudaMemcpyDeviceToHost, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return st;
}

SBQ_API int stokes_op_set_mobility(void *oph, int nbody, const int64_t *body_off, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (op->laplace)
        return fail(SBQ_EINVAL, "the mobility formulation is a Stokes formulation");
    if (nbody < 1 || !body_off || body_off[0] != 0 || body_off[nbody] != op->n)
        return fail(SBQ_EINVAL, "body offsets must run from 0 to n");
    for (int b = 0; b < nbody; ++b)
        if (body_off[b + 1] < body_off[b])
            return fail(SBQ_EINVAL, "body offsets must be non-decreasing");
    std::lock_guard<std::mutex> lk(op->mu);
    return mob_setup(op, nbody, body_off, static_cast<cudaStream_t>(stream));
}

SBQ_API int stokes_op_set_tree(void *oph, double theta, int order, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (!std::isfinite(theta))
        return fail(SBQ_EINVAL, "stokes_op_set_tree: non-finite theta");
    std::lock_guard<std::mutex> lk(op->mu);
    const int st = tree_op_attach(op, theta, order, static_cast<cudaStream_t>(stream));
    if (st == SBQ_OK)
        SBQ_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return st;
}

SBQ_API int stokes_op_set_sl_correction(void *oph, int64_t nnz, const int64_t *rowptr,
                                        const int64_t *col, const double *val, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (op->laplace)
        return fail(SBQ_EINVAL, "the single-layer correction serves the Stokes mobility problem");
    if (nnz < 0 || (nnz > 0 && (!rowptr || !col || !val)))
        return fail(SBQ_EINVAL, "negative nnz or null CSR pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(op->mu);
    op->sl_nnz = 0;
    if (nnz == 0) {
        op->sl_rowptr.release();
        op->sl_col.release();
        op->sl_val.release();
        return SBQ_OK;
    }
    const size_t rows = 3 * static_cast<size_t>(op->n);
    SBQ_TRY(op->sl_rowptr.alloc((rows + 1) * sizeof(int64_t)));
    SBQ_TRY(op->sl_col.alloc(static_cast<size_t>(nnz) * sizeof(int64_t)));
    SBQ_TRY(op->sl_val.alloc(static_cast<size_t>(nnz) * sizeof(double)));
    SBQ_CUDA(cudaMemcpyAsync(op->sl_rowptr.p, rowptr, (rows + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(op->sl_col.p, col, nnz * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(op->sl_val.p, val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    op->sl_nnz = nnz;
    return SBQ_OK;
}

SBQ_API int stokes_mobility_rhs(void *oph, const double *FT, const double *us, double *rhs,
                                int prec, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op || !op->mob)
        return fail(SBQ_EINVAL, "not a mobility operator (stokes_op_set_mobility)");
    if (!FT || (op->n > 0 && !rhs))
        return fail(SBQ_EINVAL, "null force/torque or right-hand-side pointer");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    std::lock_guard<std::mutex> lk(op->mu);
    return mob_rhs(op, FT, us, rhs, prec, static_cast<cudaStream_t>(stream));
}

SBQ_API int stokes_mobility_velocity(void *oph, const double *sigma, double *UW, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op || !op->mob)
        return fail(SBQ_EINVAL, "not a mobility operator (stokes_op_set_mobility)");
    if (!UW || (op->n > 0 && !sigma))
        return fail(SBQ_EINVAL, "null density or velocity pointer");
    std::lock_guard<std::mutex> lk(op->mu);
    return mob_velocity(op, sigma, UW, static_cast<cudaStream_t>(stream));
}

SBQ_API int stokes_matvec(const void *oph, const double *sigma, double *out, int prec, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    if (op->n > 0 && (!sigma || !out))
        return fail(SBQ_EINVAL, "null density or output pointer");
    std::lock_guard<std::mutex> lk(op->mu);
    return op_matvec(op, sigma, out, prec, static_cast<cudaStream_t>(stream));
}

SBQ_API int stokes_matvec_bounded(const void *oph, const double *sigma, double *out,
                                  double *bound, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (op->n > 0 && (!sigma || !out || !bound))
        return fail(SBQ_EINVAL, "null density, output or bound pointer");
    std::lock_guard<std::mutex> lk(op->mu);
    return op_matvec(op, sigma, out, SBQ_DF32, static_cast<cudaStream_t>(stream), bound);
}

SBQ_API int sbq_op_time_pairsum(const void *oph, const double *sigma, double *out, int prec,
                                int reps, void *stream, double *kernel_ms, double *apply_ms)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    if (reps < 1)
        return fail(SBQ_EINVAL, "reps < 1");
    if (op->n > 0 && (!sigma || !out))
        return fail(SBQ_EINVAL, "null density or output pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(op->mu);
    SBQ_TRY(op_ensure_tuned(op, prec, s));
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int st = SBQ_OK;
    for (int i = 0; i < 4 && st == SBQ_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess)
            st = fail(SBQ_ECUDA, "cudaEventCreate");
    PairsumTiming pt;
    pt.before = ev[0];
    pt.after = ev[1];
    double ksum = 0.0, asum = 0.0;
    for (int r = 0; r < reps && st == SBQ_OK; ++r) {
        cudaEventRecord(ev[2], s);
        pairsum_timing() = &pt;
        st = op_matvec(op, sigma, out, prec, s);
        pairsum_timing() = nullptr;
        cudaEventRecord(ev[3], s);
        if (st != SBQ_OK)
            break;
        cudaError_t e = cudaEventSynchronize(ev[3]);
        float k = 0.0f, a = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&k, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[2], ev[3]);
        if (e != cudaSuccess)
            st = cuda_status(e, "pair-sum timing");
        ksum += k;
        asum += a;
    }
    for (cudaEvent_t e : ev)
        if (e)
            cudaEventDestroy(e);
    if (st != SBQ_OK)
        return st;
    if (kernel_ms)
        *kernel_ms = ksum / reps;
    if (apply_ms)
        *apply_ms = asum / reps;
    return SBQ_OK;
}

SBQ_API int gmres_solve(const void *oph, const double *rhs, double *x, const sbq_gmres_opts *o,
                        sbq_gmres_report *rep, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (!o)
        return fail(SBQ_EINVAL, "null options");
    if (op->n > 0 && (!rhs || !x))
        return fail(SBQ_EINVAL, "null rhs or solution pointer");
    if (!(o->tol > 0.0) || o->restart < 1 || o->restart > 256 || o->max_iter < 1 ||
        !prec_ok(o->inner_prec))
        return fail(SBQ_EINVAL, "bad GMRES options (tol > 0, 1 <= restart <= 256, max_iter >= 1)");
    const bool mixed = (o->inner_prec == SBQ_FP32 || o->inner_prec == SBQ_FP32_COMP);
    if (mixed && (!(o->inner_tol > 0.0) || o->inner_tol >= 1.0 || o->max_outer < 1))
        return fail(SBQ_EINVAL, "bad refinement options (0 < inner_tol < 1, max_outer >= 1)");
    if (mixed && o->resid_prec != SBQ_FP64 && o->resid_prec != SBQ_DF32)
        return fail(SBQ_EINVAL, "resid_prec must be SBQ_FP64 or SBQ_DF32");
    sbq_gmres_report local{};
    sbq_gmres_report &r = rep ? *rep : local;
    if (op->n == 0) {
        r = sbq_gmres_report{};
        return SBQ_OK;
    }
    std::lock_guard<std::mutex> lk(op->mu);
    const int st = gmres_solve_impl(op, rhs, x, *o, r, static_cast<cudaStream_t>(stream));
    r.status = st;
    return st;
}

SBQ_API int sbq_autotune(void *oph, int prec, sbq_tune *out, void *stream)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op)
        return fail(SBQ_EINVAL, "not an operator handle");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    std::lock_guard<std::mutex> lk(op->mu);
    if (op->n > 0)
        SBQ_TRY(op_autotune(op, prec, static_cast<cudaStream_t>(stream)));
    if (out && op->ts[prec])
        *out = op->ts[prec]->tune;
    return SBQ_OK;
}

SBQ_API int sbq_op_tune(const void *oph, int prec, sbq_tune *out)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op || !out || !prec_ok(prec))
        return fail(SBQ_EINVAL, "bad arguments");
    if (!op->ts[prec])
        return fail(SBQ_EINVAL, "no tile shape chosen yet for this precision");
    *out = op->ts[prec]->tune;
    return SBQ_OK;
}

SBQ_API int sbq_op_stats(const void *oph, int prec, int *kernels_per_matvec, double *pairs_per_matvec)
{
    clear_error();
    Op *op = as_op(oph);
    if (!op || !prec_ok(prec))
        return fail(SBQ_EINVAL, "bad arguments");
    if (kernels_per_matvec)
        *kernels_per_matvec = op_kernels_per_matvec(op, prec);
    if (pairs_per_matvec)
        *pairs_per_matvec = op->ts[prec] ? op->ts[prec]->pairs : 0.0;
    return SBQ_OK;
}

SBQ_API int sbq_check_device(void *stream)
{
    clear_error();
    SBQ_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int *err = device_error_word();
    if (!err)
        return fail(SBQ_ENOMEM, "cannot allocate the device error word");
    int h = 0;
    SBQ_CUDA(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0)
        SBQ_CUDA(cudaMemset(err, 0, sizeof(int)));
    // the allocation-free apply keeps its own word inside its fixed scratch array
    int hn = 0;
    SBQ_TRY(noalloc_take_error(&hn));
    if ((h | hn) & DEV_ERR_TIMEOUT)
        return fail(SBQ_ETIMEOUT, "a device-side bounded wait expired");
    return SBQ_OK;
}

SBQ_API int stokes_dl_gauss_correction(int nbody, const int64_t *body_off, const double *src,
                                       const double *nrm, const double *w, int prec,
                                       int64_t *rowptr, int64_t *col, double *val, void *stream)
{
    clear_error();
    if (nbody < 1 || !body_off)
        return fail(SBQ_EINVAL, "nbody < 1 or null offsets");
    if (body_off[0] != 0)
        return fail(SBQ_EINVAL, "offsets must start at 0");
    for (int i = 0; i < nbody; ++i)
        if (body_off[i + 1] < body_off[i])
            return fail(SBQ_EINVAL, "offsets must be non-decreasing");
    const int64_t n = body_off[nbody];
    if (n > (1LL << 31) / 3)
        return fail(SBQ_EINVAL, "n above 2^31 / 3");
    if (!prec_ok(prec))
        return fail(SBQ_EINVAL, "unknown precision");
    if (!rowptr)
        return fail(SBQ_EINVAL, "null rowptr");
    if (n > 0 && (!src || !nrm || !w || !col || !val))
        return fail(SBQ_EINVAL, "null geometry or CSR pointer");
    return dl_gauss_correction(nbody, body_off, src, nrm, w, prec, rowptr, col, val,
                               static_cast<cudaStream_t>(stream));
}

SBQ_API int tube_correction(int64_t nelem, int ns, int nt, int64_t n_total, const double *src,
                            const double *nrm, const double *w, int laplace, double alpha,
                            double beta, double near_factor, int64_t *nnz_out, int64_t *rowptr,
                            int64_t *col, double *val, void *stream)
{
    clear_error();
    if (nelem < 0 || n_total < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (ns < 2 || ns > 16)
        return fail(SBQ_EINVAL, "ns must be in 2..16");
    if (nt < 4 || nt > 64 || (nt & 1))
        return fail(SBQ_EINVAL, "nt must be even and in 4..64");
    if (nelem * ns * nt > n_total)
        return fail(SBQ_EINVAL, "n_total below nelem * ns * nt");
    if (n_total > (1LL << 31) / 3)
        return fail(SBQ_EINVAL, "n_total above 2^31 / 3");
    if (laplace != 0 && laplace != 1)
        return fail(SBQ_EINVAL, "laplace must be 0 or 1");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(near_factor))
        return fail(SBQ_EINVAL, "non-finite alpha, beta or near_factor");
    if (!rowptr && !nnz_out)
        return fail(SBQ_EINVAL, "null rowptr and nnz_out");
    if (nelem > 0 && (!src || !nrm || !w))
        return fail(SBQ_EINVAL, "null geometry pointer");
    return build_tube_correction(nelem, ns, nt, n_total, src, nrm, w, 0, nullptr, laplace, alpha,
                                 beta, near_factor, nnz_out, rowptr, col, val,
                                 static_cast<cudaStream_t>(stream));
}

SBQ_API int tube_correction_targets(int64_t nelem, int ns, int nt, int64_t n_total,
                                    const double *src, const double *nrm, const double *w,
                                    int64_t ntrg, const double *trg, int laplace, double alpha,
                                    double beta, double near_factor, int64_t *nnz_out,
                                    int64_t *rowptr, int64_t *col, double *val, void *stream)
{
    clear_error();
    if (nelem < 0 || n_total < 0 || ntrg < 0)
        return fail(SBQ_EINVAL, "negative size");
    if (ns < 2 || ns > 16)
        return fail(SBQ_EINVAL, "ns must be in 2..16");
    if (nt < 4 || nt > 64 || (nt & 1))
        return fail(SBQ_EINVAL, "nt must be even and in 4..64");
    if (nelem * ns * nt > n_total)
        return fail(SBQ_EINVAL, "n_total below nelem * ns * nt");
    if (n_total > (1LL << 31) / 3 || ntrg > (1LL << 31) / 3)
        return fail(SBQ_EINVAL, "n_total or ntrg above 2^31 / 3");
    if (laplace != 0 && laplace != 1)
        return fail(SBQ_EINVAL, "laplace must be 0 or 1");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(near_factor))
        return fail(SBQ_EINVAL, "non-finite alpha, beta or near_factor");
    if (!rowptr && !nnz_out)
        return fail(SBQ_EINVAL, "null rowptr and nnz_out");
    if ((nelem > 0 && (!src || !nrm || !w)) || (ntrg > 0 && !trg))
        return fail(SBQ_EINVAL, "null geometry or target pointer");
    return build_tube_correction(nelem, ns, nt, n_total, src, nrm, w, ntrg, trg ? trg : src,
                                 laplace, alpha, beta, near_factor, nnz_out, rowptr, col, val,
                                 static_cast<cudaStream_t>(stream));
}

SBQ_API void sbq_destroy(void *handle)
{
    if (!handle)
        return;
    const uint32_t magic = *static_cast<const uint32_t *>(handle);
    if (magic == OP_MAGIC) {
        Op *op = static_cast<Op *>(handle);
        op->magic = 0;
        delete op;
    } else if (magic == PLAN_MAGIC) {
        PlanH *p = static_cast<PlanH *>(handle);
        p->magic = 0;
        delete p;
    }
}

}  // extern "C"
