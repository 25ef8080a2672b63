// GMRES for K sigma = u0 (paper Eq. stokes-bie-new), on the device, FP64 Krylov algebra.
//
// The paper solves its second-kind BIEs with unpreconditioned GMRES (Sec. 4, Sec. 5)
// without stating restart, orthogonalisation or initial guess.  This solver uses
// restarted GMRES(m) with classical Gram--Schmidt applied twice and Givens rotations;
// every quantity of the Krylov method (basis, Hessenberg matrix, rotations, residual
// estimate, solution update) is FP64 on the GPU.  Two drivers:
//   * plain FP64: every operator apply is the FP64 pair sum; a cycle ends on the
//     Givens estimate, the true FP64 residual decides the restart;
//   * iterative refinement: the FP64 residual r = b - K x is formed, K d = r is solved
//     by GMRES whose operator applies run in FP32 or compensated FP32, x += d, repeat.
// Each Arnoldi step (operator apply + CGS2 + Givens) is a fixed sequence of kernels
// that read the step index from device memory, so one captured copy of it serves every
// step: it is the body of a CUDA-graph while node, which repeats it on the device until
// the cycle ends (convergence, breakdown or m steps).
#include "engine.h"

#include <chrono>
#include <cmath>

namespace sbq {

constexpr int GB = 256;          // threads of the vector kernels
constexpr int MAX_RESTART = 256;

struct GState {
    int j;          // completed Arnoldi steps of the cycle (= index of the next column)
    int stop;       // the cycle must end
    int conv;       // Givens estimate <= tol_abs
    int brk;        // exact breakdown (h_{j+1,j} == 0)
    int m;          // step limit of this cycle
    int iters;      // Arnoldi steps since the solve began
    int nonfinite;  // a non-finite norm was seen
    int pad_;
    double tol_abs; // absolute tolerance on the residual norm of the system being solved
    double beta;    // residual norm at the start of the cycle
    double res_est; // |g_{j}| after the last step
    double res_true;// last norm computed by k_norm_fin
    double inv_hn;  // 1 / h_{j+1,j} of the last step (0 on breakdown)
};

struct GmresWS {
    int device = 0;
    int m = 0;
    long long N = 0;
    int nblk = 0;
    int ldp = 0;
    DevBuf V, H, cs, sn, g, y, hb, w, vin, r, d, ax, part, st;
    GState *hst = nullptr;             // pinned host mirror
    cudaStream_t cap = nullptr;        // capture stream
    cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    bool graph_tried[3] = {false, false, false};
    long long launches = 0;            // kernels executed by the current solve
};

int gmres_destroy(GmresWS *ws)
{
    if (!ws)
        return SBQ_OK;
    for (int i = 0; i < 3; ++i) {
        if (ws->exec[i])
            cudaGraphExecDestroy(ws->exec[i]);
        if (ws->graph[i])
            cudaGraphDestroy(ws->graph[i]);
    }
    if (ws->cap)
        cudaStreamDestroy(ws->cap);
    if (ws->hst)
        cudaFreeHost(ws->hst);
    delete ws;
    return SBQ_OK;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
namespace {

__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;   // thread 0
}

__device__ __forceinline__ void block_rows(long long N, long long &a, long long &b)
{
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    a = static_cast<long long>(blockIdx.x) * chunk;
    b = a + chunk < N ? a + chunk : N;
}

// part[b * ldp + k] = sum over the rows of block b of V[k][i] w[i], k = 0..j.
__global__ void k_dots(const double *__restrict__ V, long long N, const GState *__restrict__ st,
                       const double *__restrict__ w, double *part, int ldp)
{
    __shared__ double red[32];
    const int j = st->j;
    long long a, b;
    block_rows(N, a, b);
    for (int k0 = 0; k0 <= j; k0 += 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
            const double wi = w[i];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k0 + q <= j)
                    acc[q] = fma(V[static_cast<size_t>(k0 + q) * N + i], wi, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double s = block_sum(acc[q], red);
            if (threadIdx.x == 0 && k0 + q <= j)
                part[static_cast<size_t>(blockIdx.x) * ldp + k0 + q] = s;
        }
    }
}

// hb[k] = sum_b part[b][k] (fixed order); column j of H gets it (pass 0) or adds it (pass 1).
__global__ void k_dots_fin(const double *__restrict__ part, int nblk, int ldp, const GState *st,
                           double *H, double *hb, int pass)
{
    const int j = st->j, m1 = MAX_RESTART + 1;
    (void)m1;
    const int ld = st->m + 1;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b)
            s += part[static_cast<size_t>(b) * ldp + k];
        hb[k] = s;
        double *h = H + static_cast<size_t>(j) * ld + k;
        *h = pass ? *h + s : s;
    }
}

// w[i] -= sum_{k <= j} V[k][i] hb[k]
__global__ void k_axpy_multi(const double *__restrict__ V, long long N, const GState *__restrict__ st,
                             const double *__restrict__ hb, double *w)
{
    __shared__ double sh[MAX_RESTART + 1];
    const int j = st->j;
    for (int k = threadIdx.x; k <= j; k += blockDim.x)
        sh[k] = hb[k];
    __syncthreads();
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        double acc = w[i];
        for (int k = 0; k <= j; ++k)
            acc = fma(-V[static_cast<size_t>(k) * N + i], sh[k], acc);
        w[i] = acc;
    }
}

__global__ void k_norm_part(const double *__restrict__ x, long long N, double *part)
{
    __shared__ double red[32];
    long long a, b;
    block_rows(N, a, b);
    double acc = 0.0;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x)
        acc = fma(x[i], x[i], acc);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

__global__ void k_norm_fin(const double *__restrict__ part, int nblk, GState *st)
{
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b)
            s += part[b];
        const double r = sqrt(s);
        st->res_true = r;
        if (!isfinite(r))
            st->nonfinite = 1;
    }
}

// New column of H: h_{j+1,j}, previous rotations, new rotation, residual estimate.
__global__ void k_arnoldi_fin(const double *__restrict__ part, int nblk, GState *st, double *H,
                              double *cs, double *sn, double *g)
{
    if (threadIdx.x != 0)
        return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b)
        s += part[b];
    const double hn = sqrt(s);
    const int j = st->j, ld = st->m + 1;
    double *col = H + static_cast<size_t>(j) * ld;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = col[i], c = col[i + 1];
        col[i] = cs[i] * a + sn[i] * c;
        col[i + 1] = -sn[i] * a + cs[i] * c;
    }
    const double a = col[j], c = col[j + 1];
    const double den = hypot(a, c);
    const double cj = (den == 0.0) ? 1.0 : a / den, sj = (den == 0.0) ? 0.0 : c / den;
    cs[j] = cj;
    sn[j] = sj;
    col[j] = cj * a + sj * c;
    col[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
    const double est = fabs(g[j + 1]);
    st->res_est = est;
    st->iters += 1;
    const bool nonfinite = !isfinite(hn) || !isfinite(est);
    st->nonfinite |= nonfinite ? 1 : 0;
    st->conv = est <= st->tol_abs;
    st->brk = (hn == 0.0);
    st->inv_hn = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    st->stop = st->conv || st->brk || nonfinite || (j + 1 >= st->m);
}

__global__ void k_normalize(const double *__restrict__ w, long long N, const GState *__restrict__ st,
                            double *V)
{
    const int j = st->j;
    const double s = st->inv_hn;
    double *v = V + static_cast<size_t>(j + 1) * N;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        v[i] = w[i] * s;
}

__global__ void k_advance(GState *st, cudaGraphConditionalHandle h, int use_cond)
{
    if (threadIdx.x == 0) {
        st->j += 1;
        if (use_cond)
            cudaGraphSetConditional(h, st->stop ? 0u : 1u);
    }
}

__global__ void k_copy_col(const double *__restrict__ V, long long N, const GState *__restrict__ st,
                           double *vin)
{
    const double *v = V + static_cast<size_t>(st->j) * N;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        vin[i] = v[i];
}

// Start a cycle from the residual whose norm k_norm_fin left in res_true.
__global__ void k_cycle_init(GState *st, double *g, int m, double tol_abs)
{
    if (threadIdx.x == 0) {
        const double beta = st->res_true;
        st->beta = beta;
        st->j = 0;
        st->stop = 0;
        st->conv = 0;
        st->brk = 0;
        st->m = m;
        st->tol_abs = tol_abs;
        st->res_est = beta;
        for (int i = 0; i <= m; ++i)
            g[i] = 0.0;
        g[0] = beta;
    }
}

__global__ void k_scale_first(const double *__restrict__ r, long long N, const GState *__restrict__ st,
                              double *V)
{
    const double inv = 1.0 / st->beta;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        V[i] = r[i] * inv;
}

// y = H^{-1} g over the j completed steps (upper triangular after the rotations).
__global__ void k_solve_y(const GState *__restrict__ st, const double *__restrict__ H,
                          const double *__restrict__ g, double *y)
{
    if (threadIdx.x != 0)
        return;
    const int k = st->j, ld = st->m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l)
            s -= H[static_cast<size_t>(l) * ld + i] * y[l];
        y[i] = s / H[static_cast<size_t>(i) * ld + i];
    }
}

// x += sum_{k < j} V[k] y[k]
__global__ void k_update_x(const double *__restrict__ V, long long N, const GState *__restrict__ st,
                           const double *__restrict__ y, double *x)
{
    __shared__ double sy[MAX_RESTART];
    const int k = st->j;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        sy[i] = y[i];
    __syncthreads();
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        double acc = x[i];
        for (int l = 0; l < k; ++l)
            acc = fma(V[static_cast<size_t>(l) * N + i], sy[l], acc);
        x[i] = acc;
    }
}

__global__ void k_sub(const double *__restrict__ b, const double *__restrict__ ax, double *r,
                      long long N)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        r[i] = b[i] - ax[i];
}

__global__ void k_add(const double *__restrict__ d, double *x, long long N)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        x[i] += d[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
static int vec_grid(long long N)
{
    const long long want = (N + GB - 1) / GB;
    const long long cap = 8LL * device_props().sms;
    return static_cast<int>(std::max<long long>(1, std::min(want, cap)));
}

static int ws_ensure(Op *op, int m)
{
    if (m < 1 || m > MAX_RESTART) {
        set_error("restart must be in 1..256");
        return SBQ_EINVAL;
    }
    if (op->gm && op->gm->m >= m)
        return SBQ_OK;
    if (op->gm) {
        gmres_destroy(op->gm);
        op->gm = nullptr;
    }
    auto *ws = new GmresWS();
    ws->m = m;
    ws->N = 3 * op->n;
    const long long N = ws->N;
    ws->nblk = static_cast<int>(std::max<long long>(1, std::min<long long>(2LL * device_props().sms,
                                                                        (N + 2047) / 2048)));
    ws->ldp = m + 1;
    int s = SBQ_OK;
    if (s == SBQ_OK) s = ws->V.alloc(static_cast<size_t>(m + 1) * N * sizeof(double));
    if (s == SBQ_OK) s = ws->H.alloc(static_cast<size_t>(m + 1) * m * sizeof(double));
    if (s == SBQ_OK) s = ws->cs.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->sn.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->g.alloc((m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->y.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->hb.alloc((m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->w.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->vin.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->r.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->d.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->ax.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->part.alloc(static_cast<size_t>(ws->nblk) * (m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->st.alloc(sizeof(GState));
    if (s == SBQ_OK) {
        cudaError_t e = cudaMallocHost(&ws->hst, sizeof(GState));
        if (e != cudaSuccess)
            s = cuda_status(e, "cudaMallocHost");
    }
    if (s == SBQ_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            s = cuda_status(e, "cudaStreamCreate");
    }
    if (s == SBQ_OK) {
        cudaError_t e = cudaMemset(ws->st.p, 0, sizeof(GState));
        if (e != cudaSuccess)
            s = cuda_status(e, "cudaMemset");
    }
    if (s != SBQ_OK) {
        gmres_destroy(ws);
        return s;
    }
    cudaGetDevice(&ws->device);
    op->gm = ws;
    return SBQ_OK;
}

// Enqueue one Arnoldi step on stream s (use_cond: inside the while body).
static int enqueue_step(Op *op, GmresWS *ws, int prec, cudaStream_t s,
                        cudaGraphConditionalHandle h, int use_cond)
{
    const long long N = ws->N;
    GState *st = ws->st.as<GState>();
    const int vg = vec_grid(N);
    k_copy_col<<<vg, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->vin.as<double>());
    SBQ_CUDA(cudaGetLastError());
    SBQ_TRY(op_matvec(op, ws->vin.as<double>(), ws->w.as<double>(), prec, s));
    for (int pass = 0; pass < 2; ++pass) {
        k_dots<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->w.as<double>(),
                                       ws->part.as<double>(), ws->ldp);
        k_dots_fin<<<1, GB, 0, s>>>(ws->part.as<double>(), ws->nblk, ws->ldp, st,
                                    ws->H.as<double>(), ws->hb.as<double>(), pass);
        k_axpy_multi<<<vg, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->hb.as<double>(),
                                       ws->w.as<double>());
    }
    k_norm_part<<<ws->nblk, GB, 0, s>>>(ws->w.as<double>(), N, ws->part.as<double>());
    k_arnoldi_fin<<<1, 32, 0, s>>>(ws->part.as<double>(), ws->nblk, st, ws->H.as<double>(),
                                   ws->cs.as<double>(), ws->sn.as<double>(), ws->g.as<double>());
    k_normalize<<<vg, GB, 0, s>>>(ws->w.as<double>(), N, st, ws->V.as<double>());
    k_advance<<<1, 32, 0, s>>>(st, h, use_cond);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

// Kernels of one Arnoldi step (enqueue_step).
static int step_kernels(const Op *op, int prec) { return 1 + op_kernels_per_matvec(op, prec) + 6 + 4; }

// Build the while-node graph of one Arnoldi step for precision prec.
static int build_graph(Op *op, GmresWS *ws, int prec)
{
    ws->graph_tried[prec] = true;
    cudaGraph_t g = nullptr;
    SBQ_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "cudaGraphAddNode(while)");
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(ws->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "cudaStreamBeginCaptureToGraph");
    }
    int st = enqueue_step(op, ws, prec, ws->cap, h, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(ws->cap, &captured);
    if (st != SBQ_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (st != SBQ_OK)
            return st;
        return cuda_status(e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "cudaGraphInstantiate");
    }
    ws->graph[prec] = g;
    ws->exec[prec] = ex;
    return SBQ_OK;
}

static int read_state(GmresWS *ws, cudaStream_t s)
{
    SBQ_CUDA(cudaMemcpyAsync(ws->hst, ws->st.p, sizeof(GState), cudaMemcpyDeviceToHost, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

// ||v|| into st->res_true (and the host mirror).
static int norm_to_state(GmresWS *ws, const double *v, cudaStream_t s)
{
    k_norm_part<<<ws->nblk, GB, 0, s>>>(v, ws->N, ws->part.as<double>());
    k_norm_fin<<<1, 32, 0, s>>>(ws->part.as<double>(), ws->nblk, ws->st.as<GState>());
    SBQ_CUDA(cudaGetLastError());
    ws->launches += 2;
    return read_state(ws, s);
}

// r = b - K x in precision prec; ||r|| to the state.
static int residual(Op *op, GmresWS *ws, int prec, const double *b, const double *x, double *r,
                    cudaStream_t s)
{
    SBQ_TRY(op_matvec(op, x, ws->ax.as<double>(), prec, s));
    k_sub<<<vec_grid(ws->N), GB, 0, s>>>(b, ws->ax.as<double>(), r, ws->N);
    SBQ_CUDA(cudaGetLastError());
    ws->launches += op_kernels_per_matvec(op, prec) + 1;
    return norm_to_state(ws, r, s);
}

// One GMRES cycle from residual r (norm in the state) updating xu += V y.
static int run_cycle(Op *op, GmresWS *ws, int prec, const double *r, double *xu, int m,
                     double tol_abs, bool use_graph, cudaStream_t s, bool *graph_used)
{
    const long long N = ws->N;
    GState *st = ws->st.as<GState>();
    k_cycle_init<<<1, 32, 0, s>>>(st, ws->g.as<double>(), m, tol_abs);
    k_scale_first<<<vec_grid(N), GB, 0, s>>>(r, N, st, ws->V.as<double>());
    SBQ_CUDA(cudaGetLastError());
    bool done = false;
    if (use_graph) {
        if (!ws->graph_tried[prec]) {
            // capture happens on the internal stream: order it after the work on s
            SBQ_CUDA(cudaStreamSynchronize(s));
            int gs = build_graph(op, ws, prec);
            if (gs != SBQ_OK)
                clear_error();   // fall back to host-driven steps below
        }
        if (ws->exec[prec]) {
            SBQ_CUDA(cudaGraphLaunch(ws->exec[prec], s));
            *graph_used = true;
            done = true;
        }
    }
    if (!done) {
        for (int it = 0; it < m; ++it) {
            SBQ_TRY(enqueue_step(op, ws, prec, s, 0, 0));
            SBQ_TRY(read_state(ws, s));
            if (ws->hst->stop)
                break;
        }
    }
    k_solve_y<<<1, 32, 0, s>>>(st, ws->H.as<double>(), ws->g.as<double>(), ws->y.as<double>());
    k_update_x<<<vec_grid(N), GB, 0, s>>>(ws->V.as<double>(), N, st, ws->y.as<double>(), xu);
    SBQ_CUDA(cudaGetLastError());
    SBQ_TRY(read_state(ws, s));
    ws->launches += 4 + static_cast<long long>(ws->hst->j) * step_kernels(op, prec);
    return SBQ_OK;
}

int gmres_solve_impl(Op *op, const double *b, double *x, const sbq_gmres_opts &o,
                     sbq_gmres_report &rep, cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    rep = sbq_gmres_report{};
    const int low = o.inner_prec;
    const bool mixed = (low == SBQ_FP32 || low == SBQ_FP32_COMP);
    SBQ_TRY(ws_ensure(op, o.restart));
    GmresWS *ws = op->gm;
    ws->launches = 0;
    const long long N = ws->N;
    if (!device_error_word()) {
        set_error("cannot allocate the device error word");
        return SBQ_ENOMEM;
    }
    SBQ_TRY(op_ensure_tuned(op, SBQ_FP64, s));
    if (mixed)
        SBQ_TRY(op_ensure_tuned(op, low, s));

    SBQ_TRY(norm_to_state(ws, b, s));
    const double bnorm = ws->hst->res_true;
    if (!std::isfinite(bnorm)) {
        set_error("right-hand side is not finite");
        return SBQ_ENONFINITE;
    }
    if (bnorm == 0.0) {
        SBQ_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        SBQ_CUDA(cudaStreamSynchronize(s));
        rep.status = SBQ_OK;
        rep.n_hist = 1;
        rep.rel_res_hist[0] = 0.0;
        return SBQ_OK;
    }
    const double tol_abs = o.tol * bnorm;
    bool graph_used = false;
    auto push_hist = [&](double v) {
        if (rep.n_hist < SBQ_HIST)
            rep.rel_res_hist[rep.n_hist++] = v;
    };

    SBQ_TRY(residual(op, ws, SBQ_FP64, b, x, ws->r.as<double>(), s));
    rep.matvecs_fp64 += 1;
    double res = ws->hst->res_true;
    push_hist(res / bnorm);
    int status = SBQ_OK;
    while (res > tol_abs) {
        if (!std::isfinite(res)) {
            status = SBQ_ENONFINITE;
            set_error("residual is not finite");
            break;
        }
        if (rep.iters >= o.max_iter || (mixed && rep.outer_iters >= o.max_outer)) {
            status = SBQ_ENOCONV;
            set_error("GMRES reached its iteration cap above the tolerance");
            break;
        }
        if (!mixed) {
            const int m = std::min(o.restart, o.max_iter - rep.iters);
            SBQ_TRY(run_cycle(op, ws, SBQ_FP64, ws->r.as<double>(), x, m, tol_abs, o.use_graph != 0,
                              s, &graph_used));
            const int steps = ws->hst->j;
            rep.iters += steps;
            rep.matvecs_fp64 += steps;
            const bool brk = ws->hst->brk != 0;
            if (ws->hst->nonfinite) {
                status = SBQ_ENONFINITE;
                set_error("non-finite value in the Arnoldi process");
                break;
            }
            SBQ_TRY(residual(op, ws, SBQ_FP64, b, x, ws->r.as<double>(), s));
            rep.matvecs_fp64 += 1;
            rep.outer_iters += 1;
            const double nres = ws->hst->res_true;
            push_hist(nres / bnorm);
            if (brk && nres > tol_abs && nres >= res) {
                status = SBQ_EBREAKDOWN;
                set_error("GMRES breakdown without convergence");
                res = nres;
                break;
            }
            res = nres;
        } else {
            // inner solve K_low d = r, d = 0, to inner_tol * ||r||
            double *d = ws->d.as<double>();
            SBQ_CUDA(cudaMemsetAsync(d, 0, N * sizeof(double), s));
            const double inner_abs = o.inner_tol * res;
            double ires = res;
            const double *rin = ws->r.as<double>();
            // the inner residual lives in ws->w between restarts; the first cycle starts
            // from r itself, whose norm is in the state already
            for (;;) {
                const int m = std::min(o.restart, o.max_iter - rep.iters);
                if (m <= 0)
                    break;
                SBQ_TRY(run_cycle(op, ws, low, rin, d, m, inner_abs, o.use_graph != 0, s,
                                  &graph_used));
                const int steps = ws->hst->j;
                rep.iters += steps;
                rep.matvecs_low += steps;
                if (ws->hst->nonfinite) {
                    status = SBQ_ENONFINITE;
                    break;
                }
                if (ws->hst->conv || ws->hst->brk)
                    break;
                // restart the inner solve from its true low-precision residual
                SBQ_TRY(op_matvec(op, d, ws->ax.as<double>(), low, s));
                rep.matvecs_low += 1;
                k_sub<<<vec_grid(N), GB, 0, s>>>(ws->r.as<double>(), ws->ax.as<double>(),
                                                 ws->vin.as<double>(), N);
                SBQ_CUDA(cudaGetLastError());
                ws->launches += op_kernels_per_matvec(op, low) + 1;
                SBQ_TRY(norm_to_state(ws, ws->vin.as<double>(), s));
                const double nr = ws->hst->res_true;
                if (!(nr < ires) || nr <= inner_abs)
                    break;
                ires = nr;
                // the cycle overwrites vin (k_copy_col) only after k_scale_first has read it
                rin = ws->vin.as<double>();
            }
            if (status != SBQ_OK) {
                set_error("non-finite value in the inner solve");
                break;
            }
            k_add<<<vec_grid(N), GB, 0, s>>>(d, x, N);
            SBQ_CUDA(cudaGetLastError());
            ws->launches += 1;
            SBQ_TRY(residual(op, ws, SBQ_FP64, b, x, ws->r.as<double>(), s));
            rep.matvecs_fp64 += 1;
            rep.outer_iters += 1;
            const double nres = ws->hst->res_true;
            push_hist(nres / bnorm);
            if (!(nres < res)) {
                res = nres;
                status = SBQ_ENOCONV;
                set_error("iterative refinement stagnated above the tolerance");
                break;
            }
            res = nres;
        }
    }
    SBQ_CUDA(cudaStreamSynchronize(s));
    rep.rel_res = res / bnorm;
    rep.graph_used = graph_used ? 1 : 0;
    rep.kernel_launches = static_cast<int>(std::min<long long>(ws->launches, INT32_MAX));
    rep.status = status;
    rep.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
    return status;
}

}  // namespace sbq
