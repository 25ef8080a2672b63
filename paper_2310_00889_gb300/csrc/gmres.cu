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
// Each Arnoldi step is a fixed sequence of kernels that read the step index from device
// memory, so one captured copy of it serves every step: it is the body of a CUDA-graph
// while node, which repeats it on the device until the cycle ends (convergence,
// breakdown or m steps).  One step is: operator apply on v_j; first Gram--Schmidt
// pass (partial dots, finished by the last block); second pass fused with the first
// update of w; norm fused with the second update, whose last block also applies the
// Givens rotations; normalisation that writes v_{j+1} and the next operator input.
#include "engine.h"

#include <chrono>
#include <cmath>

namespace sbq {

constexpr int GB = 256;          // threads of the vector kernels
constexpr int MAX_RESTART = 256;
constexpr int SOLVE_SMEM_MAX_M = 200;   // back-substitution keeps R in shared memory up to this m

struct GState {
    int j;          // completed Arnoldi steps of the cycle (= index of the next column)
    int stop;       // the cycle must end
    int conv;       // Givens estimate <= tol_abs
    int brk;        // exact breakdown (h_{j+1,j} == 0)
    int m;          // step limit of this cycle
    int iters;      // Arnoldi steps since the solve began
    int nonfinite;  // a non-finite norm was seen
    unsigned int ctr;   // blocks finished in the current fused kernel
    int guard;      // steps run in this cycle, counted by k_guard
    int guard_hit;  // k_guard ended the cycle (the step counter failed to stop it)
    double tol_abs; // absolute tolerance on the residual norm of the system being solved
    double beta;    // residual norm at the start of the cycle
    double res_est; // |g_{j}| after the last step
    double res_true;// last norm computed by a norm kernel
    double inv_hn;  // 1 / h_{j+1,j} of the last step (0 on breakdown)
};

struct GmresWS {
    int device = 0;
    int m = 0;
    long long N = 0;
    int nblk = 0;
    int ldp = 0;
    size_t solve_smem = 0;
    DevBuf V, H, cs, sn, g, y, hb1, hb2, w, vin, r, d, ax, part, st;
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

// Rows [a, b) owned by this block; every fused kernel uses the same partition.
__device__ __forceinline__ void block_rows(long long N, long long &a, long long &b)
{
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    a = static_cast<long long>(blockIdx.x) * chunk;
    b = a + chunk < N ? a + chunk : N;
}

// True in the block that finishes last (all other blocks' writes are visible to it).
__device__ bool last_block(unsigned int *ctr)
{
    __shared__ unsigned int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = (atomicAdd(ctr, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last)
        __threadfence();
    return s_last != 0;
}

// part[blockIdx][k] = sum over the block's rows of V[k][i] w[i], k = 0..j: one warp per
// Krylov vector, lanes striding over the rows (coalesced), no block barrier.
__device__ void block_multi_dot(const double *__restrict__ V, long long N, int j,
                                const double *__restrict__ w, long long a, long long b,
                                double *part_row)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k <= j; k += nw) {
        const double *v = V + static_cast<size_t>(k) * N;
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
        long long i = a + lane;
        for (; i + 96 < b; i += 128) {
            acc0 = fma(v[i], w[i], acc0);
            acc1 = fma(v[i + 32], w[i + 32], acc1);
            acc2 = fma(v[i + 64], w[i + 64], acc2);
            acc3 = fma(v[i + 96], w[i + 96], acc3);
        }
        for (; i < b; i += 32)
            acc0 = fma(v[i], w[i], acc0);
        double acc = (acc0 + acc1) + (acc2 + acc3);
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0)
            part_row[k] = acc;
    }
}

// Last block: hb[k] = sum_b part[b][k] (one warp per k, lanes over the blocks, fixed
// order); column j of H gets (pass 0) or adds (pass 1) it.
__device__ void finish_dots(const double *part, int ldp, GState *st, double *H, double *hb, int pass)
{
    const int j = st->j, ld = st->m + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k <= j; k += nw) {
        double s = 0.0;
        for (int bb = lane; bb < (int)gridDim.x; bb += 32)
            s += __ldcg(part + static_cast<size_t>(bb) * ldp + k);
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            hb[k] = s;
            double *h = H + static_cast<size_t>(j) * ld + k;
            *h = pass ? *h + s : s;
        }
    }
    if (threadIdx.x == 0)
        st->ctr = 0;
}

// First Gram--Schmidt pass: h1 = V[0..j]^T w.
__global__ void k_cgs_pass1(const double *__restrict__ V, long long N, GState *st,
                            const double *__restrict__ w, double *part, int ldp, double *H,
                            double *hb1)
{
    long long a, b;
    block_rows(N, a, b);
    block_multi_dot(V, N, st->j, w, a, b, part + static_cast<size_t>(blockIdx.x) * ldp);
    if (last_block(&st->ctr))
        finish_dots(part, ldp, st, H, hb1, 0);
}

// w -= V h1 on this block's rows, then the second pass h2 = V^T w on the same rows.
__global__ void k_cgs_pass2(const double *__restrict__ V, long long N, GState *st,
                            const double *__restrict__ hb1, double *w, double *part, int ldp,
                            double *H, double *hb2)
{
    __shared__ double sh[MAX_RESTART + 1];
    const int j = st->j;
    for (int k = threadIdx.x; k <= j; k += blockDim.x)
        sh[k] = hb1[k];
    __syncthreads();
    long long a, b;
    block_rows(N, a, b);
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
        double acc = w[i];
#pragma unroll 8
        for (int k = 0; k <= j; ++k)
            acc = fma(-V[static_cast<size_t>(k) * N + i], sh[k], acc);
        w[i] = acc;
    }
    __syncthreads();   // the dots below read rows of w that other threads just updated
    block_multi_dot(V, N, j, w, a, b, part + static_cast<size_t>(blockIdx.x) * ldp);
    if (last_block(&st->ctr))
        finish_dots(part, ldp, st, H, hb2, 1);
}

// w -= V h2 and ||w||^2 on this block's rows; the last block forms h_{j+1,j}, applies the
// previous Givens rotations to column j, builds the new one and updates the residual
// estimate and the stop flags.
__global__ void k_cgs_norm_givens(const double *__restrict__ V, long long N, GState *st,
                                  const double *__restrict__ hb2, double *w, double *part,
                                  double *H, double *cs, double *sn, double *g)
{
    __shared__ double sh[MAX_RESTART + 1];
    __shared__ double red[32];
    const int j = st->j;
    for (int k = threadIdx.x; k <= j; k += blockDim.x)
        sh[k] = hb2[k];
    __syncthreads();
    long long a, b;
    block_rows(N, a, b);
    double nrm = 0.0;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
        double acc = w[i];
#pragma unroll 8
        for (int k = 0; k <= j; ++k)
            acc = fma(-V[static_cast<size_t>(k) * N + i], sh[k], acc);
        w[i] = acc;
        nrm = fma(acc, acc, nrm);
    }
    const double bs = block_sum(nrm, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = bs;
    if (!last_block(&st->ctr))
        return;
    // the last block: column j of H and the rotations into shared memory in parallel,
    // the sequential rotation sweep by one thread, results written back in parallel
    __shared__ double scol[MAX_RESTART + 1], scs[MAX_RESTART], ssn[MAX_RESTART];
    __shared__ double s_hn;
    const int ld = st->m + 1;
    double *col = H + static_cast<size_t>(j) * ld;
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        scol[i] = __ldcg(col + i);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        scs[i] = __ldcg(cs + i);
        ssn[i] = __ldcg(sn + i);
    }
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int bb = threadIdx.x; bb < (int)gridDim.x; bb += 32)
            t += __ldcg(part + bb);
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0)
            s_hn = sqrt(t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->ctr = 0;
        const double hn = s_hn;
        for (int i = 0; i < j; ++i) {
            const double x0 = scol[i], x1 = scol[i + 1];
            scol[i] = scs[i] * x0 + ssn[i] * x1;
            scol[i + 1] = -ssn[i] * x0 + scs[i] * x1;
        }
        const double x0 = scol[j], x1 = hn;
        const double den = hypot(x0, x1);
        const double cj = (den == 0.0) ? 1.0 : x0 / den, sj = (den == 0.0) ? 0.0 : x1 / den;
        cs[j] = cj;
        sn[j] = sj;
        scol[j] = cj * x0 + sj * x1;
        col[j + 1] = 0.0;
        const double gj = __ldcg(g + j);
        g[j + 1] = -sj * gj;
        g[j] = cj * gj;
        const double est = fabs(sj * gj);
        st->res_est = est;
        st->iters += 1;
        const bool nonfinite = !isfinite(hn) || !isfinite(est);
        st->nonfinite |= nonfinite ? 1 : 0;
        st->conv = est <= st->tol_abs;
        st->brk = (hn == 0.0);
        st->inv_hn = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
        st->stop = st->conv || st->brk || nonfinite || (j + 1 >= st->m);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        col[i] = scol[i];
}

// v_{j+1} = w / h_{j+1,j}, also written to the operator input buffer; the last block
// advances j and, inside the graph, sets the while condition.
__global__ void k_normalize_advance(const double *__restrict__ w, long long N, GState *st,
                                    double *V, double *vin, cudaGraphConditionalHandle h,
                                    int use_cond)
{
    const int j = st->j;
    const double s = st->inv_hn;
    double *v = V + static_cast<size_t>(j + 1) * N;
    long long a, b;
    block_rows(N, a, b);
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
        const double x = w[i] * s;
        v[i] = x;
        vin[i] = x;
    }
    if (last_block(&st->ctr) && threadIdx.x == 0) {
        st->ctr = 0;
        st->j = j + 1;
        if (use_cond)
            cudaGraphSetConditional(h, st->stop ? 0u : 1u);
    }
}

// Independent bound on the while loop: ends the cycle after `cap` steps whatever the
// other kernels did to the step counter.
__global__ void k_guard(GState *st, cudaGraphConditionalHandle h, int cap, int use_cond)
{
    if (threadIdx.x == 0) {
        st->guard += 1;
        if (st->guard >= cap || st->j >= cap) {
            if (!st->stop)
                st->guard_hit = 1;
            st->stop = 1;
            if (use_cond)
                cudaGraphSetConditional(h, 0u);
        }
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
        st->ctr = 0;
        st->guard = 0;
        st->m = m;
        st->tol_abs = tol_abs;
        st->res_est = beta;
        for (int i = 0; i <= m; ++i)
            g[i] = 0.0;
        g[0] = beta;
    }
}

// v_0 = r / beta, also the first operator input.
__global__ void k_scale_first(const double *__restrict__ r, long long N, const GState *__restrict__ st,
                              double *V, double *vin)
{
    const double inv = 1.0 / st->beta;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double x = r[i] * inv;
        V[i] = x;
        vin[i] = x;
    }
}

// y = R^{-1} g over the j completed steps, R the rotated (upper triangular) H, by
// columns from the last: y_i = g_i / R_ii, then g_l -= R_li y_i for l < i.  R sits in
// shared memory when it fits (use_smem).
__global__ void k_solve_y(const GState *__restrict__ st, const double *__restrict__ H,
                          const double *__restrict__ g, double *y, int use_smem)
{
    extern __shared__ double tri[];
    __shared__ double gs[MAX_RESTART + 1];
    const int k = st->j, ld = st->m + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        gs[i] = g[i];
    if (use_smem)
        for (int c = 0; c < k; ++c)
            for (int r = threadIdx.x; r <= c; r += blockDim.x)
                tri[c * (c + 1) / 2 + r] = H[static_cast<size_t>(c) * ld + r];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
        const double rii = use_smem ? tri[i * (i + 1) / 2 + i] : H[static_cast<size_t>(i) * ld + i];
        const double yi = gs[i] / rii;
        if (threadIdx.x == 0)
            y[i] = yi;
        for (int l = threadIdx.x; l < i; l += blockDim.x)
            gs[l] -= (use_smem ? tri[i * (i + 1) / 2 + l] : H[static_cast<size_t>(i) * ld + l]) * yi;
        __syncthreads();
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
    ws->nblk = static_cast<int>(std::max<long long>(1, std::min<long long>(4LL * device_props().sms,
                                                                        (N + 127) / 128)));
    ws->ldp = m + 1;
    ws->solve_smem = (m <= SOLVE_SMEM_MAX_M) ? static_cast<size_t>(m) * (m + 1) / 2 * sizeof(double) : 0;
    int s = SBQ_OK;
    if (s == SBQ_OK) s = ws->V.alloc(static_cast<size_t>(m + 1) * N * sizeof(double));
    if (s == SBQ_OK) s = ws->H.alloc(static_cast<size_t>(m + 1) * m * sizeof(double));
    if (s == SBQ_OK) s = ws->cs.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->sn.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->g.alloc((m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->y.alloc(m * sizeof(double));
    if (s == SBQ_OK) s = ws->hb1.alloc((m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->hb2.alloc((m + 1) * sizeof(double));
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
    if (s == SBQ_OK && ws->solve_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_solve_y, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(ws->solve_smem));
        if (e != cudaSuccess) {
            cudaGetLastError();
            ws->solve_smem = 0;   // keep R in global memory
        }
    }
    if (s != SBQ_OK) {
        gmres_destroy(ws);
        return s;
    }
    cudaGetDevice(&ws->device);
    op->gm = ws;
    return SBQ_OK;
}

// Enqueue one Arnoldi step on stream s (use_cond: inside the while body).  The operator
// input v_j is already in ws->vin (k_scale_first / k_normalize_advance put it there).
static int enqueue_step(Op *op, GmresWS *ws, int prec, cudaStream_t s,
                        cudaGraphConditionalHandle h, int use_cond)
{
    const long long N = ws->N;
    GState *st = ws->st.as<GState>();
    SBQ_TRY(op_matvec(op, ws->vin.as<double>(), ws->w.as<double>(), prec, s));
    k_cgs_pass1<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->w.as<double>(),
                                        ws->part.as<double>(), ws->ldp, ws->H.as<double>(),
                                        ws->hb1.as<double>());
    k_cgs_pass2<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->hb1.as<double>(),
                                        ws->w.as<double>(), ws->part.as<double>(), ws->ldp,
                                        ws->H.as<double>(), ws->hb2.as<double>());
    k_cgs_norm_givens<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, ws->hb2.as<double>(),
                                              ws->w.as<double>(), ws->part.as<double>(),
                                              ws->H.as<double>(), ws->cs.as<double>(),
                                              ws->sn.as<double>(), ws->g.as<double>());
    k_normalize_advance<<<ws->nblk, GB, 0, s>>>(ws->w.as<double>(), N, st, ws->V.as<double>(),
                                                ws->vin.as<double>(), h, use_cond);
    k_guard<<<1, 32, 0, s>>>(st, h, ws->m, use_cond);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

// Kernels of one Arnoldi step (enqueue_step).
static int step_kernels(const Op *op, int prec) { return op_kernels_per_matvec(op, prec) + 5; }

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
    k_scale_first<<<vec_grid(N), GB, 0, s>>>(r, N, st, ws->V.as<double>(), ws->vin.as<double>());
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
    k_solve_y<<<1, GB, ws->solve_smem, s>>>(st, ws->H.as<double>(), ws->g.as<double>(),
                                             ws->y.as<double>(), ws->solve_smem > 0 ? 1 : 0);
    k_update_x<<<vec_grid(N), GB, 0, s>>>(ws->V.as<double>(), N, st, ws->y.as<double>(), xu);
    SBQ_CUDA(cudaGetLastError());
    SBQ_TRY(read_state(ws, s));
    ws->launches += 4 + static_cast<long long>(ws->hst->j) * step_kernels(op, prec);
    if (ws->hst->guard_hit) {
        set_error("Arnoldi loop stopped by its step guard (inconsistent step counter)");
        return SBQ_ECUDA;
    }
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

    // Initial residual: b itself when x0 = 0 (no operator apply needed).
    SBQ_TRY(norm_to_state(ws, x, s));
    if (ws->hst->res_true == 0.0) {
        SBQ_CUDA(cudaMemcpyAsync(ws->r.p, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        ws->hst->res_true = bnorm;
        k_norm_part<<<ws->nblk, GB, 0, s>>>(ws->r.as<double>(), N, ws->part.as<double>());
        k_norm_fin<<<1, 32, 0, s>>>(ws->part.as<double>(), ws->nblk, ws->st.as<GState>());
        SBQ_CUDA(cudaGetLastError());
        ws->launches += 2;
        SBQ_TRY(read_state(ws, s));
    } else {
        SBQ_TRY(residual(op, ws, SBQ_FP64, b, x, ws->r.as<double>(), s));
        rep.matvecs_fp64 += 1;
    }
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
            // the inner residual lives in ws->ax's partner buffer between restarts; the
            // first cycle starts from r itself, whose norm is in the state already
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
                // restart the inner solve from its true low-precision residual r - K d,
                // kept in w (the next cycle reads it before its first step writes w)
                SBQ_TRY(op_matvec(op, d, ws->ax.as<double>(), low, s));
                rep.matvecs_low += 1;
                k_sub<<<vec_grid(N), GB, 0, s>>>(ws->r.as<double>(), ws->ax.as<double>(),
                                                 ws->w.as<double>(), N);
                SBQ_CUDA(cudaGetLastError());
                ws->launches += op_kernels_per_matvec(op, low) + 1;
                SBQ_TRY(norm_to_state(ws, ws->w.as<double>(), s));
                const double nr = ws->hst->res_true;
                if (!(nr < ires) || nr <= inner_abs)
                    break;
                ires = nr;
                rin = ws->w.as<double>();
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
