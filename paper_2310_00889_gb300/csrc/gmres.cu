// Batched GMRES for K sigma = u0 (paper Eq. stokes-bie-new), on the device, FP64 Krylov
// algebra.
//
// The paper solves its second-kind BIEs with unpreconditioned GMRES (Sec. 4, Sec. 5)
// without stating restart, orthogonalisation or initial guess.  This solver uses
// restarted GMRES(m) with classical Gram--Schmidt applied twice and Givens rotations;
// every quantity of the Krylov method (basis, Hessenberg matrix, rotations, residual
// estimate, solution update) is FP64 on the GPU.
//
// Segments.  An operator built on a batch plan is block diagonal: its segments are
// independent problems.  Each segment gets its own Krylov method (its own Hessenberg
// matrix, rotations, residual estimate and convergence test) while all segments share
// the Arnoldi step: one operator apply (one persistent launch over every segment) and
// vector kernels whose row blocks never straddle a segment; the last block of each
// segment to finish reduces that segment's partial dot products in fixed order.  A cycle
// ends when every segment has converged (or broken down) or after m steps; a solve ends
// when every segment's relative residual ||b_s - K_s x_s|| / ||b_s|| meets the tolerance.
// A single-segment operator is the ordinary GMRES.
//
// Two drivers:
//   * plain FP64: every operator apply is the FP64 pair sum; a cycle ends on the Givens
//     estimates, the true FP64 residual decides the restart;
//   * iterative refinement: the FP64 residual r = b - K x is formed, K d = r is solved by
//     GMRES whose operator applies run in FP32 or compensated FP32, x += d, repeat.
// Each Arnoldi step is a fixed sequence of kernels that read the step index from device
// memory, so one captured copy of it serves every step: it is the body of a CUDA-graph
// while node that repeats it on the device until the cycle ends.  Per step: operator
// apply on v_j; first Gram--Schmidt pass; second pass fused with the first update of w;
// norm fused with the second update, whose segment-last blocks also apply the Givens
// rotations; normalisation that writes v_{j+1} and the next operator input; a step guard.
#include "engine.h"

#include <chrono>
#include <cmath>

namespace sbq {

constexpr int GB = 256;          // threads of the vector kernels
constexpr int MAX_RESTART = 256;
constexpr int SOLVE_SMEM_MAX_M = 200;   // back-substitution keeps R in shared memory up to this m

struct GState {                  // shared by all segments
    int j;          // completed Arnoldi steps of the cycle (= index of the next column)
    int stop;       // the cycle must end
    int m;          // step limit of this cycle
    int iters;      // Arnoldi steps since the solve began
    int nonfinite;  // a non-finite norm was seen
    int guard;      // steps run in this cycle, counted by k_guard
    int guard_hit;  // k_guard ended the cycle (the step counter failed to stop it)
    int nseg;
    unsigned int ctr;       // blocks finished in the current kernel
    unsigned int seg_done;  // segments finished in the current kernel
};

struct SegState {                // one per segment
    double tol_abs;  // absolute tolerance on this segment's residual norm
    double beta;     // residual norm at the start of the cycle
    double res_est;  // Givens estimate after the last step
    double res_true; // last norm computed by the norm kernels
    double inv_hn;   // 1 / h_{j+1,j} of the last step (0 on breakdown)
    int conv;        // res_est <= tol_abs
    int brk;         // exact breakdown
    unsigned int ctr;   // this segment's blocks finished in the current kernel
    int pad_;
};

struct GmresWS {
    int device = 0;
    int m = 0;
    int nseg = 0;
    long long N = 0;
    int nblk = 0;
    int ldp = 0;      // stride of part rows (m + 1)
    int LD = 0;       // leading dimension of a Hessenberg matrix (m + 1)
    size_t solve_smem = 0;
    DevBuf V, H, cs, sn, g, y, hb1, hb2, w, vin, r, d, ax, bnd, part, st, seg, blk, segblk, tolv;
    GState *hst = nullptr;             // pinned host mirrors
    SegState *hseg = nullptr;
    double *htol = nullptr;
    cudaStream_t cap = nullptr;        // capture stream
    cudaGraph_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
    bool graph_tried[4] = {false, false, false, false};
    long long launches = 0;            // kernels executed by the current solve
};

int gmres_destroy(GmresWS *ws)
{
    if (!ws)
        return SBQ_OK;
    for (int i = 0; i < 4; ++i) {
        if (ws->exec[i])
            cudaGraphExecDestroy(ws->exec[i]);
        if (ws->graph[i])
            cudaGraphDestroy(ws->graph[i]);
    }
    if (ws->cap)
        cudaStreamDestroy(ws->cap);
    if (ws->hst)
        cudaFreeHost(ws->hst);
    if (ws->hseg)
        cudaFreeHost(ws->hseg);
    if (ws->htol)
        cudaFreeHost(ws->htol);
    delete ws;
    return SBQ_OK;
}

// ---------------------------------------------------------------------------
// Kernels (row kernels: one block per entry of the block table {row_begin, row_end, seg})
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

// True in the block that finishes last among `count` blocks counted on *ctr; all their
// writes are visible to it.  The caller resets *ctr.
__device__ bool last_of(unsigned int *ctr, unsigned int count)
{
    __shared__ unsigned int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = (atomicAdd(ctr, 1u) == count - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last)
        __threadfence();
    return s_last != 0;
}

// part_row[k] = sum over rows [a, b) of V[k][i] w[i], k = 0..j: one warp per Krylov
// vector, lanes striding over the rows (coalesced), no block barrier.
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

// Segment-last block: hb[k] = sum over the segment's blocks of part[b][k] (one warp per
// k, lanes over the blocks, fixed order); column j of the segment's H gets (pass 0) or
// adds (pass 1) it.
__device__ void finish_dots(const double *part, int ldp, int2 sb, int j, double *Hs, int LD,
                            double *hb, int pass)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k <= j; k += nw) {
        double s = 0.0;
        for (int bb = lane; bb < sb.y; bb += 32)
            s += __ldcg(part + static_cast<size_t>(sb.x + bb) * ldp + k);
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            hb[k] = s;
            double *h = Hs + static_cast<size_t>(j) * LD + k;
            *h = pass ? *h + s : s;
        }
    }
}

// First Gram--Schmidt pass: h1 = V[0..j]^T w per segment.
__global__ void k_cgs_pass1(const double *__restrict__ V, long long N, GState *st, SegState *seg,
                            const int4 *__restrict__ blk, const int2 *__restrict__ segblk,
                            const double *__restrict__ w, double *part, int ldp, double *H,
                            int LD, int M, double *hb1)
{
    const int4 bi = blk[blockIdx.x];
    const int s = bi.z, j = st->j;
    block_multi_dot(V, N, j, w, bi.x, bi.y, part + static_cast<size_t>(blockIdx.x) * ldp);
    const int2 sb = segblk[s];
    if (last_of(&seg[s].ctr, sb.y)) {
        finish_dots(part, ldp, sb, j, H + static_cast<size_t>(s) * LD * M, LD,
                    hb1 + static_cast<size_t>(s) * LD, 0);
        if (threadIdx.x == 0)
            seg[s].ctr = 0;
    }
}

// w -= V h1 on this block's rows, then the second pass h2 = V^T w on the same rows.
__global__ void k_cgs_pass2(const double *__restrict__ V, long long N, GState *st, SegState *seg,
                            const int4 *__restrict__ blk, const int2 *__restrict__ segblk,
                            const double *__restrict__ hb1, double *w, double *part, int ldp,
                            double *H, int LD, int M, double *hb2)
{
    __shared__ double sh[MAX_RESTART + 1];
    const int4 bi = blk[blockIdx.x];
    const int s = bi.z, j = st->j;
    for (int k = threadIdx.x; k <= j; k += blockDim.x)
        sh[k] = hb1[static_cast<size_t>(s) * LD + k];
    __syncthreads();
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x) {
        double acc = w[i];
#pragma unroll 8
        for (int k = 0; k <= j; ++k)
            acc = fma(-V[static_cast<size_t>(k) * N + i], sh[k], acc);
        w[i] = acc;
    }
    __syncthreads();   // the dots below read rows of w that other threads just updated
    block_multi_dot(V, N, j, w, bi.x, bi.y, part + static_cast<size_t>(blockIdx.x) * ldp);
    const int2 sb = segblk[s];
    if (last_of(&seg[s].ctr, sb.y)) {
        finish_dots(part, ldp, sb, j, H + static_cast<size_t>(s) * LD * M, LD,
                    hb2 + static_cast<size_t>(s) * LD, 1);
        if (threadIdx.x == 0)
            seg[s].ctr = 0;
    }
}

// w -= V h2 and ||w||^2 on this block's rows.  The segment-last block forms h_{j+1,j},
// applies the segment's previous Givens rotations to its column j, builds the new one and
// updates the segment's residual estimate; the last segment to finish decides whether the
// cycle stops.
__global__ void k_cgs_norm_givens(const double *__restrict__ V, long long N, GState *st,
                                  SegState *seg, const int4 *__restrict__ blk,
                                  const int2 *__restrict__ segblk, const double *__restrict__ hb2,
                                  double *w, double *part, double *H, int LD, int M, double *cs,
                                  double *sn, double *g)
{
    __shared__ double sh[MAX_RESTART + 1];
    __shared__ double red[32];
    const int4 bi = blk[blockIdx.x];
    const int s = bi.z, j = st->j;
    for (int k = threadIdx.x; k <= j; k += blockDim.x)
        sh[k] = hb2[static_cast<size_t>(s) * LD + k];
    __syncthreads();
    double nrm = 0.0;
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x) {
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
    const int2 sb = segblk[s];
    if (!last_of(&seg[s].ctr, sb.y))
        return;
    // segment-last block: column j of H and the rotations into shared memory in parallel,
    // the sequential rotation sweep by one thread, results written back in parallel
    __shared__ double scol[MAX_RESTART + 1], scs[MAX_RESTART], ssn[MAX_RESTART];
    __shared__ double s_hn;
    double *Hs = H + static_cast<size_t>(s) * LD * M;
    double *cs_s = cs + static_cast<size_t>(s) * M, *sn_s = sn + static_cast<size_t>(s) * M;
    double *g_s = g + static_cast<size_t>(s) * LD;
    double *col = Hs + static_cast<size_t>(j) * LD;
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        scol[i] = __ldcg(col + i);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        scs[i] = __ldcg(cs_s + i);
        ssn[i] = __ldcg(sn_s + i);
    }
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int bb = threadIdx.x; bb < sb.y; bb += 32)
            t += __ldcg(part + sb.x + bb);
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0)
            s_hn = sqrt(t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        SegState &ss = seg[s];
        ss.ctr = 0;
        const double hn = s_hn;
        for (int i = 0; i < j; ++i) {
            const double x0 = scol[i], x1 = scol[i + 1];
            scol[i] = scs[i] * x0 + ssn[i] * x1;
            scol[i + 1] = -ssn[i] * x0 + scs[i] * x1;
        }
        const double x0 = scol[j], x1 = hn;
        const double den = hypot(x0, x1);
        const double cj = (den == 0.0) ? 1.0 : x0 / den, sj = (den == 0.0) ? 0.0 : x1 / den;
        cs_s[j] = cj;
        sn_s[j] = sj;
        scol[j] = cj * x0 + sj * x1;
        col[j + 1] = 0.0;
        const double gj = __ldcg(g_s + j);
        g_s[j + 1] = -sj * gj;
        g_s[j] = cj * gj;
        const double est = fabs(sj * gj);
        ss.res_est = est;
        const bool nonfinite = !isfinite(hn) || !isfinite(est);
        if (nonfinite)
            st->nonfinite = 1;
        ss.conv = ss.conv || (est <= ss.tol_abs);
        ss.brk = (hn == 0.0);
        ss.inv_hn = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        col[i] = scol[i];
    // the last segment to finish decides for the whole batch
    if (last_of(&st->seg_done, static_cast<unsigned int>(st->nseg)) && threadIdx.x == 0) {
        st->seg_done = 0;
        int all_done = 1;
        for (int q = 0; q < st->nseg; ++q) {
            const SegState &o = seg[q];
            if (!(o.conv || o.brk))
                all_done = 0;
        }
        st->iters += 1;
        st->stop = all_done || st->nonfinite || (j + 1 >= st->m);
    }
}

// v_{j+1} = w / h_{j+1,j} (per segment), also written to the operator input buffer; the
// last block advances j and, inside the graph, sets the while condition.
__global__ void k_normalize_advance(const double *__restrict__ w, long long N, GState *st,
                                    const SegState *__restrict__ seg, const int4 *__restrict__ blk,
                                    double *V, double *vin, cudaGraphConditionalHandle h,
                                    int use_cond)
{
    const int4 bi = blk[blockIdx.x];
    const int j = st->j;
    const double sc = seg[bi.z].inv_hn;
    double *v = V + static_cast<size_t>(j + 1) * N;
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x) {
        const double x = w[i] * sc;
        v[i] = x;
        vin[i] = x;
    }
    if (last_of(&st->ctr, gridDim.x) && threadIdx.x == 0) {
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

// part[b] = ||x||^2 over this block's rows.
__global__ void k_norm_part(const double *__restrict__ x, const int4 *__restrict__ blk, double *part)
{
    __shared__ double red[32];
    const int4 bi = blk[blockIdx.x];
    double acc = 0.0;
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x)
        acc = fma(x[i], x[i], acc);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

// res_true of every segment from the block partials (fixed order).
__global__ void k_norm_fin(const double *__restrict__ part, const int2 *__restrict__ segblk,
                           int nseg, SegState *seg, GState *st)
{
    for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
        const int2 sb = segblk[s];
        double t = 0.0;
        for (int b = 0; b < sb.y; ++b)
            t += part[sb.x + b];
        const double r = sqrt(t);
        seg[s].res_true = r;
        if (!isfinite(r))
            st->nonfinite = 1;
    }
}

// Start a cycle from the residual whose per-segment norms are in res_true.
__global__ void k_cycle_init(GState *st, SegState *seg, const double *__restrict__ tolv, double *g,
                             int LD, int m, int nseg)
{
    if (threadIdx.x == 0) {
        st->j = 0;
        st->stop = 0;
        st->ctr = 0;
        st->seg_done = 0;
        st->guard = 0;
        st->guard_hit = 0;
        st->nonfinite = 0;   // per cycle (a norm pass before the cycle may have set it)
        st->m = m;
        st->nseg = nseg;
    }
    for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
        SegState &ss = seg[s];
        const double beta = ss.res_true;
        ss.beta = beta;
        ss.tol_abs = tolv[s];
        ss.res_est = beta;
        ss.conv = beta <= tolv[s];
        ss.brk = 0;
        ss.ctr = 0;
        ss.inv_hn = 0.0;
        double *gs = g + static_cast<size_t>(s) * LD;
        for (int i = 0; i <= m; ++i)
            gs[i] = 0.0;
        gs[0] = beta;
    }
}

// v_0 = r / beta per segment (0 for a segment with a zero residual), also the first
// operator input.
__global__ void k_scale_first(const double *__restrict__ r, const SegState *__restrict__ seg,
                              const int4 *__restrict__ blk, double *V, double *vin)
{
    const int4 bi = blk[blockIdx.x];
    const double beta = seg[bi.z].beta;
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x) {
        const double x = r[i] * inv;
        V[i] = x;
        vin[i] = x;
    }
}

// y_s = R_s^{-1} g_s over the j completed steps, R_s the segment's rotated (upper
// triangular) H, by columns from the last: y_i = g_i / R_ii, then g_l -= R_li y_i for
// l < i.  One block per segment; R sits in shared memory when it fits (use_smem).
__global__ void k_solve_y(const GState *__restrict__ st, const double *__restrict__ H,
                          const double *__restrict__ g, double *y, int LD, int M, int use_smem)
{
    extern __shared__ double tri[];
    __shared__ double gs[MAX_RESTART + 1];
    const int s = blockIdx.x;
    const int k = st->j;
    const double *Hs = H + static_cast<size_t>(s) * LD * M;
    const double *g_s = g + static_cast<size_t>(s) * LD;
    double *y_s = y + static_cast<size_t>(s) * M;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        gs[i] = g_s[i];
    if (use_smem)
        for (int c = 0; c < k; ++c)
            for (int r = threadIdx.x; r <= c; r += blockDim.x)
                tri[c * (c + 1) / 2 + r] = Hs[static_cast<size_t>(c) * LD + r];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
        const double rii = use_smem ? tri[i * (i + 1) / 2 + i] : Hs[static_cast<size_t>(i) * LD + i];
        const double yi = (rii != 0.0) ? gs[i] / rii : 0.0;
        if (threadIdx.x == 0)
            y_s[i] = yi;
        for (int l = threadIdx.x; l < i; l += blockDim.x)
            gs[l] -= (use_smem ? tri[i * (i + 1) / 2 + l] : Hs[static_cast<size_t>(i) * LD + l]) * yi;
        __syncthreads();
    }
}

// x += sum_{k < j} V[k] y_s[k] on each block's rows (segment s of the block).
__global__ void k_update_x(const double *__restrict__ V, long long N, const GState *__restrict__ st,
                           const int4 *__restrict__ blk, const double *__restrict__ y, int M,
                           double *x)
{
    __shared__ double sy[MAX_RESTART];
    const int4 bi = blk[blockIdx.x];
    const int k = st->j;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        sy[i] = y[static_cast<size_t>(bi.z) * M + i];
    __syncthreads();
    for (long long i = bi.x + threadIdx.x; i < bi.y; i += blockDim.x) {
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
    ws->N = static_cast<long long>(op->ncomp) * op->n;
    ws->nseg = op->plan.nseg;
    ws->ldp = m + 1;
    ws->LD = m + 1;
    const long long N = ws->N, n = op->n;
    const int nseg = ws->nseg;
    // Block table: rows of segment s are the component ranges c n + [o_s, o_{s+1});
    // each range is cut into chunks of about N / (8 SMs) rows, at least 256 (one row per
    // thread of the update loops).
    const long long chunk = std::max<long long>(256, N / (8LL * device_props().sms) + 1);
    std::vector<int4> hb;
    std::vector<int2> hsb(nseg);
    for (int s = 0; s < nseg; ++s) {
        hsb[s].x = static_cast<int>(hb.size());
        const long long a = op->plan.src_off[s], b = op->plan.src_off[s + 1];
        for (int c = 0; c < op->ncomp; ++c)
            for (long long r = a; r < b; r += chunk)
                hb.push_back(make_int4(static_cast<int>(c * n + r),
                                       static_cast<int>(c * n + std::min(b, r + chunk)), s, 0));
        if (b == a)   // an empty segment still owns one (empty) block
            hb.push_back(make_int4(0, 0, s, 0));
        hsb[s].y = static_cast<int>(hb.size()) - hsb[s].x;
    }
    ws->nblk = static_cast<int>(hb.size());
    ws->solve_smem = (m <= SOLVE_SMEM_MAX_M) ? static_cast<size_t>(m) * (m + 1) / 2 * sizeof(double) : 0;
    const size_t S = nseg;
    int s = SBQ_OK;
    if (s == SBQ_OK) s = ws->V.alloc(static_cast<size_t>(m + 1) * N * sizeof(double));
    if (s == SBQ_OK) s = ws->H.alloc(S * (m + 1) * m * sizeof(double));
    if (s == SBQ_OK) s = ws->cs.alloc(S * m * sizeof(double));
    if (s == SBQ_OK) s = ws->sn.alloc(S * m * sizeof(double));
    if (s == SBQ_OK) s = ws->g.alloc(S * (m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->y.alloc(S * m * sizeof(double));
    if (s == SBQ_OK) s = ws->hb1.alloc(S * (m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->hb2.alloc(S * (m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->w.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->vin.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->r.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->d.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->ax.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->bnd.alloc(N * sizeof(double));
    if (s == SBQ_OK) s = ws->part.alloc(static_cast<size_t>(ws->nblk) * (m + 1) * sizeof(double));
    if (s == SBQ_OK) s = ws->st.alloc(sizeof(GState));
    if (s == SBQ_OK) s = ws->seg.alloc(S * sizeof(SegState));
    if (s == SBQ_OK) s = ws->blk.alloc(hb.size() * sizeof(int4));
    if (s == SBQ_OK) s = ws->segblk.alloc(S * sizeof(int2));
    if (s == SBQ_OK) s = ws->tolv.alloc(S * sizeof(double));
    if (s == SBQ_OK) {
        cudaError_t e = cudaMallocHost(&ws->hst, sizeof(GState));
        if (e == cudaSuccess) e = cudaMallocHost(&ws->hseg, S * sizeof(SegState));
        if (e == cudaSuccess) e = cudaMallocHost(&ws->htol, S * sizeof(double));
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
        if (e == cudaSuccess) e = cudaMemset(ws->seg.p, 0, S * sizeof(SegState));
        if (e == cudaSuccess)
            e = cudaMemcpy(ws->blk.p, hb.data(), hb.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ws->segblk.p, hsb.data(), S * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            s = cuda_status(e, "gmres workspace set-up");
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
    SegState *sg = ws->seg.as<SegState>();
    const int4 *blk = ws->blk.as<int4>();
    const int2 *sb = ws->segblk.as<int2>();
    SBQ_TRY(op_matvec(op, ws->vin.as<double>(), ws->w.as<double>(), prec, s));
    k_cgs_pass1<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, sg, blk, sb, ws->w.as<double>(),
                                        ws->part.as<double>(), ws->ldp, ws->H.as<double>(), ws->LD,
                                        ws->m, ws->hb1.as<double>());
    k_cgs_pass2<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, sg, blk, sb, ws->hb1.as<double>(),
                                        ws->w.as<double>(), ws->part.as<double>(), ws->ldp,
                                        ws->H.as<double>(), ws->LD, ws->m, ws->hb2.as<double>());
    k_cgs_norm_givens<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), N, st, sg, blk, sb,
                                              ws->hb2.as<double>(), ws->w.as<double>(),
                                              ws->part.as<double>(), ws->H.as<double>(), ws->LD,
                                              ws->m, ws->cs.as<double>(), ws->sn.as<double>(),
                                              ws->g.as<double>());
    k_normalize_advance<<<ws->nblk, GB, 0, s>>>(ws->w.as<double>(), N, st, sg, blk,
                                                ws->V.as<double>(), ws->vin.as<double>(), h,
                                                use_cond);
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
    SBQ_CUDA(cudaMemcpyAsync(ws->hseg, ws->seg.p, ws->nseg * sizeof(SegState),
                             cudaMemcpyDeviceToHost, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

// Per-segment ||v|| into res_true (device and host mirrors).
static int norm_to_state(GmresWS *ws, const double *v, cudaStream_t s)
{
    k_norm_part<<<ws->nblk, GB, 0, s>>>(v, ws->blk.as<int4>(), ws->part.as<double>());
    k_norm_fin<<<1, GB, 0, s>>>(ws->part.as<double>(), ws->segblk.as<int2>(), ws->nseg,
                                ws->seg.as<SegState>(), ws->st.as<GState>());
    SBQ_CUDA(cudaGetLastError());
    ws->launches += 2;
    return read_state(ws, s);
}

static void copy_res(const GmresWS *ws, std::vector<double> &out)
{
    out.resize(ws->nseg);
    for (int i = 0; i < ws->nseg; ++i)
        out[i] = ws->hseg[i].res_true;
}

// r = b - K x in precision prec; per-segment ||r|| to the state.  bound (double-float
// only, nullable): per entry a bound on the rounding error of K x.
static int residual(Op *op, GmresWS *ws, int prec, const double *b, const double *x, double *r,
                    cudaStream_t s, double *bound = nullptr)
{
    SBQ_TRY(op_matvec(op, x, ws->ax.as<double>(), prec, s, bound));
    k_sub<<<vec_grid(ws->N), GB, 0, s>>>(b, ws->ax.as<double>(), r, ws->N);
    SBQ_CUDA(cudaGetLastError());
    ws->launches += op_kernels_per_matvec(op, prec) + 1;
    return norm_to_state(ws, r, s);
}

// One GMRES cycle from residual r (per-segment norms in the state) updating xu += V y;
// tol_abs[s] is each segment's absolute residual target.
static int run_cycle(Op *op, GmresWS *ws, int prec, const double *r, double *xu, int m,
                     const std::vector<double> &tol_abs, bool use_graph, cudaStream_t s,
                     bool *graph_used)
{
    GState *st = ws->st.as<GState>();
    for (int i = 0; i < ws->nseg; ++i)
        ws->htol[i] = tol_abs[i];
    SBQ_CUDA(cudaMemcpyAsync(ws->tolv.p, ws->htol, ws->nseg * sizeof(double), cudaMemcpyHostToDevice,
                             s));
    k_cycle_init<<<1, GB, 0, s>>>(st, ws->seg.as<SegState>(), ws->tolv.as<double>(),
                                  ws->g.as<double>(), ws->LD, m, ws->nseg);
    k_scale_first<<<ws->nblk, GB, 0, s>>>(r, ws->seg.as<SegState>(), ws->blk.as<int4>(),
                                          ws->V.as<double>(), ws->vin.as<double>());
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
    k_solve_y<<<ws->nseg, GB, ws->solve_smem, s>>>(st, ws->H.as<double>(), ws->g.as<double>(),
                                                    ws->y.as<double>(), ws->LD, ws->m,
                                                    ws->solve_smem > 0 ? 1 : 0);
    k_update_x<<<ws->nblk, GB, 0, s>>>(ws->V.as<double>(), ws->N, st, ws->blk.as<int4>(),
                                       ws->y.as<double>(), ws->m, xu);
    SBQ_CUDA(cudaGetLastError());
    SBQ_TRY(read_state(ws, s));
    ws->launches += 5 + static_cast<long long>(ws->hst->j) * step_kernels(op, prec);
    if (ws->hst->guard_hit) {
        set_error("Arnoldi loop stopped by its step guard (inconsistent step counter)");
        return SBQ_ECUDA;
    }
    return SBQ_OK;
}

// The residual that decides convergence, in precision hp.  A double-float residual comes
// with a bound on the rounding error of K x (the kernel's running sum of term
// magnitudes times the per-term error bound).  Where that bound exceeds a quarter of a
// segment's tolerance the double-float residual cannot certify the tolerance: it is
// recomputed in FP64 and the rest of the solve stays in FP64.  Otherwise each segment's
// residual norm is taken as its double-float value plus the bound (an upper bound of the
// exact residual of the returned x up to FP64 rounding).
static int decisive_residual(Op *op, GmresWS *ws, int &hp, const double *b, const double *x,
                             double tol, const std::vector<double> &bnorm,
                             std::vector<double> &res, sbq_gmres_report &rep, cudaStream_t s)
{
    if (hp == SBQ_DF32) {
        SBQ_TRY(residual(op, ws, SBQ_DF32, b, x, ws->r.as<double>(), s, ws->bnd.as<double>()));
        rep.matvecs_fp64 += 1;
        std::vector<double> bn;
        copy_res(ws, res);
        SBQ_TRY(norm_to_state(ws, ws->bnd.as<double>(), s));
        copy_res(ws, bn);
        bool trusted = true;
        for (size_t i = 0; i < res.size(); ++i)
            trusted = trusted && !(bn[i] > 0.25 * tol * bnorm[i]);
        if (trusted) {
            for (size_t i = 0; i < res.size(); ++i)
                res[i] += bn[i];
            // the state keeps the residual norms for the next cycle
            SBQ_TRY(norm_to_state(ws, ws->r.as<double>(), s));
            return SBQ_OK;
        }
        hp = SBQ_FP64;
        rep.resid_fallbacks += 1;
        SBQ_TRY(op_ensure_tuned(op, SBQ_FP64, s));
    }
    SBQ_TRY(residual(op, ws, hp, b, x, ws->r.as<double>(), s));
    rep.matvecs_fp64 += 1;
    copy_res(ws, res);
    return SBQ_OK;
}

// max over segments of res[s] / ref[s] (segments with ref 0 count as 0)
static double max_rel(const std::vector<double> &res, const std::vector<double> &ref)
{
    double m = 0.0;
    for (size_t i = 0; i < res.size(); ++i) {
        const double v = ref[i] > 0.0 ? res[i] / ref[i] : (res[i] > 0.0 ? INFINITY : 0.0);
        if (!(v <= m))
            m = v;   // also propagates NaN
    }
    return m;
}

static bool all_finite(const std::vector<double> &v)
{
    for (double x : v)
        if (!std::isfinite(x))
            return false;
    return true;
}

int gmres_solve_impl(Op *op, const double *b, double *x, const sbq_gmres_opts &o,
                     sbq_gmres_report &rep, cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    rep = sbq_gmres_report{};
    const int low = o.inner_prec;
    const bool mixed = (low == SBQ_FP32 || low == SBQ_FP32_COMP);
    // the precision of the residuals that decide convergence (and of the plain solve)
    int hp = mixed ? o.resid_prec : low;
    SBQ_TRY(ws_ensure(op, o.restart));
    GmresWS *ws = op->gm;
    ws->launches = 0;
    const long long N = ws->N;
    const int nseg = ws->nseg;
    if (!device_error_word()) {
        set_error("cannot allocate the device error word");
        return SBQ_ENOMEM;
    }
    SBQ_TRY(op_ensure_tuned(op, hp, s));
    if (mixed && !(low == SBQ_FP32 && op->tree))   // an attached treecode needs no tile shape
        SBQ_TRY(op_ensure_tuned(op, low, s));

    std::vector<double> bnorm, res, tol_abs(nseg);
    SBQ_TRY(norm_to_state(ws, b, s));
    copy_res(ws, bnorm);
    if (!all_finite(bnorm)) {
        set_error("right-hand side is not finite");
        return SBQ_ENONFINITE;
    }
    bool bzero = true;
    for (double v : bnorm)
        bzero = bzero && (v == 0.0);
    if (bzero) {
        SBQ_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        SBQ_CUDA(cudaStreamSynchronize(s));
        rep.status = SBQ_OK;
        rep.n_hist = 1;
        rep.rel_res_hist[0] = 0.0;
        return SBQ_OK;
    }
    bool graph_used = false;
    auto push_hist = [&](double v) {
        if (rep.n_hist < SBQ_HIST)
            rep.rel_res_hist[rep.n_hist++] = v;
    };

    // Initial residual: b itself when x0 = 0 (no operator apply needed).
    SBQ_TRY(norm_to_state(ws, x, s));
    bool xzero = true;
    for (int i = 0; i < nseg; ++i)
        xzero = xzero && (ws->hseg[i].res_true == 0.0);
    if (xzero) {
        SBQ_CUDA(cudaMemcpyAsync(ws->r.p, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SBQ_TRY(norm_to_state(ws, ws->r.as<double>(), s));
        copy_res(ws, res);
    } else {
        SBQ_TRY(decisive_residual(op, ws, hp, b, x, o.tol, bnorm, res, rep, s));
    }
    double rel = max_rel(res, bnorm);
    push_hist(rel);
    int status = SBQ_OK;
    while (rel > o.tol) {
        if (!std::isfinite(rel)) {
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
            for (int i = 0; i < nseg; ++i)
                tol_abs[i] = o.tol * bnorm[i];
            SBQ_TRY(run_cycle(op, ws, hp, ws->r.as<double>(), x, m, tol_abs,
                              o.use_graph != 0, s, &graph_used));
            const int steps = ws->hst->j;
            rep.iters += steps;
            rep.matvecs_fp64 += steps;
            bool any_brk = false;
            for (int i = 0; i < nseg; ++i)
                any_brk = any_brk || ws->hseg[i].brk;
            if (ws->hst->nonfinite) {
                status = SBQ_ENONFINITE;
                set_error("non-finite value in the Arnoldi process");
                break;
            }
            SBQ_TRY(decisive_residual(op, ws, hp, b, x, o.tol, bnorm, res, rep, s));
            rep.outer_iters += 1;
            const double nrel = max_rel(res, bnorm);
            push_hist(nrel);
            if (any_brk && nrel > o.tol && nrel >= rel) {
                status = SBQ_EBREAKDOWN;
                set_error("GMRES breakdown without convergence");
                rel = nrel;
                break;
            }
            rel = nrel;
        } else {
            // inner solve K_low d = r, d = 0, to inner_tol * ||r_s|| per segment
            double *d = ws->d.as<double>();
            SBQ_CUDA(cudaMemsetAsync(d, 0, N * sizeof(double), s));
            // a segment need not go below half the outer target
            for (int i = 0; i < nseg; ++i)
                tol_abs[i] = std::max(o.inner_tol * res[i], 0.5 * o.tol * bnorm[i]);
            std::vector<double> ires = res;
            const double *rin = ws->r.as<double>();
            for (;;) {
                const int m = std::min(o.restart, o.max_iter - rep.iters);
                if (m <= 0)
                    break;
                SBQ_TRY(run_cycle(op, ws, low, rin, d, m, tol_abs, o.use_graph != 0, s,
                                  &graph_used));
                const int steps = ws->hst->j;
                rep.iters += steps;
                rep.matvecs_low += steps;
                if (ws->hst->nonfinite) {
                    status = SBQ_ENONFINITE;
                    break;
                }
                bool all_done = true;
                for (int i = 0; i < nseg; ++i)
                    all_done = all_done && (ws->hseg[i].conv || ws->hseg[i].brk);
                if (all_done)
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
                std::vector<double> nr;
                copy_res(ws, nr);
                bool progress = false, reached = true;
                for (int i = 0; i < nseg; ++i) {
                    progress = progress || (nr[i] < ires[i]);
                    reached = reached && (nr[i] <= tol_abs[i]);
                }
                if (!progress || reached)
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
            SBQ_TRY(decisive_residual(op, ws, hp, b, x, o.tol, bnorm, res, rep, s));
            rep.outer_iters += 1;
            const double nrel = max_rel(res, bnorm);
            push_hist(nrel);
            if (!(nrel < rel)) {
                rel = nrel;
                status = SBQ_ENOCONV;
                set_error("iterative refinement stagnated above the tolerance");
                break;
            }
            rel = nrel;
        }
    }
    SBQ_CUDA(cudaStreamSynchronize(s));
    rep.rel_res = rel;
    rep.graph_used = graph_used ? 1 : 0;
    rep.kernel_launches = static_cast<int>(std::min<long long>(ws->launches, INT32_MAX));
    rep.status = status;
    rep.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
    return status;
}

}  // namespace sbq
