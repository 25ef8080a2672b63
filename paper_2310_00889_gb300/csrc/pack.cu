// Packing, reduction and sparse-correction kernels of the pair-sum engine.
//
//  * source geometry pack (once per operator): positions relative to the tile centre
//    (FP32) or absolute (FP64), unit normals, padding of ragged tiles, tile radius;
//  * density pack (every apply): q = w sigma, the quadrature weight of paper
//    Eq. nystrom-no-correction folded into the density;
//  * target pack (FP32, once per tile shape): positions relative to the target tile
//    centre;
//  * fixed-order reduction of chunk partials with the prefactor and the diagonal term
//    diag * sigma of K = I/2 + D + eta S (Eq. stokes-bie-new);
//  * CSR apply y += E x of the local correction (Eq. nystrom-correction).
#include "sbq_common.cuh"

namespace sbq {

namespace {

// Block-wide max of a non-negative double (blockDim.x a multiple of 32, <= 1024).
__device__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1)
            v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;   // valid in thread 0
}

// Block-wide min and max of x, y, z (blockDim.x a multiple of 32); lo/hi valid in all
// threads on return.  Threads without a point pass +inf / -inf.
__device__ void block_bbox(double (&lo)[3], double (&hi)[3], double (*red)[32])
{
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
        for (int c = 0; c < 3; ++c) {
            red[c][warp] = lo[c];
            red[3 + c][warp] = hi[c];
        }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        lo[c] = red[c][0];
        hi[c] = red[3 + c][0];
        for (int w = 1; w < nw; ++w) {
            lo[c] = fmin(lo[c], red[c][w]);
            hi[c] = fmax(hi[c], red[3 + c][w]);
        }
    }
}

// Centre of a tile: the midpoint of its points' bounding box (the tile's bounding sphere
// about it is at most half the box diagonal, smaller than about any member node).
__device__ void tile_centre(const double *__restrict__ pts, long long stride, long long begin,
                            int count, int tile_size, double (*red)[32], double &cx, double &cy,
                            double &cz)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = threadIdx.x; j < tile_size; j += blockDim.x)
        if (j < count)
            for (int c = 0; c < 3; ++c) {
                const double v = pts[c * stride + begin + j];
                lo[c] = fmin(lo[c], v);
                hi[c] = fmax(hi[c], v);
            }
    block_bbox(lo, hi, red);
    cx = 0.5 * (lo[0] + hi[0]);
    cy = 0.5 * (lo[1] + hi[1]);
    cz = 0.5 * (lo[2] + hi[2]);
}

// Radius rounded up so that the FP32 value bounds every FP64 distance.
__device__ float radius_up(double d2max)
{
    const double r = sqrt(d2max) * (1.0 + 1.0e-6) + 1.0e-300;
    return __double2float_ru(r);
}

__global__ void pack_src_geom_f32(const double *__restrict__ src, const double *__restrict__ nrm,
                                  double nscale, long long ns, TileInfo *stiles, float4 *spack)
{
    constexpr int TS = TS_F32;
    __shared__ double red[32];
    __shared__ double bb[6][32];
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    double cx, cy, cz;
    tile_centre(src, ns, begin, count, TS, bb, cx, cy, cz);
    float *tile = reinterpret_cast<float *>(spack + static_cast<size_t>(k) * F32_TILE_F4);
    double d2 = 0.0;
    if (j < count) {
        const long long s = begin + j;
        const double dx = src[s] - cx, dy = src[ns + s] - cy, dz = src[2 * ns + s] - cz;
        const float fx = static_cast<float>(dx), fy = static_cast<float>(dy),
                    fz = static_cast<float>(dz);
        tile[f32_slot(FX, j)] = fx;
        tile[f32_slot(FY, j)] = fy;
        tile[f32_slot(FZ, j)] = fz;
        tile[f32_slot(FLX, j)] = static_cast<float>(dx - fx);
        tile[f32_slot(FLY, j)] = static_cast<float>(dy - fy);
        tile[f32_slot(FLZ, j)] = static_cast<float>(dz - fz);
        tile[f32_slot(FNX, j)] = nrm ? static_cast<float>(nscale * nrm[s]) : 0.0f;
        tile[f32_slot(FNY, j)] = nrm ? static_cast<float>(nscale * nrm[ns + s]) : 0.0f;
        tile[f32_slot(FNZ, j)] = nrm ? static_cast<float>(nscale * nrm[2 * ns + s]) : 0.0f;
        d2 = dx * dx + dy * dy + dz * dz;
    } else {
        tile[f32_slot(FX, j)] = tile[f32_slot(FY, j)] = tile[f32_slot(FZ, j)] = PAD_POS_F32;
        for (int f = FQX; f <= FLZ; ++f)
            tile[f32_slot(f, j)] = 0.0f;
    }
    const double m = block_max(d2, red);
    if (j == 0) {
        stiles[k].cx = cx;
        stiles[k].cy = cy;
        stiles[k].cz = cz;
        stiles[k].rad = radius_up(m);
    }
}

__global__ void pack_src_geom_f64(const double *__restrict__ src, const double *__restrict__ nrm,
                                  double nscale, long long ns, TileInfo *stiles, double *spack)
{
    constexpr int TS = TS_F64;
    __shared__ double red[32];
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    const long long c = begin + min(TS / 2, count - 1);
    const double cx = src[c], cy = src[ns + c], cz = src[2 * ns + c];
    double *tile = spack + static_cast<size_t>(k) * 9 * TS;
    double d2 = 0.0;
    if (j < count) {
        const long long s = begin + j;
        tile[j] = src[s];
        tile[TS + j] = src[ns + s];
        tile[2 * TS + j] = src[2 * ns + s];
        tile[6 * TS + j] = nrm ? nscale * nrm[s] : 0.0;
        tile[7 * TS + j] = nrm ? nscale * nrm[ns + s] : 0.0;
        tile[8 * TS + j] = nrm ? nscale * nrm[2 * ns + s] : 0.0;
        const double dx = src[s] - cx, dy = src[ns + s] - cy, dz = src[2 * ns + s] - cz;
        d2 = dx * dx + dy * dy + dz * dz;
    } else {
        tile[j] = tile[TS + j] = tile[2 * TS + j] = PAD_POS_F64;
        tile[3 * TS + j] = tile[4 * TS + j] = tile[5 * TS + j] = 0.0;
        tile[6 * TS + j] = tile[7 * TS + j] = tile[8 * TS + j] = 0.0;
    }
    const double m = block_max(d2, red);
    if (j == 0) {
        stiles[k].cx = cx;
        stiles[k].cy = cy;
        stiles[k].cz = cz;
        stiles[k].rad = radius_up(m);
    }
}

__global__ void pack_src_q_f32(const double *__restrict__ w, const double *__restrict__ sigma,
                               long long ns, const TileInfo *__restrict__ stiles, float4 *spack,
                               int *counter, const int *__restrict__ perm, int scalar)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && counter)
        *counter = 0;
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    float qx = 0.0f, qy = 0.0f, qz = 0.0f;
    if (j < count) {
        const long long s = begin + j;
        const long long u = perm ? perm[s] : s;   // caller's index of internal node s
        const double ww = w[s];
        qx = static_cast<float>(ww * sigma[u]);
        if (!scalar) {   // scalar (Laplace) densities: one component, in qx
            qy = static_cast<float>(ww * sigma[ns + u]);
            qz = static_cast<float>(ww * sigma[2 * ns + u]);
        }
    }
    float *tile = reinterpret_cast<float *>(spack + static_cast<size_t>(k) * F32_TILE_F4);
    tile[f32_slot(FQX, j)] = qx;
    tile[f32_slot(FQY, j)] = qy;
    tile[f32_slot(FQZ, j)] = qz;
}

__global__ void pack_src_q_f64(const double *__restrict__ w, const double *__restrict__ sigma,
                               long long ns, const TileInfo *__restrict__ stiles, double *spack,
                               int *counter, const int *__restrict__ perm, int scalar)
{
    constexpr int TS = TS_F64;
    if (blockIdx.x == 0 && threadIdx.x == 0 && counter)
        *counter = 0;
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    double *tile = spack + static_cast<size_t>(k) * 9 * TS;
    double qx = 0.0, qy = 0.0, qz = 0.0;
    if (j < count) {
        const long long s = begin + j;
        const long long u = perm ? perm[s] : s;
        const double ww = w[s];
        qx = ww * sigma[u];
        if (!scalar) {
            qy = ww * sigma[ns + u];
            qz = ww * sigma[2 * ns + u];
        }
    }
    tile[3 * TS + j] = qx;
    tile[4 * TS + j] = qy;
    tile[5 * TS + j] = qz;
}

// Double-float source tiles (record layout in pairsum_df.cuh): float index of field f of
// source j.  Fields: 0 xh 1 yh 2 zh 3 qxh 4 qyh 5 qzh 6 nxh 7 nyh 8 nzh 9 xm 10 ym 11 zm
// 12 qxl 13 qyl 14 qzl 15 nxl 16 nyl 17 nzl 18 |q|_1 19 |n|_1 (both rounded up; they feed
// the rounding-error bound only) 20 xl 21 yl 22 zl (23 unused).
__device__ __forceinline__ int df_slot(int f, int j) { return 24 * j + f; }

__device__ __forceinline__ void split_df(double v, float &h, float &l)
{
    h = static_cast<float>(v);
    l = static_cast<float>(v - static_cast<double>(h));
}

// a - b = h + m + l to about 2^-72 |a - b|: the FP64 difference with its exact rounding
// error (TwoSum), split into three FP32 parts.
__device__ __forceinline__ void split3(double a, double b, float &h, float &m, float &l)
{
    const double s = a - b;
    const double bb = s - a;
    const double e = (a - (s - bb)) - (b + bb);
    h = static_cast<float>(s);
    const double r1 = s - static_cast<double>(h);
    m = static_cast<float>(r1);
    l = static_cast<float>((r1 - static_cast<double>(m)) + e);
}

__global__ void pack_src_geom_df(const double *__restrict__ src, const double *__restrict__ nrm,
                                 double nscale, long long ns, TileInfo *stiles, float4 *spack)
{
    constexpr int TS = TS_DF;
    __shared__ double red[32];
    __shared__ double bb[6][32];
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    double cx, cy, cz;
    tile_centre(src, ns, begin, count, TS, bb, cx, cy, cz);
    float *tile = reinterpret_cast<float *>(spack + static_cast<size_t>(k) * DF_TILE_F4);
    double d2 = 0.0;
    float v[24];
    for (int f = 0; f < 24; ++f)
        v[f] = 0.0f;
    if (j < count) {
        const long long s = begin + j;
        const double dx = src[s] - cx, dy = src[ns + s] - cy, dz = src[2 * ns + s] - cz;
        split3(src[s], cx, v[0], v[9], v[20]);
        split3(src[ns + s], cy, v[1], v[10], v[21]);
        split3(src[2 * ns + s], cz, v[2], v[11], v[22]);
        if (nrm) {
            split_df(nscale * nrm[s], v[6], v[15]);
            split_df(nscale * nrm[ns + s], v[7], v[16]);
            split_df(nscale * nrm[2 * ns + s], v[8], v[17]);
            v[19] = __double2float_ru(fabs(nscale) * (fabs(nrm[s]) + fabs(nrm[ns + s]) +
                                                      fabs(nrm[2 * ns + s])) * (1.0 + 1e-12));
        }
        d2 = dx * dx + dy * dy + dz * dz;
    } else {
        v[0] = v[1] = v[2] = PAD_POS_F32;
    }
    for (int f = 0; f < 24; ++f)
        if (f < 3 || f > 5)
            if ((f < 12 || f > 14) && f != 18)
                tile[df_slot(f, j)] = v[f];
    const double m = block_max(d2, red);
    if (j == 0) {
        stiles[k].cx = cx;
        stiles[k].cy = cy;
        stiles[k].cz = cz;
        stiles[k].rad = radius_up(m);
    }
}

__global__ void pack_src_q_df(const double *__restrict__ w, const double *__restrict__ sigma,
                               long long ns, const TileInfo *__restrict__ stiles, float4 *spack,
                               int *counter, const int *__restrict__ perm, int scalar)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && counter)
        *counter = 0;
    const int k = blockIdx.x, j = threadIdx.x;
    const long long begin = stiles[k].begin;
    const int count = stiles[k].count;
    float qh[3] = {0.0f, 0.0f, 0.0f}, ql[3] = {0.0f, 0.0f, 0.0f}, qn = 0.0f;
    if (j < count) {
        const long long s = begin + j;
        const long long u = perm ? perm[s] : s;
        const double ww = w[s];
        double a = 0.0;
        for (int c = 0; c < (scalar ? 1 : 3); ++c) {
            const double q = ww * sigma[c * ns + u];
            split_df(q, qh[c], ql[c]);
            a += fabs(q);
        }
        qn = __double2float_ru(a * (1.0 + 1e-12));
    }
    float *tile = reinterpret_cast<float *>(spack + static_cast<size_t>(k) * DF_TILE_F4);
    for (int c = 0; c < 3; ++c) {
        tile[df_slot(3 + c, j)] = qh[c];
        tile[df_slot(12 + c, j)] = ql[c];
    }
    tile[df_slot(18, j)] = qn;
}

__global__ void pack_trg_f32(const double *__restrict__ trg, long long nt, TileInfo *ttiles, int TT,
                             float4 *tpack, float4 *tpack_lo, float4 *tpack_l2)
{
    __shared__ double red[32];
    __shared__ double bb[6][32];
    const int k = blockIdx.x;
    const long long begin = ttiles[k].begin;
    const int count = ttiles[k].count;
    double cx, cy, cz;
    tile_centre(trg, nt, begin, count, TT, bb, cx, cy, cz);
    double d2 = 0.0;
    for (int j = threadIdx.x; j < TT; j += blockDim.x) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f), l = v, l2 = v;
        if (j < count) {
            const long long t = begin + j;
            const double dx = trg[t] - cx, dy = trg[nt + t] - cy, dz = trg[2 * nt + t] - cz;
            split3(trg[t], cx, v.x, l.x, l2.x);
            split3(trg[nt + t], cy, v.y, l.y, l2.y);
            split3(trg[2 * nt + t], cz, v.z, l.z, l2.z);
            d2 = fmax(d2, dx * dx + dy * dy + dz * dz);
        }
        tpack[static_cast<size_t>(k) * TT + j] = v;
        if (tpack_lo)
            tpack_lo[static_cast<size_t>(k) * TT + j] = l;
        if (tpack_l2)
            tpack_l2[static_cast<size_t>(k) * TT + j] = l2;
    }
    const double m = block_max(d2, red);
    if (threadIdx.x == 0) {
        ttiles[k].cx = cx;
        ttiles[k].cy = cy;
        ttiles[k].cz = cz;
        ttiles[k].rad = radius_up(m);
    }
}

__global__ void reduce_partials_kernel(const TileInfo *__restrict__ ttiles, int TT,
                                       const double *__restrict__ partial, long long nt,
                                       double *out, double scale, double diag,
                                       const double *__restrict__ diag_sigma,
                                       const int *__restrict__ perm, int ncomp)
{
    const TileInfo ti = ttiles[blockIdx.x];
    if (ti.slot_begin < 0)
        return;
    for (int loc = threadIdx.x; loc < ti.count; loc += blockDim.x) {
        const long long t0 = ti.begin + loc;
        const long long t = perm ? perm[t0] : t0;   // caller's index of internal target t0
        for (int c = 0; c < ncomp; ++c) {
            double s = 0.0;
            for (int q = 0; q < ti.slot_count; ++q)
                s += partial[(static_cast<size_t>(ti.slot_begin + q) * 3 + c) * TT + loc];
            double o = scale * s;
            if (diag_sigma)
                o += diag * diag_sigma[c * nt + t];
            out[c * nt + t] = o;
        }
    }
}

// FP32 partials: (hi, lo) float pairs per (slot, component, target).  Compensated sums
// (comp 1) are merged across slots with TwoSum in FP32, plain ones (comp 0) with FP32 adds,
// double-float ones (comp 2) in FP64; the FP64 result gets the prefactor and the diagonal
// term.  Block (tile, component); four slot loads in
// flight per thread.
__device__ __forceinline__ void merge_partial(float &hi, float &lo, float2 v, int comp)
{
    if (comp) {
        const float s = hi + v.x;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (v.x - bb)) + v.y;
        hi = s;
    } else {
        hi += v.x;
    }
}

__global__ void reduce_partials_f32_kernel(const TileInfo *__restrict__ ttiles, int TT,
                                           const float2 *__restrict__ partial, long long nt,
                                           double *out, double scale, double diag,
                                           const double *__restrict__ diag_sigma, int comp,
                                           double *bound, const int *__restrict__ perm)
{
    const TileInfo ti = ttiles[blockIdx.x];
    const int c = blockIdx.y;
    const int nq = ti.slot_count;
    for (int loc = threadIdx.x; loc < ti.count; loc += blockDim.x) {
        const long long t0 = ti.begin + loc;
        const long long t = perm ? perm[t0] : t0;
        const float2 *pp = partial + (static_cast<size_t>(ti.slot_begin) * 3 + c) * TT + loc;
        const size_t qs = static_cast<size_t>(3) * TT;   // stride between slots
        if (comp == 2) {
            // double-float partials (hi, lo, error bound): each slot's hi + lo is exact in
            // FP64; add in FP64
            const float4 *p4 = reinterpret_cast<const float4 *>(partial) +
                               (static_cast<size_t>(ti.slot_begin) * 3 + c) * TT + loc;
            double acc = 0.0, mag = 0.0;
            for (int q = 0; q < nq; ++q) {
                const float4 v = p4[q * qs];
                acc += static_cast<double>(v.x) + static_cast<double>(v.y);
                mag += static_cast<double>(v.z);
            }
            double o = scale * acc;
            if (diag_sigma)
                o += diag * diag_sigma[c * nt + t];
            out[c * nt + t] = o;
            if (bound)
                bound[c * nt + t] = fabs(scale) * mag * (1.0 + 1e-6);
            continue;
        }
        float hi = 0.0f, lo = 0.0f;
        int q = 0;
        for (; q + 4 <= nq; q += 4) {
            const float2 v0 = pp[q * qs], v1 = pp[(q + 1) * qs], v2 = pp[(q + 2) * qs],
                         v3 = pp[(q + 3) * qs];
            merge_partial(hi, lo, v0, comp);
            merge_partial(hi, lo, v1, comp);
            merge_partial(hi, lo, v2, comp);
            merge_partial(hi, lo, v3, comp);
        }
        for (; q < nq; ++q)
            merge_partial(hi, lo, pp[q * qs], comp);
        double o = scale * (static_cast<double>(hi) + static_cast<double>(lo));
        if (diag_sigma)
            o += diag * diag_sigma[c * nt + t];
        out[c * nt + t] = o;
    }
}

__global__ void csr_apply_kernel(long long nrows, const int64_t *__restrict__ rowptr,
                                 const int64_t *__restrict__ col, const double *__restrict__ val,
                                 const double *__restrict__ x, double *y)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < nrows;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += val[k] * x[col[k]];
        y[i] += acc;
    }
}

}  // namespace

cudaError_t launch_pack_src_geom(int prec, const double *src, const double *nrm, double nscale,
                                 long long ns, TileInfo *stiles, int n_stiles, void *spack,
                                 cudaStream_t s)
{
    if (n_stiles <= 0)
        return cudaSuccess;
    if (prec == SBQ_FP64)
        pack_src_geom_f64<<<n_stiles, TS_F64, 0, s>>>(src, nrm, nscale, ns, stiles,
                                                       static_cast<double *>(spack));
    else if (prec == SBQ_DF32)
        pack_src_geom_df<<<n_stiles, TS_DF, 0, s>>>(src, nrm, nscale, ns, stiles,
                                                     static_cast<float4 *>(spack));
    else
        pack_src_geom_f32<<<n_stiles, TS_F32, 0, s>>>(src, nrm, nscale, ns, stiles,
                                                       static_cast<float4 *>(spack));
    return cudaGetLastError();
}

cudaError_t launch_pack_src_q(int prec, const double *w, const double *sigma, long long ns,
                              const TileInfo *stiles, int n_stiles, void *spack, int *counter,
                              const int *perm, int scalar, cudaStream_t s)
{
    if (n_stiles <= 0)
        return cudaSuccess;
    if (prec == SBQ_FP64)
        pack_src_q_f64<<<n_stiles, TS_F64, 0, s>>>(w, sigma, ns, stiles,
                                                    static_cast<double *>(spack), counter,
                                                    perm, scalar);
    else if (prec == SBQ_DF32)
        pack_src_q_df<<<n_stiles, TS_DF, 0, s>>>(w, sigma, ns, stiles,
                                                  static_cast<float4 *>(spack), counter,
                                                    perm, scalar);
    else
        pack_src_q_f32<<<n_stiles, TS_F32, 0, s>>>(w, sigma, ns, stiles,
                                                    static_cast<float4 *>(spack), counter,
                                                    perm, scalar);
    return cudaGetLastError();
}

cudaError_t launch_pack_trg(const double *trg, long long nt, TileInfo *ttiles, int n_ttiles, int TT,
                            float4 *tpack, float4 *tpack_lo, float4 *tpack_l2, cudaStream_t s)
{
    if (n_ttiles <= 0)
        return cudaSuccess;
    pack_trg_f32<<<n_ttiles, 256, 0, s>>>(trg, nt, ttiles, TT, tpack, tpack_lo, tpack_l2);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const TileInfo *ttiles, int n_ttiles, int TT,
                                   const double *partial, long long nt, double *out, double scale,
                                   double diag, const double *diag_sigma, const int *perm,
                                   int ncomp, cudaStream_t s)
{
    if (n_ttiles <= 0)
        return cudaSuccess;
    reduce_partials_kernel<<<n_ttiles, 256, 0, s>>>(ttiles, TT, partial, nt, out, scale, diag,
                                                     diag_sigma, perm, ncomp);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials_f32(const TileInfo *ttiles, int n_ttiles, int TT,
                                       const void *partial, long long nt, double *out,
                                       double scale, double diag, const double *diag_sigma,
                                       int comp, double *bound, const int *perm, int ncomp,
                                       cudaStream_t s)
{
    if (n_ttiles <= 0)
        return cudaSuccess;
    reduce_partials_f32_kernel<<<dim3(n_ttiles, ncomp), 256, 0, s>>>(ttiles, TT,
                                                         static_cast<const float2 *>(partial), nt,
                                                         out, scale, diag, diag_sigma, comp,
                                                         bound, perm);
    return cudaGetLastError();
}

cudaError_t launch_csr_apply(long long nrows, const int64_t *rowptr, const int64_t *col,
                             const double *val, const double *x, double *y, cudaStream_t s)
{
    if (nrows <= 0)
        return cudaSuccess;
    long long blocks = (nrows + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    csr_apply_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(nrows, rowptr, col, val, x, y);
    return cudaGetLastError();
}

cudaError_t launch_pairsum_sl(int, int, int, int, const PairsumParams &, cudaStream_t);
cudaError_t launch_pairsum_dl(int, int, int, int, const PairsumParams &, cudaStream_t);
cudaError_t launch_pairsum_cf(int, int, int, int, const PairsumParams &, cudaStream_t);
int occupancy_pairsum_sl(int, int, int);
int occupancy_pairsum_dl(int, int, int);
int occupancy_pairsum_cf(int, int, int);

cudaError_t launch_pairsum(int kind, int prec, int R, int W, int grid, const PairsumParams &p,
                           cudaStream_t s)
{
    switch (kind) {
    case KIND_SL: return launch_pairsum_sl(prec, R, W, grid, p, s);
    case KIND_DL: return launch_pairsum_dl(prec, R, W, grid, p, s);
    case KIND_CF: return launch_pairsum_cf(prec, R, W, grid, p, s);
    case KIND_LSL:
    case KIND_LDL:
    case KIND_LCF: return launch_pairsum_laplace(kind, prec, R, W, grid, p, s);
    default: return cudaErrorInvalidValue;
    }
}

int pairsum_blocks_per_sm(int kind, int prec, int R, int W)
{
    switch (kind) {
    case KIND_SL: return occupancy_pairsum_sl(prec, R, W);
    case KIND_DL: return occupancy_pairsum_dl(prec, R, W);
    case KIND_CF: return occupancy_pairsum_cf(prec, R, W);
    case KIND_LSL:
    case KIND_LDL:
    case KIND_LCF: return occupancy_pairsum_laplace(kind, prec, R, W);
    default: return 0;
    }
}

bool pairsum_shape_supported(int prec, int R, int W)
{
    if (prec == SBQ_FP64)
        return W == 4 && (R == 1 || R == 2);
    if (prec == SBQ_DF32)
        return (W == 4 && (R == 1 || R == 2 || R == 4)) || (W == 8 && R == 2);
    return (W == 4 && (R == 1 || R == 2 || R == 4 || R == 8)) || (W == 8 && (R == 1 || R == 4)) ||
           (W == 2 && (R == 4 || R == 8));
}

size_t pairsum_smem_bytes(int prec)
{
    if (prec == SBQ_FP64)
        return 2 * 9 * TS_F64 * sizeof(double);
    if (prec == SBQ_DF32)
        return 2 * DF_TILE_F4 * sizeof(float4);
    return 2 * F32_TILE_F4 * sizeof(float4);
}

}  // namespace sbq
