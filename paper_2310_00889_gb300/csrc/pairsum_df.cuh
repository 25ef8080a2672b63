// Double-float pair sums: FP64-class results from FP32 arithmetic.
//
// Every quantity is an unevaluated sum h + l of two FP32 numbers (about 48 significant
// bits).  Sums and products use error-free transformations: TwoSum (Knuth) for a + b,
// Fast2Sum (Dekker) when the larger operand is known, and the FMA residual
// a*b - fl(a*b) for products (Dekker's product, FMA form).  1/|r| starts from the SFU
// estimate and takes one Newton step evaluated with the exact square of the estimate,
// with its second-order term.  Each pair then carries a relative error of a few 2^-46
// against the exact kernel, so the sums reach about 1e-13 of the largest term, where the
// FP64 kernel reaches about 1e-15, while GB300 issues FP32 operations 64 times faster
// than FP64 ones.
//
// All arithmetic below goes through the __f*_rn intrinsics: the compiler never fuses or
// reorders them, which the error-free transformations rely on.
//
// Source tile layout (TS_DF sources, six float4 per source, source-major):
//   {xh, yh, zh, qxh} {qyh, qzh, nxh, nyh} {nzh, xm, ym, zm} {qxl, qyl, qzl, nxl}
//   {nyl, nzl, |q|, |n|} {xl, yl, zl, 0}
// positions relative to the tile centre in three FP32 parts h + m + l (to about 2^-72 of
// the offset), q = w sigma and the scaled normals in two parts, and the 1-norms of q and
// of the scaled normal (rounded up, for the error bound).  Targets use the FP32 target
// tiles with their second and third parts (tpack, tpack_lo, tpack_l2).
//
// Forming r.  Each target is rebased once per tile pair onto the source tile's centre as
// T + C + D (T one float, C the next 24 bits, D the rest).  Where the closest possible pair
// of the two tiles is at least DF_EXACT_R of (radii + centre distance) away, r = (T - y_h)
// + (C + D - y_m), within about 2^-46 of |r|.  Nearer tile pairs form r exactly from all
// three parts (two more TwoSums), so close pairs in wide tiles keep 2^-48 of |r| too.
//
// Rounding-error bound.  Every pair adds its envelope E = |q| ri (2 + |n| ri) (SL: 2 |q| ri,
// DL: |q| |n| ri^2), which bounds the magnitude of every intermediate product of the pair
// whatever cancels, to a running sum; an item's bound is DF_TERM_REL x that sum.
#pragma once

#include "sbq_common.cuh"

namespace sbq {

struct dfl {
    float h, l;
};

__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ff(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// a + b = s + e exactly (TwoSum)
__device__ __forceinline__ float df_two_sum(float a, float b, float &e)
{
    const float s = fa(a, b);
    const float bb = fs(s, a);
    e = fa(fs(a, fs(s, bb)), fs(b, bb));
    return s;
}

// a + b = s + e exactly when |a| >= |b| (Fast2Sum)
__device__ __forceinline__ float df_fast_two_sum(float a, float b, float &e)
{
    const float s = fa(a, b);
    e = fs(b, fs(s, a));
    return s;
}

__device__ __forceinline__ dfl df_norm(dfl a)
{
    float e;
    const float s = df_fast_two_sum(a.h, a.l, e);
    return {s, e};
}

// (a.h + a.l)(b.h + b.l), dropping a.l b.l
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = fm(a.h, b.h);
    float e = ff(a.h, b.h, -p);
    e = ff(a.h, b.l, e);
    e = ff(a.l, b.h, e);
    return {p, e};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float e;
    const float s = df_two_sum(a.h, b.h, e);
    return {s, fa(e, fa(a.l, b.l))};
}

// (hi, lo) += t
__device__ __forceinline__ void df_acc(float &hi, float &lo, dfl t)
{
    float e;
    hi = df_two_sum(hi, t.h, e);
    lo = fa(lo, fa(e, t.l));
}

// One pair in double-float.  Target: T + C + D (the target rebased onto the source tile's
// centre, see above); source record a..f (layout above).  Accumulates the same folded
// kernels as the FP32 and FP64 paths:
//   SL: ri q + (r.q) ri^3 r;  DL: (r.q)(r.n) ri^5 r;  CF: ri q + (r.q) ri^3 (1 + (r.n') ri^2) r
//   Laplace (scalar q): LSL ri q, LDL (r.n) ri^3 q, LCF ri q (1 + (r.n') ri^2)
// and the pair's envelope into env (see the error bound above; Laplace: |q| ri,
// |q| |n| ri^2, |q| ri (1 + |n| ri)).
template <int KIND, bool CHECK, bool EXACT>
__device__ __forceinline__ void pair_df(const float (&T)[3], const float (&C)[3],
                                        const float (&D)[3], const float4 a, const float4 b,
                                        const float4 c, const float4 d, const float4 e,
                                        const float4 f, float thr2, float (&acc)[6], float &env)
{
    const float ph[3] = {a.x, a.y, a.z}, pm[3] = {c.y, c.z, c.w}, pl[3] = {f.x, f.y, f.z};
    dfl rv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float e1;
        const float s1 = df_two_sum(T[k], -ph[k], e1);
        if (EXACT) {
            float e2, e3;
            const float s2 = df_two_sum(C[k], -pm[k], e2);
            const float h = df_two_sum(s1, s2, e3);
            rv[k] = df_norm({h, fa(fa(e1, e2), fa(e3, fs(D[k], pl[k])))});
        } else {
            rv[k] = df_norm({s1, fa(e1, fs(fa(C[k], D[k]), pm[k]))});
        }
    }
    const dfl rx = rv[0], ry = rv[1], rz = rv[2];
    // r^2: exact squares of the high parts, cross terms 2 h l, two TwoSums
    dfl r2;
    {
        const float px = fm(rx.h, rx.h), py = fm(ry.h, ry.h), pz = fm(rz.h, rz.h);
        float ex = ff(rx.h, rx.h, -px), ey = ff(ry.h, ry.h, -py), ez = ff(rz.h, rz.h, -pz);
        ex = ff(fa(rx.h, rx.h), rx.l, ex);
        ey = ff(fa(ry.h, ry.h), ry.l, ey);
        ez = ff(fa(rz.h, rz.h), rz.l, ez);
        float e1, e2;
        const float s1 = df_two_sum(px, py, e1);
        const float s2 = df_two_sum(s1, pz, e2);
        r2 = {s2, fa(fa(ex, ey), fa(fa(ez, e1), e2))};
    }
    // 1/|r| = y (1 + t/2 + 3 t^2 / 8), y the SFU estimate, t = 1 - r^2 y^2 (y^2 exact)
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2.h));
    if (CHECK)
        y = (r2.h > thr2) ? y : 0.0f;
    const float yy = fm(y, y);
    const float yl = ff(y, y, -yy);
    // t: the O(1) cancellation in one FMA, the two small terms summed first
    const float t = fa(ff(-r2.h, yy, 1.0f), ff(-r2.h, yl, -fm(r2.l, yy)));
    const dfl ri = {y, fm(fm(y, t), ff(0.375f, t, 0.5f))};
    // ri^2 = y^2 + 2 y ril (+ ril^2, dropped): the exact y^2 is already at hand
    const dfl ri2 = {yy, ff(fa(y, y), ri.l, yl)};
    const dfl ri3 = df_mul(ri2, ri);
    const dfl qx = {a.w, d.x}, qy = {b.x, d.y}, qz = {b.y, d.z};
    if (kind_laplace(KIND)) {   // scalar q in qx, one output component
        dfl tq;
        if (KIND == KIND_LSL) {
            tq = ri;
            env = ff(e.z, y, env);
        } else {
            const dfl nx = {b.z, d.w}, ny = {b.w, e.x}, nz = {c.x, e.y};
            const dfl rn = df_norm(df_add(df_add(df_mul(rx, nx), df_mul(ry, ny)), df_mul(rz, nz)));
            if (KIND == KIND_LDL) {
                tq = df_mul(rn, ri3);
                env = ff(fm(e.z, e.w), yy, env);
            } else {
                const dfl m = df_mul(rn, ri2);
                float eg;
                const float gh = df_two_sum(1.0f, m.h, eg);
                tq = df_mul(ri, df_norm({gh, fa(eg, m.l)}));
                env = ff(fm(e.z, y), ff(e.w, y, 1.0f), env);
            }
        }
        df_acc(acc[0], acc[3], df_mul(tq, qx));
        return;
    }
    const dfl rq = df_norm(df_add(df_add(df_mul(rx, qx), df_mul(ry, qy)), df_mul(rz, qz)));
    dfl bc;
    if (KIND == KIND_SL) {
        bc = df_mul(rq, ri3);
    } else {
        const dfl nx = {b.z, d.w}, ny = {b.w, e.x}, nz = {c.x, e.y};
        const dfl rn = df_norm(df_add(df_add(df_mul(rx, nx), df_mul(ry, ny)), df_mul(rz, nz)));
        if (KIND == KIND_DL) {
            bc = df_mul(df_mul(rq, rn), df_mul(ri3, ri2));
        } else {
            const dfl m = df_mul(rn, ri2);
            float eg;
            const float gh = df_two_sum(1.0f, m.h, eg);
            const dfl g = df_norm({gh, fa(eg, m.l)});
            bc = df_mul(df_mul(rq, ri3), g);
        }
    }
    if (KIND != KIND_DL) {
        df_acc(acc[0], acc[3], df_mul(ri, qx));
        df_acc(acc[1], acc[4], df_mul(ri, qy));
        df_acc(acc[2], acc[5], df_mul(ri, qz));
    }
    df_acc(acc[0], acc[3], df_mul(bc, rx));
    df_acc(acc[1], acc[4], df_mul(bc, ry));
    df_acc(acc[2], acc[5], df_mul(bc, rz));
    if (KIND == KIND_SL)
        env = ff(fa(e.z, e.z), y, env);
    else if (KIND == KIND_DL)
        env = ff(fm(e.z, e.w), yy, env);
    else
        env = ff(fm(e.z, y), ff(e.w, y, 2.0f), env);
}

// Parameters of one (target tile, source tile) pair for the double-float kernel.
struct __align__(16) DfPairParams {
    float dh[3], dm[3], dl[3];   // c_T - c_S = dh + dm + dl
    float thr2;                  // squared coincidence threshold
    int flags;                   // TP_NEAR (coincidence test) | TP_EXACT (exact r)
    float pad_;
};
constexpr int TP_EXACT = 4;

__device__ __forceinline__ void df_split3(double a, double b, float &h, float &m, float &l)
{
    const double s = a - b;
    const double bb = s - a;
    const double e = (a - (s - bb)) - (b + bb);
    h = static_cast<float>(s);
    const double r1 = s - static_cast<double>(h);
    m = static_cast<float>(r1);
    l = static_cast<float>((r1 - static_cast<double>(m)) + e);
}

__device__ __forceinline__ void tile_pair_setup_df(DfPairParams &tp, double tcx, double tcy,
                                                   double tcz, float trad, const TileInfo &si)
{
    const double ddx = tcx - si.cx, ddy = tcy - si.cy, ddz = tcz - si.cz;
    const double dist = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
    const double lim = static_cast<double>(trad) + static_cast<double>(si.rad);
    int flags = 0;
    if ((dist - lim) <= 1.0e-5 * (dist + lim) + 1.0e-30)
        flags |= TP_NEAR | TP_EXACT;
    if ((dist - lim) < DF_EXACT_R * (dist + lim))
        flags |= TP_EXACT;
    tp.flags = flags;
    df_split3(tcx, si.cx, tp.dh[0], tp.dm[0], tp.dl[0]);
    df_split3(tcy, si.cy, tp.dh[1], tp.dm[1], tp.dl[1]);
    df_split3(tcz, si.cz, tp.dh[2], tp.dm[2], tp.dl[2]);
    const float thr = static_cast<float>(DF_COINCIDENT_REL * lim);
    tp.thr2 = thr * thr;
}

template <int KIND, int R, bool CHECK, bool EXACT>
__device__ __forceinline__ void tile_df(const float4 *__restrict__ sp, float thr2,
                                        const float (&T)[R][3], const float (&C)[R][3],
                                        const float (&D)[R][3], float (&acc)[R][6],
                                        float (&env)[R])
{
#pragma unroll 2
    for (int j = 0; j < TS_DF; ++j) {
        const float4 *rec = sp + 6 * j;
        const float4 a = rec[0], b = rec[1], c = rec[2], d = rec[3], e = rec[4], f = rec[5];
#pragma unroll
        for (int r = 0; r < R; ++r)
            pair_df<KIND, CHECK, EXACT>(T[r], C[r], D[r], a, b, c, d, e, f, thr2, acc[r], env[r]);
    }
}

// Persistent double-float pair-sum kernel: same work list, ring protocol and bounded
// waits as pairsum_f32_kernel; every item writes its (hi, lo) sums and the magnitude sum
// of its terms to its partial slot as float4 [slot][3][TT], and reduce_partials_f32
// (double-float mode) adds the slots in FP64.
template <int KIND, int R, int W>
__global__ void __launch_bounds__(W * 32) pairsum_df_kernel(const PairsumParams p)
{
    constexpr int NT = W * 32;
    constexpr int TT = NT * R;
    constexpr uint32_t TILE_BYTES = DF_TILE_F4 * sizeof(float4);
    constexpr int STAGE = DF_TILE_F4;

    extern __shared__ __align__(128) float4 sbuf[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int4 s_item;
    __shared__ DfPairParams s_tp[2];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const float4 *__restrict__ spack = static_cast<const float4 *>(p.spack);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t g = 0;
    double tcx = 0.0, tcy = 0.0, tcz = 0.0;
    float trad = 0.0f;
    int4 pending = make_int4(-1, 0, 0, 0);
    bool have_pending = false;

    auto claim_and_issue = [&](int st) -> int4 {
        const int i = atomicAdd(p.counter, 1);
        const int4 nx = (i < p.n_items) ? p.items[i] : make_int4(-1, 0, 0, 0);
        if (nx.x >= 0) {
            const TileInfo tt = p.ttiles[nx.x];
            tcx = tt.cx;
            tcy = tt.cy;
            tcz = tt.cz;
            trad = tt.rad;
            tile_pair_setup_df(s_tp[st], tcx, tcy, tcz, trad, p.stiles[nx.y]);
            mbar_arrive_expect_tx(&bar[st], TILE_BYTES);
            bulk_copy_g2s(sbuf + st * STAGE, spack + static_cast<size_t>(nx.y) * STAGE, TILE_BYTES,
                          &bar[st]);
        }
        return nx;
    };

    for (;;) {
        if (tid == 0) {
            if (have_pending) {
                s_item = pending;
                have_pending = false;
            } else {
                s_item = claim_and_issue(g & 1);
            }
        }
        __syncthreads();
        const int4 it = s_item;
        if (it.x < 0)
            break;

        float th[R][3], tm[R][3], tl[R][3];   // target - c_T in three parts
        const size_t toff = static_cast<size_t>(it.x) * TT + warp * 32 * R + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 v = p.tpack[toff + r * 32];
            const float4 m = p.tpack_lo[toff + r * 32];
            const float4 l = p.tpack_l2[toff + r * 32];
            th[r][0] = v.x;
            th[r][1] = v.y;
            th[r][2] = v.z;
            tm[r][0] = m.x;
            tm[r][1] = m.y;
            tm[r][2] = m.z;
            tl[r][0] = l.x;
            tl[r][1] = l.y;
            tl[r][2] = l.z;
        }
        float acc[R][6], env[R];   // item sums; sum of the pair envelopes
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int q = 0; q < 6; ++q)
                acc[r][q] = 0.0f;
            env[r] = 0.0f;
        }

        const int nk = it.z - it.y;
        for (int k = 0; k < nk; ++k) {
            const uint32_t gk = g + k;
            const int st = gk & 1;
            const bool timed_out = !mbar_wait_bounded(&bar[st], (gk >> 1) & 1);
            if (__syncthreads_or(timed_out)) {
                if (tid == 0)
                    atomicOr(p.err, DEV_ERR_TIMEOUT);
                mbar_wait_bounded(&bar[st], (gk >> 1) & 1, 100000000ull);
                return;
            }
            if (tid == 0) {
                const int sn = (gk + 1) & 1;
                if (k + 1 < nk) {
                    tile_pair_setup_df(s_tp[sn], tcx, tcy, tcz, trad, p.stiles[it.y + k + 1]);
                    mbar_arrive_expect_tx(&bar[sn], TILE_BYTES);
                    bulk_copy_g2s(sbuf + sn * STAGE,
                                  spack + static_cast<size_t>(it.y + k + 1) * STAGE, TILE_BYTES,
                                  &bar[sn]);
                } else {
                    pending = claim_and_issue(sn);
                    have_pending = true;
                }
            }
            const DfPairParams tp = s_tp[st];
            // target rebased onto the source tile's centre: T + C + D
            float T[R][3], C[R][3], D[R][3];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float e1, e2, e3;
                    T[r][q] = df_two_sum(th[r][q], tp.dh[q], e1);
                    const float c0 = df_two_sum(tm[r][q], tp.dm[q], e2);
                    C[r][q] = df_two_sum(c0, e1, e3);
                    D[r][q] = fa(fa(tl[r][q], tp.dl[q]), fa(e2, e3));
                }
            // the tile's sums start from zero and join the item's sums with a full
            // double-float addition, so rounding inside a tile stays relative to that
            // tile's own sum, not to the running sum of thousands of tiles
            float tacc[R][6];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    tacc[r][q] = 0.0f;
            const float4 *sp = sbuf + st * STAGE;
            if (tp.flags & TP_NEAR)
                tile_df<KIND, R, true, true>(sp, tp.thr2, T, C, D, tacc, env);
            else if (tp.flags & TP_EXACT)
                tile_df<KIND, R, false, true>(sp, tp.thr2, T, C, D, tacc, env);
            else
                tile_df<KIND, R, false, false>(sp, tp.thr2, T, C, D, tacc, env);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const dfl v = df_norm(df_add({acc[r][q], acc[r][q + 3]},
                                                 df_norm({tacc[r][q], tacc[r][q + 3]})));
                    acc[r][q] = v.h;
                    acc[r][q + 3] = v.l;
                }
        }
        g += nk;

        float4 *pp = reinterpret_cast<float4 *>(p.partial) + static_cast<size_t>(it.w) * 3 * TT +
                     warp * 32 * R + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float bd = fm(static_cast<float>(DF_TERM_REL), env[r]);
            pp[r * 32] = make_float4(acc[r][0], acc[r][3], bd, 0.0f);
            pp[TT + r * 32] = make_float4(acc[r][1], acc[r][4], bd, 0.0f);
            pp[2 * TT + r * 32] = make_float4(acc[r][2], acc[r][5], bd, 0.0f);
        }
    }
}

}  // namespace sbq
