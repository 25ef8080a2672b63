// Pair-sum kernels: the uncorrected Nystrom sum of paper Eq. nystrom-no-correction for
// the Stokes single layer (Eq. stokes-sl), double layer (Eq. stokes-dl, sign such that
// int D[e] = -e inside) and their combination eta S + D (Eq. stokes-bie-new).
//
// Work decomposition (both precisions): a persistent grid claims work items
// {target tile, first source tile, end source tile, partial slot} from a list with an
// atomic counter.  A target tile holds TT = 32 * W * R targets; thread (warp w, lane l)
// keeps targets w*32*R + r*32 + l (r < R) in registers.  Source tiles stream through
// a two-stage shared-memory ring filled by one bulk async copy per tile (TMA engine)
// that completes on an mbarrier; every thread reads each source by broadcast and
// applies it to its R targets.  An item writes its sums straight to the output when it
// covers the whole source range of its target tile, else to its partial slot, which a
// fixed-order reduction adds up later (deterministic results).
//
// FP32 path: the inner loop takes two sources per step with the packed FP32x2
// instructions (one issue slot for two FP32 operations), each thread applying them to its
// R targets.  Targets and sources are stored relative to their tile centre (FP64
// subtraction, then rounding), and per (target tile, source tile) the FP64 offset of
// the two centres is rounded once and added to the targets.  Pairs whose tiles cannot
// contain coincident points skip the r^2 == 0 test.  The compensated variant
//  * sums runs of COMP_RUN sources in FP32 and merges each run into a (hi, lo) pair
//    with TwoSum, and
//  * in tile pairs whose tiles come within one tile extent of each other (where the
//    rounding of the centred coordinates is not small next to the pair distance) forms
//    r = x - y from high and low FP32 parts of both points and of the centre offset, so
//    that the difference of nearby points keeps its full FP32 accuracy.
#pragma once

#include "sbq_common.cuh"

namespace sbq {

// 1/sqrt(x) on the SFU, denormals flushed (x is a squared distance between distinct
// points, far above the FP32 denormal range for any admissible input).
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32 pairs: one 64-bit register holds the values of two sources (2m, 2m + 1);
// the f32x2 instructions process both in one issue slot.
using f2 = unsigned long long;

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// 1/x on the SFU, denormals flushed (x as for rsqrt_sfu).
__device__ __forceinline__ float rcp_sfu(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-pair arithmetic for one target against two sources at once, given r = (dx, dy, dz)
// (packed).  Accumulates (folded prefactors, see the launcher):
//   SL: ri (q + (r.q) ri^2 r)
//   DL: (r.q)(r.n) ri^5 r
//   CF: ri (q + (r.q) ri^2 (1 + (r.n') ri^2) r),  n' = kappa n stored by the pack
//   Laplace (scalar q): LSL ri q, LDL (r.n) ri^3 q, LCF ri q (1 + (r.n') ri^2)
// ri^2 comes from the SFU reciprocal of r^2 (a second SFU operation per pair in place of
// an FP32-pipe multiply: the FP32 pipe is the kernel's bound, the SFU has room), except
// in tile pairs that may hold coincident points (CHECK), where ri is zeroed for skipped
// pairs and ri^2 = ri ri inherits that zero.  Per two pairs the combined field takes 21
// packed FP32 operations (3 sub, 13 fma, 5 mul) and 4 SFU operations.
template <int KIND, bool CHECK>
__device__ __forceinline__ void pair2(f2 dx, f2 dy, f2 dz, f2 QX, f2 QY, f2 QZ, f2 NX, f2 NY, f2 NZ,
                                      float thr2, f2 &ax, f2 &ay, f2 &az)
{
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float r2a, r2b;
    f2_unpack(r2, r2a, r2b);
    float ra = rsqrt_sfu(r2a), rb = rsqrt_sfu(r2b);
    if (CHECK) {
        ra = (r2a > thr2) ? ra : 0.0f;
        rb = (r2b > thr2) ? rb : 0.0f;
    }
    const f2 ri = f2_pack(ra, rb);
    auto inv_r2 = [&]() -> f2 {
        return CHECK ? f2_mul(ri, ri) : f2_pack(rcp_sfu(r2a), rcp_sfu(r2b));
    };
    if (KIND == KIND_SL) {
        const f2 rq = f2_fma(dx, QX, f2_fma(dy, QY, f2_mul(dz, QZ)));
        const f2 b = f2_mul(rq, inv_r2());
        ax = f2_fma(ri, f2_fma(b, dx, QX), ax);
        ay = f2_fma(ri, f2_fma(b, dy, QY), ay);
        az = f2_fma(ri, f2_fma(b, dz, QZ), az);
    } else if (KIND == KIND_DL) {
        const f2 rq = f2_fma(dx, QX, f2_fma(dy, QY, f2_mul(dz, QZ)));
        const f2 rn = f2_fma(dx, NX, f2_fma(dy, NY, f2_mul(dz, NZ)));
        const f2 ri2 = inv_r2();
        const f2 b = f2_mul(f2_mul(f2_mul(rq, ri2), f2_mul(rn, ri2)), ri);
        ax = f2_fma(b, dx, ax);
        ay = f2_fma(b, dy, ay);
        az = f2_fma(b, dz, az);
    } else if (KIND == KIND_CF) {
        const f2 one = f2_pack(1.0f, 1.0f);
        const f2 rq = f2_fma(dx, QX, f2_fma(dy, QY, f2_mul(dz, QZ)));
        const f2 rn = f2_fma(dx, NX, f2_fma(dy, NY, f2_mul(dz, NZ)));
        const f2 ri2 = inv_r2();
        const f2 b = f2_mul(f2_mul(rq, ri2), f2_fma(rn, ri2, one));
        ax = f2_fma(ri, f2_fma(b, dx, QX), ax);
        ay = f2_fma(ri, f2_fma(b, dy, QY), ay);
        az = f2_fma(ri, f2_fma(b, dz, QZ), az);
    } else if (KIND == KIND_LSL) {   // Laplace: scalar q in QX, sum in ax
        ax = f2_fma(ri, QX, ax);
    } else if (KIND == KIND_LDL) {
        const f2 rn = f2_fma(dx, NX, f2_fma(dy, NY, f2_mul(dz, NZ)));
        ax = f2_fma(f2_mul(rn, f2_mul(inv_r2(), ri)), QX, ax);
    } else {                         // KIND_LCF: ri q (1 + (r.n') ri^2), n' = kappa n
        const f2 one = f2_pack(1.0f, 1.0f);
        const f2 rn = f2_fma(dx, NX, f2_fma(dy, NY, f2_mul(dz, NZ)));
        ax = f2_fma(f2_mul(ri, f2_fma(rn, inv_r2(), one)), QX, ax);
    }
}

// Error-free transformation a + b = s + e (Knuth's TwoSum); folds e into lo.
__device__ __forceinline__ void two_sum_merge(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += e;
}

// Fold a packed accumulator (even- and odd-indexed sources) into a scalar sum.
__device__ __forceinline__ void fold_packed(f2 &acc, float &hi, float &lo, bool comp)
{
    float a, b;
    f2_unpack(acc, a, b);
    if (comp) {
        two_sum_merge(hi, lo, a);
        two_sum_merge(hi, lo, b);
    } else {
        hi += a + b;
    }
    acc = 0ull;
}

// One staged source tile (pair layout, see sbq_common.cuh) applied to the thread's R
// targets, two sources per step.  HILO: targets carry low parts (xl, yl, zl) and r is
// formed from high and low parts.  CHECK: pairs with r^2 <= thr2 count as coincident.
// COMP: packed partial sums are merged into (hi, lo) with TwoSum every COMP_RUN sources;
// otherwise they are folded into hi once per tile.
template <int KIND, int R, bool CHECK, bool COMP, bool HILO>
__device__ __forceinline__ void tile_f32(const float4 *__restrict__ sp, float thr2,
                                         const float (&xh)[R], const float (&yh)[R],
                                         const float (&zh)[R], const float (&xl)[R],
                                         const float (&yl)[R], const float (&zl)[R],
                                         float (&hx)[R], float (&hy)[R], float (&hz)[R],
                                         float (&lx)[R], float (&ly)[R], float (&lz)[R])
{
    constexpr int H = TS_F32 / 2;           // source pairs per tile
    constexpr int RUN = COMP ? COMP_RUN / 2 : H;
    const ulonglong2 *__restrict__ s2 = reinterpret_cast<const ulonglong2 *>(sp);
    f2 XT[R], YT[R], ZT[R], XL[R], YL[R], ZL[R], ax[R], ay[R], az[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        XT[r] = f2_pack(xh[r], xh[r]);
        YT[r] = f2_pack(yh[r], yh[r]);
        ZT[r] = f2_pack(zh[r], zh[r]);
        if (HILO) {
            XL[r] = f2_pack(xl[r], xl[r]);
            YL[r] = f2_pack(yl[r], yl[r]);
            ZL[r] = f2_pack(zl[r], zl[r]);
        }
        ax[r] = ay[r] = az[r] = 0ull;
    }
#pragma unroll 1
    for (int m0 = 0; m0 < H; m0 += RUN) {
#pragma unroll 4
        for (int m = m0; m < m0 + RUN; ++m) {
            const ulonglong2 a0 = s2[m];           // X, Y
            const ulonglong2 a1 = s2[H + m];       // Z, QX
            const ulonglong2 a2 = s2[2 * H + m];   // QY, QZ
            ulonglong2 b0, b1, b2;
            if (kind_has_normals(KIND) || HILO)
                b1 = s2[4 * H + m];                // NZ, LX
            if (kind_has_normals(KIND))
                b0 = s2[3 * H + m];                // NX, NY
            if (HILO)
                b2 = s2[5 * H + m];                // LY, LZ
#pragma unroll
            for (int r = 0; r < R; ++r) {
                f2 dx = f2_sub(XT[r], a0.x), dy = f2_sub(YT[r], a0.y), dz = f2_sub(ZT[r], a1.x);
                if (HILO) {
                    dx = f2_add(dx, f2_sub(XL[r], b1.y));
                    dy = f2_add(dy, f2_sub(YL[r], b2.x));
                    dz = f2_add(dz, f2_sub(ZL[r], b2.y));
                }
                pair2<KIND, CHECK>(dx, dy, dz, a1.y, a2.x, a2.y, b0.x, b0.y, b1.x, thr2, ax[r],
                                   ay[r], az[r]);
            }
        }
        if (COMP) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                fold_packed(ax[r], hx[r], lx[r], true);
                fold_packed(ay[r], hy[r], ly[r], true);
                fold_packed(az[r], hz[r], lz[r], true);
            }
        }
    }
    if (!COMP) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            fold_packed(ax[r], hx[r], lx[r], false);
            fold_packed(ay[r], hy[r], ly[r], false);
            fold_packed(az[r], hz[r], lz[r], false);
        }
    }
}

// x + d = s + e exactly (TwoSum), returning s; e is added to lo.
__device__ __forceinline__ float two_sum_add(float x, float d, float &lo)
{
    const float s = x + d;
    const float bb = s - x;
    lo += (x - (s - bb)) + (d - bb);
    return s;
}

// Parameters of one (target tile, source tile) pair, computed once per pair by the
// thread that issues the source tile's copy and read by all threads from shared memory.
struct __align__(16) TilePairParams {
    float sx, sy, sz;      // centre offset c_T - c_S rounded to FP32
    float thr2;            // squared coincidence threshold
    float lx, ly, lz;      // part of the offset lost to that rounding
    int flags;             // TP_NEAR | TP_HILO
};
constexpr int TP_NEAR = 1;   // the tiles may hold coincident points: test r^2 > thr2
constexpr int TP_HILO = 2;   // form r from high and low parts (compensated kernels)
// Compensated kernels use high/low differences for tile pairs whose centres are closer
// than HILO_REL x (sum of the tile radii): there the FP32 centring error is not small
// next to the shortest pair distances.
constexpr double HILO_REL = 1.0;

template <bool COMP>
__device__ __forceinline__ void tile_pair_setup(TilePairParams &tp, double tcx, double tcy,
                                                double tcz, float trad, const TileInfo &si)
{
    const double ddx = tcx - si.cx, ddy = tcy - si.cy, ddz = tcz - si.cz;
    const double dist = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
    const double lim = static_cast<double>(trad) + static_cast<double>(si.rad);
    int flags = 0;
    if ((dist - lim) <= 1.0e-5 * (dist + lim) + 1.0e-30)
        flags |= TP_NEAR;
    if (COMP && dist <= HILO_REL * lim)
        flags |= TP_HILO | TP_NEAR;
    const float sx = static_cast<float>(ddx), sy = static_cast<float>(ddy),
                sz = static_cast<float>(ddz);
    tp.sx = sx;
    tp.sy = sy;
    tp.sz = sz;
    tp.lx = static_cast<float>(ddx - static_cast<double>(sx));
    tp.ly = static_cast<float>(ddy - static_cast<double>(sy));
    tp.lz = static_cast<float>(ddz - static_cast<double>(sz));
    const float thr = static_cast<float>(COINCIDENT_REL * lim);
    tp.thr2 = thr * thr;
    tp.flags = flags;
}

// Resident CTAs per SM the FP32 kernel is compiled for: the 128-thread shapes are held to
// the register budget of 5 (R = 2) or 8 (R = 1) CTAs per SM; the others take what their
// registers allow.
__host__ __device__ constexpr int f32_min_blocks(int R, int W)
{
    return (W == 4 && R == 2) ? 5 : ((W == 4 && R == 1) ? 8 : 1);
}

// FP32 kernels write every item's sums to its partial slot as (hi, lo) float pairs,
// [slot][3][TT] float2; reduce_partials_f32 adds the slots of a target tile and applies
// the prefactor and the diagonal term in FP64 (no FP64 work in this kernel's loop).
template <int KIND, int R, int W, bool COMP>
__global__ void __launch_bounds__(W * 32, f32_min_blocks(R, W)) pairsum_f32_kernel(const PairsumParams p)
{
    constexpr int NT = W * 32;
    constexpr int TT = NT * R;
    constexpr int TS = TS_F32;
    // blocks of TS/2 float4 to copy: SL {X,Y} {Z,QX} {QY,QZ}; DL/CF add {NX,NY} {NZ,LX};
    // compensated kernels also need {LY,LZ} (and LX)
    constexpr int NB = COMP ? F32_TILE_BLOCKS
                            : ((KIND == KIND_SL || KIND == KIND_LSL) ? 3 : 5);
    constexpr uint32_t TILE_BYTES = NB * (TS / 2) * sizeof(float4);
    constexpr int STAGE = F32_TILE_BLOCKS * (TS / 2);   // float4 per smem stage
    constexpr int GSTRIDE = F32_TILE_BLOCKS * (TS / 2); // float4 per packed tile

    extern __shared__ __align__(128) float4 sbuf[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int4 s_item;
    __shared__ TilePairParams s_tp[2];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const float4 *__restrict__ spack = static_cast<const float4 *>(p.spack);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Ring protocol (two stages, one barrier per tile): the copy of the next tile is
    // issued right after the barrier that follows the wait for the current tile, when
    // every thread has finished the tile that last used the other stage.  During an item's
    // last tile, thread 0 already claims the next item and issues its first tile.
    uint32_t g = 0;                  // source tiles consumed by this CTA (ring position)
    double tcx = 0.0, tcy = 0.0, tcz = 0.0;   // thread 0: centre and radius of the target tile
    float trad = 0.0f;
    int4 pending = make_int4(-1, 0, 0, 0);   // thread 0: next item, first tile already issued
    bool have_pending = false;

    // thread 0: claim an item and issue its first source tile into stage `st`
    auto claim_and_issue = [&](int st) -> int4 {
        const int i = atomicAdd(p.counter, 1);
        const int4 nx = (i < p.n_items) ? p.items[i] : make_int4(-1, 0, 0, 0);
        if (nx.x >= 0) {
            const TileInfo tt = p.ttiles[nx.x];
            tcx = tt.cx;
            tcy = tt.cy;
            tcz = tt.cz;
            trad = tt.rad;
            tile_pair_setup<COMP>(s_tp[st], tcx, tcy, tcz, trad, p.stiles[nx.y]);
            mbar_arrive_expect_tx(&bar[st], TILE_BYTES);
            bulk_copy_g2s(sbuf + st * STAGE, spack + static_cast<size_t>(nx.y) * GSTRIDE,
                          TILE_BYTES, &bar[st]);
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

        float tx[R], ty[R], tz[R];
        const size_t toff = static_cast<size_t>(it.x) * TT + warp * 32 * R + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 v = p.tpack[toff + r * 32];
            tx[r] = v.x;
            ty[r] = v.y;
            tz[r] = v.z;
        }
        float hx[R], hy[R], hz[R], lx[R], ly[R], lz[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            hx[r] = hy[r] = hz[r] = 0.0f;
            lx[r] = ly[r] = lz[r] = 0.0f;
        }

        const int nk = it.z - it.y;
        for (int k = 0; k < nk; ++k) {
            const uint32_t gk = g + k;
            const int st = gk & 1;
            const bool timed_out = !mbar_wait_bounded(&bar[st], (gk >> 1) & 1);
            if (__syncthreads_or(timed_out)) {
                // The copy never landed: flag it, give it a bounded chance to land, and
                // leave without touching the output (no other copy is in flight here).
                if (tid == 0)
                    atomicOr(p.err, DEV_ERR_TIMEOUT);
                mbar_wait_bounded(&bar[st], (gk >> 1) & 1, 100000000ull);
                return;
            }
            // every thread is past tile gk - 1: the other stage can be refilled
            if (tid == 0) {
                const int sn = (gk + 1) & 1;
                if (k + 1 < nk) {
                    tile_pair_setup<COMP>(s_tp[sn], tcx, tcy, tcz, trad, p.stiles[it.y + k + 1]);
                    mbar_arrive_expect_tx(&bar[sn], TILE_BYTES);
                    bulk_copy_g2s(sbuf + sn * STAGE,
                                  spack + static_cast<size_t>(it.y + k + 1) * GSTRIDE, TILE_BYTES,
                                  &bar[sn]);
                } else {
                    pending = claim_and_issue(sn);
                    have_pending = true;
                }
            }
            const TilePairParams tp = s_tp[st];
            float xh[R], yh[R], zh[R], xl[R], yl[R], zl[R];
            const float4 *sp = sbuf + st * STAGE;
            if (COMP && (tp.flags & TP_HILO)) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 l = p.tpack_lo[toff + r * 32];   // only hilo tiles need it
                    xl[r] = l.x + tp.lx;
                    yl[r] = l.y + tp.ly;
                    zl[r] = l.z + tp.lz;
                    xh[r] = two_sum_add(tx[r], tp.sx, xl[r]);
                    yh[r] = two_sum_add(ty[r], tp.sy, yl[r]);
                    zh[r] = two_sum_add(tz[r], tp.sz, zl[r]);
                }
                tile_f32<KIND, R, true, COMP, COMP>(sp, tp.thr2, xh, yh, zh, xl, yl, zl, hx, hy, hz,
                                                     lx, ly, lz);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    xh[r] = tx[r] + tp.sx;
                    yh[r] = ty[r] + tp.sy;
                    zh[r] = tz[r] + tp.sz;
                    xl[r] = yl[r] = zl[r] = 0.0f;
                }
                if (tp.flags & TP_NEAR)
                    tile_f32<KIND, R, true, COMP, false>(sp, tp.thr2, xh, yh, zh, xl, yl, zl, hx, hy,
                                                         hz, lx, ly, lz);
                else
                    tile_f32<KIND, R, false, COMP, false>(sp, tp.thr2, xh, yh, zh, xl, yl, zl, hx,
                                                          hy, hz, lx, ly, lz);
            }
        }
        g += nk;

        // Epilogue: (hi, lo) pairs to the item's partial slot (padded targets included).
        float2 *pp = reinterpret_cast<float2 *>(p.partial) + static_cast<size_t>(it.w) * 3 * TT +
                     warp * 32 * R + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pp[r * 32] = make_float2(hx[r], lx[r]);
            pp[TT + r * 32] = make_float2(hy[r], ly[r]);
            pp[2 * TT + r * 32] = make_float2(hz[r], lz[r]);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void pair_f64(double x, double y, double z, const double *__restrict__ s,
                                         int j, double &ax, double &ay, double &az)
{
    constexpr int TS = TS_F64;
    const double dx = x - s[j], dy = y - s[TS + j], dz = z - s[2 * TS + j];
    const double qx = s[3 * TS + j], qy = s[4 * TS + j], qz = s[5 * TS + j];
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double ri = (r2 > 0.0) ? rsqrt(r2) : 0.0;
    const double rq = fma(dx, qx, fma(dy, qy, dz * qz));
    const double ri2 = ri * ri;
    if (KIND == KIND_SL) {
        const double b = (rq * ri2) * ri;
        ax = fma(ri, qx, ax);
        ay = fma(ri, qy, ay);
        az = fma(ri, qz, az);
        ax = fma(b, dx, ax);
        ay = fma(b, dy, ay);
        az = fma(b, dz, az);
    } else if (KIND == KIND_LSL) {
        ax = fma(ri, qx, ax);
    } else if (KIND == KIND_LDL || KIND == KIND_LCF) {
        const double rn = fma(dx, s[6 * TS + j], fma(dy, s[7 * TS + j], dz * s[8 * TS + j]));
        if (KIND == KIND_LDL)
            ax = fma(rn * (ri2 * ri), qx, ax);
        else
            ax = fma(ri * fma(rn, ri2, 1.0), qx, ax);
    } else {
        const double rn = fma(dx, s[6 * TS + j], fma(dy, s[7 * TS + j], dz * s[8 * TS + j]));
        if (KIND == KIND_DL) {
            const double b = ((rq * ri2) * (rn * ri2)) * ri;
            ax = fma(b, dx, ax);
            ay = fma(b, dy, ay);
            az = fma(b, dz, az);
        } else {
            const double gg = fma(rn, ri2, 1.0);
            const double b = (rq * ri2) * (ri * gg);
            ax = fma(ri, qx, ax);
            ay = fma(ri, qy, ay);
            az = fma(ri, qz, az);
            ax = fma(b, dx, ax);
            ay = fma(b, dy, ay);
            az = fma(b, dz, az);
        }
    }
}

template <int KIND, int R, int W>
__global__ void __launch_bounds__(W * 32) pairsum_f64_kernel(const PairsumParams p)
{
    constexpr int NT = W * 32;
    constexpr int TT = NT * R;
    constexpr int TS = TS_F64;
    constexpr int NF = (KIND == KIND_SL || KIND == KIND_LSL) ? 6 : 9;
    constexpr uint32_t TILE_BYTES = NF * TS * sizeof(double);
    constexpr int STAGE = 9 * TS;   // doubles per stage (and per packed tile)

    extern __shared__ __align__(128) double dbuf[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int4 s_item;

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const double *__restrict__ spack = static_cast<const double *>(p.spack);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t g = 0;
    for (;;) {
        if (tid == 0) {
            const int i = atomicAdd(p.counter, 1);
            s_item = (i < p.n_items) ? p.items[i] : make_int4(-1, 0, 0, 0);
        }
        __syncthreads();
        const int4 it = s_item;
        if (it.x < 0)
            break;
        const TileInfo tt = p.ttiles[it.x];

        double tx[R], ty[R], tz[R], ax[R], ay[R], az[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int loc = warp * 32 * R + r * 32 + lane;
            const long long t = tt.begin + (loc < tt.count ? loc : 0);
            tx[r] = p.trg[t];
            ty[r] = p.trg[p.nt + t];
            tz[r] = p.trg[2 * p.nt + t];
            ax[r] = ay[r] = az[r] = 0.0;
        }

        const int nk = it.z - it.y;
        if (tid == 0) {
            const int st = g & 1;
            mbar_arrive_expect_tx(&bar[st], TILE_BYTES);
            bulk_copy_g2s(dbuf + st * STAGE, spack + static_cast<size_t>(it.y) * STAGE, TILE_BYTES,
                          &bar[st]);
        }
        for (int k = 0; k < nk; ++k) {
            const uint32_t gk = g + k;
            const int st = gk & 1;
            if (tid == 0 && k + 1 < nk) {
                const int sn = (gk + 1) & 1;
                mbar_arrive_expect_tx(&bar[sn], TILE_BYTES);
                bulk_copy_g2s(dbuf + sn * STAGE, spack + static_cast<size_t>(it.y + k + 1) * STAGE,
                              TILE_BYTES, &bar[sn]);
            }
            const bool timed_out = !mbar_wait_bounded(&bar[st], (gk >> 1) & 1);
            if (__syncthreads_or(timed_out)) {
                if (tid == 0)
                    atomicOr(p.err, DEV_ERR_TIMEOUT);
                mbar_wait_bounded(&bar[st], (gk >> 1) & 1, 100000000ull);
                if (k + 1 < nk)
                    mbar_wait_bounded(&bar[(gk + 1) & 1], ((gk + 1) >> 1) & 1, 100000000ull);
                return;
            }
            const double *sp = dbuf + st * STAGE;
#pragma unroll 2
            for (int j = 0; j < TS; ++j) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    pair_f64<KIND>(tx[r], ty[r], tz[r], sp, j, ax[r], ay[r], az[r]);
            }
            __syncthreads();
        }
        g += nk;

#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int loc = warp * 32 * R + r * 32 + lane;
            if (it.w < 0) {
                if (loc < tt.count) {
                    const long long t = p.perm ? p.perm[tt.begin + loc] : tt.begin + loc;
                    double ox = p.scale * ax[r], oy = p.scale * ay[r], oz = p.scale * az[r];
                    if (kind_laplace(KIND)) {
                        if (p.diag_sigma)
                            ox += p.diag * p.diag_sigma[t];
                        p.out[t] = ox;
                        continue;
                    }
                    if (p.diag_sigma) {
                        ox += p.diag * p.diag_sigma[t];
                        oy += p.diag * p.diag_sigma[p.nt + t];
                        oz += p.diag * p.diag_sigma[2 * p.nt + t];
                    }
                    p.out[t] = ox;
                    p.out[p.nt + t] = oy;
                    p.out[2 * p.nt + t] = oz;
                }
            } else {
                double *pp = p.partial + static_cast<size_t>(it.w) * 3 * TT + loc;
                pp[0] = ax[r];
                pp[TT] = ay[r];
                pp[2 * TT] = az[r];
            }
        }
    }
}

}  // namespace sbq

#include "pairsum_df.cuh"

namespace sbq {

// ---------------------------------------------------------------------------
// Launch table for one kind
// ---------------------------------------------------------------------------
template <int KIND>
struct KindLauncher {
    template <int R, int W, bool COMP>
    static cudaError_t f32(int grid, const PairsumParams &p, cudaStream_t s)
    {
        const size_t smem = pairsum_smem_bytes(COMP ? SBQ_FP32_COMP : SBQ_FP32);
        pairsum_f32_kernel<KIND, R, W, COMP><<<grid, W * 32, smem, s>>>(p);
        return cudaGetLastError();
    }
    template <int R, int W>
    static cudaError_t f64(int grid, const PairsumParams &p, cudaStream_t s)
    {
        const size_t smem = 2 * 9 * TS_F64 * sizeof(double);
        pairsum_f64_kernel<KIND, R, W><<<grid, W * 32, smem, s>>>(p);
        return cudaGetLastError();
    }
    template <int R, int W>
    static cudaError_t df(int grid, const PairsumParams &p, cudaStream_t s)
    {
        pairsum_df_kernel<KIND, R, W><<<grid, W * 32, pairsum_smem_bytes(SBQ_DF32), s>>>(p);
        return cudaGetLastError();
    }
    template <int R, int W>
    static int occdf()
    {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pairsum_df_kernel<KIND, R, W>, W * 32,
                                                      pairsum_smem_bytes(SBQ_DF32));
        return b;
    }
    template <int R, int W, bool COMP>
    static int occ32()
    {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pairsum_f32_kernel<KIND, R, W, COMP>, W * 32,
                                                      pairsum_smem_bytes(COMP ? SBQ_FP32_COMP
                                                                              : SBQ_FP32));
        return b;
    }
    template <int R, int W>
    static int occ64()
    {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pairsum_f64_kernel<KIND, R, W>, W * 32,
                                                      2 * 9 * TS_F64 * sizeof(double));
        return b;
    }

// Supported tile shapes.  FP32: (R, W) in {(1,4), (1,8), (2,4), (4,4), (8,4), (4,8), (4,2),
// (8,2)}; FP64: (1,4), (2,4); double-float: (1,4), (2,4), (4,4), (2,8).
#define SBQ_F32_SHAPES(X) X(1, 4) X(1, 8) X(2, 4) X(4, 4) X(8, 4) X(4, 8) X(4, 2) X(8, 2)
#define SBQ_F64_SHAPES(X) X(1, 4) X(2, 4)
#define SBQ_DF_SHAPES(X) X(1, 4) X(2, 4) X(4, 4) X(2, 8)

    static cudaError_t launch(int prec, int R, int W, int grid, const PairsumParams &p, cudaStream_t s)
    {
        if (prec == SBQ_FP64) {
#define X(r, w) \
    if (R == r && W == w) return f64<r, w>(grid, p, s);
            SBQ_F64_SHAPES(X)
#undef X
        } else if (prec == SBQ_DF32) {
#define X(r, w) \
    if (R == r && W == w) return df<r, w>(grid, p, s);
            SBQ_DF_SHAPES(X)
#undef X
        } else {
            const bool comp = (prec == SBQ_FP32_COMP);
#define X(r, w)                                      \
    if (R == r && W == w)                            \
        return comp ? f32<r, w, true>(grid, p, s) : f32<r, w, false>(grid, p, s);
            SBQ_F32_SHAPES(X)
#undef X
        }
        return cudaErrorInvalidValue;
    }
    static int occupancy(int prec, int R, int W)
    {
        if (prec == SBQ_FP64) {
#define X(r, w) \
    if (R == r && W == w) return occ64<r, w>();
            SBQ_F64_SHAPES(X)
#undef X
        } else if (prec == SBQ_DF32) {
#define X(r, w) \
    if (R == r && W == w) return occdf<r, w>();
            SBQ_DF_SHAPES(X)
#undef X
        } else {
            const bool comp = (prec == SBQ_FP32_COMP);
#define X(r, w) \
    if (R == r && W == w) return comp ? occ32<r, w, true>() : occ32<r, w, false>();
            SBQ_F32_SHAPES(X)
#undef X
        }
        return 0;
    }
};

}  // namespace sbq
