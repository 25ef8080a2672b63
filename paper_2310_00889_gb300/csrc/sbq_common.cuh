// Internal definitions shared by the CUDA translation units of libsbq.
// Not part of the public ABI (include/sbq.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

#include "../../include/sbq.h"

namespace sbq {

// Pair-sum kernel kinds: Stokes single layer, double layer, combined field
// (paper Eqs. stokes-sl, stokes-dl, stokes-bie-new) and the Laplace ones (Sec. 4.1: kernels
// G = 1/(4 pi |r|) and dG/dn_y, combined field of Eq. laplace-bie-rep-new).  Laplace kinds
// carry a scalar density in the first charge component and produce one output component.
enum Kind { KIND_SL = 0, KIND_DL = 1, KIND_CF = 2, KIND_LSL = 3, KIND_LDL = 4, KIND_LCF = 5 };
__host__ __device__ constexpr bool kind_laplace(int k) { return k >= KIND_LSL; }
__host__ __device__ constexpr bool kind_has_normals(int k)
{
    return k == KIND_DL || k == KIND_CF || k == KIND_LDL || k == KIND_LCF;
}

// Sources per shared-memory tile.
// FP32 tiles store every field as packed pairs (value of source 2m, value of source 2m+1)
// so that one 64-bit operand feeds the f32x2 instructions.  Fields, in order:
// x, y, z, qx, qy, qz, nx, ny, nz, lx, ly, lz (l: the part of the centred FP64 position
// lost when rounding it to FP32).  Two fields share a float4; six blocks of TS/2 float4
// make a tile: {x,y} {z,qx} {qy,qz} {nx,ny} {nz,lx} {ly,lz}.
// FP64 tiles hold 9 doubles per source {x, y, z, qx, qy, qz, nx, ny, nz}, each field a
// run of TS.
constexpr int TS_F32 = 256;
constexpr int F32_TILE_BLOCKS = 6;            // blocks of TS_F32 / 2 float4 per tile
constexpr int F32_TILE_F4 = F32_TILE_BLOCKS * (TS_F32 / 2);
enum F32Field { FX = 0, FY, FZ, FQX, FQY, FQZ, FNX, FNY, FNZ, FLX, FLY, FLZ };
// float index of field f of source j within a packed FP32 tile
__host__ __device__ constexpr int f32_slot(int f, int j)
{
    return ((f >> 1) * (TS_F32 / 2) + (j >> 1)) * 4 + (f & 1) * 2 + (j & 1);
}
constexpr int TS_F64 = 128;
// Double-float tiles: TS_DF sources, six float4 per source (layout in pairsum_df.cuh).
constexpr int TS_DF = 128;
constexpr int DF_TILE_F4 = 6 * TS_DF;
// Double-float path: pairs closer than this fraction of the sum of their tile radii are
// coincident.  Centring in double-float leaves a coincident pair a few 2^-48 of that sum
// apart; distinct nodes of any admissible discretisation are orders of magnitude farther.
constexpr double DF_COINCIDENT_REL = 1.0e-10;
// Rounding-error bound of one double-float pair term, relative to the term's envelope
// |q|_1 ri (2 + |n'|_1 ri) (which bounds every intermediate product, cancellations
// included): 2^-41, several times the sum of the ten or so double-float steps of
// 2^-46..2^-48 a term goes through, r included (formed to 2^-46 of |r| or better, see
// DF_EXACT_R).
constexpr double DF_TERM_REL = 4.547473508864641e-13;
// Tile pairs whose closest possible pair distance is below this fraction of (radii +
// centre distance) form r from three-part coordinates exactly; elsewhere the two-part
// form is within 2^-48 x 2 of |r| (each coordinate part within 2^-48 of the extent).
constexpr double DF_EXACT_R = 0.5;
// Compensated FP32: plain FP32 sums over runs of this many sources are merged into
// the (hi, lo) pair with TwoSum.  Each packed lane sums COMP_RUN / 2 terms in FP32 per run.
constexpr int COMP_RUN = 128;
// FP32 paths: pairs closer than this fraction of the sum of their two tile radii are
// taken as coincident (skipped).  The FP32 centring rounds a coincident pair to at most
// ~5 ulps of that sum (3e-7 of it), well below this threshold; distinct nodes of any
// admissible discretisation are far above it.
constexpr double COINCIDENT_REL = 4.0e-6;
// Position of padding sources in the last (ragged) tile of a segment.  Their weight
// and normal are zero, so every term they produce is an exact zero.
constexpr float PAD_POS_F32 = 1.0e15f;
constexpr double PAD_POS_F64 = 1.0e100;

// Device error word bits.
constexpr int DEV_ERR_TIMEOUT = 1;

// Geometry of one source or target tile.
struct __align__(16) TileInfo {
    double cx, cy, cz;   // FP64 centre (a member node); FP32 tiles store coordinates relative to it
    float rad;           // max |member - centre| (rounded up), for the self-pair test
    int count;           // valid members (<= tile size)
    long long begin;     // global index of the first member
    int seg;             // segment of the tile
    int slot_begin;      // target tiles: first partial slot, -1 when the tile has one chunk
    int slot_count;      // target tiles: number of chunk partials
    int pad_;
};
static_assert(sizeof(TileInfo) == 64, "TileInfo layout");

// Arguments of one pair-sum launch (all pointers are device pointers).
struct PairsumParams {
    const void *spack;          // packed source tiles
    const TileInfo *stiles;     // source tile table
    const float4 *tpack;        // FP32 paths: packed targets [ttile][TT] (x - c, y - c, z - c, 0)
    const float4 *tpack_lo;     // FP32 paths: parts of the centred targets lost to rounding
    const float4 *tpack_l2;     // double-float: third parts of the centred targets
    const TileInfo *ttiles;     // target tile table
    const double *trg;          // FP64 path: targets (SoA, stride nt)
    long long nt;               // global number of targets (stride of trg / out / diag_sigma)
    const int4 *items;          // work list {ttile, stile_begin, stile_end, slot (-1: direct)}
    int n_items;
    int *counter;               // work-claim counter, zeroed by the density pack kernel
    int *err;                   // device error word
    double *out;                // (3, nt) FP64 output
    double *partial;            // chunk partials: FP64 [slot][3][TT] (FP64 kernel) or
                                // float2 (hi, lo) [slot][3][TT] (FP32 kernels)
    const double *diag_sigma;   // nullable: out += diag * diag_sigma (same indexing as out)
    const int *perm;            // nullable: caller's index of each internal target (FP64
                                // kernel's direct output)
    int ncomp;                  // output components: 3 (Stokes) or 1 (Laplace)
    double diag;
    double scale;               // prefactor applied to the accumulated sum
    double kappa;               // combined field: 6 beta / alpha (folded into the packed normals)
    int TT;                     // targets per target tile
};

// ---------------------------------------------------------------------------
// Inline PTX: mbarrier + bulk async copy (TMA engine, non-tensor form)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bulk copy global -> shared that signals `bar` with its byte count on landing.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((i & 255u) == 255u && global_timer_ns() - t0 > limit_ns)
            return false;
    }
}

// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
void clear_error();
int cuda_status(cudaError_t e, const char *what);   // records the message, returns status

#define SBQ_CUDA(call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess)                                 \
            return ::sbq::cuda_status(e_, #call);              \
    } while (0)

#define SBQ_TRY(call)                                          \
    do {                                                       \
        int s_ = (call);                                       \
        if (s_ != SBQ_OK)                                      \
            return s_;                                         \
    } while (0)

struct DeviceProps {
    int sms = 0, cc_major = 0, cc_minor = 0;
};
const DeviceProps &device_props();
int *device_error_word();   // per-device error word (allocated once per device)
// noalloc.cu: bits of the allocation-free apply's error word on the current device, read
// and cleared (0 if that entry point never ran on the device).  Synchronous.
int noalloc_take_error(int *bits);

// Launchers implemented per kind (pairsum_{sl,dl,cf}.cu).  prec: sbq_prec.
// Return cudaErrorInvalidValue for an unsupported (R, W).
cudaError_t launch_pairsum(int kind, int prec, int R, int W, int grid, const PairsumParams &p,
                           cudaStream_t s);
// pairsum_laplace.cu
cudaError_t launch_pairsum_laplace(int kind, int prec, int R, int W, int grid,
                                   const PairsumParams &p, cudaStream_t s);
int occupancy_pairsum_laplace(int kind, int prec, int R, int W);
int pairsum_blocks_per_sm(int kind, int prec, int R, int W);
bool pairsum_shape_supported(int prec, int R, int W);
size_t pairsum_smem_bytes(int prec);

// pack.cu
// nscale multiplies the packed normals (the combined-field kernels read kappa * n).
cudaError_t launch_pack_src_geom(int prec, const double *src, const double *nrm, double nscale,
                                 long long ns, TileInfo *stiles, int n_stiles, void *spack,
                                 cudaStream_t s);
// perm (nullable): caller's index of each internal node; sigma is read through it (w and
// the tiles are in internal order).
cudaError_t launch_pack_src_q(int prec, const double *w, const double *sigma, long long ns,
                              const TileInfo *stiles, int n_stiles, void *spack, int *counter,
                              const int *perm, int scalar, cudaStream_t s);
// tpack_l2 (nullable): third parts; then tpack / tpack_lo / tpack_l2 hold x - c as
// h + m + l to about 2^-72 of |x - c|.
cudaError_t launch_pack_trg(const double *trg, long long nt, TileInfo *ttiles, int n_ttiles,
                            int TT, float4 *tpack, float4 *tpack_lo, float4 *tpack_l2,
                            cudaStream_t s);
// perm (nullable): out, diag_sigma and bound are indexed by the caller's index of each
// internal target.
cudaError_t launch_reduce_partials(const TileInfo *ttiles, int n_ttiles, int TT,
                                   const double *partial, long long nt, double *out,
                                   double scale, double diag, const double *diag_sigma,
                                   const int *perm, int ncomp, cudaStream_t s);
// FP32 partial sums ((hi, lo) float pairs) of every slot of a target tile -> FP64 output.
// comp: 0 plain FP32, 1 compensated, 2 double-float (float4 partials carrying each item's
// error bound; bound, when not null, receives |scale| x the sum of the items' bounds).
cudaError_t launch_reduce_partials_f32(const TileInfo *ttiles, int n_ttiles, int TT,
                                       const void *partial, long long nt, double *out,
                                       double scale, double diag, const double *diag_sigma,
                                       int comp, double *bound, const int *perm, int ncomp,
                                       cudaStream_t s);
cudaError_t launch_csr_apply(long long nrows, const int64_t *rowptr, const int64_t *col,
                             const double *val, const double *x, double *y, cudaStream_t s);

}  // namespace sbq
