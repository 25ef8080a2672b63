// Allocation-free variant of the single-layer apply (stokes_sl_apply_noalloc).
//
// Some callers cannot allocate GPU memory at the point where they need the sum: code
// running under a strict memory budget or a pre-reserved pool, real-time loops that
// must not hit the allocator's synchronisation, or hosts that forbid cudaMalloc /
// cudaFree (or torch's allocator) after start-up.  stokes_sl_apply takes its scratch
// (packed tiles, tile tables, work list, partial sums) from the stream-ordered pool on
// every call; this entry point instead uses one fixed array in device global memory
// that the library declares at file scope, so a call allocates nothing.
//
// The array is part of the library's device image: every GPU that loads the library
// holds NOALLOC_SCRATCH_BYTES of it until the process exits.  All calls on a device
// share it and it keeps the last call's contents, so each call rewrites everything it
// reads (tables, packed tiles, counters) before use, and two calls whose work overlaps
// on the GPU (different streams without ordering, or several host threads) race on it.
#include "engine.h"

#include <algorithm>
#include <mutex>

using namespace sbq;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
constexpr long long NOALLOC_MAX_POINTS = 131072;             // per side (sources, targets)
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device.
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch layout of one call (byte offsets from the start of the array).
struct Layout {
    size_t err, counter, stiles, ttiles, items, spack, tpack, tpack_lo, partial, end;
};

Layout make_layout(int prec, int n_st, int n_tt, int TT, int n_items, long long n_slots)
{
    Layout L{};
    size_t o = 0;
    L.err = o;
    o = align256(o + sizeof(int));
    L.counter = o;
    o = align256(o + sizeof(int));
    L.stiles = o;
    o = align256(o + size_t(n_st) * sizeof(TileInfo));
    L.ttiles = o;
    o = align256(o + size_t(n_tt) * sizeof(TileInfo));
    L.items = o;
    o = align256(o + size_t(n_items) * sizeof(int4));
    L.spack = o;
    const size_t per_tile = (prec == SBQ_FP64) ? 9 * TS_F64 * sizeof(double)
                                               : F32_TILE_F4 * sizeof(float4);
    o = align256(o + size_t(n_st) * per_tile);
    L.tpack = o;
    if (prec != SBQ_FP64)
        o = align256(o + size_t(n_tt) * TT * sizeof(float4));
    L.tpack_lo = o;
    if (prec == SBQ_FP32_COMP)
        o = align256(o + size_t(n_tt) * TT * sizeof(float4));
    L.partial = o;
    o = align256(o + size_t(n_slots) * 3 * TT * sizeof(double));
    L.end = o;
    return L;
}

// Tile tables and work list of a single segment, written on the device so that the call
// needs no host staging buffer either; zeroes the claim counter.  The error word at the
// start of the array is left alone: a bounded wait that expired in an earlier call stays
// recorded until sbq_check_device() reads and clears it.
__global__ void noalloc_tables(unsigned char *base, Layout L, long long ns, long long nt, int TS,
                               int TT, int n_st, int n_tt, int n_chunks, int C, int slots)
{
    TileInfo *stiles = reinterpret_cast<TileInfo *>(base + L.stiles);
    TileInfo *ttiles = reinterpret_cast<TileInfo *>(base + L.ttiles);
    int4 *items = reinterpret_cast<int4 *>(base + L.items);
    const long long tid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    if (tid == 0)
        *reinterpret_cast<int *>(base + L.counter) = 0;
    for (long long k = tid; k < n_st; k += stride) {
        TileInfo ti{};
        ti.begin = k * TS;
        ti.count = static_cast<int>(min(static_cast<long long>(TS), ns - ti.begin));
        ti.seg = 0;
        ti.slot_begin = -1;
        ti.slot_count = 0;
        stiles[k] = ti;
    }
    for (long long k = tid; k < n_tt; k += stride) {
        TileInfo ti{};
        ti.begin = k * TT;
        ti.count = static_cast<int>(min(static_cast<long long>(TT), nt - ti.begin));
        ti.seg = 0;
        ti.slot_begin = slots ? static_cast<int>(k * n_chunks) : -1;
        ti.slot_count = slots ? n_chunks : 0;
        ttiles[k] = ti;
    }
    const long long n_items = static_cast<long long>(n_tt) * n_chunks;
    for (long long i = tid; i < n_items; i += stride) {
        const int k = static_cast<int>(i / n_chunks), c = static_cast<int>(i % n_chunks);
        const int a = c * C, b = min(n_st, a + C);
        items[i] = make_int4(k, a, b, slots ? k * n_chunks + c : -1);
    }
}

}  // namespace

namespace sbq {

// Error word of the allocation-free apply on the current device (offset 0 of its array):
// returns the bits set since the last call and clears them.  0 when the entry point has
// not been used on this device (the array was never addressed: nothing to read).
int noalloc_take_error(int *bits)
{
    *bits = 0;
    int dev = 0;
    SBQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return SBQ_OK;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        p = g_noalloc_ptr[dev];
    }
    if (!p)
        return SBQ_OK;
    int h = 0;
    SBQ_CUDA(cudaMemcpy(&h, p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0)
        SBQ_CUDA(cudaMemset(p, 0, sizeof(int)));
    *bits = h;
    return SBQ_OK;
}

}  // namespace sbq

extern "C" SBQ_API int stokes_sl_apply_noalloc(int64_t ns, const double *src, const double *w,
                                               const double *sigma, int64_t nt,
                                               const double *trg, double *u, int prec,
                                               void *stream)
{
    clear_error();
    if (ns < 0 || nt < 0) {
        set_error("negative size");
        return SBQ_EINVAL;
    }
    if (prec != SBQ_FP64 && prec != SBQ_FP32 && prec != SBQ_FP32_COMP) {
        set_error("unknown precision");
        return SBQ_EINVAL;
    }
    if (ns > NOALLOC_MAX_POINTS || nt > NOALLOC_MAX_POINTS) {
        set_error("stokes_sl_apply_noalloc: ns and nt must each be at most 131072 (the fixed "
                  "32 MiB scratch); use stokes_sl_apply for larger problems");
        return SBQ_EINVAL;
    }
    if (nt > 0 && (!trg || !u)) {
        set_error("null target or output pointer");
        return SBQ_EINVAL;
    }
    if (ns > 0 && nt > 0 && (!src || !w || !sigma)) {
        set_error("null source, weight or density pointer");
        return SBQ_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nt == 0)
        return SBQ_OK;
    if (ns == 0) {
        SBQ_CUDA(cudaMemsetAsync(u, 0, 3 * static_cast<size_t>(nt) * sizeof(double), s));
        return SBQ_OK;
    }

    // Set-up, once per device with that device current: the device address of the array.
    int dev = 0;
    SBQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device index out of range for the no-alloc scratch table");
        return SBQ_EINVAL;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                   "cudaGetSymbolAddress(no-alloc scratch)");
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }

    // Fixed tile shape (targets per CTA = 256) and a chunking that fits the scratch.
    const int R = 2, W = 4, TT = 32 * W * R;
    const int TS = (prec == SBQ_FP64) ? TS_F64 : TS_F32;
    const int n_st = static_cast<int>((ns + TS - 1) / TS);
    const int n_tt = static_cast<int>((nt + TT - 1) / TT);
    int sms = 0;
    SBQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int occ = pairsum_blocks_per_sm(KIND_SL, prec, R, W);
    if (occ < 1)
        occ = 1;
    const long long slots = static_cast<long long>(sms > 0 ? sms : 1) * occ;
    // about 4 work items per resident CTA, fewer chunks if the partial sums do not fit
    int n_chunks = static_cast<int>(std::min<long long>(
        n_st, std::max<long long>(1, (4 * slots + n_tt - 1) / n_tt)));
    Layout L{};
    for (;;) {
        const int C = (n_st + n_chunks - 1) / n_chunks;
        n_chunks = (n_st + C - 1) / C;
        L = make_layout(prec, n_st, n_tt, TT, n_tt * n_chunks,
                        (n_chunks > 1 || prec != SBQ_FP64) ? static_cast<long long>(n_tt) * n_chunks
                                                           : 0);
        if (L.end <= NOALLOC_SCRATCH_BYTES || n_chunks == 1)
            break;
        n_chunks = std::max(1, n_chunks / 2);
    }
    if (L.end > NOALLOC_SCRATCH_BYTES) {
        set_error("stokes_sl_apply_noalloc: problem does not fit the 32 MiB scratch");
        return SBQ_EINVAL;
    }
    const int C = (n_st + n_chunks - 1) / n_chunks;
    const int n_items = n_tt * n_chunks;
    unsigned char *b8 = static_cast<unsigned char *>(base);

    const int tb = 256;
    const int tg = static_cast<int>(std::min<long long>(
        1024, std::max<long long>(1, (std::max<long long>(n_items, std::max(n_st, n_tt)) + tb - 1) / tb)));
    // FP32 kernels always write partial slots; the FP64 kernel only with several chunks
    const int use_slots = (n_chunks > 1 || prec != SBQ_FP64) ? 1 : 0;
    noalloc_tables<<<tg, tb, 0, s>>>(b8, L, ns, nt, TS, TT, n_st, n_tt, n_chunks, C, use_slots);
    SBQ_CUDA(cudaGetLastError());
    TileInfo *stiles = reinterpret_cast<TileInfo *>(b8 + L.stiles);
    TileInfo *ttiles = reinterpret_cast<TileInfo *>(b8 + L.ttiles);
    SBQ_CUDA(launch_pack_src_geom(prec == SBQ_FP64 ? SBQ_FP64 : SBQ_FP32, src, nullptr, 1.0, ns, stiles,
                                  n_st, b8 + L.spack, s));
    int *counter = reinterpret_cast<int *>(b8 + L.counter);
    SBQ_CUDA(launch_pack_src_q(prec == SBQ_FP64 ? SBQ_FP64 : SBQ_FP32, w, sigma, ns, stiles, n_st,
                               b8 + L.spack, counter, nullptr, 0, s));
    if (prec != SBQ_FP64)
        SBQ_CUDA(launch_pack_trg(trg, nt, ttiles, n_tt, TT, reinterpret_cast<float4 *>(b8 + L.tpack),
                                 prec == SBQ_FP32_COMP ? reinterpret_cast<float4 *>(b8 + L.tpack_lo)
                                                       : nullptr,
                                 nullptr, s));
    int kind;
    double scale, kappa;
    kind_and_scale(1.0, 0.0, &kind, &scale, &kappa);
    PairsumParams p{};
    p.spack = b8 + L.spack;
    p.stiles = stiles;
    p.tpack = reinterpret_cast<const float4 *>(b8 + L.tpack);
    p.tpack_lo = reinterpret_cast<const float4 *>(b8 + L.tpack_lo);
    p.ttiles = ttiles;
    p.trg = trg;
    p.nt = nt;
    p.items = reinterpret_cast<const int4 *>(b8 + L.items);
    p.n_items = n_items;
    p.counter = counter;
    p.err = reinterpret_cast<int *>(b8 + L.err);
    p.out = u;
    p.partial = reinterpret_cast<double *>(b8 + L.partial);
    p.diag_sigma = nullptr;
    p.diag = 0.0;
    p.scale = scale;
    p.kappa = kappa;
    p.TT = TT;
    const int grid = static_cast<int>(std::min<long long>(n_items, slots));
    SBQ_CUDA(launch_pairsum(kind, prec, R, W, grid, p, s));
    if (prec != SBQ_FP64)
        SBQ_CUDA(launch_reduce_partials_f32(ttiles, n_tt, TT, p.partial, nt, u, scale, 0.0, nullptr,
                                            prec == SBQ_FP32_COMP ? 1 : 0, nullptr, nullptr, 3, s));
    else if (n_chunks > 1)
        SBQ_CUDA(launch_reduce_partials(ttiles, n_tt, TT, p.partial, nt, u, scale, 0.0, nullptr,
                                        nullptr, 3, s));
    return SBQ_OK;
}
