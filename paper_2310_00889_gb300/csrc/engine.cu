// Host-side engine: tile tables, work lists, pair-sum launches, operator matvec and the
// tile-shape autotuner.
#include "engine.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>

namespace sbq {

// ---------------------------------------------------------------------------
// Errors, device properties
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
const char *last_error_cstr() { return g_last_error.c_str(); }

int cuda_status(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return (e == cudaErrorMemoryAllocation) ? SBQ_ENOMEM : SBQ_ECUDA;
}

static std::mutex g_dev_mu;
static std::map<int, DeviceProps> g_props;
static std::map<int, int *> g_err_words;

const DeviceProps &device_props()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_props.find(dev);
    if (it == g_props.end()) {
        DeviceProps p;
        cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&p.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&p.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (p.sms <= 0)
            p.sms = 1;
        it = g_props.emplace(dev, p).first;
    }
    return it->second;
}

int *device_error_word()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_err_words.find(dev);
    if (it != g_err_words.end())
        return it->second;
    int *p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess)
        return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(p);
        return nullptr;
    }
    g_err_words[dev] = p;
    return p;
}

static thread_local bool g_async_on = false;
static thread_local cudaStream_t g_async_stream = nullptr;

AsyncAllocScope::AsyncAllocScope(cudaStream_t s) : prev(g_async_stream), prev_on(g_async_on)
{
    g_async_stream = s;
    g_async_on = true;
}

AsyncAllocScope::~AsyncAllocScope()
{
    g_async_stream = prev;
    g_async_on = prev_on;
}

int DevBuf::alloc(size_t n)
{
    release();
    if (n == 0)
        n = 16;
    cudaError_t e;
    if (g_async_on) {
        e = cudaMallocAsync(&p, n, g_async_stream);
        async = true;
        stream = g_async_stream;
    } else {
        e = cudaMalloc(&p, n);
        async = false;
        stream = nullptr;
    }
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_status(e, async ? "cudaMallocAsync" : "cudaMalloc");
    }
    bytes = n;
    return SBQ_OK;
}

void DevBuf::release()
{
    if (p) {
        if (async)
            cudaFreeAsync(p, stream);
        else
            cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    async = false;
    stream = nullptr;
}

Op::~Op()
{
    if (gm)
        gmres_destroy(gm);
    tree_op_free(this);
}

// ---------------------------------------------------------------------------
// Prefactors
// ---------------------------------------------------------------------------
static const double kPi = 3.14159265358979323846264338327950288;

void laplace_kind_and_scale(double alpha, double beta, int *kind, double *scale, double *kappa)
{
    // alpha S + beta D with S = 1/(4 pi |r|), D = (r.n_y)/(4 pi |r|^3).
    *kappa = 0.0;
    if (beta == 0.0) {
        *kind = KIND_LSL;
        *scale = alpha / (4.0 * kPi);
    } else if (alpha == 0.0) {
        *kind = KIND_LDL;
        *scale = beta / (4.0 * kPi);
    } else {
        *kind = KIND_LCF;
        *scale = alpha / (4.0 * kPi);
        *kappa = beta / alpha;
    }
}

void kind_and_scale(double alpha, double beta, int *kind, double *scale, double *kappa)
{
    // alpha S + beta D with S = (1/8pi)(...), D = (3/4pi)(...).
    *kappa = 0.0;
    if (beta == 0.0) {
        *kind = KIND_SL;
        *scale = alpha / (8.0 * kPi);
    } else if (alpha == 0.0) {
        *kind = KIND_DL;
        *scale = 3.0 * beta / (4.0 * kPi);
    } else {
        *kind = KIND_CF;
        *scale = alpha / (8.0 * kPi);
        *kappa = 6.0 * beta / alpha;
    }
}

sbq_tune default_tune(int prec, long long nt)
{
    sbq_tune t{};
    if (prec == SBQ_FP64 || prec == SBQ_DF32) {
        t.r = 2;
        t.warps = 4;
    } else {
        t.r = (nt >= 65536) ? 4 : 2;
        t.warps = 4;
    }
    t.chunk_tiles = 0;
    return t;
}

// ---------------------------------------------------------------------------
// Tile tables and work lists
// ---------------------------------------------------------------------------
int build_src_pack(SrcPack &sp, int layout, const std::vector<int64_t> &src_off, const double *src,
                   const double *nrm, double nscale, long long ns, cudaStream_t s)
{
    sp.layout = layout;
    sp.TS = (layout == SBQ_FP64) ? TS_F64 : (layout == SBQ_DF32) ? TS_DF : TS_F32;
    const int nseg = static_cast<int>(src_off.size()) - 1;
    std::vector<TileInfo> h;
    sp.seg_tile_begin.assign(nseg, 0);
    sp.seg_tile_count.assign(nseg, 0);
    for (int i = 0; i < nseg; ++i) {
        const long long a = src_off[i], b = src_off[i + 1];
        sp.seg_tile_begin[i] = static_cast<int>(h.size());
        for (long long t = a; t < b; t += sp.TS) {
            TileInfo ti{};
            ti.begin = t;
            ti.count = static_cast<int>(std::min<long long>(sp.TS, b - t));
            ti.seg = i;
            ti.slot_begin = -1;
            h.push_back(ti);
        }
        sp.seg_tile_count[i] = static_cast<int>(h.size()) - sp.seg_tile_begin[i];
    }
    sp.n_stiles = static_cast<int>(h.size());
    if (h.size() > static_cast<size_t>(INT32_MAX / 2)) {
        set_error("too many source tiles");
        return SBQ_EINVAL;
    }
    SBQ_TRY(sp.stiles.alloc(h.size() * sizeof(TileInfo)));
    const size_t per_tile = (layout == SBQ_FP64)   ? 9 * TS_F64 * sizeof(double)
                            : (layout == SBQ_DF32) ? DF_TILE_F4 * sizeof(float4)
                                                   : F32_TILE_F4 * sizeof(float4);
    SBQ_TRY(sp.spack.alloc(h.size() * per_tile));
    if (!h.empty()) {
        SBQ_CUDA(cudaMemcpyAsync(sp.stiles.p, h.data(), h.size() * sizeof(TileInfo),
                                 cudaMemcpyHostToDevice, s));
        SBQ_CUDA(launch_pack_src_geom(layout, src, nrm, nscale, ns, sp.stiles.as<TileInfo>(), sp.n_stiles,
                                      sp.spack.p, s));
    }
    return SBQ_OK;
}

static long long persistent_slots(int kind, int prec, const sbq_tune &t)
{
    int occ = pairsum_blocks_per_sm(kind, prec, t.r, t.warps);
    if (occ <= 0)
        occ = 1;
    return static_cast<long long>(device_props().sms) * occ;
}

// Source tiles per work item: about 16 items per resident CTA over the whole batch.
int auto_chunk_tiles(int kind, int prec, const sbq_tune &t, const SrcPack &sp,
                     const std::vector<int64_t> &trg_off)
{
    const int TT = 32 * t.warps * t.r;
    const int nseg = static_cast<int>(trg_off.size()) - 1;
    double total_tp = 0.0;
    for (int i = 0; i < nseg; ++i) {
        const long long nti = trg_off[i + 1] - trg_off[i];
        total_tp += static_cast<double>((nti + TT - 1) / TT) * sp.seg_tile_count[i];
    }
    const double want_items = 16.0 * static_cast<double>(persistent_slots(kind, prec, t));
    long long C = std::llround(total_tp / want_items);
    return static_cast<int>(std::max<long long>(1, std::min<long long>(C, 1 << 20)));
}

int build_trg_set(TrgSet &ts, int kind, int prec, const sbq_tune &tune, const SrcPack &sp,
                  const std::vector<int64_t> &trg_off, const double *trg, long long nt,
                  const std::vector<int64_t> &src_off, cudaStream_t s)
{
    if (!pairsum_shape_supported(prec, tune.r, tune.warps)) {
        set_error("unsupported tile shape r=" + std::to_string(tune.r) +
                  " warps=" + std::to_string(tune.warps));
        return SBQ_EINVAL;
    }
    ts.tune = tune;
    ts.TT = 32 * tune.warps * tune.r;
    const int TT = ts.TT;
    const int nseg = static_cast<int>(trg_off.size()) - 1;
    const long long slots = persistent_slots(kind, prec, tune);

    std::vector<int> seg_ntt(nseg);
    ts.pairs = 0.0;
    for (int i = 0; i < nseg; ++i) {
        const long long nti = trg_off[i + 1] - trg_off[i];
        const long long nsi = src_off[i + 1] - src_off[i];
        seg_ntt[i] = static_cast<int>((nti + TT - 1) / TT);
        ts.pairs += static_cast<double>(nti) * static_cast<double>(nsi);
        if (nti > 0 && nsi == 0) {
            set_error("segment " + std::to_string(i) + " has targets but no sources");
            return SBQ_EINVAL;
        }
    }
    int C = tune.chunk_tiles;
    if (C <= 0)
        C = auto_chunk_tiles(kind, prec, tune, sp, trg_off);
    ts.tune.chunk_tiles = C;

    std::vector<TileInfo> ht;
    struct Item {
        int4 v;
        int cost;
        double pairs;
    };
    std::vector<Item> items;
    int slot = 0;
    for (int i = 0; i < nseg; ++i) {
        const int sb = sp.seg_tile_begin[i], sn = sp.seg_tile_count[i];
        const int ci = std::max(1, std::min(C, sn));
        const int nchunk = (sn + ci - 1) / ci;
        // FP32 kernels always write partial slots (their FP64 epilogue is the reduction)
        const bool slots = nchunk > 1 || prec != SBQ_FP64;
        for (int k = 0; k < seg_ntt[i]; ++k) {
            TileInfo ti{};
            ti.begin = trg_off[i] + static_cast<long long>(k) * TT;
            ti.count = static_cast<int>(std::min<long long>(TT, trg_off[i + 1] - ti.begin));
            ti.seg = i;
            const int tidx = static_cast<int>(ht.size());
            if (slots) {
                ti.slot_begin = slot;
                ti.slot_count = nchunk;
            } else {
                ti.slot_begin = -1;
                ti.slot_count = 0;
            }
            for (int c = 0; c < nchunk; ++c) {
                const int a = sb + c * ci, b = std::min(sb + sn, a + ci);
                Item it;
                it.v = make_int4(tidx, a, b, slots ? slot + c : -1);
                it.cost = b - a;
                const long long src_a = src_off[i] + static_cast<long long>(a - sb) * sp.TS;
                const long long src_b = std::min<long long>(
                    src_off[i + 1], src_off[i] + static_cast<long long>(b - sb) * sp.TS);
                it.pairs = static_cast<double>(ti.count) * static_cast<double>(src_b - src_a);
                items.push_back(it);
            }
            if (slots)
                slot += nchunk;
            ht.push_back(ti);
        }
    }
    // Longest items first (list scheduling of the persistent grid).
    std::stable_sort(items.begin(), items.end(),
                     [](const Item &x, const Item &y) { return x.cost > y.cost; });
    std::vector<int4> hv(items.size());
    ts.item_pairs.resize(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        hv[i] = items[i].v;
        ts.item_pairs[i] = items[i].pairs;
    }

    ts.n_ttiles = static_cast<int>(ht.size());
    ts.n_items = static_cast<int>(hv.size());
    ts.needs_reduce = slot > 0;
    ts.grid = static_cast<int>(std::min<long long>(std::max(ts.n_items, 1), slots));
    SBQ_TRY(ts.ttiles.alloc(ht.size() * sizeof(TileInfo)));
    SBQ_TRY(ts.items.alloc(hv.size() * sizeof(int4)));
    // FP64: one double per entry; FP32: (hi, lo) float2; double-float: (hi, lo, |.|, -) float4
    const size_t pbytes = (prec == SBQ_DF32) ? sizeof(float4) : sizeof(double);
    SBQ_TRY(ts.partial.alloc(static_cast<size_t>(slot) * 3 * TT * pbytes));
    SBQ_TRY(ts.counter.alloc(sizeof(int)));
    if (prec != SBQ_FP64)
        SBQ_TRY(ts.tpack.alloc(ht.size() * static_cast<size_t>(TT) * sizeof(float4)));
    else
        ts.tpack.release();
    if (prec == SBQ_FP32_COMP || prec == SBQ_DF32)
        SBQ_TRY(ts.tpack_lo.alloc(ht.size() * static_cast<size_t>(TT) * sizeof(float4)));
    else
        ts.tpack_lo.release();
    if (prec == SBQ_DF32)
        SBQ_TRY(ts.tpack_l2.alloc(ht.size() * static_cast<size_t>(TT) * sizeof(float4)));
    else
        ts.tpack_l2.release();
    if (!ht.empty()) {
        SBQ_CUDA(cudaMemcpyAsync(ts.ttiles.p, ht.data(), ht.size() * sizeof(TileInfo),
                                 cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(ts.items.p, hv.data(), hv.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s));
    }
    SBQ_CUDA(cudaMemsetAsync(ts.counter.p, 0, sizeof(int), s));
    if (prec != SBQ_FP64 && ts.n_ttiles > 0)
        SBQ_CUDA(launch_pack_trg(trg, nt, ts.ttiles.as<TileInfo>(), ts.n_ttiles, TT,
                                 ts.tpack.as<float4>(), ts.tpack_lo.as<float4>(),
                                 ts.tpack_l2.as<float4>(), s));
    return SBQ_OK;
}

PairsumTiming *&pairsum_timing()
{
    static thread_local PairsumTiming *t = nullptr;
    return t;
}

int run_pairsum(int kind, int prec, const SrcPack &sp, const TrgSet &ts, const double *w,
                const double *sigma, long long ns, const double *trg, long long nt, double *out,
                double scale, double kappa, double diag, const double *diag_sigma, cudaStream_t s,
                double *bound, const int *perm)
{
    if (ts.n_items == 0)
        return SBQ_OK;
    int *err = device_error_word();
    if (!err) {
        set_error("cannot allocate the device error word");
        return SBQ_ENOMEM;
    }
    const int ncomp = kind_laplace(kind) ? 1 : 3;
    SBQ_CUDA(launch_pack_src_q(prec, w, sigma, ns, sp.stiles.as<TileInfo>(), sp.n_stiles, sp.spack.p,
                               ts.counter.as<int>(), perm, ncomp == 1, s));
    PairsumParams p{};
    p.spack = sp.spack.p;
    p.stiles = sp.stiles.as<TileInfo>();
    p.tpack = ts.tpack.as<float4>();
    p.tpack_lo = ts.tpack_lo.as<float4>();
    p.tpack_l2 = ts.tpack_l2.as<float4>();
    p.ttiles = ts.ttiles.as<TileInfo>();
    p.trg = trg;
    p.nt = nt;
    p.items = ts.items.as<int4>();
    p.n_items = ts.n_items;
    p.counter = ts.counter.as<int>();
    p.err = err;
    p.out = out;
    p.partial = ts.partial.as<double>();
    p.diag_sigma = diag_sigma;
    p.perm = perm;
    p.ncomp = ncomp;
    p.diag = diag;
    p.scale = scale;
    p.kappa = kappa;
    p.TT = ts.TT;
    PairsumTiming *pt = pairsum_timing();
    if (pt)
        SBQ_CUDA(cudaEventRecord(pt->before, s));
    SBQ_CUDA(launch_pairsum(kind, prec, ts.tune.r, ts.tune.warps, ts.grid, p, s));
    if (pt)
        SBQ_CUDA(cudaEventRecord(pt->after, s));
    if (prec != SBQ_FP64)
        SBQ_CUDA(launch_reduce_partials_f32(ts.ttiles.as<TileInfo>(), ts.n_ttiles, ts.TT,
                                            ts.partial.p, nt, out, scale, diag, diag_sigma,
                                            prec == SBQ_FP32_COMP ? 1 : (prec == SBQ_DF32 ? 2 : 0),
                                            prec == SBQ_DF32 ? bound : nullptr, perm, ncomp, s));
    else if (ts.needs_reduce)
        SBQ_CUDA(launch_reduce_partials(ts.ttiles.as<TileInfo>(), ts.n_ttiles, ts.TT,
                                        ts.partial.as<double>(), nt, out, scale, diag, diag_sigma,
                                        perm, ncomp, s));
    return SBQ_OK;
}

// ---------------------------------------------------------------------------
// Operator
// ---------------------------------------------------------------------------
static const SrcPack &op_srcpack(const Op *op, int prec)
{
    return prec == SBQ_FP64 ? op->sp64 : (prec == SBQ_DF32 ? op->spdf : op->sp32);
}

int op_kernels_per_matvec(const Op *op, int prec)
{
    const TrgSet *ts = op->ts[prec].get();
    int k = 0;
    if (ts && ts->n_items > 0)
        k += 2 + ((ts->needs_reduce || prec != SBQ_FP64) ? 1 : 0);
    if (op->nnz > 0)
        k += 1;
    if (op->mob)
        k += 4;   // moments, rigid motions, sigma - L sigma, + L sigma
    return k;
}

static int op_kind(const Op *op, int *kind, double *scale, double *kappa)
{
    if (op->laplace)
        laplace_kind_and_scale(op->eta, 1.0, kind, scale, kappa);
    else
        kind_and_scale(op->eta, 1.0, kind, scale, kappa);
    return SBQ_OK;
}

// Autotune cache shared by all operators of the process.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, long long, long long, int>, sbq_tune> g_tune_cache;

static std::tuple<int, int, int, long long, long long, int> tune_key(const Op *op, int kind,
                                                                      int prec)
{
    long long maxseg = 0;
    for (int i = 0; i < op->plan.nseg; ++i)
        maxseg = std::max<long long>(maxseg, op->plan.src_off[i + 1] - op->plan.src_off[i]);
    return std::make_tuple(kind, prec, op->plan.nseg, static_cast<long long>(op->n), maxseg,
                           device_props().sms);
}

// Kernel time of the pair sums over the first `items` work items of ts (the longest ones:
// the list is sorted by cost), from events recorded around the pair-sum launch; the pack
// and reduction kernels run as in an apply.  Returns pair interactions per millisecond.
static int time_prefix(int kind, int prec, const SrcPack &sp, TrgSet &ts, const Op *op,
                       const double *zs, double *zo, double scale, double kappa, int items,
                       cudaStream_t s, double *rate, float *kernel_ms)
{
    const int saved = ts.n_items;
    items = std::max(1, std::min(items, saved));
    double pairs = 0.0;
    for (int i = 0; i < items; ++i)
        pairs += ts.item_pairs[i];
    PairsumTiming pt;
    SBQ_CUDA(cudaEventCreate(&pt.before));
    cudaError_t ce = cudaEventCreate(&pt.after);
    if (ce != cudaSuccess) {
        cudaEventDestroy(pt.before);
        return cuda_status(ce, "autotune");
    }
    // warm-up over one item: the first launch of a kernel loads its module
    ts.n_items = 1;
    int st = run_pairsum(kind, prec, sp, ts, op->w.as<double>(), zs, op->n, op->src.as<double>(),
                         op->n, zo, scale, kappa, 0.0, nullptr, s);
    PairsumTiming *prev = pairsum_timing();
    pairsum_timing() = &pt;
    ts.n_items = items;
    if (st == SBQ_OK)
        st = run_pairsum(kind, prec, sp, ts, op->w.as<double>(), zs, op->n, op->src.as<double>(),
                         op->n, zo, scale, kappa, 0.0, nullptr, s);
    ts.n_items = saved;
    pairsum_timing() = prev;
    float ms = 0.0f;
    if (st == SBQ_OK) {
        ce = cudaEventSynchronize(pt.after);
        if (ce == cudaSuccess)
            ce = cudaEventElapsedTime(&ms, pt.before, pt.after);
        if (ce != cudaSuccess)
            st = cuda_status(ce, "autotune");
    }
    cudaEventDestroy(pt.before);
    cudaEventDestroy(pt.after);
    *kernel_ms = ms;
    *rate = (ms > 0.0f) ? pairs / ms : 0.0;
    return st;
}

// Tile-shape autotuner.  Small problems: every candidate (shape, chunking) is timed on
// whole applies (pack, pair sums, reduction), which includes the tail of the persistent
// grid.  Large problems (an apply of the first candidate estimated above 20 ms): each
// shape, at its default chunking (where the tail is a small part of the apply), is timed
// on two waves of its longest work items (two items per resident CTA), whose cost is
// representative of the whole list, best of two runs, and the candidates are compared by
// pair interactions per millisecond.  If one wave of the first candidate already takes
// longer than 250 ms (FP64 at a million nodes), it is kept untimed.
static int autotune_op(Op *op, int prec, cudaStream_t s)
{
    int kind;
    double scale, kappa;
    op_kind(op, &kind, &scale, &kappa);
    const SrcPack &sp = op_srcpack(op, prec);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(op, kind, prec));
        if (it != g_tune_cache.end()) {
            auto ts = std::make_unique<TrgSet>();
            SBQ_TRY(build_trg_set(*ts, kind, prec, it->second, sp, op->plan.src_off,
                                  op->src.as<double>(), op->n, op->plan.src_off, s));
            op->ts[prec] = std::move(ts);
            op->tuned[prec] = true;
            return SBQ_OK;
        }
    }
    std::vector<sbq_tune> shapes;
    if (prec == SBQ_FP64) {
        shapes = {{2, 4, 0}, {1, 4, 0}};
    } else if (prec == SBQ_DF32) {
        shapes = {{2, 4, 0}, {1, 4, 0}, {4, 4, 0}, {2, 8, 0}};
    } else {
        shapes = {{2, 4, 0}, {4, 2, 0}, {4, 4, 0}, {1, 4, 0}, {1, 8, 0}, {8, 2, 0}, {8, 4, 0},
                  {4, 8, 0}};
    }
    DevBuf zs, zo;
    SBQ_TRY(zs.alloc(3 * static_cast<size_t>(op->n) * sizeof(double)));
    SBQ_TRY(zo.alloc(3 * static_cast<size_t>(op->n) * sizeof(double)));
    SBQ_CUDA(cudaMemsetAsync(zs.p, 0, zs.bytes, s));
    cudaEvent_t e0, e1;
    SBQ_CUDA(cudaEventCreate(&e0));
    SBQ_CUDA(cudaEventCreate(&e1));
    auto done = [&](int st) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    };
    double best_rate = -1.0;       // pair interactions per ms (higher is better)
    std::unique_ptr<TrgSet> best;
    double budget_ms = 0.0;
    int mode = 0;                  // 0: undecided, 1: whole applies, 2: two-wave prefixes
    for (size_t si = 0; si < shapes.size() && budget_ms < 4000.0; ++si) {
        const int c0 = auto_chunk_tiles(kind, prec, shapes[si], sp, op->plan.src_off);
        std::vector<int> cands = {c0};
        if (mode != 2) {
            if (c0 > 1)
                cands.push_back(std::max(1, c0 / 2));
            cands.push_back(2 * c0);
        }
        for (int C : cands) {
            sbq_tune t = shapes[si];
            t.chunk_tiles = C;
            auto ts = std::make_unique<TrgSet>();
            int st = build_trg_set(*ts, kind, prec, t, sp, op->plan.src_off, op->src.as<double>(),
                                   op->n, op->plan.src_off, s);
            if (st != SBQ_OK)
                return done(st);
            if (ts->n_items == 0) {   // nothing to time
                best = std::move(ts);
                budget_ms = 1e30;
                break;
            }
            double rate = 0.0;
            if (mode != 1) {
                float kms = 0.0f;
                if (mode == 0) {
                    // one wave decides how to time the candidates
                    st = time_prefix(kind, prec, sp, *ts, op, zs.as<double>(), zo.as<double>(),
                                     scale, kappa, ts->grid, s, &rate, &kms);
                    if (st != SBQ_OK)
                        return done(st);
                    budget_ms += kms;
                    const double est_full_ms = rate > 0.0 ? ts->pairs / rate : 0.0;
                    if (kms > 250.0f) {   // too long to tune: keep the first candidate
                        best = std::move(ts);
                        budget_ms = 1e30;
                        break;
                    }
                    mode = (est_full_ms > 20.0 && ts->n_items > 4 * ts->grid) ? 2 : 1;
                }
                if (mode == 2) {
                    // the measurement: two waves, best of two runs
                    rate = 0.0;
                    for (int rep = 0; rep < 2; ++rep) {
                        double r2 = 0.0;
                        st = time_prefix(kind, prec, sp, *ts, op, zs.as<double>(), zo.as<double>(),
                                         scale, kappa, 2 * ts->grid, s, &r2, &kms);
                        if (st != SBQ_OK)
                            return done(st);
                        budget_ms += kms;
                        rate = std::max(rate, r2);
                    }
                }
            }
            if (mode == 1) {
                // one warm-up apply, then three timed ones
                const int reps = 3;
                for (int r = 0; r <= reps && st == SBQ_OK; ++r) {
                    if (r == 1)
                        cudaEventRecord(e0, s);
                    st = run_pairsum(kind, prec, sp, *ts, op->w.as<double>(), zs.as<double>(),
                                     op->n, op->src.as<double>(), op->n, zo.as<double>(), scale,
                                     kappa, 0.0, nullptr, s);
                }
                cudaEventRecord(e1, s);
                if (st == SBQ_OK) {
                    cudaError_t ce = cudaEventSynchronize(e1);
                    if (ce != cudaSuccess)
                        st = cuda_status(ce, "autotune");
                }
                if (st != SBQ_OK)
                    return done(st);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                budget_ms += ms * (reps + 1);
                rate = ms > 0.0f ? ts->pairs / ms : 0.0;
            }
            if (rate > best_rate) {
                best_rate = rate;
                best = std::move(ts);
            }
            if (budget_ms >= 4000.0)
                break;
        }
    }
    done(SBQ_OK);
    if (!best) {
        set_error("autotune found no runnable tile shape");
        return SBQ_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(op, kind, prec)] = best->tune;
    }
    op->ts[prec] = std::move(best);
    op->tuned[prec] = true;
    return SBQ_OK;
}

int op_prepare_untimed(Op *op, int prec, const sbq_tune *tune, cudaStream_t s)
{
    int kind;
    double scale, kappa;
    op_kind(op, &kind, &scale, &kappa);
    sbq_tune t = default_tune(prec, op->n);
    if (tune && tune->r != 0) {
        t = *tune;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(op, kind, prec));
        if (it != g_tune_cache.end())
            t = it->second;
    }
    auto ts = std::make_unique<TrgSet>();
    SBQ_TRY(build_trg_set(*ts, kind, prec, t, op_srcpack(op, prec), op->plan.src_off,
                          op->src.as<double>(), op->n, op->plan.src_off, s));
    op->ts[prec] = std::move(ts);
    return SBQ_OK;
}

int op_ensure_tuned(Op *op, int prec, cudaStream_t s)
{
    if (op->ts[prec])
        return SBQ_OK;
    int kind;
    double scale, kappa;
    op_kind(op, &kind, &scale, &kappa);
    if (op->plan.has_tune) {
        auto ts = std::make_unique<TrgSet>();
        sbq_tune t = op->plan.tune;
        if (!pairsum_shape_supported(prec, t.r, t.warps)) {
            const int chunk = t.chunk_tiles;
            t = default_tune(prec, op->n);   // the plan's shape exists for the other precision
            t.chunk_tiles = chunk;
        }
        SBQ_TRY(build_trg_set(*ts, kind, prec, t, op_srcpack(op, prec), op->plan.src_off,
                              op->src.as<double>(), op->n, op->plan.src_off, s));
        op->ts[prec] = std::move(ts);
        return SBQ_OK;
    }
    return autotune_op(op, prec, s);
}

int op_autotune(Op *op, int prec, cudaStream_t s)
{
    op->ts[prec].reset();
    op->tuned[prec] = false;
    {
        int kind;
        double scale, kappa;
        op_kind(op, &kind, &scale, &kappa);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache.erase(tune_key(op, kind, prec));
    }
    return autotune_op(op, prec, s);
}

int op_matvec(Op *op, const double *sigma, double *out, int prec, cudaStream_t s, double *bound)
{
    // an attached treecode takes the plain FP32 applies (inner solves)
    const bool tree = prec == SBQ_FP32 && op->tree != nullptr && bound == nullptr;
    if (!tree)
        SBQ_TRY(op_ensure_tuned(op, prec, s));
    int kind;
    double scale, kappa;
    op_kind(op, &kind, &scale, &kappa);
    const long long n = op->n;
    if (n == 0)
        return SBQ_OK;
    // mobility: K (sigma - L sigma) + L sigma, with y = sigma - L sigma in the state's scratch
    const double *y = sigma;
    if (op->mob) {
        SBQ_TRY(mob_project(op, sigma, 1.0, s));
        SBQ_TRY(mob_field(op, sigma, -1.0, op->mob->y.as<double>(), s));
        y = op->mob->y.as<double>();
    }
    if (tree)
        SBQ_TRY(tree_op_apply(op, y, out, s));
    else
        SBQ_TRY(run_pairsum(kind, prec, op_srcpack(op, prec), *op->ts[prec], op->w.as<double>(), y,
                            n, op->src.as<double>(), n, out, scale, kappa, op->diag, y, s,
                            bound, op->perm.as<int>()));
    if (op->nnz > 0)
        SBQ_CUDA(launch_csr_apply(op->ncomp * n, op->rowptr.as<int64_t>(), op->col.as<int64_t>(),
                                  op->val.as<double>(), y, out, s));
    if (op->mob)
        SBQ_TRY(mob_field(op, out, 1.0, out, s));
    return SBQ_OK;
}

}  // namespace sbq
