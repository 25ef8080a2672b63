// Far-field acceleration of the layer sums alpha S + beta D for large N (the paper evaluates
// its far field with an FMM, Sec. 3.2, and states the O(N^2) direct cost it replaces,
// Sec. 3.4): a barycentric Lagrange treecode on the GPU.
//
// Setup (host, once per geometry): an octree over the sources (Morton order, tight boxes,
// leaves of at most TR_LEAF sources) and one over the targets (the same tree when the
// targets are the sources); every cell gets a tensor grid of Chebyshev points of the second
// kind on its box, n_d points along dimension d with n_d ~ order * (h_d / h_max)^(1/3) (a
// slender cell needs few points across); targets in blocks of up to 128 consecutive points
// in Morton order inside one cell of at most 512 targets, and for every block a list: the
// proxy grid of every cell that is far (acceptance: distance between the centres minus the
// block's radius positive and >= cell radius / theta, and the cell holds more sources than
// proxies) and
// the sources of every leaf it reaches.
// Apply (GPU, per density): charge records of the sources (q = w sigma scaled for the single
// layer and, with the double layer, the tensor (w sigma) n^T); proxy charges q_m = sum_k
// L_m(y_k) q_k, L_m the tensor Lagrange basis of the grid (barycentric form), for the cells
// some list takes as far; then one CTA per target block sums the kernel over its list, each
// list entry in FP32 and the entries' sums in FP64.  Positions are kept in FP32 relative to
// the centre of their leaf (sources), block (targets) or cell (proxies), and each entry
// carries the offset between its frame and the target block's, so that near pairs lose no
// digits to large absolute coordinates; with the double layer, source leaves also take the
// rounding residuals of the positions and of the offsets, so that r keeps its FP32 accuracy
// relative to |r| itself, since on the surface r . n is O(|r|^2).  Pairs of a leaf and a
// block closer than 4e-6 x the sum of their radii count as coincident and are skipped, as
// in the direct FP32 sums.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <utility>
#include <vector>

struct sbq_tree_s {
    uint32_t magic = 0x53425454u;   // "SBTT"
    int device = 0;
    long long ns = 0, nt = 0;
    bool same = false;              // targets are the sources (one tree)
    double theta = 0.0;
    int order = 0;
    long long n_cells = 0, n_proxies = 0, n_entries = 0, n_tleaves = 0;
    double pairs = 0.0;             // kernel evaluations per apply
    // device data
    sbq::DevBuf perm_s, perm_t;     // sorted position -> original index
    sbq::DevBuf w_sorted;           // FP64 weights, sorted order
    sbq::DevBuf n_sorted;           // FP64 normals (3 x ns, sorted), double layer only
    double alpha = 1.0, beta = 0.0; // u = alpha S + beta D
    int nq = 1;                     // float4 charge records per point: 1 (S), 3 (S and D)
    sbq::DevBuf src_loc;            // float4: source - its leaf centre (sorted order)
    sbq::DevBuf src_abs;            // double: absolute source positions (3 x ns, sorted)
    sbq::DevBuf trg_loc;            // float4: target - its block centre (sorted order)
    sbq::DevBuf trg_lo, src_lo;     // float4: rounding residuals of trg_loc and src_loc
    sbq::DevBuf q;                  // nq float4 charge records per source, sorted order
    sbq::DevBuf cells;              // TrCellDev per cell
    sbq::DevBuf prox_loc;           // float4: proxy - its cell centre
    sbq::DevBuf prox_q;             // nq float4 charge records per proxy
    sbq::DevBuf chunks;             // int4 (cell, first source, count, 0): P2M work items
    long long n_chunks = 0;
    sbq::DevBuf tleaf;              // int4 (first target, count, first entry, entry count)
    sbq::DevBuf entries;            // TrEntry
};

namespace sbq {

namespace {

constexpr int TR_LEAF = 128;       // sources (targets) per leaf at most
constexpr int TR_NMAX = 16;        // proxy points per dimension at most
constexpr int TR_THREADS = 128;
constexpr int TR_CHUNK = 512;      // sources per P2M work item
constexpr int TR_BLOCKCELL = 512;  // target blocks: runs of TR_THREADS inside cells this small
constexpr int TR_MAXLEV = 21;
constexpr double TR_PI = 3.14159265358979323846;
// Pairs of a source leaf and a target block closer than this fraction of the sum of their
// radii count as coincident and are skipped (the direct FP32 sums' rule): the rounding of
// the FP32 frame coordinates moves a coincident pair (a node and itself on the surface) by
// a few ulps of that sum, far below it.
constexpr double TR_COINCIDENT_REL = 4.0e-6;
constexpr float TR_R2MIN = 1.17549435e-38f;   // FLT_MIN: the SFU rsqrt flushes below it

struct TrCellDev {
    double c[3], h[3];
    int n[3], pfirst;
};

struct alignas(16) TrEntry {
    int first, count, kind;        // kind 0: sources [first, first + count); 1: proxies
    int cell;                      // the source cell (set up on the host; unused on the device)
    float dx, dy, dz;              // block frame centre minus target block centre (FP32)
    float thr2;                    // kind 0: squared distance below which a pair is skipped
    float lx, ly, lz, pad3;        // and the rounding residual of that offset
};
static_assert(sizeof(TrEntry) % sizeof(int4) == 0, "entries are read as int4 heads");

// thr: pairs of a source leaf closer than this count as coincident (skipped)
inline TrEntry make_entry(int first, int count, int kind, double thr, const double *cb, const double *ct)
{
    TrEntry e{};
    e.first = first;
    e.count = count;
    e.kind = kind;
    const double d[3] = {cb[0] - ct[0], cb[1] - ct[1], cb[2] - ct[2]};
    e.dx = static_cast<float>(d[0]);
    e.dy = static_cast<float>(d[1]);
    e.dz = static_cast<float>(d[2]);
    e.lx = static_cast<float>(d[0] - e.dx);
    e.ly = static_cast<float>(d[1] - e.dy);
    e.lz = static_cast<float>(d[2] - e.dz);
    e.thr2 = std::max(static_cast<float>(thr * thr), TR_R2MIN);
    return e;
}

// a float and its rounding residual (the pair holds a double to ~48 bits)
inline float4 hi4(double x, double y, double z)
{
    return make_float4(static_cast<float>(x), static_cast<float>(y), static_cast<float>(z), 0.0f);
}
inline float4 lo4(double x, double y, double z)
{
    return make_float4(static_cast<float>(x - static_cast<float>(x)), static_cast<float>(y - static_cast<float>(y)),
                       static_cast<float>(z - static_cast<float>(z)), 0.0f);
}

struct HostCell {
    double c[3], h[3], rad;
    int first, count, level;
    int child[8], nchild;
    int n[3], pfirst, nprox;
};

struct HostTree {
    std::vector<int> perm;          // sorted position -> original index
    std::vector<HostCell> cells;    // cells[0] is the root
    std::vector<int> leaf_of;       // sorted position -> leaf cell
    std::vector<int> leaves;        // leaf cells in sorted order
};

inline uint64_t spread21(uint64_t v)
{
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// fn(lo, hi) over [0, count) split into contiguous ranges of at least `grain` items run by
// up to 16 host threads (in the calling thread alone when threads cannot be started); fn
// writes disjoint outputs
template <class Fn>
void host_parallel(long long count, long long grain, Fn fn)
{
    const long long hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int nth = static_cast<int>(std::max(1LL, std::min(hw, count / std::max(1LL, grain))));
    const long long per = (count + nth - 1) / nth;
    std::vector<std::thread> th;
    long long done_to = 0;   // ranges below this were handed to threads
    try {
        for (int i = 1; i < nth && i * per < count; ++i) {
            const long long lo = i * per, hi = std::min(count, lo + per);
            th.emplace_back([=, &fn] { fn(lo, hi); });
            done_to = hi;
        }
    } catch (...) {
    }
    fn(0, std::min(count, per));
    if (done_to < count)   // ranges no thread took
        for (long long lo = std::max(per, done_to); lo < count; lo += per)
            fn(lo, std::min(count, lo + per));
    for (std::thread &t : th)
        t.join();
}

// Octree over n points (SoA x, y, z): Morton sort, then cells split by the next three key
// bits until at most `leaf` points remain; tight boxes.  The topology comes from the sorted
// keys alone (octant boundaries by binary search), the boxes bottom-up: leaves from their
// points, every other cell from its children.
void build_host_tree(const std::vector<double> &x, long long n, int leaf, HostTree &T)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long k = 0; k < n; ++k)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], x[d * n + k]);
            hi[d] = std::max(hi[d], x[d * n + k]);
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d)
        ext = std::max(ext, hi[d] - lo[d]);
    ext = ext > 0.0 ? ext * (1.0 + 1e-9) : 1.0;
    // sort (key, index) pairs: chunks in parallel, then pairwise merges (the order is the
    // total order of the pairs, whatever the chunking)
    std::vector<std::pair<uint64_t, int>> kp(n);
    constexpr long long PGRAIN = 32768;   // points per thread at least
    host_parallel(n, PGRAIN, [&](long long b, long long e) {
        for (long long k = b; k < e; ++k) {
            uint64_t kk = 0;
            for (int d = 0; d < 3; ++d) {
                double u = (x[d * n + k] - lo[d]) / ext * 2097152.0;
                uint64_t q = static_cast<uint64_t>(std::min(std::max(u, 0.0), 2097151.0));
                kk |= spread21(q) << (2 - d);
            }
            kp[k] = {kk, static_cast<int>(k)};
        }
    });
    const long long nchunk = n >= 16 * PGRAIN ? 16 : 1, per = std::max(1LL, (n + nchunk - 1) / nchunk);
    host_parallel(nchunk, 1, [&](long long b, long long e) {
        for (long long c = b; c < e; ++c)
            std::sort(kp.begin() + std::min(n, c * per), kp.begin() + std::min(n, (c + 1) * per));
    });
    for (long long w = per; w < n; w *= 2)
        host_parallel((n + 2 * w - 1) / (2 * w), 1, [&](long long b, long long e) {
            for (long long c = b; c < e; ++c) {
                const long long a0 = c * 2 * w, m = std::min(n, a0 + w), b0 = std::min(n, a0 + 2 * w);
                std::inplace_merge(kp.begin() + a0, kp.begin() + m, kp.begin() + b0);
            }
        });
    T.perm.resize(n);
    std::vector<uint64_t> ks(n);
    std::vector<double> xs(3 * n);   // coordinates in sorted order
    host_parallel(n, PGRAIN, [&](long long b, long long e) {
        for (long long k = b; k < e; ++k) {
            T.perm[k] = kp[k].second;
            ks[k] = kp[k].first;
            for (int d = 0; d < 3; ++d)
                xs[d * n + k] = x[d * n + kp[k].second];
        }
    });
    // topology, depth first (cell indices in creation order: children after their parent)
    T.cells.clear();
    T.leaves.clear();
    T.leaf_of.assign(n, -1);
    HostCell root{};
    root.first = 0;
    root.count = static_cast<int>(n);
    root.level = 0;
    T.cells.push_back(root);
    std::vector<int> stack{0};
    while (!stack.empty()) {
        const int ci = stack.back();
        stack.pop_back();
        HostCell c = T.cells[ci];
        c.nchild = 0;
        if (c.count > leaf && c.level < TR_MAXLEV) {
            const int shift = 3 * (TR_MAXLEV - 1 - c.level);
            // the keys of a cell share their bits above `shift + 3`, so the octant is
            // non-decreasing along the cell's sorted range
            const auto beg = ks.begin() + c.first, end = beg + c.count;
            auto it = beg;
            while (it != end) {
                const uint64_t oct = (*it >> shift) & 7ULL;
                const auto nx = std::partition_point(it, end, [&](uint64_t v) { return ((v >> shift) & 7ULL) <= oct; });
                HostCell ch{};
                ch.first = static_cast<int>(it - ks.begin());
                ch.count = static_cast<int>(nx - it);
                ch.level = c.level + 1;
                c.child[c.nchild++] = static_cast<int>(T.cells.size());
                T.cells.push_back(ch);
                it = nx;
            }
            // a cell whose points share one octant keeps splitting through its child
        }
        T.cells[ci] = c;
        if (c.nchild == 0) {
            T.leaves.push_back(ci);
            for (int k = c.first; k < c.first + c.count; ++k)
                T.leaf_of[k] = ci;
        } else {
            for (int k = c.nchild - 1; k >= 0; --k)
                stack.push_back(c.child[k]);
        }
    }
    // tight boxes: leaves from their points (in parallel), then every other cell from its
    // children, in reverse creation order
    const long long nc = static_cast<long long>(T.cells.size());
    std::vector<double> blo(3 * nc, INFINITY), bhi(3 * nc, -INFINITY);
    host_parallel(static_cast<long long>(T.leaves.size()), PGRAIN / TR_LEAF, [&](long long b, long long e) {
        for (long long li = b; li < e; ++li) {
            const HostCell &c = T.cells[T.leaves[li]];
            double *l = &blo[3 * T.leaves[li]], *h = &bhi[3 * T.leaves[li]];
            for (int k = c.first; k < c.first + c.count; ++k)
                for (int d = 0; d < 3; ++d) {
                    l[d] = std::min(l[d], xs[d * n + k]);
                    h[d] = std::max(h[d], xs[d * n + k]);
                }
        }
    });
    for (long long ci = nc - 1; ci >= 0; --ci) {
        HostCell &c = T.cells[ci];
        for (int j = 0; j < c.nchild; ++j)
            for (int d = 0; d < 3; ++d) {
                blo[3 * ci + d] = std::min(blo[3 * ci + d], blo[3 * c.child[j] + d]);
                bhi[3 * ci + d] = std::max(bhi[3 * ci + d], bhi[3 * c.child[j] + d]);
            }
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            c.c[d] = 0.5 * (blo[3 * ci + d] + bhi[3 * ci + d]);
            c.h[d] = 0.5 * (bhi[3 * ci + d] - blo[3 * ci + d]);
            r2 += c.h[d] * c.h[d];
        }
        c.rad = std::sqrt(r2);
    }
    std::sort(T.leaves.begin(), T.leaves.end(),
              [&](int a, int b) { return T.cells[a].first < T.cells[b].first; });
}

// ---------------------------------------------------------------------------------------
// device kernels

// Chebyshev points of the second kind, cos(pi j / (n - 1)), for n = 2..TR_NMAX (row n)
__constant__ float c_cheb[TR_NMAX + 1][TR_NMAX];

// 1D Lagrange basis values of the n-point grid at xi (barycentric form in FP32: the proxy
// charges need ~1e-7, and the FP64 form's divisions made this the apply's second kernel)
__device__ void lagrange_1d(float xi, int n, float *out)
{
    if (n == 1) {
        out[0] = 1.0f;
        return;
    }
    float den = 0.0f;
    int hit = -1;
    for (int j = 0; j < n; ++j) {
        const float d = xi - c_cheb[n][j];
        if (d == 0.0f)
            hit = j;
        float w = (j & 1) ? -1.0f : 1.0f;
        if (j == 0 || j == n - 1)
            w *= 0.5f;
        out[j] = w / d;
        den += out[j];
    }
    const float inv = 1.0f / den;
    for (int j = 0; j < n; ++j)
        out[j] = hit >= 0 ? (j == hit ? 1.0f : 0.0f) : out[j] * inv;
}

// charge records of source k (sorted order): q = w sigma scaled by alpha / (8 pi) and, for
// the double layer, the tensor d = m n^T, m = w sigma scaled by 3 beta / (4 pi): record 0
// (q_x, q_y, q_z, d00), record 1 (d01, d02, d10, d11), record 2 (d12, d20, d21, d22), each
// product formed in FP64 and rounded once.  (The near sums in the rank-one form (r . m)(r . n)
// from FP32 m and n were tried: twice the error of the combined field at 1M nodes.)
template <int NQ>
__global__ void k_tree_charges(long long ns, const int *__restrict__ perm, const double *__restrict__ w,
                               const double *__restrict__ nrm, const double *__restrict__ sigma,
                               double a, double b, float4 *q)
{
    const long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (k >= ns)
        return;
    const long long o = perm[k];
    const double ww = w[k];
    const double s0 = ww * sigma[o], s1 = ww * sigma[ns + o], s2 = ww * sigma[2 * ns + o];
    if (NQ == 1) {
        q[k] = make_float4(static_cast<float>(a * s0), static_cast<float>(a * s1), static_cast<float>(a * s2), 0.0f);
        return;
    }
    const double n0 = nrm[k], n1 = nrm[ns + k], n2 = nrm[2 * ns + k];
    const double m0 = b * s0, m1 = b * s1, m2 = b * s2;
    q[3 * k] = make_float4(static_cast<float>(a * s0), static_cast<float>(a * s1), static_cast<float>(a * s2),
                           static_cast<float>(m0 * n0));
    q[3 * k + 1] = make_float4(static_cast<float>(m0 * n1), static_cast<float>(m0 * n2),
                               static_cast<float>(m1 * n0), static_cast<float>(m1 * n1));
    q[3 * k + 2] = make_float4(static_cast<float>(m1 * n2), static_cast<float>(m2 * n0),
                               static_cast<float>(m2 * n1), static_cast<float>(m2 * n2));
}

// proxy charges of one cell from one chunk of its sources (atomically accumulated)
template <int NQ>
__global__ void __launch_bounds__(TR_THREADS)
k_tree_p2m(const int4 *__restrict__ chunks, const TrCellDev *__restrict__ cells,
           const double *__restrict__ src_abs, long long ns, const float4 *__restrict__ q,
           float4 *prox_q)
{
    __shared__ float Lx[TR_THREADS][TR_NMAX], Ly[TR_THREADS][TR_NMAX], Lz[TR_THREADS][TR_NMAX];
    __shared__ float4 sq[TR_THREADS * NQ];
    const int4 ck = chunks[blockIdx.x];
    const TrCellDev c = cells[ck.x];
    const int np = c.n[0] * c.n[1] * c.n[2];
    double ih[3];   // the cell's offset from its centre in half-widths (0 on a flat axis)
    for (int d = 0; d < 3; ++d)
        ih[d] = c.h[d] > 0.0 ? 1.0 / c.h[d] : 0.0;
    constexpr int MPT = 8;   // proxies per thread: 8 x 128 = 1024 >= 10^3, the largest grid
    float acc[MPT][4 * NQ];
    for (int m = 0; m < MPT; ++m)
        for (int v = 0; v < 4 * NQ; ++v)
            acc[m][v] = 0.0f;
    for (int base = 0; base < ck.z; base += TR_THREADS) {
        const int k = base + threadIdx.x;
        if (k < ck.z) {
            const long long s = ck.y + k;
            float xi[3];
            for (int d = 0; d < 3; ++d)
                xi[d] = static_cast<float>((src_abs[d * ns + s] - c.c[d]) * ih[d]);
            lagrange_1d(xi[0], c.n[0], Lx[threadIdx.x]);
            lagrange_1d(xi[1], c.n[1], Ly[threadIdx.x]);
            lagrange_1d(xi[2], c.n[2], Lz[threadIdx.x]);
            for (int r = 0; r < NQ; ++r)
                sq[threadIdx.x * NQ + r] = q[s * NQ + r];
        } else {
            for (int r = 0; r < NQ; ++r)
                sq[threadIdx.x * NQ + r] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int j = 0; j < TR_NMAX; ++j)
                Lx[threadIdx.x][j] = Ly[threadIdx.x][j] = Lz[threadIdx.x][j] = 0.0f;
        }
        __syncthreads();
        const int cnt = min(TR_THREADS, ck.z - base);
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int pm = threadIdx.x + m * TR_THREADS;
            if (pm < np) {
                const int a = pm / (c.n[1] * c.n[2]), b = (pm / c.n[2]) % c.n[1], cc = pm % c.n[2];
                for (int kk = 0; kk < cnt; ++kk) {
                    const float l = Lx[kk][a] * Ly[kk][b] * Lz[kk][cc];
#pragma unroll
                    for (int r = 0; r < NQ; ++r) {
                        const float4 qq = sq[kk * NQ + r];
                        acc[m][4 * r] = fmaf(l, qq.x, acc[m][4 * r]);
                        acc[m][4 * r + 1] = fmaf(l, qq.y, acc[m][4 * r + 1]);
                        acc[m][4 * r + 2] = fmaf(l, qq.z, acc[m][4 * r + 2]);
                        acc[m][4 * r + 3] = fmaf(l, qq.w, acc[m][4 * r + 3]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < MPT; ++m) {
        const int pm = threadIdx.x + m * TR_THREADS;
        if (pm < np) {
            float *dst = reinterpret_cast<float *>(prox_q + static_cast<size_t>(c.pfirst + pm) * NQ);
#pragma unroll
            for (int v = 0; v < 4 * NQ; ++v)
                if (NQ > 1 || v < 3)
                    atomicAdd(dst + v, acc[m][v]);
        }
    }
}

// Packed FP32 pairs: one 64-bit register holds the values of two sources; the f32x2
// instructions process both in one issue slot.
using tf2 = unsigned long long;

__device__ __forceinline__ tf2 tf2_fma(tf2 a, tf2 b, tf2 c)
{
    tf2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ tf2 tf2_mul(tf2 a, tf2 b)
{
    tf2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ tf2 tf2_sub(tf2 a, tf2 b)
{
    tf2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ tf2 tf2_add(tf2 a, tf2 b)
{
    tf2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ tf2 tf2_pack(float lo, float hi)
{
    tf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void tf2_unpack(tf2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Shared-memory tile of TR_THREADS points as packed pairs: field f of points 2m and 2m + 1
// at f2 index f * (TR_THREADS / 2) + m.  Fields: 0..2 position, 3..5 single-layer charge,
// then (NQ == 3) 6..14 the double layer's tensor d_jl and 15..17 the position residuals.
constexpr int TR_HALF = TR_THREADS / 2;

template <int NQ>
__host__ __device__ constexpr int tree_fields()
{
    return NQ == 3 ? 18 : 6;
}

// 1/sqrt(x) on the SFU, denormals flushed (callers pass squared distances of at least
// FLT_MIN, or select the result away)
__device__ __forceinline__ float tr_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 4-byte asynchronous copy global -> shared (no register holds the value on its way)
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Stage point k of a list entry, head en = (first, count, kind), into column t of the
// shared tile, copied asynchronously; a point past the entry's end is written directly
// (zero charge, far away).  Fields: 0..2 position, 3..5 single-layer charge q; with the
// double layer, the tensor d in 6..14 (d00 d01 d02 d10 d11 d12 d20 d21 d22, the records'
// floats 3..11 in order) and, for a source leaf, the position's rounding residual in
// 15..17.
template <int NQ>
__device__ __forceinline__ void tr_stage(float *sf, int t, const int4 &en, int k,
                                         const float4 *__restrict__ src_loc, const float4 *__restrict__ q,
                                         const float4 *__restrict__ prox_loc,
                                         const float4 *__restrict__ prox_q, const float4 *__restrict__ src_lo)
{
    constexpr int NF = tree_fields<NQ>();
    if (k < en.y) {
        const float *P = reinterpret_cast<const float *>((en.z ? prox_loc : src_loc) + en.x + k);
        const float *Q = reinterpret_cast<const float *>((en.z ? prox_q : q) +
                                                         static_cast<size_t>(en.x + k) * NQ);
        for (int f = 0; f < 3; ++f)
            cp_async4(sf + f * TR_THREADS + t, P + f);
        for (int f = 0; f < 3 * NQ + (NQ == 3 ? 3 : 0); ++f)
            cp_async4(sf + (3 + f) * TR_THREADS + t, Q + f);
        if (NQ == 3 && en.z == 0) {
            const float *L = reinterpret_cast<const float *>(src_lo + en.x + k);
            for (int f = 15; f < 18; ++f)
                cp_async4(sf + f * TR_THREADS + t, L + (f - 15));
        }
    } else {
        for (int f = 0; f < NF; ++f)
            sf[f * TR_THREADS + t] = f < 3 ? 1e15f : 0.0f;
    }
}

// The staged points 0 .. 2 cnt2 - 1 of one entry against the thread's target, two per packed
// operation.  NEAR (a source leaf): pairs closer than the entry's coincidence distance (the
// target's own node on the surface among them) add nothing; with the double layer, r is
// formed from high and low parts, since on the surface r . n = O(|r|^2): the target in the
// leaf's frame as an exact (hi, lo) pair (TwoSum, once per entry), then r = (x_hi - y_hi) +
// (x_lo - y_lo), accurate to an ulp of r itself rather than of the frames.  Far entries
// (proxy grids) need neither: with d > 0 the distance between the centres less the block's
// radius, their acceptance (d theta >= cell radius) keeps every target at least
// (1 - theta) d from every proxy point.
template <int NQ, bool NEAR>
__device__ __forceinline__ void tr_tile(const tf2 *__restrict__ F, int cnt2, const float4 &x,
                                        const float4 &xl, const TrEntry &en, tf2 &ax, tf2 &ay, tf2 &az)
{
    constexpr bool HILO = NEAR && NQ == 3;
    const float thr2 = en.thr2;
    float xh[3], xo[3];
    {
        const float xv[3] = {x.x, x.y, x.z}, xlv[3] = {xl.x, xl.y, xl.z};
        const float ev[3] = {en.dx, en.dy, en.dz}, elv[3] = {en.lx, en.ly, en.lz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xh[d] = xv[d] - ev[d];
            if (HILO) {   // x - e = xh + err exactly
                const float bb = xh[d] - xv[d];
                const float err = (xv[d] - (xh[d] - bb)) - (ev[d] + bb);
                xo[d] = (xlv[d] - elv[d]) + err;
            }
        }
    }
    const tf2 X2 = tf2_pack(xh[0], xh[0]), Y2 = tf2_pack(xh[1], xh[1]), Z2 = tf2_pack(xh[2], xh[2]);
    tf2 XL2 = 0ull, YL2 = 0ull, ZL2 = 0ull;
    if (HILO) {
        XL2 = tf2_pack(xo[0], xo[0]);
        YL2 = tf2_pack(xo[1], xo[1]);
        ZL2 = tf2_pack(xo[2], xo[2]);
    }
    // unrolled twice for the single layer; the double layer's loop holds enough registers
    constexpr int UNROLL = NQ == 3 ? 1 : 2;
#pragma unroll UNROLL
    for (int m = 0; m < cnt2; ++m) {
        tf2 dx = tf2_sub(X2, F[0 * TR_HALF + m]);
        tf2 dy = tf2_sub(Y2, F[1 * TR_HALF + m]);
        tf2 dz = tf2_sub(Z2, F[2 * TR_HALF + m]);
        if (HILO) {
            dx = tf2_add(dx, tf2_sub(XL2, F[15 * TR_HALF + m]));
            dy = tf2_add(dy, tf2_sub(YL2, F[16 * TR_HALF + m]));
            dz = tf2_add(dz, tf2_sub(ZL2, F[17 * TR_HALF + m]));
        }
        const tf2 QX = F[3 * TR_HALF + m], QY = F[4 * TR_HALF + m], QZ = F[5 * TR_HALF + m];
        const tf2 r2 = tf2_fma(dx, dx, tf2_fma(dy, dy, tf2_mul(dz, dz)));
        float r2a, r2b;
        tf2_unpack(r2, r2a, r2b);
        float ra = tr_rsqrt(r2a), rb = tr_rsqrt(r2b);
        if (NEAR) {
            ra = r2a >= thr2 ? ra : 0.0f;
            rb = r2b >= thr2 ? rb : 0.0f;
        }
        const tf2 ri = tf2_pack(ra, rb);
        const tf2 ri2 = tf2_mul(ri, ri);
        const tf2 rq = tf2_fma(dx, QX, tf2_fma(dy, QY, tf2_mul(dz, QZ)));
        // u = ri (q + r [(r . q) ri^2 + (r^T d r) ri^4])
        tf2 bq = tf2_mul(rq, ri2);
        if (NQ == 3) {
            const tf2 a0 = tf2_fma(F[6 * TR_HALF + m], dx, tf2_fma(F[7 * TR_HALF + m], dy,
                                                                   tf2_mul(F[8 * TR_HALF + m], dz)));
            const tf2 a1 = tf2_fma(F[9 * TR_HALF + m], dx, tf2_fma(F[10 * TR_HALF + m], dy,
                                                                   tf2_mul(F[11 * TR_HALF + m], dz)));
            const tf2 a2 = tf2_fma(F[12 * TR_HALF + m], dx, tf2_fma(F[13 * TR_HALF + m], dy,
                                                                    tf2_mul(F[14 * TR_HALF + m], dz)));
            const tf2 rdr = tf2_fma(dx, a0, tf2_fma(dy, a1, tf2_mul(dz, a2)));
            bq = tf2_fma(rdr, tf2_mul(ri2, ri2), bq);
        }
        ax = tf2_fma(ri, tf2_fma(bq, dx, QX), ax);
        ay = tf2_fma(ri, tf2_fma(bq, dy, QY), ay);
        az = tf2_fma(ri, tf2_fma(bq, dz, QZ), az);
    }
}

// Sums over the list of a target block: one CTA per block, one thread per target.  The list
// is walked in chunks of up to TR_THREADS points of one entry; chunks alternate between two
// shared-memory buffers, and every thread's asynchronous copies of its point of the next
// chunk are in flight while the current one is summed (one barrier per chunk).  Each entry is summed in FP32, two
// sources per packed FP32x2 operation, and the entries' sums are added in FP64.
template <int NQ>
__global__ void __launch_bounds__(TR_THREADS)
k_tree_eval(const int4 *__restrict__ tleaf, const TrEntry *__restrict__ entries,
            const float4 *__restrict__ trg_loc, const float4 *__restrict__ src_loc,
            const float4 *__restrict__ q, const float4 *__restrict__ prox_loc,
            const float4 *__restrict__ prox_q, const int *__restrict__ perm_t, long long nt,
            const float4 *__restrict__ trg_lo, const float4 *__restrict__ src_lo, double *u)
{
    constexpr int NF = tree_fields<NQ>();
    __shared__ __align__(16) float sf[2][NF * TR_THREADS];
    const int4 tl = tleaf[blockIdx.x];
    const int t = threadIdx.x;
    const bool live = t < tl.y;
    const float4 x = live ? trg_loc[tl.x + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xl = (NQ == 3 && live) ? trg_lo[tl.x + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (tl.w > 0) {
        // (first, count, kind): the leading fields of an entry, all the staging needs
        const int4 *ehead = reinterpret_cast<const int4 *>(entries + tl.z);
        constexpr int ESTRIDE = sizeof(TrEntry) / sizeof(int4);
        int e = 0, base = 0, buf = 0;
        TrEntry en = entries[tl.z];
        tr_stage<NQ>(sf[0], t, make_int4(en.first, en.count, en.kind, 0), t, src_loc, q, prox_loc,
                     prox_q, src_lo);
        cp_async_commit();
        tf2 ax = 0ull, ay = 0ull, az = 0ull;   // packed (0.f, 0.f)
        for (;;) {
            cp_async_wait_all();
            __syncthreads();   // chunk in sf[buf] complete; sf[buf ^ 1] free (its sums are done)
            // the next chunk: the rest of this entry, else the next entry's first points
            int e_n = e, base_n = base + TR_THREADS;
            int4 hn = make_int4(en.first, en.count, en.kind, 0);
            if (base_n >= en.count) {
                e_n = e + 1;
                base_n = 0;
                if (e_n < tl.w)
                    hn = ehead[e_n * ESTRIDE];
            }
            const bool more = e_n < tl.w;
            if (more) {
                tr_stage<NQ>(sf[buf ^ 1], t, hn, base_n + t, src_loc, q, prox_loc, prox_q, src_lo);
                cp_async_commit();
            }
            const tf2 *F = reinterpret_cast<const tf2 *>(sf[buf]);
            const int cnt2 = (min(TR_THREADS, en.count - base) + 1) / 2;
            if (en.kind == 0)
                tr_tile<NQ, true>(F, cnt2, x, xl, en, ax, ay, az);
            else
                tr_tile<NQ, false>(F, cnt2, x, xl, en, ax, ay, az);
            if (e_n != e) {   // the entry is complete: its FP32 sum into the FP64 total
                float a0, a1;
                tf2_unpack(ax, a0, a1);
                v0 += static_cast<double>(a0) + static_cast<double>(a1);
                tf2_unpack(ay, a0, a1);
                v1 += static_cast<double>(a0) + static_cast<double>(a1);
                tf2_unpack(az, a0, a1);
                v2 += static_cast<double>(a0) + static_cast<double>(a1);
                ax = ay = az = 0ull;
            }
            if (!more)
                break;
            if (e_n != e)
                en = entries[tl.z + e_n];
            e = e_n;
            base = base_n;
            buf ^= 1;
        }
    }
    if (live) {
        const long long o = perm_t[tl.x + t];
        u[o] = v0;
        u[nt + o] = v1;
        u[2 * nt + o] = v2;
    }
}

int proxies_per_dim(const HostCell &c, int order, int n[3])
{
    const double hm = std::max(c.h[0], std::max(c.h[1], c.h[2]));
    for (int d = 0; d < 3; ++d) {
        if (c.h[d] <= 0.0 || hm <= 0.0) {
            n[d] = 1;
            continue;
        }
        const int v = static_cast<int>(std::ceil(order * std::cbrt(c.h[d] / hm)));
        n[d] = std::max(2, std::min(order, v));
    }
    return n[0] * n[1] * n[2];
}

}  // namespace

static int tree_create_impl(long long ns, const double *src, const double *nrm, const double *w,
                            long long nt, const double *trg, double alpha, double beta,
                            double theta, int order, sbq_tree_s *T, cudaStream_t s)
{
    T->alpha = alpha;
    T->beta = beta;
    T->nq = beta != 0.0 ? 3 : 1;
    T->ns = ns;
    T->nt = nt;
    T->same = trg == src && nt == ns;
    T->theta = theta;
    T->order = order;
    if (ns == 0 || nt == 0)
        return SBQ_OK;   // nothing to build: the apply writes zeros (no sources) or nothing
    std::vector<double> hs(3 * ns), hw(ns), ht, hn;
    SBQ_CUDA(cudaMemcpyAsync(hs.data(), src, 3 * ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (T->nq == 3) {
        hn.resize(3 * ns);
        SBQ_CUDA(cudaMemcpyAsync(hn.data(), nrm, 3 * ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    SBQ_CUDA(cudaMemcpyAsync(hw.data(), w, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!T->same) {
        ht.resize(3 * nt);
        SBQ_CUDA(cudaMemcpyAsync(ht.data(), trg, 3 * nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    SBQ_CUDA(cudaStreamSynchronize(s));
    HostTree S, TT;
    build_host_tree(hs, ns, TR_LEAF, S);
    if (!T->same)
        build_host_tree(ht, nt, TR_LEAF, TT);
    const HostTree &Tt = T->same ? S : TT;
    const std::vector<double> &xt = T->same ? hs : ht;

    // Chebyshev points for the proxy-charge kernel (the same values on every call)
    {
        float tab[TR_NMAX + 1][TR_NMAX] = {};
        for (int n = 2; n <= TR_NMAX; ++n)
            for (int j = 0; j < n; ++j)
                tab[n][j] = static_cast<float>(std::cos(TR_PI * j / (n - 1)));
        SBQ_CUDA(cudaMemcpyToSymbolAsync(c_cheb, tab, sizeof(tab), 0, cudaMemcpyHostToDevice, s));
    }
    // proxies of every cell
    long long np = 0;
    for (size_t ci = 0; ci < S.cells.size(); ++ci) {
        HostCell &c = S.cells[ci];
        c.nprox = proxies_per_dim(c, order, c.n);
        c.pfirst = static_cast<int>(np);
        np += c.nprox;
    }
    if (np > 0x7fffffffLL) {
        set_error("stokes_tree_create: too many proxy points");
        return SBQ_EINVAL;
    }
    // Chebyshev points of the second kind, cos(pi j / (n - 1)), row n
    double cheb[TR_NMAX + 1][TR_NMAX] = {};
    for (int m = 2; m <= TR_NMAX; ++m)
        for (int j = 0; j < m; ++j)
            cheb[m][j] = std::cos(TR_PI * j / (m - 1));
    std::vector<float4> h_ploc(np);
    std::vector<TrCellDev> h_cells(S.cells.size());
    host_parallel(static_cast<long long>(S.cells.size()), 256, [&](long long cb, long long ce) {
        for (long long ci = cb; ci < ce; ++ci) {
            const HostCell &c = S.cells[ci];
            TrCellDev &dc = h_cells[ci];
            for (int d = 0; d < 3; ++d) {
                dc.c[d] = c.c[d];
                dc.h[d] = c.h[d];
                dc.n[d] = c.n[d];
            }
            dc.pfirst = c.pfirst;
            auto pt = [&](int j, int m) { return m > 1 ? cheb[m][j] : 0.0; };
            for (int a = 0; a < c.n[0]; ++a)
                for (int b = 0; b < c.n[1]; ++b)
                    for (int e = 0; e < c.n[2]; ++e) {
                        const int m = (a * c.n[1] + b) * c.n[2] + e;
                        h_ploc[c.pfirst + m] = make_float4(static_cast<float>(c.h[0] * pt(a, c.n[0])),
                                                           static_cast<float>(c.h[1] * pt(b, c.n[1])),
                                                           static_cast<float>(c.h[2] * pt(e, c.n[2])), 0.0f);
                    }
        }
    });
    // sources: FP32 offsets from their leaf's centre, FP64 absolute positions, weights
    std::vector<float4> h_sloc(ns), h_slo(ns);
    std::vector<double> h_sabs(3 * ns), h_ws(ns), h_ns(T->nq == 3 ? 3 * ns : 0);
    host_parallel(ns, 32768, [&](long long kb, long long ke) {
        for (long long k = kb; k < ke; ++k) {
            const int o = S.perm[k];
            const HostCell &L = S.cells[S.leaf_of[k]];
            h_sloc[k] = hi4(hs[o] - L.c[0], hs[ns + o] - L.c[1], hs[2 * ns + o] - L.c[2]);
            h_slo[k] = lo4(hs[o] - L.c[0], hs[ns + o] - L.c[1], hs[2 * ns + o] - L.c[2]);
            for (int d = 0; d < 3; ++d) {
                h_sabs[d * ns + k] = hs[d * ns + o];
                if (T->nq == 3)
                    h_ns[d * ns + k] = hn[d * ns + o];
            }
            h_ws[k] = hw[o];
        }
    });
    // target blocks: runs of TR_THREADS consecutive targets in Morton order, each with its
    // own tight box; target positions in FP32 relative to their block's centre
    struct TBlock {
        double c[3], rad;
        int first, count;
    };
    // (runs never leave a cell of at most TR_BLOCKCELL targets, so that a block is as compact
    // as such a cell: a run across a jump of the Morton order would be spread over the domain
    // and its FP32 offsets would lose the digits the near pairs need)
    std::vector<TBlock> tb;
    std::vector<float4> h_tloc(nt), h_tlo(nt);
    std::vector<std::pair<int, int>> runs;
    {
        std::vector<int> st{0};
        while (!st.empty()) {
            const HostCell &C = Tt.cells[st.back()];
            st.pop_back();
            if (C.count <= TR_BLOCKCELL || C.nchild == 0) {
                for (int b = 0; b < C.count; b += TR_THREADS)
                    runs.emplace_back(C.first + b, std::min(TR_THREADS, C.count - b));
            } else {
                for (int k = C.nchild - 1; k >= 0; --k)
                    st.push_back(C.child[k]);
            }
        }
    }
    tb.resize(runs.size());
    host_parallel(static_cast<long long>(runs.size()), 256, [&](long long rb, long long re) {
        for (long long ri = rb; ri < re; ++ri) {
            TBlock &B = tb[ri];
            B.first = runs[ri].first;
            B.count = runs[ri].second;
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int k = B.first; k < B.first + B.count; ++k)
                for (int d = 0; d < 3; ++d) {
                    const double v = xt[d * nt + Tt.perm[k]];
                    lo[d] = std::min(lo[d], v);
                    hi[d] = std::max(hi[d], v);
                }
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                B.c[d] = 0.5 * (lo[d] + hi[d]);
                r2 += 0.25 * (hi[d] - lo[d]) * (hi[d] - lo[d]);
            }
            B.rad = std::sqrt(r2);
            for (int k = B.first; k < B.first + B.count; ++k) {
                const int o = Tt.perm[k];
                h_tloc[k] = hi4(xt[o] - B.c[0], xt[nt + o] - B.c[1], xt[2 * nt + o] - B.c[2]);
                h_tlo[k] = lo4(xt[o] - B.c[0], xt[nt + o] - B.c[1], xt[2 * nt + o] - B.c[2]);
            }
        }
    });
    // lists: per target block, a traversal of the source tree (blocks in parallel ranges,
    // each range's entries concatenated in block order)
    const long long nblk = static_cast<long long>(tb.size());
    const long long nrange = std::min<long long>(64, std::max<long long>(1, nblk));
    const long long bper = (nblk + nrange - 1) / nrange;
    std::vector<std::vector<TrEntry>> rent(nrange);
    std::vector<int> rcount(nblk, 0);
    std::vector<double> rpairs(nrange, 0.0);
    host_parallel(nrange, nblk >= 256 ? 1 : nrange, [&](long long rlo, long long rhi) {
        std::vector<int> stack;
        for (long long r = rlo; r < rhi; ++r) {
            std::vector<TrEntry> &ent = rent[r];
            for (long long bi = r * bper; bi < std::min(nblk, (r + 1) * bper); ++bi) {
                const TBlock &L = tb[bi];
                const size_t e0 = ent.size();
                stack.assign(1, 0);
                while (!stack.empty()) {
                    const int cidx = stack.back();
                    const HostCell &C = S.cells[cidx];
                    stack.pop_back();
                    double d2 = 0.0;
                    for (int d = 0; d < 3; ++d)
                        d2 += (C.c[d] - L.c[d]) * (C.c[d] - L.c[d]);
                    const double dist = std::sqrt(d2) - L.rad;
                    if (dist > 0.0 && dist * theta >= C.rad && C.count > C.nprox) {
                        ent.push_back(make_entry(C.pfirst, C.nprox, 1, 0.0, C.c, L.c));
                        ent.back().cell = cidx;
                        rpairs[r] += static_cast<double>(C.nprox) * L.count;
                    } else if (C.nchild == 0) {
                        ent.push_back(make_entry(C.first, C.count, 0, TR_COINCIDENT_REL * (L.rad + C.rad),
                                                 C.c, L.c));
                        ent.back().cell = cidx;
                        rpairs[r] += static_cast<double>(C.count) * L.count;
                    } else {
                        for (int k = C.nchild - 1; k >= 0; --k)
                            stack.push_back(C.child[k]);
                    }
                }
                rcount[bi] = static_cast<int>(ent.size() - e0);
            }
        }
    });
    std::vector<int4> h_tleaf;
    std::vector<TrEntry> h_ent;
    double pairs = 0.0;
    for (long long r = 0; r < nrange; ++r) {
        h_ent.insert(h_ent.end(), rent[r].begin(), rent[r].end());
        pairs += rpairs[r];
    }
    if (h_ent.size() > 0x7fffffffULL) {
        set_error("stokes_tree_create: too many list entries");
        return SBQ_EINVAL;
    }
    {
        long long e0 = 0;
        for (long long bi = 0; bi < nblk; ++bi) {
            h_tleaf.push_back(make_int4(tb[bi].first, tb[bi].count, static_cast<int>(e0), rcount[bi]));
            e0 += rcount[bi];
        }
    }
    // P2M work items: the cells some list takes as far (the others need no proxy charges),
    // their sources in chunks
    std::vector<char> used(S.cells.size(), 0);
    for (const TrEntry &en : h_ent)
        if (en.kind == 1)
            used[en.cell] = 1;
    std::vector<int4> h_chunks;
    for (size_t ci = 0; ci < S.cells.size(); ++ci) {
        if (!used[ci])
            continue;
        const HostCell &c = S.cells[ci];
        for (int b = 0; b < c.count; b += TR_CHUNK)
            h_chunks.push_back(make_int4(static_cast<int>(ci), c.first + b, std::min(TR_CHUNK, c.count - b), 0));
    }
    T->n_cells = static_cast<long long>(S.cells.size());
    T->n_proxies = np;
    T->n_entries = static_cast<long long>(h_ent.size());
    T->n_tleaves = static_cast<long long>(h_tleaf.size());
    T->n_chunks = static_cast<long long>(h_chunks.size());
    T->pairs = pairs;

    SBQ_TRY(T->perm_s.alloc(ns * sizeof(int)));
    SBQ_TRY(T->perm_t.alloc(nt * sizeof(int)));
    SBQ_TRY(T->w_sorted.alloc(ns * sizeof(double)));
    SBQ_TRY(T->src_loc.alloc(ns * sizeof(float4)));
    SBQ_TRY(T->src_abs.alloc(3 * ns * sizeof(double)));
    SBQ_TRY(T->trg_loc.alloc(nt * sizeof(float4)));
    SBQ_TRY(T->trg_lo.alloc(nt * sizeof(float4)));
    SBQ_TRY(T->src_lo.alloc(ns * sizeof(float4)));
    SBQ_CUDA(cudaMemcpyAsync(T->trg_lo.p, h_tlo.data(), nt * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->src_lo.p, h_slo.data(), ns * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBQ_TRY(T->q.alloc(ns * T->nq * sizeof(float4)));
    if (T->nq == 3) {
        SBQ_TRY(T->n_sorted.alloc(3 * ns * sizeof(double)));
        SBQ_CUDA(cudaMemcpyAsync(T->n_sorted.p, h_ns.data(), 3 * ns * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    SBQ_TRY(T->cells.alloc(h_cells.size() * sizeof(TrCellDev)));
    SBQ_TRY(T->prox_loc.alloc(std::max<long long>(np, 1) * sizeof(float4)));
    SBQ_TRY(T->prox_q.alloc(std::max<long long>(np, 1) * T->nq * sizeof(float4)));
    SBQ_TRY(T->chunks.alloc(std::max<size_t>(h_chunks.size(), 1) * sizeof(int4)));
    SBQ_TRY(T->tleaf.alloc(std::max<size_t>(h_tleaf.size(), 1) * sizeof(int4)));
    SBQ_TRY(T->entries.alloc(std::max<size_t>(h_ent.size(), 1) * sizeof(TrEntry)));
    SBQ_CUDA(cudaMemcpyAsync(T->perm_s.p, S.perm.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->perm_t.p, Tt.perm.data(), nt * sizeof(int), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->w_sorted.p, h_ws.data(), ns * sizeof(double), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->src_loc.p, h_sloc.data(), ns * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->src_abs.p, h_sabs.data(), 3 * ns * sizeof(double), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->trg_loc.p, h_tloc.data(), nt * sizeof(float4), cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaMemcpyAsync(T->cells.p, h_cells.data(), h_cells.size() * sizeof(TrCellDev),
                             cudaMemcpyHostToDevice, s));
    if (np > 0)
        SBQ_CUDA(cudaMemcpyAsync(T->prox_loc.p, h_ploc.data(), np * sizeof(float4), cudaMemcpyHostToDevice, s));
    if (!h_chunks.empty())
        SBQ_CUDA(cudaMemcpyAsync(T->chunks.p, h_chunks.data(), h_chunks.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s));
    if (!h_tleaf.empty())
        SBQ_CUDA(cudaMemcpyAsync(T->tleaf.p, h_tleaf.data(), h_tleaf.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s));
    if (!h_ent.empty())
        SBQ_CUDA(cudaMemcpyAsync(T->entries.p, h_ent.data(), h_ent.size() * sizeof(TrEntry),
                                 cudaMemcpyHostToDevice, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

template <int NQ>
static int tree_apply_nq(sbq_tree_s *T, const double *sigma, double *u, cudaStream_t s)
{
    const unsigned g = static_cast<unsigned>((T->ns + 255) / 256);
    k_tree_charges<NQ><<<g, 256, 0, s>>>(T->ns, T->perm_s.as<int>(), T->w_sorted.as<double>(),
                                         T->n_sorted.as<double>(), sigma, T->alpha / (8.0 * TR_PI),
                                         3.0 * T->beta / (4.0 * TR_PI), T->q.as<float4>());
    SBQ_CUDA(cudaGetLastError());
    SBQ_CUDA(cudaMemsetAsync(T->prox_q.p, 0, std::max<long long>(T->n_proxies, 1) * NQ * sizeof(float4), s));
    if (T->n_chunks > 0) {
        k_tree_p2m<NQ><<<static_cast<unsigned>(T->n_chunks), TR_THREADS, 0, s>>>(
            T->chunks.as<int4>(), T->cells.as<TrCellDev>(), T->src_abs.as<double>(), T->ns,
            T->q.as<float4>(), T->prox_q.as<float4>());
        SBQ_CUDA(cudaGetLastError());
    }
    k_tree_eval<NQ><<<static_cast<unsigned>(T->n_tleaves), TR_THREADS, 0, s>>>(
        T->tleaf.as<int4>(), T->entries.as<TrEntry>(), T->trg_loc.as<float4>(), T->src_loc.as<float4>(),
        T->q.as<float4>(), T->prox_loc.as<float4>(), T->prox_q.as<float4>(), T->perm_t.as<int>(), T->nt,
        T->trg_lo.as<float4>(), T->src_lo.as<float4>(), u);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

static int tree_apply_impl(sbq_tree_s *T, const double *sigma, double *u, cudaStream_t s)
{
    if (T->ns == 0 || T->nt == 0) {
        if (T->nt > 0)
            SBQ_CUDA(cudaMemsetAsync(u, 0, 3 * T->nt * sizeof(double), s));
        return SBQ_OK;
    }
    return T->nq == 3 ? tree_apply_nq<3>(T, sigma, u, s) : tree_apply_nq<1>(T, sigma, u, s);
}

// ---- a treecode attached to an operator (engine.h): the operator's K = diag I + D + eta S
// with the pair sum by the treecode, in the caller's node order

__global__ void k_tree_unperm(long long n, const int *__restrict__ perm, const double *__restrict__ in,
                              double *out)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n)
        return;
    const long long o = perm[i];
    for (int d = 0; d < 3; ++d)
        out[d * n + o] = in[d * n + i];
}

__global__ void k_tree_add_diag(long long m, double diag, const double *__restrict__ y, double *out)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < m)
        out[i] += diag * y[i];
}

void tree_op_free(Op *op)
{
    delete static_cast<sbq_tree_s *>(op->tree);
    op->tree = nullptr;
}

static int tree_op_attach_impl(Op *op, double theta, int order, cudaStream_t s)
{
    tree_op_free(op);
    if (theta <= 0.0)
        return SBQ_OK;
    if (op->laplace) {
        set_error("stokes_op_set_tree: the treecode serves the Stokes operator");
        return SBQ_EINVAL;
    }
    if (op->plan.nseg > 1) {
        set_error("stokes_op_set_tree: a batched operator (independent segments) takes no treecode");
        return SBQ_EINVAL;
    }
    if (!(theta < 1.0) || order < 2 || order > 10) {
        set_error("stokes_op_set_tree: theta must be in (0, 1) and order in 2..10");
        return SBQ_EINVAL;
    }
    const long long n = op->n;
    DevBuf src, nrm, w;
    SBQ_TRY(src.alloc(3 * std::max<long long>(n, 1) * sizeof(double)));
    SBQ_TRY(nrm.alloc(3 * std::max<long long>(n, 1) * sizeof(double)));
    SBQ_TRY(w.alloc(std::max<long long>(n, 1) * sizeof(double)));
    if (n > 0) {
        const unsigned g = static_cast<unsigned>((n + 255) / 256);
        k_tree_unperm<<<g, 256, 0, s>>>(n, op->perm.as<int>(), op->src.as<double>(), src.as<double>());
        k_tree_unperm<<<g, 256, 0, s>>>(n, op->perm.as<int>(), op->nrm.as<double>(), nrm.as<double>());
        SBQ_CUDA(cudaGetLastError());
        // weights: one component
        std::vector<int> hp(n);
        std::vector<double> hw(n), hwo(n);
        SBQ_CUDA(cudaMemcpyAsync(hp.data(), op->perm.p, n * sizeof(int), cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaMemcpyAsync(hw.data(), op->w.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaStreamSynchronize(s));
        for (long long i = 0; i < n; ++i)
            hwo[hp[i]] = hw[i];
        SBQ_CUDA(cudaMemcpyAsync(w.p, hwo.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    sbq_tree_s *T = new sbq_tree_s();
    cudaGetDevice(&T->device);
    int st;
    try {
        st = tree_create_impl(n, src.as<double>(), nrm.as<double>(), w.as<double>(), n,
                              src.as<double>(), op->eta, 1.0, theta, order, T, s);
    } catch (...) {
        delete T;
        throw;
    }
    if (st != SBQ_OK) {
        delete T;
        return st;
    }
    op->tree = T;
    return SBQ_OK;
}

int tree_op_attach(Op *op, double theta, int order, cudaStream_t s)
{
    try {   // the host build allocates; nothing may be thrown across the C ABI
        return tree_op_attach_impl(op, theta, order, s);
    } catch (const std::bad_alloc &) {
        set_error("stokes_op_set_tree: out of host memory");
        return SBQ_ENOMEM;
    }
}

int tree_op_apply(Op *op, const double *y, double *out, cudaStream_t s)
{
    sbq_tree_s *T = static_cast<sbq_tree_s *>(op->tree);
    SBQ_TRY(tree_apply_impl(T, y, out, s));
    const long long m = 3 * op->n;
    if (m > 0 && op->diag != 0.0) {
        k_tree_add_diag<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(m, op->diag, y, out);
        SBQ_CUDA(cudaGetLastError());
    }
    return SBQ_OK;
}

}  // namespace sbq

namespace {
int tree_fail(int code, const char *msg)
{
    sbq::set_error(msg);
    return code;
}
}  // namespace

extern "C" __attribute__((visibility("default"))) int stokes_tree_create(
    int64_t ns, const double *src, const double *nrm, const double *w, int64_t nt,
    const double *trg, double alpha, double beta, double theta, int order, sbq_tree_s **out,
    void *stream)
{
    sbq::clear_error();
    if (!out)
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: null out");
    *out = nullptr;
    if (ns < 0 || nt < 0 || ns > 0x3fffffffLL || nt > 0x3fffffffLL)
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: sizes must be in 0..2^30 - 1");
    if ((ns > 0 && (!src || !w)) || (nt > 0 && !trg) || (ns > 0 && beta != 0.0 && !nrm))
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: null pointer");
    if (!std::isfinite(alpha) || !std::isfinite(beta))
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: non-finite alpha or beta");
    if (!(theta > 0.0 && theta < 1.0))
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: theta must be in (0, 1)");
    if (order < 2 || order > 10)
        return tree_fail(SBQ_EINVAL, "stokes_tree_create: order must be in 2..10");
    sbq_tree_s *T = new (std::nothrow) sbq_tree_s();
    if (!T)
        return tree_fail(SBQ_ENOMEM, "stokes_tree_create: out of host memory");
    cudaGetDevice(&T->device);
    int st;
    try {   // the host build allocates; nothing may be thrown across the C ABI
        st = sbq::tree_create_impl(ns, src, nrm, w, nt, trg, alpha, beta, theta, order, T,
                                   static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        st = tree_fail(SBQ_ENOMEM, "stokes_tree_create: out of host memory");
    }
    if (st != SBQ_OK) {
        delete T;
        return st;
    }
    *out = T;
    return SBQ_OK;
}

extern "C" __attribute__((visibility("default"))) int stokes_tree_apply(sbq_tree_s *T,
                                                                           const double *sigma,
                                                                           double *u, void *stream)
{
    sbq::clear_error();
    if (!T || T->magic != 0x53425454u)
        return tree_fail(SBQ_EINVAL, "stokes_tree_apply: not a tree handle");
    if ((T->ns > 0 && !sigma) || (T->nt > 0 && !u))
        return tree_fail(SBQ_EINVAL, "stokes_tree_apply: null pointer");
    return sbq::tree_apply_impl(T, sigma, u, static_cast<cudaStream_t>(stream));
}

extern "C" __attribute__((visibility("default"))) int stokes_tree_stats(const sbq_tree_s *T,
                                                                           double *pairs,
                                                                           int64_t *counts)
{
    sbq::clear_error();
    if (!T || T->magic != 0x53425454u)
        return tree_fail(SBQ_EINVAL, "stokes_tree_stats: not a tree handle");
    if (pairs)
        *pairs = T->pairs;
    if (counts) {
        counts[0] = T->n_cells;
        counts[1] = T->n_proxies;
        counts[2] = T->n_entries;
        counts[3] = T->n_tleaves;
    }
    return SBQ_OK;
}

extern "C" __attribute__((visibility("default"))) int stokes_tree_destroy(sbq_tree_s *T)
{
    sbq::clear_error();
    if (!T)
        return SBQ_OK;
    if (T->magic != 0x53425454u)
        return tree_fail(SBQ_EINVAL, "stokes_tree_destroy: not a tree handle");
    T->magic = 0;
    delete T;
    return SBQ_OK;
}
