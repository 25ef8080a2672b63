// Quadrature correction E of tube elements (paper Sec. 3.2.1-3.2.4, Eq. nystrom-correction).
//
// For every tube node x (an on-surface target) and every element k whose near region holds
// x, the element's uncorrected sum is replaced by an accurate integral over the element:
//   E_ij(x) = sum_m P_mi w^s_m h_j(x, t_m) - G(x, y_ij) w_ij,
// the coincident node left out of the subtracted term (the pair sums leave it out).
//   * geometry: each GL row of an element's nodes lies on a circle y = c_i + a_i cos(theta) +
//     b_i sin(theta) (Eq. surface-coord); c, a, b come from the nodes (Fourier modes 0 and
//     1) and are interpolated in the panel parameter t with the Lagrange basis of the GL
//     nodes;
//   * h_j (Sec. 3.2.2, Eqs. modal-greens-fn-coeff / modal-greens-fn-wts): the modal
//     integrals of G e^{i l theta} J, l = 0..N_theta/2, over a composite Gauss-Legendre rule
//     in theta - theta_0 refined dyadically towards the circle point closest to x until the
//     smallest panel is no longer than the relative distance alpha; then an inverse DFT;
//   * outer rule in t (Sec. 3.2.3 / 3.2.4): dyadic towards the target's own parameter with a
//     rule for p log|t - t0| + q on the panel next to it (own element), or dyadic towards the
//     nearest parameter t* until the panel next to it is no longer than the distance d*.
// For the own element the offsets y - x are formed from exact parameter offsets (partition of
// unity of the Lagrange basis, product formulas for the trigonometric differences), so they
// keep their relative accuracy on the s-nodes that lie within rounding distance of x.
//
// Work decomposition: one 128-thread CTA per (target, near element) item, FP64 throughout.
// The outer rule's s-nodes are taken in batches: one thread per s-node forms the
// interpolation basis, the circle there, the closest angle and the relative distance alpha
// of the target, and picks the angular rule with the fewest nodes among (Sec. 3.2.2):
//   * the periodic trapezoidal rule of M = k N_theta equispaced angles (k = 1 .. 8), with k
//     the smallest whose aliasing bound keeps the error of every mode below ~1e-14 (for
//     far targets, where the paper takes the trapezoidal rule on the N_theta angles
//     themselves); the modal transform and inverse DFT of such a rule collapse to fixed
//     weights D_k[(m - k j) mod M], and these s-nodes go through the CTA 128 / M at a
//     time, one thread per (s-node, node);
//   * the compressed rule of alpha's dyadic level (generalized Chebyshev rules, App. B,
//     compiled into the library), and the dyadically refined Gauss-Legendre rule, each
//     followed by the modal coefficients (a reduction over the rule's nodes) and the
//     inverse DFT, one s-node at a time.
// The first two assume that the area element is resolved by a few modes beyond N_theta / 2;
// at s-nodes where a bound on its complex singularities says otherwise (a bend whose radius
// of curvature nears the tube's radius) the dyadically refined rule is taken.
#include "engine.h"

// compressed angular rules compiled in from rules/angular_l*.txt (kRuleTables, kRuleL0,
// kRuleCnt, kRuleData), written by build.py
#include "angular_rules_tables.inc"
// whole-element singular rules compiled in from rules/singular_ns*_l*.txt (kSingTables, kSingNs,
// kSingL0, kSingLo, kSingHi, kSingCnt, kSingOff, kSingData), written by build.py
#include "singular_rules_tables.inc"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace sbq {

namespace {

constexpr int TQ_THREADS = 128;
constexpr int TQ_Q = 16;           // GL nodes per panel (angular and outer rules)
constexpr int TQ_SING_N = 24;      // log-singular rule: GL in u after t = u^6
constexpr int TQ_SING_G = 6;
constexpr double TQ_SING_TURN = 0.2;  // largest tangent turning (rad) of an element that
                                      // takes a whole-element singular rule
constexpr int TQ_LMAX = 60;        // deepest dyadic level
constexpr int TQ_NS_MAX = 16;
constexpr int TQ_REFINE = 3;       // rounds of 128-point refinement of t*: bracket ~2e-7
constexpr int TQ_PARAB = 3;        // then parabolic rounds on the squared distance
constexpr int TQ_RULE_SLOT = 128;  // nodes reserved per level of a compressed angular rule
constexpr int TQ_RULE_MAXLEV = 52; // compressed rules serve levels 0..52: 2^-52 <= alpha < 2
static_assert(kRuleLevels == TQ_RULE_MAXLEV + 1, "compiled-in rule tables and TQ_RULE_MAXLEV disagree");
constexpr int TQ_SB = 64;          // s-nodes per batch
constexpr int TQ_TRAP_KMAX = 8;    // trapezoidal angular rules of k N_theta nodes, k <= 8
// aliasing bound of the trapezoidal rule: its error on G e^{i l theta} decays like
// exp(-a (M - l)), a = acosh(1 + alpha^2 / (2 (1 + alpha))) the distance of the nearest
// complex singularity of G(x, y(theta)) from the real axis (target in the circle's plane,
// outside it: the worst position at relative distance alpha); M - l0 >= TQ_TRAP_LOG / a
// keeps it below e^-TQ_TRAP_LOG ~ 1e-14
constexpr double TQ_TRAP_LOG = 32.3;
// The area element J = |y_theta x y_t| has its own complex singularities: the zeros of J^2, a
// trigonometric polynomial of degree 4, which approach the real axis where the tube bends
// with a radius of curvature close to its own radius.  Both faster rules assume J is resolved
// by a few modes beyond N_theta / 2 (the premise of the paper's angular rules); where the
// width a_g of J^2's zero-free strip is small that premise fails and the dyadically refined
// rule is kept.  The trapezoidal rule takes a = min(a, a_g) in its bound and needs a_g >=
// TQ_GEOM_TRAP; the compressed rules (modes l <= N_theta / 2 + 4 of the circle's kernel) need
// a_g >= TQ_GEOM_TABLE.  Thresholds from a sweep of a random slender loop's sharpest bend:
// above them the dyadic rule and the compressed rule agree with a converged trapezoidal
// reference (M = 512) to ~1e-13.
constexpr double TQ_GEOM_TRAP = 1.0;
constexpr double TQ_GEOM_TABLE = 2.0;

// reach sphere of an element: centre and radius
struct Reach {
    double x, y, z, r;
};

struct ElemGeo {
    double c[3][TQ_NS_MAX], a[3][TQ_NS_MAX], b[3][TQ_NS_MAX];
    double cl[3][TQ_NS_MAX + 2];   // centreline samples: c_i and C(-1), C(+1)
    double rho_max, speed_max, sgn, pad;
    double ag[33];                 // strip width a_g of J^2's zeros at t = -1 + q / 16
    double spd[TQ_NS_MAX];         // |C'(t_i)|: the centreline's speed at the GL nodes
    double rho[TQ_NS_MAX];         // radius of row i
    double turn;                   // turning angle of the centreline's tangent over [-1, 1]
};
constexpr int TQ_AG_N = 33;

struct TQParams {
    double tn[TQ_NS_MAX];                  // element GL nodes on [-1, 1]
    double invd[TQ_NS_MAX][TQ_NS_MAX];     // 1 / (tn_i - tn_k), 0 on the diagonal
    double gx[TQ_Q], gw[TQ_Q];             // GL on [0, 1]
    double sx[TQ_SING_N], sw[TQ_SING_N];   // singular rule on [0, 1]
    double alpha, beta;
    long long ntot;
    int ns, nt, per;
    // compressed angular rules: level lev (alpha in [2^-lev, 2^(1-lev)), 0 <= lev < rnlev)
    // holds rcnt[lev] <= TQ_RULE_SLOT nodes rphi[lev * TQ_RULE_SLOT + m], weights rw[...]
    const double *rphi, *rw;
    const int *rcnt;
    int rnlev;
    // trapezoidal rules of M = k N_theta nodes at the angles 2 pi m / M: the weights that
    // map the M integrand values to h_j (Eq. modal-greens-fn-wts composed with Eq.
    // modal-greens-fn-coeff on that grid) depend on (m - k j) mod M only:
    // dtab[N_theta k (k - 1) / 2 + q], q < k N_theta
    const double *dtab;
    int kmax;
    // whole-element singular rules (Sec. 3.2.4) for own-element targets: for aspect level
    // b (2 |C'(t_i0)| / radius_i0 in [2^b, 2^(b+1)), slo <= b <= shi) and position i0, scnt[(b -
    // slo) ns + i0] nodes from soff[...]: offsets sdel (t - t_i0) and weights swt; scnt null:
    // none (dyadic panels and the graded panel next to t0 instead)
    const int *scnt, *soff;
    const double *sdel, *swt;
    int slo, shi;
};

struct Item {
    int t, k, slot, pad;
};

// ---------------------------------------------------------------------------------------
// Lagrange basis of the GL nodes (product form)

__device__ __forceinline__ double lag(const double *tn, int ns, int i, double t)
{
    double v = 1.0;
    for (int k = 0; k < ns; ++k)
        if (k != i)
            v *= (t - tn[k]) / (tn[i] - tn[k]);
    return v;
}

__device__ __forceinline__ double dlag(const double *tn, int ns, int i, double t)
{
    double s = 0.0;
    for (int m = 0; m < ns; ++m) {
        if (m == i)
            continue;
        double v = 1.0 / (tn[i] - tn[m]);
        for (int k = 0; k < ns; ++k)
            if (k != i && k != m)
                v *= (t - tn[k]) / (tn[i] - tn[k]);
        s += v;
    }
    return s;
}

__device__ __forceinline__ double dot3(const double *u, const double *v)
{
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

// Kernel components: Stokes (6: xx yy zz xy xz yz of the symmetric 3 x 3) or Laplace (1).
template <int NC>
__device__ __forceinline__ void kern(const double r[3], const double n[3], double alpha,
                                     double beta, double K[NC])
{
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double ri = rsqrt(r2);
    const double rn = r[0] * n[0] + r[1] * n[1] + r[2] * n[2];
    constexpr double PI_ = 3.14159265358979323846;
    if (NC == 1) {
        K[0] = alpha * ri / (4.0 * PI_) + beta * rn * ri * ri * ri / (4.0 * PI_);
    } else {
        const double ri3 = ri * ri * ri;
        const double s1 = alpha / (8.0 * PI_);
        const double f = s1 * ri3 + beta * 3.0 / (4.0 * PI_) * rn * ri3 * ri * ri;
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int c = 0; c < NC; ++c)
            K[c] = f * r[ia[c]] * r[ib[c]] + (c < 3 ? s1 * ri : 0.0);
    }
}

__device__ __forceinline__ int dyadic_levels(double phys, double scale)
{
    if (phys <= scale)
        return 0;
    if (scale <= 0.0)
        return TQ_LMAX;
    return min(TQ_LMAX, static_cast<int>(ceil(log2(phys / scale))));
}

// ---------------------------------------------------------------------------------------
// element geometry: one thread per element

__global__ void k_elem_setup(long long nelem, TQParams p, const double *__restrict__ src,
                             const double *__restrict__ nrm, ElemGeo *geo, int *bad)
{
    const long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (k >= nelem)
        return;
    const int ns = p.ns, nt = p.nt;
    const long long N = p.ntot, base = k * p.per;
    ElemGeo &g = geo[k];
    double rho_max = 0.0, dev = 0.0;
    for (int i = 0; i < ns; ++i) {
        double c[3] = {0, 0, 0}, a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
        for (int j = 0; j < nt; ++j) {
            double sn, cs;
            sincospi(2.0 * j / nt, &sn, &cs);
            for (int d = 0; d < 3; ++d) {
                const double y = src[d * N + base + i * nt + j];
                c[d] += y;
                a[d] += y * cs;
                b[d] += y * sn;
            }
        }
        for (int d = 0; d < 3; ++d) {
            g.c[d][i] = c[d] / nt;
            g.a[d][i] = 2.0 * a[d] / nt;
            g.b[d][i] = 2.0 * b[d] / nt;
        }
        const double rho = sqrt(0.5 * (g.a[0][i] * g.a[0][i] + g.a[1][i] * g.a[1][i] + g.a[2][i] * g.a[2][i]
                                       + g.b[0][i] * g.b[0][i] + g.b[1][i] * g.b[1][i] + g.b[2][i] * g.b[2][i]));
        rho_max = fmax(rho_max, rho);
        for (int j = 0; j < nt; ++j) {
            double sn, cs;
            sincospi(2.0 * j / nt, &sn, &cs);
            for (int d = 0; d < 3; ++d)
                dev = fmax(dev, fabs(g.c[d][i] + g.a[d][i] * cs + g.b[d][i] * sn
                                     - src[d * N + base + i * nt + j]));
        }
    }
    if (!(dev <= 1e-9 * rho_max))
        atomicExch(bad, 1);
    double speed = 0.0;
    for (int i = 0; i < ns; ++i) {
        double v[3] = {0, 0, 0};
        for (int m = 0; m < ns; ++m) {
            const double dl = dlag(p.tn, ns, m, p.tn[i]);
            for (int d = 0; d < 3; ++d)
                v[d] += dl * g.c[d][m];
        }
        g.spd[i] = sqrt(dot3(v, v));
        g.rho[i] = sqrt(0.5 * (g.a[0][i] * g.a[0][i] + g.a[1][i] * g.a[1][i] + g.a[2][i] * g.a[2][i]
                               + g.b[0][i] * g.b[0][i] + g.b[1][i] * g.b[1][i] + g.b[2][i] * g.b[2][i]));
        speed = fmax(speed, g.spd[i]);
    }
    // tangent turning between consecutive GL nodes, scaled from [t_0, t_ns-1] to [-1, 1]
    double turn = 0.0, tprev[3] = {0, 0, 0};
    for (int i = 0; i < ns; ++i) {
        double v[3] = {0, 0, 0};
        for (int m = 0; m < ns; ++m) {
            const double dl = dlag(p.tn, ns, m, p.tn[i]);
            for (int d = 0; d < 3; ++d)
                v[d] += dl * g.c[d][m];
        }
        const double inv = 1.0 / sqrt(dot3(v, v));
        for (int d = 0; d < 3; ++d)
            v[d] *= inv;
        if (i > 0) {
            const double cr[3] = {tprev[1] * v[2] - tprev[2] * v[1], tprev[2] * v[0] - tprev[0] * v[2],
                                  tprev[0] * v[1] - tprev[1] * v[0]};
            turn += atan2(sqrt(dot3(cr, cr)), dot3(tprev, v));
        }
        for (int d = 0; d < 3; ++d)
            tprev[d] = v[d];
    }
    g.turn = turn * 2.0 / (p.tn[ns - 1] - p.tn[0]);
    // orientation: sign of (y_theta x y_t) . n at node (0, 0): y_theta = b_0, y_t = C'(t_0) + A'(t_0)
    double yt[3] = {0, 0, 0}, yth[3];
    for (int m = 0; m < ns; ++m) {
        const double dl = dlag(p.tn, ns, m, p.tn[0]);
        for (int d = 0; d < 3; ++d)
            yt[d] += dl * (g.c[d][m] + g.a[d][m]);
    }
    for (int d = 0; d < 3; ++d)
        yth[d] = g.b[d][0];
    const double cr[3] = {yth[1] * yt[2] - yth[2] * yt[1], yth[2] * yt[0] - yth[0] * yt[2],
                          yth[0] * yt[1] - yth[1] * yt[0]};
    const double n0[3] = {nrm[base], nrm[N + base], nrm[2 * N + base]};
    g.sgn = dot3(cr, n0) >= 0.0 ? 1.0 : -1.0;
    g.rho_max = rho_max;
    g.speed_max = speed;
    for (int i = 0; i < ns; ++i)
        for (int d = 0; d < 3; ++d)
            g.cl[d][i] = g.c[d][i];
    for (int e = 0; e < 2; ++e) {
        const double te = e ? 1.0 : -1.0;
        for (int d = 0; d < 3; ++d) {
            double v = 0.0;
            for (int m = 0; m < ns; ++m)
                v += lag(p.tn, ns, m, te) * g.c[d][m];
            g.cl[d][ns + e] = v;
        }
    }
}

// Near region of element k (the approximation of Sec. 3.2.1 by spheres around samples):
// closer than radius + f max(length, 2 radius) to a centreline sample.
__device__ __forceinline__ bool is_near(const ElemGeo &g, int ns, const double x[3], double f)
{
    double d2 = 1e300;
    for (int i = 0; i < ns + 2; ++i) {
        const double dx = x[0] - g.cl[0][i], dy = x[1] - g.cl[1][i], dz = x[2] - g.cl[2][i];
        d2 = fmin(d2, dx * dx + dy * dy + dz * dz);
    }
    const double lim = g.rho_max + f * fmax(2.0 * g.speed_max, 2.0 * g.rho_max);
    return lim > 0.0 && d2 < lim * lim;
}

// Reach sphere of an element: centre = mean of its centreline samples, radius = the largest
// distance of a sample from it plus the near-region radius.  Every target near the element
// (is_near) lies inside it.
__global__ void k_elem_reach(long long nelem, int ns, double f, const ElemGeo *__restrict__ geo,
                             Reach *reach)
{
    const long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (k >= nelem)
        return;
    const ElemGeo &g = geo[k];
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < ns + 2; ++i)
        for (int d = 0; d < 3; ++d)
            c[d] += g.cl[d][i];
    for (int d = 0; d < 3; ++d)
        c[d] /= (ns + 2);
    double r2 = 0.0;
    for (int i = 0; i < ns + 2; ++i) {
        const double dx = g.cl[0][i] - c[0], dy = g.cl[1][i] - c[1], dz = g.cl[2][i] - c[2];
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
    }
    const double lim = g.rho_max + f * fmax(2.0 * g.speed_max, 2.0 * g.rho_max);
    reach[k] = Reach{c[0], c[1], c[2], sqrt(r2) + fmax(lim, 0.0)};
}

// Spatial grid of the element reach spheres (the near search of Sec. 3.3, in place of a
// brute-force pass over all pairs): cells of side h >= the largest reach radius, elements
// sorted by the Morton key of the cell holding their centre; a target meets only the
// elements of the 27 cells around its own.
struct NearGrid {
    double lo[3];
    double inv_h;
    int dim;                                   // cells per axis (power of two, <= 2^21)
    const unsigned long long *keys;            // sorted Morton keys, one per element
    const int *elem;                           // element of each sorted key
    long long nelem;
};

__host__ __device__ inline unsigned long long morton_spread(unsigned v)
{
    unsigned long long x = v & 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

__host__ __device__ inline unsigned long long morton_key(int ix, int iy, int iz)
{
    return morton_spread(static_cast<unsigned>(ix)) | (morton_spread(static_cast<unsigned>(iy)) << 1)
           | (morton_spread(static_cast<unsigned>(iz)) << 2);
}

__device__ __forceinline__ long long lower_bound_key(const unsigned long long *keys, long long n,
                                                     unsigned long long k)
{
    long long a = 0, b = n;
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (keys[m] < k)
            a = m + 1;
        else
            b = m;
    }
    return a;
}

// Targets: the tube nodes (trg == nullptr; each has its own element) or an array of
// off-surface points trg (SoA, ntarget points, no own element).  Pass 1 (off == nullptr)
// counts each target's near elements, pass 2 writes them, in increasing element order.
__global__ void k_near(long long ntarget, TQParams p, double f, const double *__restrict__ src,
                       const double *__restrict__ trg, const ElemGeo *__restrict__ geo,
                       NearGrid grid, const long long *__restrict__ off, int *out)
{
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (t >= ntarget)
        return;
    double x[3];
    long long own = -1;
    if (trg) {
        x[0] = trg[t];
        x[1] = trg[ntarget + t];
        x[2] = trg[2 * ntarget + t];
    } else {
        x[0] = src[t];
        x[1] = src[p.ntot + t];
        x[2] = src[2 * p.ntot + t];
        own = t / p.per;
    }
    int ic[3];
    bool inside = true;
    for (int d = 0; d < 3; ++d) {
        const double u = (x[d] - grid.lo[d]) * grid.inv_h;
        if (!(u > -2.0 && u < grid.dim + 1.0))
            inside = false;
        ic[d] = inside ? static_cast<int>(floor(u)) : 0;
    }
    int c = 0;
    // the own element first if it precedes every near element, else in order: collect in
    // increasing element index by a merge over the candidates (few per target)
    int cand[64];
    int nc = 0;
    bool overflow = false;
    if (inside) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int jx = ic[0] + dx, jy = ic[1] + dy, jz = ic[2] + dz;
                    if (jx < 0 || jy < 0 || jz < 0 || jx >= grid.dim || jy >= grid.dim || jz >= grid.dim)
                        continue;
                    const unsigned long long key = morton_key(jx, jy, jz);
                    for (long long q = lower_bound_key(grid.keys, grid.nelem, key);
                         q < grid.nelem && grid.keys[q] == key; ++q) {
                        const int k = grid.elem[q];
                        if (k == own || !is_near(geo[k], p.ns, x, f))
                            continue;
                        if (nc < 64)
                            cand[nc++] = k;
                        else
                            overflow = true;
                    }
                }
    }
    if (own >= 0) {
        bool has = false;
        for (int q = 0; q < nc; ++q)
            has = has || cand[q] == own;
        if (!has && nc < 64)
            cand[nc++] = static_cast<int>(own);
        else if (!has)
            overflow = true;
    }
    // insertion sort: rows list their near elements in increasing order
    for (int a = 1; a < nc; ++a) {
        const int v = cand[a];
        int b = a - 1;
        while (b >= 0 && cand[b] > v) {
            cand[b + 1] = cand[b];
            --b;
        }
        cand[b + 1] = v;
    }
    if (overflow) {
        // more than 64 near elements: a linear pass over the grid's elements in index order
        // (rare: elements much shorter than their near region)
        c = 0;
        for (long long k = 0; k < grid.nelem; ++k) {
            if (k == own || is_near(geo[k], p.ns, x, f)) {
                if (off)
                    out[off[t] + c] = static_cast<int>(k);
                ++c;
            }
        }
        if (!off)
            out[t] = c;
        return;
    }
    c = nc;
    if (off)
        for (int q = 0; q < nc; ++q)
            out[off[t] + q] = cand[q];
    else
        out[t] = c;
}

// ---------------------------------------------------------------------------------------
// the correction blocks

// Lagrange basis of the GL nodes and its derivative at t, by products with the precomputed
// reciprocals 1 / (t_i - t_k) (no division): with b_k = (t - t_k) / (t_i - t_k),
//   l_i(t) = prod_{k != i} b_k,   l_i'(t) = sum_{m != i} 1 / (t_i - t_m) prod_{k != i, m} b_k,
// the partial products from a suffix array and a running prefix.  own: for i != i0, l_i from
// the exact offset delta = t - t_i0 (the factor k = i0 is delta itself, the others
// (t_i0 - t_k) + delta), so that l_i keeps its relative accuracy for tiny delta; l_i0 is set
// by the caller from the partition of unity.
__device__ __forceinline__ void basis_at(const TQParams &p, int ns, double t, bool own, int i0,
                                         double delta, double *L, double *dL)
{
    for (int i = 0; i < ns; ++i) {
        double suf[TQ_NS_MAX + 1];
        suf[ns] = 1.0;
        for (int k = ns - 1; k >= 0; --k)
            suf[k] = suf[k + 1] * (k == i ? 1.0 : (t - p.tn[k]) * p.invd[i][k]);
        double pre = 1.0, d = 0.0;
        for (int m = 0; m < ns; ++m) {
            if (m == i)
                continue;
            d += p.invd[i][m] * pre * suf[m + 1];
            pre *= (t - p.tn[m]) * p.invd[i][m];
        }
        dL[i] = d;
        if (own) {
            double v = 1.0;
            for (int k = 0; k < ns; ++k) {
                if (k == i)
                    continue;
                v *= (k == i0 ? delta : (p.tn[i0] - p.tn[k]) + delta) * p.invd[i][k];
            }
            L[i] = (i == i0) ? 0.0 : v;
        } else {
            L[i] = pre;
        }
    }
}

// l_i(t) alone (the nearest-parameter search).
__device__ __forceinline__ double lag_fast(const TQParams &p, int ns, int i, double t)
{
    double v = 1.0;
    for (int k = 0; k < ns; ++k)
        if (k != i)
            v *= (t - p.tn[k]) * p.invd[i][k];
    return v;
}

// Per s-node geometry in shared memory: C A B (circle at t), C' A' B' (their t-derivatives),
// dC dA dB (own element: sum_{i != i0} l_i (v_i - v_i0), the exact offsets from row i0).
constexpr int SG_STRIDE = 27;

// cos and sin of l theta, l = 1..4, from those of theta
__device__ __forceinline__ void trig_multiples(double c1, double s1, double cs[4], double sn[4])
{
    cs[0] = c1;
    sn[0] = s1;
    cs[1] = 2.0 * c1 * c1 - 1.0;
    sn[1] = 2.0 * s1 * c1;
    cs[2] = cs[1] * c1 - sn[1] * s1;
    sn[2] = sn[1] * c1 + cs[1] * s1;
    cs[3] = 2.0 * cs[1] * cs[1] - 1.0;
    sn[3] = 2.0 * sn[1] * cs[1];
}

// min over 64 real theta of Re J^2(theta + i y) = p0 + sum_l (re_l cos l theta + im_l sin l
// theta) cosh(l y)
__device__ double strip_re_min(double p0, const double re[4], const double im[4], double y)
{
    const double e = exp(y), ei = 1.0 / e;
    double ch[4], el = e, eil = ei;
    for (int l = 0; l < 4; ++l) {
        ch[l] = 0.5 * (el + eil);
        el *= e;
        eil *= ei;
    }
    double m = 1e300;
    for (int q = 0; q < 64; ++q) {
        double sn1, cs1, cs[4], sn[4];
        sincospi(q / 32.0, &sn1, &cs1);
        trig_multiples(cs1, sn1, cs, sn);
        double v = p0;
        for (int l = 0; l < 4; ++l)
            v += (re[l] * cs[l] + im[l] * sn[l]) * ch[l];
        m = fmin(m, v);
    }
    return m;
}

// Width a_g of a strip |Im theta| < a_g free of zeros of J^2 = |y_theta x y_t|^2, for the
// circle y = C + A cos + B sin at parameter t (G[3..8] = A, B; G[9..17] = C_t, A_t, B_t).
// J^2 = p0 + sum_{l=1..4} (re_l cos l theta + im_l sin l theta) exactly (16 samples resolve
// it).  A zero at theta + i y needs Re J^2(theta + i y) = 0, so J^2 has none at height y while
// min_theta Re J^2(theta + i y) > 0.  Start: the strip in which sum_l |p_l| (e^{l y} - 1) stays
// below min J^2 on the real line (zero-free by the triangle inequality); then raised in steps
// of 1.2 while the real-part test holds at the next height, and bisected.  For a circular
// torus of aspect e the exact distance is acosh(1 / e); this gives 0.84 of it at e = 0.25.
__device__ double geom_strip(const double *G)
{
    constexpr int NQ = 16;
    double p0 = 0.0, re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0}, c[4];
    for (int q = 0; q < NQ; ++q) {
        double sn1, cs1;
        sincospi(q / 8.0, &sn1, &cs1);
        double yth[3], yt[3];
        for (int d = 0; d < 3; ++d) {
            yth[d] = -G[3 + d] * sn1 + G[6 + d] * cs1;
            yt[d] = G[9 + d] + G[12 + d] * cs1 + G[15 + d] * sn1;
        }
        const double c0 = yth[1] * yt[2] - yth[2] * yt[1];
        const double c1 = yth[2] * yt[0] - yth[0] * yt[2];
        const double c2 = yth[0] * yt[1] - yth[1] * yt[0];
        const double j2 = c0 * c0 + c1 * c1 + c2 * c2;
        double cs[4], sn[4];
        trig_multiples(cs1, sn1, cs, sn);
        p0 += j2;
        for (int l = 0; l < 4; ++l) {
            re[l] += j2 * cs[l];
            im[l] += j2 * sn[l];
        }
    }
    p0 /= NQ;
    for (int l = 0; l < 4; ++l) {
        re[l] *= 2.0 / NQ;
        im[l] *= 2.0 / NQ;
        c[l] = sqrt(re[l] * re[l] + im[l] * im[l]);
    }
    const double m = strip_re_min(p0, re, im, 0.0);
    if (!(m > 0.0))
        return 0.0;
    constexpr double YMAX = 12.0;
    // largest z = e^y with sum_l c_l (z^l - 1) <= m, by bisection on [1, e^YMAX]
    double lo = 1.0, hi = exp(YMAX);
    for (int it = 0; it < 48; ++it) {
        const double z = 0.5 * (lo + hi);
        const double z2 = z * z;
        const double f = c[0] * (z - 1.0) + c[1] * (z2 - 1.0) + c[2] * (z2 * z - 1.0)
                         + c[3] * (z2 * z2 - 1.0);
        if (f > m)
            hi = z;
        else
            lo = z;
    }
    double y = fmax(log(lo), 1e-3);
    while (y < YMAX && strip_re_min(p0, re, im, 1.2 * y) > 0.0)
        y *= 1.2;
    if (y >= YMAX)
        return YMAX;
    double ylo = y, yhi = 1.2 * y;
    for (int it = 0; it < 24; ++it) {
        const double ym = 0.5 * (ylo + yhi);
        if (strip_re_min(p0, re, im, ym) > 0.0)
            ylo = ym;
        else
            yhi = ym;
    }
    return ylo;
}

// a_g at the TQ_AG_N parameters t = -1 + 2 q / (TQ_AG_N - 1) of every element: one thread
// per (element, sample)
__global__ void k_elem_strip(long long nelem, TQParams p, ElemGeo *geo)
{
    const long long gi = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (gi >= nelem * TQ_AG_N)
        return;
    const long long k = gi / TQ_AG_N;
    const int q = static_cast<int>(gi % TQ_AG_N);
    const int ns = p.ns;
    const double t = -1.0 + 2.0 * q / (TQ_AG_N - 1);
    double L[TQ_NS_MAX], dL[TQ_NS_MAX];
    basis_at(p, ns, t, false, 0, 0.0, L, dL);
    ElemGeo &g = geo[k];
    double G[18];
    for (int d = 0; d < 3; ++d) {
        double a = 0.0, b = 0.0, ct = 0.0, at = 0.0, bt = 0.0;
        for (int i = 0; i < ns; ++i) {
            a += L[i] * g.a[d][i];
            b += L[i] * g.b[d][i];
            ct += dL[i] * g.c[d][i];
            at += dL[i] * g.a[d][i];
            bt += dL[i] * g.b[d][i];
        }
        G[d] = 0.0;
        G[3 + d] = a;
        G[6 + d] = b;
        G[9 + d] = ct;
        G[12 + d] = at;
        G[15 + d] = bt;
    }
    g.ag[q] = geom_strip(G);
}

// a_g near parameter t: the smallest of the four samples around it
__device__ __forceinline__ double strip_at(const ElemGeo &g, double t)
{
    const int i = min(TQ_AG_N - 2, max(0, static_cast<int>(floor((t + 1.0) * 0.5 * (TQ_AG_N - 1)))));
    return fmin(fmin(g.ag[max(i - 1, 0)], g.ag[i]), fmin(g.ag[i + 1], g.ag[min(i + 2, TQ_AG_N - 1)]));
}

// y - x, the unit normal and J at one angle of the circle at an s-node, and the kernel times
// J times the angular weight om.  cs, sn: cos and sin of the angle; own: dcos, dsin are
// cos(angle) - cos(theta_j0) and sin(angle) - sin(theta_j0) formed from half-angle
// products, a0, b0 the circle coefficients of row i0.
template <int NC>
__device__ __forceinline__ void node_value(const double *G, bool own, const double *a0,
                                           const double *b0, const double x[3], double cs,
                                           double sn, double dcos, double dsin, double sgn,
                                           double alpha, double beta, double om, double out[NC])
{
    double ymx[3], yt[3], yth[3];
    for (int d = 0; d < 3; ++d) {
        if (own)
            ymx[d] = G[18 + d] + G[21 + d] * cs + a0[d] * dcos + G[24 + d] * sn + b0[d] * dsin;
        else
            ymx[d] = G[d] + G[3 + d] * cs + G[6 + d] * sn - x[d];
        yt[d] = G[9 + d] + G[12 + d] * cs + G[15 + d] * sn;
        yth[d] = -G[3 + d] * sn + G[6 + d] * cs;
    }
    const double cr[3] = {yth[1] * yt[2] - yth[2] * yt[1], yth[2] * yt[0] - yth[0] * yt[2],
                          yth[0] * yt[1] - yth[1] * yt[0]};
    const double J2 = dot3(cr, cr);
    const double invJ = rsqrt(J2);
    const double J = J2 * invJ;
    const double inv = sgn * invJ;
    const double nn[3] = {cr[0] * inv, cr[1] * inv, cr[2] * inv};
    const double r[3] = {-ymx[0], -ymx[1], -ymx[2]};
    double K[NC];
    kern<NC>(r, nn, alpha, beta, K);
    const double jw = J * om;
#pragma unroll
    for (int c = 0; c < NC; ++c)
        out[c] = K[c] * jw;
}

struct Smem {
    double *sc, *sa, *sb;      // [3][ns] each: circle coefficients of the element's rows
    double *SG;                // [SB][27] per s-node geometry
    double *SP;                // [SB][ns] outer weight times the interpolation basis
    double *SX;                // [SB][2] closest angle (own: offset from theta_j0), alpha
    double *V;                 // [128][NC] integrand values of one chunk of angular nodes
    double *CS;                // [128][MO][2] e^{i l theta} of those nodes
    double *RED;               // [256]
    double *HH;                // [NC][MO][2] modal coefficients
    double *W;                 // [2 nt][2] cos, sin of pi q / nt
    double *H;                 // [NC][nt] angular weights h_j
    double *H2;                // [128 / nt][NC][nt] angular weights of a chunk of s-nodes
    double *EB;                // [NC][ns][nt] element block
    double *SD;                // [128] scratch (nearest-parameter search)
    int *MODE;                 // [SB] -k trapezoid of k N_theta nodes, 0 dyadic, lev + 1
                               // compressed rule lev
    int *CNT;                  // [SB] angular nodes (dyadic: levels in DLEV)
    int *DLEV;                 // [SB]
    int *LT, *LM;              // [SB] trapezoid and modal s-node lists
    int *NL;                   // [4] list lengths
};

__host__ __device__ inline size_t tq_smem_doubles(int NC, int ns, int nt)
{
    const int MO = nt / 2 + 1;
    return 9 * ns + static_cast<size_t>(SG_STRIDE + ns + 2) * TQ_SB + 128 * NC + 128 * MO * 2
           + 256 + NC * MO * 2 + 4 * nt + NC * nt + 128 * NC + static_cast<size_t>(NC) * ns * nt
           + 128 + (5 * TQ_SB + 4 + 1) / 2 + 2;
}

template <int NC>
__global__ void __launch_bounds__(TQ_THREADS)
k_tube_items(TQParams p, const Item *__restrict__ items, const ElemGeo *__restrict__ geo,
             const double *__restrict__ src, const double *__restrict__ nrm,
             const double *__restrict__ wgt, const double *__restrict__ trg, long long ntarget,
             const int64_t *__restrict__ rowptr, int64_t *__restrict__ col,
             double *__restrict__ val)
{
    extern __shared__ double sm[];
    const int tid = threadIdx.x;
    const int ns = p.ns, nt = p.nt, per = p.per, MO = nt / 2 + 1;
    const long long N = p.ntot;
    Smem s;
    {
        double *q = sm;
        s.sc = q; q += 3 * ns;
        s.sa = q; q += 3 * ns;
        s.sb = q; q += 3 * ns;
        s.SG = q; q += SG_STRIDE * TQ_SB;
        s.SP = q; q += ns * TQ_SB;
        s.SX = q; q += 2 * TQ_SB;
        s.V = q; q += 128 * NC;
        s.CS = q; q += 128 * MO * 2;
        s.RED = q; q += 256;
        s.HH = q; q += NC * MO * 2;
        s.W = q; q += 4 * nt;
        s.H = q; q += NC * nt;
        s.H2 = q; q += 128 * NC;
        s.EB = q; q += NC * ns * nt;
        s.SD = q; q += 128;
        int *qi = reinterpret_cast<int *>(q);
        s.MODE = qi; qi += TQ_SB;
        s.CNT = qi; qi += TQ_SB;
        s.DLEV = qi; qi += TQ_SB;
        s.LT = qi; qi += TQ_SB;
        s.LM = qi; qi += TQ_SB;
        s.NL = qi;
    }
    const Item it = items[blockIdx.x];
    const ElemGeo &g = geo[it.k];
    for (int e = tid; e < 3 * ns; e += TQ_THREADS) {
        const int d = e / ns, i = e % ns;
        s.sc[e] = g.c[d][i];
        s.sa[e] = g.a[d][i];
        s.sb[e] = g.b[d][i];
    }
    for (int q = tid; q < 2 * nt; q += TQ_THREADS) {
        double sn, cs;
        sincospi(static_cast<double>(q) / nt, &sn, &cs);
        s.W[2 * q] = cs;
        s.W[2 * q + 1] = sn;
    }
    for (int e = tid; e < NC * ns * nt; e += TQ_THREADS)
        s.EB[e] = 0.0;
    // rows: component-major over the targets (the nodes: stride N; off-surface: ntarget)
    const long long RS = trg ? ntarget : N;
    const double x[3] = {trg ? trg[it.t] : src[it.t], trg ? trg[ntarget + it.t] : src[N + it.t],
                         trg ? trg[2 * ntarget + it.t] : src[2 * N + it.t]};
    const bool own = !trg && (it.t / per) == it.k;
    const int i0 = own ? (it.t % per) / nt : 0, j0 = own ? it.t % nt : 0;
    const double sgn = g.sgn, rho_max = g.rho_max, speed = g.speed_max;
    constexpr double PI_ = 3.14159265358979323846;
    const double thj0 = 2.0 * PI_ * j0 / nt;
    double sj0, cj0;
    sincospi(2.0 * j0 / nt, &sj0, &cj0);
    __syncthreads();

    // ---- nearest parameter t* of an element that does not hold x: sampling, grid refinement,
    // then parabolic refinement of the squared distance (smooth at its minimum even where
    // the distance itself is not)
    double t0 = own ? p.tn[i0] : 0.0, dstar = 0.0;
    if (!own) {
        // distance from x to the circle at parameter tt (closest angle by Newton)
        auto dist_at = [&](double tt) {
            double C[3] = {0, 0, 0}, A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
            for (int i = 0; i < ns; ++i) {
                const double l = lag_fast(p, ns, i, tt);
                for (int d = 0; d < 3; ++d) {
                    C[d] += l * s.sc[d * ns + i];
                    A[d] += l * s.sa[d * ns + i];
                    B[d] += l * s.sb[d * ns + i];
                }
            }
            const double dx[3] = {x[0] - C[0], x[1] - C[1], x[2] - C[2]};
            double th = atan2(dot3(dx, B), dot3(dx, A));
            for (int itn = 0; itn < 3; ++itn) {
                double sn, cs;
                sincos(th, &sn, &cs);
                double ymx[3], yth[3], ythth[3];
                for (int d = 0; d < 3; ++d) {
                    ymx[d] = C[d] + A[d] * cs + B[d] * sn - x[d];
                    yth[d] = -A[d] * sn + B[d] * cs;
                    ythth[d] = -A[d] * cs - B[d] * sn;
                }
                const double fp = dot3(yth, yth) + dot3(ymx, ythth);
                if (fp <= 0.0)
                    break;
                th -= dot3(ymx, yth) / fp;
            }
            double sn, cs;
            sincos(th, &sn, &cs);
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double v = C[d] + A[d] * cs + B[d] * sn - x[d];
                r2 += v * v;
            }
            return sqrt(r2);
        };
        double lo = -1.0, hi = 1.0, best_t = 0.0, best_d = 1e300;
        for (int round = 0; round <= TQ_REFINE; ++round) {
            const int np = round == 0 ? 65 : 128;
            double dist = 1e300, tt = 0.0;
            if (tid < np) {
                tt = round == 0 ? -1.0 + 2.0 * tid / 64.0 : lo + (hi - lo) * tid / 127.0;
                dist = dist_at(tt);
            }
            s.SD[tid] = dist;
            s.RED[tid] = tt;
            __syncthreads();
            int kb = 0;
            for (int q = 1; q < np; ++q)
                if (s.SD[q] < s.SD[kb])
                    kb = q;
            if (s.SD[kb] < best_d) {
                best_d = s.SD[kb];
                best_t = s.RED[kb];
            }
            const double nlo = s.RED[max(kb - 1, 0)], nhi = s.RED[min(kb + 1, np - 1)];
            lo = nlo;
            hi = nhi;
            __syncthreads();
        }
        // parabolas through d^2 at best_t - h, best_t, best_t + h: the bracket of ~2e-7 shrinks
        // to ~1e-13 in TQ_PARAB rounds of three evaluations
        double h = 0.25 * (hi - lo);
        for (int pr = 0; pr < TQ_PARAB && h > 0.0; ++pr) {
            if (tid < 3) {
                const double tt = fmin(1.0, fmax(-1.0, best_t + (tid - 1) * h));
                const double dd = dist_at(tt);
                s.SD[tid] = dd;
                s.RED[tid] = tt;
            }
            __syncthreads();
            const double f0 = s.SD[0] * s.SD[0], f1 = s.SD[1] * s.SD[1], f2 = s.SD[2] * s.SD[2];
            // a clamped end point (t* at the element's end): no parabola
            const bool clamped = s.RED[0] != s.RED[1] - h || s.RED[2] != s.RED[1] + h;
            for (int q = 0; q < 3; ++q)
                if (s.SD[q] < best_d) {
                    best_d = s.SD[q];
                    best_t = s.RED[q];
                }
            __syncthreads();
            const double curv = f2 - 2.0 * f1 + f0;
            if (!(curv > 0.0) || clamped)
                break;
            const double tv = s.RED[1] - h * fmin(1.0, fmax(-1.0, 0.5 * (f2 - f0) / curv));
            if (tid == 0) {
                const double tt = fmin(1.0, fmax(-1.0, tv));
                s.SD[0] = dist_at(tt);
                s.RED[0] = tt;
            }
            __syncthreads();
            if (s.SD[0] < best_d) {
                best_d = s.SD[0];
                best_t = s.RED[0];
            }
            __syncthreads();
            h *= 1.0 / 64.0;
        }
        t0 = best_t;
        dstar = best_d;
    }

    // ---- outer rule (Sec. 3.2.3 / 3.2.4): each side of t0 split dyadically towards t0; the
    // panel next to t0 takes the log-singular rule on the own element.  Flat s-node index:
    // side 0 first, innermost panel first.
    double ell[2];
    int lev[2], nside[2];
    for (int side = 0; side < 2; ++side) {
        ell[side] = side == 0 ? 1.0 - t0 : -1.0 - t0;
        lev[side] = dyadic_levels(fabs(ell[side]) * speed, own ? rho_max : dstar);
        nside[side] = ell[side] == 0.0 ? 0 : (lev[side] + 1) * TQ_Q + (own ? TQ_SING_N - TQ_Q : 0);
    }
    // own element: the whole-element singular rule of the element's local aspect ratio at
    // t0, when one is compiled in for it and the element is nearly straight (the rules come
    // from straight cylinders: within 7e-11 of the dyadic rule on slender-loop elements
    // turning up to 0.15 rad, but 1e-8..3e-6 off on elements turning 0.4..1.3 rad)
    int srule = -1, scount = 0;
    if (own && p.scnt && g.turn <= TQ_SING_TURN) {
        const double asp = 2.0 * g.spd[i0] / g.rho[i0];
        if (asp > 0.0 && isfinite(asp)) {
            const int b = static_cast<int>(floor(log2(asp)));
            if (b >= p.slo && b <= p.shi) {
                const int r = (b - p.slo) * ns + i0;
                if (p.scnt[r] > 0) {
                    srule = p.soff[r];
                    scount = p.scnt[r];
                }
            }
        }
    }
    const int nsn = srule >= 0 ? scount : nside[0] + nside[1];
    const int nb = max(2, (nt + 7) / 8);
    const double lb = PI_ / nb;
    const int NO = NC * MO;
    const int GR = NO <= TQ_THREADS ? TQ_THREADS / NO : 1;
    const double a0v[3] = {s.sa[i0], s.sa[ns + i0], s.sa[2 * ns + i0]};
    const double b0v[3] = {s.sb[i0], s.sb[ns + i0], s.sb[2 * ns + i0]};

    for (int base = 0; base < nsn; base += TQ_SB) {
        const int nb_sn = min(TQ_SB, nsn - base);
        // ---- one thread per s-node: basis, circle, closest angle, rule
        if (tid < nb_sn) {
            const int gidx = base + tid;
            const int side = gidx < nside[0] ? 0 : 1;
            const int gs = side == 0 ? gidx : gidx - nside[0];
            int pan, q;
            if (own) {
                pan = gs < TQ_SING_N ? 0 : 1 + (gs - TQ_SING_N) / TQ_Q;
                q = gs < TQ_SING_N ? gs : (gs - TQ_SING_N) % TQ_Q;
            } else {
                pan = gs / TQ_Q;
                q = gs % TQ_Q;
            }
            const double el = ell[side];
            const int lv = lev[side];
            double plo, phi_;
            if (pan == 0) {
                plo = 0.0;
                phi_ = ldexp(el, -lv);
            } else {
                const int kk = lv - pan;
                plo = ldexp(el, -(kk + 1));
                phi_ = ldexp(el, -kk);
            }
            const bool sing = own && pan == 0;
            const double delta = srule >= 0 ? p.sdel[srule + gidx]
                                 : sing ? phi_ * p.sx[q] : plo + (phi_ - plo) * p.gx[q];
            const double wt = srule >= 0 ? p.swt[srule + gidx]
                              : sing ? fabs(phi_) * p.sw[q] : fabs(phi_ - plo) * p.gw[q];
            const double t = t0 + delta;
            double L[TQ_NS_MAX], dL[TQ_NS_MAX];
            basis_at(p, ns, t, own, i0, delta, L, dL);
            double *G = s.SG + tid * SG_STRIDE;
            if (own) {
                double sum = 0.0;
                for (int i = 0; i < ns; ++i)
                    sum += L[i];
                for (int d = 0; d < 3; ++d) {
                    double ac = 0.0, aa = 0.0, ab = 0.0;
                    for (int i = 0; i < ns; ++i) {
                        if (i == i0)
                            continue;
                        ac += L[i] * (s.sc[d * ns + i] - s.sc[d * ns + i0]);
                        aa += L[i] * (s.sa[d * ns + i] - s.sa[d * ns + i0]);
                        ab += L[i] * (s.sb[d * ns + i] - s.sb[d * ns + i0]);
                    }
                    G[18 + d] = ac;
                    G[21 + d] = aa;
                    G[24 + d] = ab;
                }
                L[i0] = 1.0 - sum;
            }
            for (int d = 0; d < 3; ++d) {
                double c = 0.0, a = 0.0, b = 0.0, ct = 0.0, at = 0.0, bt = 0.0;
                for (int i = 0; i < ns; ++i) {
                    c += L[i] * s.sc[d * ns + i];
                    a += L[i] * s.sa[d * ns + i];
                    b += L[i] * s.sb[d * ns + i];
                    ct += dL[i] * s.sc[d * ns + i];
                    at += dL[i] * s.sa[d * ns + i];
                    bt += dL[i] * s.sb[d * ns + i];
                }
                G[d] = c;
                G[3 + d] = a;
                G[6 + d] = b;
                G[9 + d] = ct;
                G[12 + d] = at;
                G[15 + d] = bt;
            }
            for (int i = 0; i < ns; ++i)
                s.SP[tid * ns + i] = wt * L[i];
            // closest angle: Newton on (y - x) . y_theta (own: as an offset psi from theta_j0)
            double th0, ymx0[3];
            if (own) {
                th0 = 0.0;
                for (int itn = 0; itn < 4; ++itn) {
                    const double ang = thj0 + th0;
                    double sn, cs, sh, ch;
                    sincos(ang, &sn, &cs);
                    sincos(thj0 + 0.5 * th0, &sh, &ch);
                    const double s2 = sin(0.5 * th0);
                    const double dcos = -2.0 * sh * s2, dsin = 2.0 * ch * s2;
                    double ymx[3], yth[3], ythth[3];
                    for (int d = 0; d < 3; ++d) {
                        ymx[d] = G[18 + d] + G[21 + d] * cs + a0v[d] * dcos + G[24 + d] * sn
                                 + b0v[d] * dsin;
                        yth[d] = -G[3 + d] * sn + G[6 + d] * cs;
                        ythth[d] = -G[3 + d] * cs - G[6 + d] * sn;
                    }
                    const double fp = dot3(yth, yth) + dot3(ymx, ythth);
                    if (fp <= 0.0)
                        break;
                    th0 -= dot3(ymx, yth) / fp;
                }
                double sn, cs, sh, ch;
                sincos(thj0 + th0, &sn, &cs);
                sincos(thj0 + 0.5 * th0, &sh, &ch);
                const double s2 = sin(0.5 * th0);
                for (int d = 0; d < 3; ++d)
                    ymx0[d] = G[18 + d] + G[21 + d] * cs + a0v[d] * (-2.0 * sh * s2) + G[24 + d] * sn
                              + b0v[d] * (2.0 * ch * s2);
            } else {
                const double dx[3] = {x[0] - G[0], x[1] - G[1], x[2] - G[2]};
                th0 = atan2(dot3(dx, G + 6), dot3(dx, G + 3));
                for (int itn = 0; itn < 3; ++itn) {
                    double sn, cs;
                    sincos(th0, &sn, &cs);
                    double ymx[3], yth[3], ythth[3];
                    for (int d = 0; d < 3; ++d) {
                        ymx[d] = G[d] + G[3 + d] * cs + G[6 + d] * sn - x[d];
                        yth[d] = -G[3 + d] * sn + G[6 + d] * cs;
                        ythth[d] = -G[3 + d] * cs - G[6 + d] * sn;
                    }
                    const double fp = dot3(yth, yth) + dot3(ymx, ythth);
                    if (fp <= 0.0)
                        break;
                    th0 -= dot3(ymx, yth) / fp;
                }
                double sn, cs;
                sincos(th0, &sn, &cs);
                for (int d = 0; d < 3; ++d)
                    ymx0[d] = G[d] + G[3 + d] * cs + G[6 + d] * sn - x[d];
            }
            double rho2 = 0.0;
            for (int d = 0; d < 3; ++d)
                rho2 += G[3 + d] * G[3 + d] + G[6 + d] * G[6 + d];
            const double rel = sqrt(dot3(ymx0, ymx0)) / sqrt(0.5 * rho2);
            // the cheapest accurate rule: dyadic Gauss-Legendre, the compressed rule of the
            // level, or the trapezoidal rule of the fewest k N_theta nodes its aliasing bound
            // allows
            int mode = 0, cnt = 0, dl = 0;
            if (rel >= lb)
                dl = 0;
            else if (rel <= 0.0)
                dl = TQ_LMAX;
            else
                dl = min(TQ_LMAX, static_cast<int>(ceil(log2(lb / rel))));
            cnt = 2 * TQ_Q * (dl + nb);
            const double ag = strip_at(g, t);
            if (p.rcnt && ag >= TQ_GEOM_TABLE && rel > 0.0 && rel < 2.0
                && rel >= ldexp(1.0, -TQ_RULE_MAXLEV)) {
                const int tl = max(0, min(TQ_RULE_MAXLEV, static_cast<int>(ceil(-log2(rel)))));
                if (tl < p.rnlev && p.rcnt[tl] > 0 && p.rcnt[tl] < cnt) {
                    mode = tl + 1;
                    cnt = p.rcnt[tl];
                }
            }
            if (rel > 0.0 && ag >= TQ_GEOM_TRAP) {
                const double a = fmin(ag, acosh(1.0 + rel * rel / (2.0 * (1.0 + rel))));
                const double mreq = (nt / 2 + 2) + TQ_TRAP_LOG / a;
                const int k = max(1, static_cast<int>(ceil(mreq / nt)));
                if (k <= p.kmax && k * nt < cnt) {
                    mode = -k;
                    cnt = k * nt;
                }
            }
            s.SX[2 * tid] = th0;
            s.SX[2 * tid + 1] = rel;
            s.MODE[tid] = mode;
            s.CNT[tid] = cnt;
            s.DLEV[tid] = dl;
        }
        __syncthreads();
        if (tid == 0) {
            int nM = 0;
            for (int m = 0; m < nb_sn; ++m)
                if (s.MODE[m] >= 0)
                    s.LM[nM++] = m;
            s.NL[1] = nM;
        }
        __syncthreads();
        const int nM = s.NL[1];

        // ---- trapezoidal s-nodes, grouped by k: M = k N_theta nodes at 2 pi m / M, 128 / M
        // s-nodes per chunk, one thread per (s-node, node); h_j = sum_m v_m D_k[(m - k j) mod M]
        for (int k = 1; k <= p.kmax; ++k) {
            const int M = k * nt;
            const int spk = TQ_THREADS / M;
            if (tid == 0) {
                int nT = 0;
                for (int m = 0; m < nb_sn; ++m)
                    if (s.MODE[m] == -k)
                        s.LT[nT++] = m;
                s.NL[0] = nT;
            }
            __syncthreads();
            const int nT = s.NL[0];
            const double *D = p.dtab + nt * k * (k - 1) / 2;
            const double om_trap = 2.0 * PI_ / M;
            for (int cb = 0; cb < nT; cb += spk) {
                const int mm = tid / M, q = tid % M;
                double out[NC];
                if (mm < spk && cb + mm < nT) {
                    const int m = s.LT[cb + mm];
                    double sn, cs, dcos = 0.0, dsin = 0.0;
                    if (own) {
                        // psi = 2 pi (q - k j0) / M: its half angle, the rest by angle addition
                        double s2, c2;
                        sincospi(static_cast<double>(q - k * j0) / M, &s2, &c2);
                        const double spsi = 2.0 * s2 * c2, cpsi = 1.0 - 2.0 * s2 * s2;
                        sn = sj0 * cpsi + cj0 * spsi;
                        cs = cj0 * cpsi - sj0 * spsi;
                        const double sh = sj0 * c2 + cj0 * s2, ch = cj0 * c2 - sj0 * s2;
                        dcos = -2.0 * sh * s2;
                        dsin = 2.0 * ch * s2;
                    } else {
                        sincospi(2.0 * q / M, &sn, &cs);
                    }
                    node_value<NC>(s.SG + m * SG_STRIDE, own, a0v, b0v, x, cs, sn, dcos, dsin, sgn,
                                   p.alpha, p.beta, om_trap, out);
                } else {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        out[c] = 0.0;
                }
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    s.V[tid * NC + c] = out[c];
                __syncthreads();
                const int cnt = min(spk, nT - cb);
                for (int e = tid; e < cnt * NC * nt; e += TQ_THREADS) {
                    const int mm2 = e / (NC * nt), rem = e % (NC * nt);
                    const int c = rem / nt, j = rem % nt;
                    const double *v = s.V + mm2 * M * NC + c;
                    double h = 0.0;
                    for (int q2 = 0; q2 < M; ++q2)
                        h += v[q2 * NC] * D[((q2 - k * j) % M + M) % M];
                    s.H2[e] = h;
                }
                __syncthreads();
                for (int e = tid; e < NC * ns * nt; e += TQ_THREADS) {
                    const int c = e / (ns * nt), rem = e % (ns * nt);
                    const int i = rem / nt, j = rem % nt;
                    double acc = 0.0;
                    for (int mm2 = 0; mm2 < cnt; ++mm2)
                        acc += s.SP[s.LT[cb + mm2] * ns + i] * s.H2[(mm2 * NC + c) * nt + j];
                    s.EB[e] += acc;
                }
                __syncthreads();
            }
            __syncthreads();   // every thread has read NL[0] and LT before the next k's lists
        }

        // ---- modal s-nodes, one at a time: compressed or dyadic rule, modal coefficients
        // (Eq. modal-greens-fn-coeff), inverse DFT (Eq. modal-greens-fn-wts)
        for (int mi = 0; mi < nM; ++mi) {
            const int m = s.LM[mi];
            const double *G = s.SG + m * SG_STRIDE;
            const double th0 = s.SX[2 * m];
            const int mode = s.MODE[m], M = s.CNT[m], L = s.DLEV[m];
            const int Mh = TQ_Q * (L + nb);
            double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
            for (int cb = 0; cb < M; cb += TQ_THREADS) {
                const int kq = cb + tid;
                if (kq < M) {
                    double phi, om;
                    if (mode > 0) {
                        phi = p.rphi[(mode - 1) * TQ_RULE_SLOT + kq];
                        om = p.rw[(mode - 1) * TQ_RULE_SLOT + kq];
                    } else {
                        const int sidek = kq / Mh, kp = kq % Mh;
                        const int pn = kp / TQ_Q, qq = kp % TQ_Q;
                        double lo, hi;
                        if (pn == 0) {
                            lo = 0.0;
                            hi = ldexp(lb, -L);
                        } else if (pn <= L) {
                            lo = ldexp(lb, -(L - pn + 1));
                            hi = ldexp(lb, -(L - pn));
                        } else {
                            lo = lb * (pn - L);
                            hi = lb * (pn - L + 1);
                        }
                        phi = lo + (hi - lo) * p.gx[qq];
                        om = (hi - lo) * p.gw[qq];
                        if (sidek == 0)
                            phi = -phi;
                    }
                    const double psi = th0 + phi;   // own: offset from theta_j0
                    double sn, cs, dcos = 0.0, dsin = 0.0;
                    if (own) {
                        // one sincos: half-angle of psi, the rest by angle addition
                        double s2, c2;
                        sincos(0.5 * psi, &s2, &c2);
                        const double spsi = 2.0 * s2 * c2, cpsi = 1.0 - 2.0 * s2 * s2;
                        sn = sj0 * cpsi + cj0 * spsi;
                        cs = cj0 * cpsi - sj0 * spsi;
                        const double sh = sj0 * c2 + cj0 * s2;   // sin(theta_j0 + psi / 2)
                        const double ch = cj0 * c2 - sj0 * s2;   // cos(theta_j0 + psi / 2)
                        dcos = -2.0 * sh * s2;
                        dsin = 2.0 * ch * s2;
                    } else {
                        sincos(psi, &sn, &cs);
                    }
                    double out[NC];
                    node_value<NC>(G, own, a0v, b0v, x, cs, sn, dcos, dsin, sgn, p.alpha, p.beta,
                                   om, out);
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        s.V[tid * NC + c] = out[c];
                    double er = 1.0, ei = 0.0;
                    double *csd = s.CS + static_cast<size_t>(tid) * MO * 2;
                    csd[0] = 1.0;
                    csd[1] = 0.0;
                    for (int l = 1; l < MO; ++l) {
                        const double nr = er * cs - ei * sn;
                        ei = er * sn + ei * cs;
                        er = nr;
                        csd[2 * l] = er;
                        csd[2 * l + 1] = ei;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        s.V[tid * NC + c] = 0.0;
                    double *csd = s.CS + static_cast<size_t>(tid) * MO * 2;
                    for (int l = 0; l < 2 * MO; ++l)
                        csd[l] = 0.0;
                }
                __syncthreads();
                const int cnt = min(TQ_THREADS, M - cb);
                if (NO <= TQ_THREADS) {
                    if (tid < GR * NO) {
                        const int gg = tid / NO, o = tid % NO;
                        const int c = o / MO, l = o % MO;
                        for (int kk = gg; kk < cnt; kk += GR) {
                            const double v = s.V[kk * NC + c];
                            acc[0][0] += v * s.CS[(kk * MO + l) * 2];
                            acc[0][1] += v * s.CS[(kk * MO + l) * 2 + 1];
                        }
                    }
                } else {
                    for (int h = 0; h < 2; ++h) {
                        const int o = tid + h * TQ_THREADS;
                        if (o < NO) {
                            const int c = o / MO, l = o % MO;
                            for (int kk = 0; kk < cnt; ++kk) {
                                const double v = s.V[kk * NC + c];
                                acc[h][0] += v * s.CS[(kk * MO + l) * 2];
                                acc[h][1] += v * s.CS[(kk * MO + l) * 2 + 1];
                            }
                        }
                    }
                }
                __syncthreads();
            }
            if (NO <= TQ_THREADS) {
                s.RED[2 * tid] = acc[0][0];
                s.RED[2 * tid + 1] = acc[0][1];
                __syncthreads();
                if (tid < NO) {
                    double re = 0.0, im = 0.0;
                    for (int gg = 0; gg < GR; ++gg) {
                        re += s.RED[2 * (gg * NO + tid)];
                        im += s.RED[2 * (gg * NO + tid) + 1];
                    }
                    s.HH[2 * tid] = re;
                    s.HH[2 * tid + 1] = im;
                }
            } else {
                for (int h = 0; h < 2; ++h) {
                    const int o = tid + h * TQ_THREADS;
                    if (o < NO) {
                        s.HH[2 * o] = acc[h][0];
                        s.HH[2 * o + 1] = acc[h][1];
                    }
                }
            }
            __syncthreads();
            // inverse DFT (Eq. modal-greens-fn-wts), the Nyquist mode as cos(N theta / 2)
            for (int e = tid; e < NC * nt; e += TQ_THREADS) {
                const int c = e / nt, j = e % nt;
                const double *hh = s.HH + 2 * c * MO;
                double h = hh[0];
                for (int l = 1; l < MO - 1; ++l) {
                    const int q = (2 * l * j) % (2 * nt);
                    h += 2.0 * (hh[2 * l] * s.W[2 * q] + hh[2 * l + 1] * s.W[2 * q + 1]);
                }
                const int qn = (2 * (MO - 1) * j) % (2 * nt);
                h += hh[2 * (MO - 1)] * s.W[2 * qn];
                s.H[e] = h / nt;
            }
            __syncthreads();
            for (int e = tid; e < NC * ns * nt; e += TQ_THREADS) {
                const int c = e / (ns * nt), rem = e % (ns * nt);
                const int i = rem / nt, j = rem % nt;
                s.EB[e] += s.SP[m * ns + i] * s.H[c * nt + j];
            }
            __syncthreads();
        }
    }

    // ---- subtract the uncorrected sum's terms (the coincident node is not in it)
    for (int e = tid; e < per; e += TQ_THREADS) {
        if (own && e == i0 * nt + j0)
            continue;
        const long long gnode = static_cast<long long>(it.k) * per + e;
        const double r[3] = {x[0] - src[gnode], x[1] - src[N + gnode], x[2] - src[2 * N + gnode]};
        const double nn[3] = {nrm[gnode], nrm[N + gnode], nrm[2 * N + gnode]};
        double K[NC];
        kern<NC>(r, nn, p.alpha, p.beta, K);
        const double wv = wgt[gnode];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            s.EB[c * per + e] -= K[c] * wv;
    }
    __syncthreads();
    // ---- scatter into the CSR rows of this target
    const long long kbase = static_cast<long long>(it.k) * per;
    if (NC == 1) {
        const int64_t r0 = rowptr[it.t] + static_cast<int64_t>(it.slot) * per;
        for (int e = tid; e < per; e += TQ_THREADS) {
            col[r0 + e] = kbase + e;
            val[r0 + e] = s.EB[e];
        }
    } else {
        const int sym[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        for (int e = tid; e < 9 * per; e += TQ_THREADS) {
            const int a = e / (3 * per), rem = e % (3 * per);
            const int b = rem / per, node = rem % per;
            const int64_t pos = rowptr[a * RS + it.t] + static_cast<int64_t>(it.slot) * 3 * per
                                + static_cast<int64_t>(b) * per + node;
            col[pos] = b * N + kbase + node;
            val[pos] = s.EB[sym[a][b] * per + node];
        }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton on the three-term recurrence of P_n
// in long double.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double PI_L = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = std::cos(PI_L * (i + 0.75L) / (n + 0.5L));
        long double dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
            const long double dz = p1 / dp;
            z -= dz;
            if (std::fabs(static_cast<double>(dz)) < 1e-19)
                break;
        }
        {
            long double p0 = 1.0L, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
        }
        // ascending order
        x[n - 1 - i] = static_cast<double>(z);
        w[n - 1 - i] = static_cast<double>(2.0L / ((1.0L - z * z) * dp * dp));
    }
}

}  // namespace

int build_tube_correction(long long nelem, int ns, int nt, long long ntot, const double *src,
                          const double *nrm, const double *w, long long ntrg, const double *trg,
                          int laplace, double alpha, double beta, double near_factor,
                          int64_t *nnz_out, int64_t *rowptr, int64_t *col, double *val,
                          cudaStream_t s, int rules_nlev, const double *rules_phi,
                          const double *rules_w, const int *rules_cnt)
{
    const long long per = static_cast<long long>(ns) * nt;
    const long long ntube = nelem * per;
    // targets: the tube nodes (rows over all ntot nodes, tube nodes first) or ntrg
    // off-surface points
    const long long ntarget = trg ? ntrg : ntube;
    const long long nrows_per_comp = trg ? ntrg : ntot;
    const int nc_rows = laplace ? 1 : 3;
    TQParams p{};
    {
        std::vector<double> x, wv;
        gauss_legendre(ns, x, wv);
        for (int i = 0; i < ns; ++i)
            p.tn[i] = x[i];
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < ns; ++k)
                p.invd[i][k] = (i == k) ? 0.0 : 1.0 / (x[i] - x[k]);
        gauss_legendre(TQ_Q, x, wv);
        for (int i = 0; i < TQ_Q; ++i) {
            p.gx[i] = 0.5 * (x[i] + 1.0);
            p.gw[i] = 0.5 * wv[i];
        }
        gauss_legendre(TQ_SING_N, x, wv);
        for (int i = 0; i < TQ_SING_N; ++i) {
            const double u = 0.5 * (x[i] + 1.0);
            p.sx[i] = std::pow(u, TQ_SING_G);
            p.sw[i] = TQ_SING_G * std::pow(u, TQ_SING_G - 1) * 0.5 * wv[i];
        }
    }
    p.alpha = alpha;
    p.beta = beta;
    p.ntot = ntot;
    p.ns = ns;
    p.nt = nt;
    p.per = static_cast<int>(per);
    p.rphi = p.rw = nullptr;
    p.scnt = p.soff = nullptr;
    p.sdel = p.swt = nullptr;
    p.slo = 0;
    p.shi = -1;
    p.rcnt = nullptr;
    p.rnlev = 0;
    // weights of the trapezoidal rules of k N_theta nodes: D_k[q] = (1/N)(1 + 2 sum_{l=1}^{N/2-1}
    // cos(l phi) + cos(N phi / 2)), phi = 2 pi q / (k N)
    p.kmax = std::max(1, std::min(TQ_TRAP_KMAX, TQ_THREADS / nt));
    std::vector<double> h_dtab;
    for (int k = 1; k <= p.kmax; ++k)
        for (int q = 0; q < k * nt; ++q) {
            const long double PI_L = 3.141592653589793238462643383279502884L;
            const long double phi = 2.0L * PI_L * q / (static_cast<long double>(k) * nt);
            long double d = 1.0L + std::cos(0.5L * nt * phi);
            for (int l = 1; l < nt / 2; ++l)
                d += 2.0L * std::cos(l * phi);
            h_dtab.push_back(static_cast<double>(d / nt));
        }

    AsyncAllocScope scope(s);
    std::vector<long long> cnt_off;
    std::vector<int> h_cnt, h_list;
    DevBuf d_geo, d_bad, d_cnt, d_off, d_list, d_keys, d_elem;
    if (ntube > 0 && ntarget > 0) {
        SBQ_TRY(d_geo.alloc(nelem * sizeof(ElemGeo)));
        SBQ_TRY(d_bad.alloc(sizeof(int)));
        SBQ_TRY(d_cnt.alloc(ntarget * sizeof(int)));
        SBQ_CUDA(cudaMemsetAsync(d_bad.p, 0, sizeof(int), s));
        const unsigned ge = static_cast<unsigned>((nelem + 63) / 64);
        k_elem_setup<<<ge, 64, 0, s>>>(nelem, p, src, nrm, d_geo.as<ElemGeo>(), d_bad.as<int>());
        SBQ_CUDA(cudaGetLastError());
        k_elem_strip<<<static_cast<unsigned>((nelem * TQ_AG_N + 127) / 128), 128, 0, s>>>(
            nelem, p, d_geo.as<ElemGeo>());
        SBQ_CUDA(cudaGetLastError());
        const unsigned gt = static_cast<unsigned>((ntarget + 127) / 128);
        // spatial grid of the element reach spheres
        DevBuf d_reach;
        SBQ_TRY(d_reach.alloc(nelem * sizeof(Reach)));
        k_elem_reach<<<ge, 64, 0, s>>>(nelem, ns, near_factor, d_geo.as<ElemGeo>(),
                                       d_reach.as<Reach>());
        SBQ_CUDA(cudaGetLastError());
        std::vector<Reach> h_reach(nelem);
        SBQ_CUDA(cudaMemcpyAsync(h_reach.data(), d_reach.p, nelem * sizeof(Reach),
                                 cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaStreamSynchronize(s));
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double h = 0.0;
        for (const Reach &r : h_reach) {
            lo[0] = std::min(lo[0], r.x);
            lo[1] = std::min(lo[1], r.y);
            lo[2] = std::min(lo[2], r.z);
            hi[0] = std::max(hi[0], r.x);
            hi[1] = std::max(hi[1], r.y);
            hi[2] = std::max(hi[2], r.z);
            h = std::max(h, r.r);
        }
        const double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 0.0});
        if (!(h > 0.0) || !std::isfinite(h) || !std::isfinite(span)) {
            set_error("tube_correction: degenerate element geometry");
            return SBQ_EINVAL;
        }
        int dim = 1;
        while (dim < (1 << 20) && dim * h < span)
            dim *= 2;
        h = std::max(h, span / dim);
        NearGrid grid{};
        for (int d = 0; d < 3; ++d)
            grid.lo[d] = (d == 0 ? lo[0] : d == 1 ? lo[1] : lo[2]);
        grid.inv_h = 1.0 / h;
        grid.dim = dim;
        grid.nelem = nelem;
        std::vector<std::pair<unsigned long long, int>> kv(nelem);
        for (long long k = 0; k < nelem; ++k) {
            const Reach &r = h_reach[k];
            const double cc[3] = {r.x, r.y, r.z};
            int ic[3];
            for (int d = 0; d < 3; ++d)
                ic[d] = std::min(dim - 1, std::max(0, static_cast<int>(std::floor((cc[d] - grid.lo[d]) * grid.inv_h))));
            kv[k] = {morton_key(ic[0], ic[1], ic[2]), static_cast<int>(k)};
        }
        std::sort(kv.begin(), kv.end());
        std::vector<unsigned long long> h_keys(nelem);
        std::vector<int> h_elem(nelem);
        for (long long k = 0; k < nelem; ++k) {
            h_keys[k] = kv[k].first;
            h_elem[k] = kv[k].second;
        }
        SBQ_TRY(d_keys.alloc(nelem * sizeof(unsigned long long)));
        SBQ_TRY(d_elem.alloc(nelem * sizeof(int)));
        SBQ_CUDA(cudaMemcpyAsync(d_keys.p, h_keys.data(), nelem * sizeof(unsigned long long),
                                 cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_elem.p, h_elem.data(), nelem * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
        grid.keys = d_keys.as<unsigned long long>();
        grid.elem = d_elem.as<int>();
        k_near<<<gt, 128, 0, s>>>(ntarget, p, near_factor, src, trg, d_geo.as<ElemGeo>(), grid,
                                  nullptr, d_cnt.as<int>());
        SBQ_CUDA(cudaGetLastError());
        int bad = 0;
        h_cnt.resize(ntarget);
        SBQ_CUDA(cudaMemcpyAsync(&bad, d_bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaMemcpyAsync(h_cnt.data(), d_cnt.p, ntarget * sizeof(int), cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaStreamSynchronize(s));
        if (bad) {
            set_error("tube_correction: element rows of nodes are not circles (nodes must be "
                      "panel-major, then GL node, then equispaced angle)");
            return SBQ_EINVAL;
        }
        cnt_off.assign(ntarget + 1, 0);
        for (long long t = 0; t < ntarget; ++t)
            cnt_off[t + 1] = cnt_off[t] + h_cnt[t];
        SBQ_TRY(d_off.alloc((ntarget + 1) * sizeof(long long)));
        SBQ_TRY(d_list.alloc(std::max<long long>(cnt_off[ntarget], 1) * sizeof(int)));
        SBQ_CUDA(cudaMemcpyAsync(d_off.p, cnt_off.data(), (ntarget + 1) * sizeof(long long),
                                 cudaMemcpyHostToDevice, s));
        k_near<<<gt, 128, 0, s>>>(ntarget, p, near_factor, src, trg, d_geo.as<ElemGeo>(), grid,
                                  d_off.as<long long>(), d_list.as<int>());
        SBQ_CUDA(cudaGetLastError());
        h_list.resize(cnt_off[ntarget]);
        SBQ_CUDA(cudaMemcpyAsync(h_list.data(), d_list.p, cnt_off[ntarget] * sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
        SBQ_CUDA(cudaStreamSynchronize(s));
    } else {
        h_cnt.assign(ntarget, 0);
        cnt_off.assign(ntarget + 1, 0);
    }
    // rows: component-major over all ntot nodes; a tube target's row holds its near
    // elements' nodes (times the three source components for Stokes)
    std::vector<int64_t> h_rowptr(static_cast<size_t>(nc_rows) * nrows_per_comp + 1, 0);
    const int64_t row_mul = laplace ? per : 3 * per;
    for (int a = 0; a < nc_rows; ++a)
        for (long long t = 0; t < nrows_per_comp; ++t) {
            const size_t r = static_cast<size_t>(a) * nrows_per_comp + t;
            h_rowptr[r + 1] = h_rowptr[r] + (t < ntarget ? h_cnt[t] * row_mul : 0);
        }
    const int64_t nnz = h_rowptr.back();
    if (nnz_out)
        *nnz_out = nnz;
    if (!rowptr)
        return SBQ_OK;
    if (nnz > 0 && (!col || !val)) {
        set_error("tube_correction: null col or val");
        return SBQ_EINVAL;
    }
    SBQ_CUDA(cudaMemcpyAsync(rowptr, h_rowptr.data(), h_rowptr.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
    const long long n_items = cnt_off[ntarget];
    if (n_items == 0) {
        SBQ_CUDA(cudaStreamSynchronize(s));
        return SBQ_OK;
    }
    if (n_items > 0x7fffffffLL) {
        set_error("tube_correction: too many (target, element) pairs");
        return SBQ_EINVAL;
    }
    std::vector<Item> h_items(n_items);
    for (long long t = 0; t < ntarget; ++t)
        for (int q = 0; q < h_cnt[t]; ++q)
            h_items[cnt_off[t] + q] = Item{static_cast<int>(t), h_list[cnt_off[t] + q], q, 0};
    // angular rules: the caller's tables (rules_nlev > 0), none (rules_nlev < 0), or the
    // compiled-in table with the smallest mode count l0 >= nt / 2 + 4 (rules_nlev == 0): the
    // integrands are G J e^{i l theta}, l <= nt / 2, and the area element J (and the normal)
    // of a tube whose radius or frame varies along it has small Fourier modes beyond +-1
    std::vector<double> b_phi, b_w;
    std::vector<int> b_cnt;
    if (rules_nlev == 0) {
        int best = -1;
        long long off = 0, best_off = 0;
        for (int tb = 0; tb < kRuleTables; ++tb) {
            long long tot = 0;
            for (int l = 0; l <= TQ_RULE_MAXLEV; ++l)
                tot += kRuleCnt[tb][l];
            if (kRuleL0[tb] >= nt / 2 + 4 && (best < 0 || kRuleL0[tb] < kRuleL0[best])) {
                best = tb;
                best_off = off;
            }
            off += 2 * tot;
        }
        if (best >= 0) {
            const int nl = TQ_RULE_MAXLEV + 1;
            b_phi.assign(static_cast<size_t>(nl) * TQ_RULE_SLOT, 0.0);
            b_w.assign(static_cast<size_t>(nl) * TQ_RULE_SLOT, 0.0);
            b_cnt.assign(nl, 0);
            long long q = best_off;
            for (int l = 0; l < nl; ++l) {
                b_cnt[l] = std::min(kRuleCnt[best][l], TQ_RULE_SLOT);
                for (int m = 0; m < kRuleCnt[best][l]; ++m, q += 2) {
                    if (m < TQ_RULE_SLOT) {
                        b_phi[l * TQ_RULE_SLOT + m] = kRuleData[q];
                        b_w[l * TQ_RULE_SLOT + m] = kRuleData[q + 1];
                    }
                }
            }
            rules_nlev = nl;
            rules_phi = b_phi.data();
            rules_w = b_w.data();
            rules_cnt = b_cnt.data();
        }
    }
    // whole-element singular rules for own-element targets: the compiled-in table when it
    // serves this ns and mode count (l0 >= nt / 2 + 4) and compressed rules are on
    DevBuf d_scnt, d_soff, d_sdat;
    std::vector<double> h_sdel, h_swt;
    if (rules_nlev >= 0 && kSingTables && ns == kSingNs && nt / 2 + 4 <= kSingL0) {
        const int nr = (kSingHi - kSingLo + 1) * kSingNs;
        int tot = 0;
        for (int r = 0; r < nr; ++r)
            tot = std::max(tot, kSingOff[r] + kSingCnt[r]);
        h_sdel.resize(2 * static_cast<size_t>(tot));
        for (int m = 0; m < tot; ++m) {
            h_sdel[m] = kSingData[2 * m];
            h_sdel[tot + m] = kSingData[2 * m + 1];
        }
        SBQ_TRY(d_scnt.alloc(nr * sizeof(int)));
        SBQ_TRY(d_soff.alloc(nr * sizeof(int)));
        SBQ_TRY(d_sdat.alloc(2 * static_cast<size_t>(tot) * sizeof(double)));
        SBQ_CUDA(cudaMemcpyAsync(d_scnt.p, kSingCnt, nr * sizeof(int), cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_soff.p, kSingOff, nr * sizeof(int), cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_sdat.p, h_sdel.data(), 2 * static_cast<size_t>(tot) * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
        p.scnt = d_scnt.as<int>();
        p.soff = d_soff.as<int>();
        p.sdel = d_sdat.as<double>();
        p.swt = d_sdat.as<double>() + tot;
        p.slo = kSingLo;
        p.shi = kSingHi;
    }
    DevBuf d_rphi, d_rw, d_rcnt;
    if (rules_nlev > 0) {
        const size_t nd = static_cast<size_t>(rules_nlev) * TQ_RULE_SLOT;
        SBQ_TRY(d_rphi.alloc(nd * sizeof(double)));
        SBQ_TRY(d_rw.alloc(nd * sizeof(double)));
        SBQ_TRY(d_rcnt.alloc(rules_nlev * sizeof(int)));
        SBQ_CUDA(cudaMemcpyAsync(d_rphi.p, rules_phi, nd * sizeof(double), cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_rw.p, rules_w, nd * sizeof(double), cudaMemcpyHostToDevice, s));
        SBQ_CUDA(cudaMemcpyAsync(d_rcnt.p, rules_cnt, rules_nlev * sizeof(int), cudaMemcpyHostToDevice, s));
        p.rphi = d_rphi.as<double>();
        p.rw = d_rw.as<double>();
        p.rcnt = d_rcnt.as<int>();
        p.rnlev = rules_nlev;
    }
    DevBuf d_dtab;
    SBQ_TRY(d_dtab.alloc(h_dtab.size() * sizeof(double)));
    SBQ_CUDA(cudaMemcpyAsync(d_dtab.p, h_dtab.data(), h_dtab.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    p.dtab = d_dtab.as<double>();
    DevBuf d_items;
    SBQ_TRY(d_items.alloc(n_items * sizeof(Item)));
    SBQ_CUDA(cudaMemcpyAsync(d_items.p, h_items.data(), n_items * sizeof(Item),
                             cudaMemcpyHostToDevice, s));
    const int NC = laplace ? 1 : 6;
    const size_t smem = tq_smem_doubles(NC, ns, nt) * sizeof(double);
    if (laplace) {
        SBQ_CUDA(cudaFuncSetAttribute(k_tube_items<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
        k_tube_items<1><<<static_cast<unsigned>(n_items), TQ_THREADS, smem, s>>>(
            p, d_items.as<Item>(), d_geo.as<ElemGeo>(), src, nrm, w, trg, ntarget, rowptr, col,
            val);
    } else {
        SBQ_CUDA(cudaFuncSetAttribute(k_tube_items<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
        k_tube_items<6><<<static_cast<unsigned>(n_items), TQ_THREADS, smem, s>>>(
            p, d_items.as<Item>(), d_geo.as<ElemGeo>(), src, nrm, w, trg, ntarget, rowptr, col,
            val);
    }
    SBQ_CUDA(cudaGetLastError());
    // the host vectors above go out of scope here: wait until the copies have been made
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

size_t tube_correction_smem_bytes(int laplace, int ns, int nt)
{
    return tq_smem_doubles(laplace ? 1 : 6, ns, nt) * sizeof(double);
}

}  // namespace sbq

// Quadrature correction with the caller's angular rules (see sbq.h): the same builder with
// the caller's tables in place of the compiled-in ones, or (nlev == 0) with no compressed
// rules at all (dyadically refined Gauss-Legendre rules below two radii).
extern "C" __attribute__((visibility("default"))) int tube_correction_rules(
    int64_t nelem, int ns, int nt, int64_t n_total, const double *src, const double *nrm,
    const double *w, int64_t ntrg, const double *trg, int laplace, double alpha, double beta,
    double near_factor, int nlev, int rule_l0, const double *rule_phi, const double *rule_w,
    const int *rule_cnt, int64_t *nnz_out, int64_t *rowptr, int64_t *col, double *val,
    void *stream)
{
    using namespace sbq;
    clear_error();
    auto bad = [](const char *m) { set_error(m); return static_cast<int>(SBQ_EINVAL); };
    if (nelem < 0 || n_total < 0 || ntrg < 0)
        return bad("negative size");
    if (ns < 2 || ns > 16)
        return bad("ns must be in 2..16");
    if (nt < 4 || nt > 64 || (nt & 1))
        return bad("nt must be even and in 4..64");
    if (nelem * ns * nt > n_total)
        return bad("n_total below nelem * ns * nt");
    if (n_total > (1LL << 31) / 3 || ntrg > (1LL << 31) / 3)
        return bad("n_total or ntrg above 2^31 / 3");
    if (laplace != 0 && laplace != 1)
        return bad("laplace must be 0 or 1");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(near_factor))
        return bad("non-finite alpha, beta or near_factor");
    if (!rowptr && !nnz_out)
        return bad("null rowptr and nnz_out");
    if (nelem > 0 && (!src || !nrm || !w))
        return bad("null geometry pointer");
    if (nlev < 0 || nlev > TQ_RULE_MAXLEV + 1)
        return bad("rules: nlev must be in 0..31");
    if (nlev > 0) {
        if (!rule_phi || !rule_w || !rule_cnt)
            return bad("rules: null table");
        if (rule_l0 < nt / 2 + 1)
            return bad("rules: the table's mode count l0 is below nt / 2 + 1 (it does not "
                       "integrate every mode of this N_theta)");
        for (int l = 0; l < nlev; ++l) {
            if (rule_cnt[l] < 0 || rule_cnt[l] > TQ_RULE_SLOT)
                return bad("rules: a level holds more than 128 nodes");
            for (int m = 0; m < rule_cnt[l]; ++m) {
                const double a = rule_phi[l * TQ_RULE_SLOT + m], b = rule_w[l * TQ_RULE_SLOT + m];
                if (!std::isfinite(a) || !std::isfinite(b) || std::fabs(a) > 3.14159265358979323846)
                    return bad("rules: non-finite entry or offset outside [-pi, pi]");
            }
        }
    }
    return build_tube_correction(nelem, ns, nt, n_total, src, nrm, w, trg ? ntrg : 0, trg,
                                 laplace, alpha, beta, near_factor, nnz_out, rowptr, col, val,
                                 static_cast<cudaStream_t>(stream), nlev > 0 ? nlev : -1,
                                 rule_phi, rule_w, rule_cnt);
}
