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
// Per s-node the angular nodes go through shared memory in chunks of 128 (kernel value x J x
// weight and e^{i l theta}); the modal coefficients are a small reduction over the chunk.
#include "engine.h"

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
constexpr int TQ_LMAX = 60;        // deepest dyadic level
constexpr int TQ_NS_MAX = 16;
constexpr int TQ_REFINE = 3;       // rounds of 128-point refinement of t*
constexpr int TQ_RULE_SLOT = 64;   // nodes reserved per level of a compressed angular rule
constexpr int TQ_RULE_MAXLEV = 30; // compressed rules serve 2^-30 <= alpha < 1

struct ElemGeo {
    double c[3][TQ_NS_MAX], a[3][TQ_NS_MAX], b[3][TQ_NS_MAX];
    double cl[3][TQ_NS_MAX + 2];   // centreline samples: c_i and C(-1), C(+1)
    double rho_max, speed_max, sgn, pad;
};

struct TQParams {
    double tn[TQ_NS_MAX];                  // element GL nodes on [-1, 1]
    double gx[TQ_Q], gw[TQ_Q];             // GL on [0, 1]
    double sx[TQ_SING_N], sw[TQ_SING_N];   // singular rule on [0, 1]
    double alpha, beta;
    long long ntot;
    int ns, nt, per;
    // optional compressed angular rules: level lev (alpha in [2^-lev, 2^(1-lev))) holds
    // rcnt[lev] <= TQ_RULE_SLOT nodes rphi[lev * TQ_RULE_SLOT + m] with weights rw[...]
    const double *rphi, *rw;
    const int *rcnt;
    int rnlev;
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

// l_i(t_i0 + delta) for i != i0 with the factor (t - t_i0) taken as delta itself.
__device__ __forceinline__ double lag_off(const double *tn, int ns, int i, int i0, double delta)
{
    double v = 1.0;
    for (int k = 0; k < ns; ++k) {
        if (k == i)
            continue;
        const double f = (k == i0) ? delta : (tn[i0] - tn[k]) + delta;
        v *= f / (tn[i] - tn[k]);
    }
    return v;
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
        speed = fmax(speed, sqrt(dot3(v, v)));
    }
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

// Targets: the tube nodes (trg == nullptr; each has its own element) or an array of
// off-surface points trg (SoA, ntarget points, no own element).
__global__ void k_near(long long ntarget, long long nelem, TQParams p, double f,
                       const double *__restrict__ src, const double *__restrict__ trg,
                       const ElemGeo *__restrict__ geo, const long long *__restrict__ off, int *out)
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
    int c = 0;
    for (long long k = 0; k < nelem; ++k) {
        if (k == own || is_near(geo[k], p.ns, x, f)) {
            if (off)
                out[off[t] + c] = static_cast<int>(k);
            ++c;
        }
    }
    if (!off)
        out[t] = c;
}

// ---------------------------------------------------------------------------------------
// the correction blocks

struct Smem {
    double *sc, *sa, *sb;      // [3][ns] each
    double *L, *dL;            // [ns]
    double *G;                 // 27: C A B C' A' B' dC dA dB
    double *V;                 // [128][NC]
    double *CS;                // [128][MO][2]
    double *RED;               // [256]
    double *HH;                // [NC][MO][2]
    double *W;                 // [nt][2]
    double *H;                 // [NC][nt]
    double *EB;                // [NC][ns][nt]
    double *SD;                // [128] distances, then misc
};

__host__ __device__ inline size_t tq_smem_doubles(int NC, int ns, int nt)
{
    const int MO = nt / 2 + 1;
    return 9 * ns + 2 * ns + 27 + 128 * NC + 128 * MO * 2 + 256 + NC * MO * 2 + 2 * nt + NC * nt
           + static_cast<size_t>(NC) * ns * nt + 128 + 8;
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
        s.L = q; q += ns;
        s.dL = q; q += ns;
        s.G = q; q += 27;
        s.V = q; q += 128 * NC;
        s.CS = q; q += 128 * MO * 2;
        s.RED = q; q += 256;
        s.HH = q; q += NC * MO * 2;
        s.W = q; q += 2 * nt;
        s.H = q; q += NC * nt;
        s.EB = q; q += NC * ns * nt;
        s.SD = q;
    }
    const Item it = items[blockIdx.x];
    const ElemGeo &g = geo[it.k];
    for (int e = tid; e < 3 * ns; e += TQ_THREADS) {
        const int d = e / ns, i = e % ns;
        s.sc[e] = g.c[d][i];
        s.sa[e] = g.a[d][i];
        s.sb[e] = g.b[d][i];
    }
    for (int q = tid; q < nt; q += TQ_THREADS) {
        double sn, cs;
        sincospi(2.0 * q / nt, &sn, &cs);
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
    double sj0, cj0;
    sincospi(2.0 * j0 / nt, &sj0, &cj0);
    constexpr double PI_ = 3.14159265358979323846;
    __syncthreads();

    // ---- nearest parameter t* of an element that does not hold x (sampling + refinement)
    double t0 = own ? p.tn[i0] : 0.0, dstar = 0.0;
    if (!own) {
        double lo = -1.0, hi = 1.0, best_t = 0.0, best_d = 1e300;
        for (int round = 0; round <= TQ_REFINE; ++round) {
            const int np = round == 0 ? 65 : 128;
            double dist = 1e300, tt = 0.0;
            if (tid < np) {
                tt = round == 0 ? -1.0 + 2.0 * tid / 64.0 : lo + (hi - lo) * tid / 127.0;
                double C[3] = {0, 0, 0}, A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
                for (int i = 0; i < ns; ++i) {
                    const double l = lag(p.tn, ns, i, tt);
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
                dist = sqrt(r2);
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
        t0 = best_t;
        dstar = best_d;
    }

    // ---- outer rule: both sides of t0, innermost panel first
    const int NO = NC * MO;
    const int G = NO <= TQ_THREADS ? TQ_THREADS / NO : 1;
    const int nb = max(2, (nt + 7) / 8);
    const double lb = PI_ / nb;
    for (int side = 0; side < 2; ++side) {
        const double ell = side == 0 ? 1.0 - t0 : -1.0 - t0;
        if (ell == 0.0)
            continue;
        const int lev = dyadic_levels(fabs(ell) * speed, own ? rho_max : dstar);
        for (int pan = 0; pan <= lev; ++pan) {
            double plo, phi_;
            if (pan == 0) {
                plo = 0.0;
                phi_ = ldexp(ell, -lev);
            } else {
                const int kk = lev - pan;
                plo = ldexp(ell, -(kk + 1));
                phi_ = ldexp(ell, -kk);
            }
            const bool sing = own && pan == 0;
            const int nq = sing ? TQ_SING_N : TQ_Q;
            for (int q = 0; q < nq; ++q) {
                const double delta = sing ? phi_ * p.sx[q] : plo + (phi_ - plo) * p.gx[q];
                const double wt = sing ? fabs(phi_) * p.sw[q] : fabs(phi_ - plo) * p.gw[q];
                const double t = t0 + delta;
                // basis at t (own: offsets for i != i0, partition of unity for i0)
                if (tid < ns) {
                    s.L[tid] = own ? (tid == i0 ? 0.0 : lag_off(p.tn, ns, tid, i0, delta))
                                   : lag(p.tn, ns, tid, t);
                    s.dL[tid] = dlag(p.tn, ns, tid, t);
                }
                __syncthreads();
                if (own && tid == 0) {
                    double sum = 0.0;
                    for (int i = 0; i < ns; ++i)
                        sum += s.L[i];
                    s.SD[0] = sum;   // sum of l_i, i != i0
                }
                __syncthreads();
                if (own && tid < 9) {
                    // dC, dA, dB = sum_{i != i0} l_i (v_i - v_i0)
                    const int which = tid / 3, d = tid % 3;
                    const double *v = which == 0 ? s.sc : which == 1 ? s.sa : s.sb;
                    double acc = 0.0;
                    for (int i = 0; i < ns; ++i)
                        if (i != i0)
                            acc += s.L[i] * (v[d * ns + i] - v[d * ns + i0]);
                    s.G[18 + tid] = acc;
                }
                __syncthreads();
                if (own && tid == 0)
                    s.L[i0] = 1.0 - s.SD[0];
                __syncthreads();
                if (tid < 18) {
                    const int which = tid / 3, d = tid % 3;
                    const double *v = (which % 3 == 0) ? s.sc : (which % 3 == 1) ? s.sa : s.sb;
                    const double *basis = which < 3 ? s.L : s.dL;
                    double acc = 0.0;
                    for (int i = 0; i < ns; ++i)
                        acc += basis[i] * v[d * ns + i];
                    s.G[tid] = acc;
                }
                __syncthreads();
                const double *C = s.G, *A = s.G + 3, *B = s.G + 6;
                const double *Ct = s.G + 9, *At = s.G + 12, *Bt = s.G + 15;
                const double *dC = s.G + 18, *dA = s.G + 21, *dB = s.G + 24;
                const double thj0 = 2.0 * PI_ * j0 / nt;
                const double *a0 = nullptr, *b0 = nullptr;
                double a0v[3], b0v[3];
                if (own) {
                    for (int d = 0; d < 3; ++d) {
                        a0v[d] = s.sa[d * ns + i0];
                        b0v[d] = s.sb[d * ns + i0];
                    }
                    a0 = a0v;
                    b0 = b0v;
                }
                // y - x at angle th (own: th = thj0 + psi), offsets for the own element
                auto ymx_at = [&](double ang, double psi, double out[3]) {
                    double sn, cs;
                    sincos(ang, &sn, &cs);
                    if (own) {
                        const double sh = sin(0.5 * psi);
                        double s2, c2;
                        sincos(thj0 + 0.5 * psi, &s2, &c2);
                        const double dcos = -2.0 * s2 * sh, dsin = 2.0 * c2 * sh;
                        for (int d = 0; d < 3; ++d)
                            out[d] = dC[d] + dA[d] * cs + a0[d] * dcos + dB[d] * sn + b0[d] * dsin;
                    } else {
                        for (int d = 0; d < 3; ++d)
                            out[d] = C[d] + A[d] * cs + B[d] * sn - x[d];
                    }
                };
                // closest angle (Newton on (y - x) . y_theta; own: as an offset psi from thj0),
                // relative distance and depth of the angular rule: one thread, broadcast
                if (tid == 0) {
                    double th0;
                    if (own) {
                        th0 = 0.0;   // psi
                        for (int itn = 0; itn < 4; ++itn) {
                            const double ang = thj0 + th0;
                            double ymx[3];
                            ymx_at(ang, th0, ymx);
                            double sn, cs;
                            sincos(ang, &sn, &cs);
                            double yth[3], ythth[3];
                            for (int d = 0; d < 3; ++d) {
                                const double Ad = a0[d] + dA[d], Bd = b0[d] + dB[d];
                                yth[d] = -Ad * sn + Bd * cs;
                                ythth[d] = -Ad * cs - Bd * sn;
                            }
                            const double fp = dot3(yth, yth) + dot3(ymx, ythth);
                            if (fp <= 0.0)
                                break;
                            th0 -= dot3(ymx, yth) / fp;
                        }
                    } else {
                        const double dx[3] = {x[0] - C[0], x[1] - C[1], x[2] - C[2]};
                        th0 = atan2(dot3(dx, B), dot3(dx, A));
                        for (int itn = 0; itn < 3; ++itn) {
                            double sn, cs;
                            sincos(th0, &sn, &cs);
                            double ymx[3], yth[3], ythth[3];
                            for (int d = 0; d < 3; ++d) {
                                ymx[d] = C[d] + A[d] * cs + B[d] * sn - x[d];
                                yth[d] = -A[d] * sn + B[d] * cs;
                                ythth[d] = -A[d] * cs - B[d] * sn;
                            }
                            const double fp = dot3(yth, yth) + dot3(ymx, ythth);
                            if (fp <= 0.0)
                                break;
                            th0 -= dot3(ymx, yth) / fp;
                        }
                    }
                    double rho2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double Ad = own ? a0[d] + dA[d] : A[d];
                        const double Bd = own ? b0[d] + dB[d] : B[d];
                        rho2 += Ad * Ad + Bd * Bd;
                    }
                    const double rho = sqrt(0.5 * rho2);
                    double ymx[3];
                    ymx_at(own ? thj0 + th0 : th0, th0, ymx);
                    const double alpha_rel = sqrt(dot3(ymx, ymx)) / rho;
                    int Lv;
                    if (alpha_rel >= lb)
                        Lv = 0;
                    else if (alpha_rel <= 0.0)
                        Lv = TQ_LMAX;
                    else
                        Lv = min(TQ_LMAX, static_cast<int>(ceil(log2(lb / alpha_rel))));
                    int tl = 0;
                    if (p.rcnt && alpha_rel < 1.0 && alpha_rel >= ldexp(1.0, -TQ_RULE_MAXLEV)) {
                        tl = static_cast<int>(ceil(-log2(alpha_rel)));
                        tl = max(1, min(TQ_RULE_MAXLEV, tl));
                        if (tl >= p.rnlev || p.rcnt[tl] <= 0 || p.rcnt[tl] > TQ_RULE_SLOT)
                            tl = 0;
                    }
                    s.SD[1] = th0;
                    s.SD[2] = static_cast<double>(Lv);
                    s.SD[3] = static_cast<double>(tl);
                }
                __syncthreads();
                const double th0 = s.SD[1];
                const int L = static_cast<int>(s.SD[2]);
                const int TL = static_cast<int>(s.SD[3]);   // > 0: compressed rule of that level
                const int Mh = TQ_Q * (L + nb);
                const int M = TL ? p.rcnt[TL] : 2 * Mh;
                double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
                for (int base = 0; base < M; base += TQ_THREADS) {
                    const int kq = base + tid;
                    if (kq < M) {
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
                        double phi = lo + (hi - lo) * p.gx[qq];
                        double om = (hi - lo) * p.gw[qq];
                        if (sidek == 0)
                            phi = -phi;
                        if (TL) {
                            phi = p.rphi[TL * TQ_RULE_SLOT + kq];
                            om = p.rw[TL * TQ_RULE_SLOT + kq];
                        }
                        const double psi = th0 + phi;                 // own: offset from thj0
                        double sn, cs, ymx[3];
                        if (own) {
                            // one sincos: half-angle of psi, the rest by angle addition
                            double s2, c2;
                            sincos(0.5 * psi, &s2, &c2);
                            const double spsi = 2.0 * s2 * c2, cpsi = 1.0 - 2.0 * s2 * s2;
                            sn = sj0 * cpsi + cj0 * spsi;
                            cs = cj0 * cpsi - sj0 * spsi;
                            const double sh = sj0 * c2 + cj0 * s2;   // sin(thj0 + psi / 2)
                            const double ch = cj0 * c2 - sj0 * s2;   // cos(thj0 + psi / 2)
                            const double dcos = -2.0 * sh * s2, dsin = 2.0 * ch * s2;
                            for (int d = 0; d < 3; ++d)
                                ymx[d] = dC[d] + dA[d] * cs + a0[d] * dcos + dB[d] * sn + b0[d] * dsin;
                        } else {
                            sincos(psi, &sn, &cs);
                            for (int d = 0; d < 3; ++d)
                                ymx[d] = C[d] + A[d] * cs + B[d] * sn - x[d];
                        }
                        double yt[3], yth[3];
                        for (int d = 0; d < 3; ++d) {
                            yt[d] = Ct[d] + At[d] * cs + Bt[d] * sn;
                            yth[d] = -A[d] * sn + B[d] * cs;
                        }
                        double cr[3] = {yth[1] * yt[2] - yth[2] * yt[1], yth[2] * yt[0] - yth[0] * yt[2],
                                        yth[0] * yt[1] - yth[1] * yt[0]};
                        const double J2 = dot3(cr, cr);
                        const double invJ = rsqrt(J2);
                        const double J = J2 * invJ;
                        const double inv = sgn * invJ;
                        const double nn[3] = {cr[0] * inv, cr[1] * inv, cr[2] * inv};
                        const double r[3] = {-ymx[0], -ymx[1], -ymx[2]};
                        double K[NC];
                        kern<NC>(r, nn, p.alpha, p.beta, K);
                        const double jw = J * om;
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                            s.V[tid * NC + c] = K[c] * jw;
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
                    const int cnt = min(TQ_THREADS, M - base);
                    if (NO <= TQ_THREADS) {
                        if (tid < G * NO) {
                            const int gg = tid / NO, o = tid % NO;
                            const int c = o / MO, l = o % MO;
                            for (int kk = gg; kk < cnt; kk += G) {
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
                // modal coefficients hhat[c][l] (Eq. modal-greens-fn-coeff)
                if (NO <= TQ_THREADS) {
                    s.RED[2 * tid] = acc[0][0];
                    s.RED[2 * tid + 1] = acc[0][1];
                    __syncthreads();
                    if (tid < NO) {
                        double re = 0.0, im = 0.0;
                        for (int gg = 0; gg < G; ++gg) {
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
                        const int q = (l * j) % nt;
                        h += 2.0 * (hh[2 * l] * s.W[2 * q] + hh[2 * l + 1] * s.W[2 * q + 1]);
                    }
                    const int qn = ((MO - 1) * j) % nt;
                    h += hh[2 * (MO - 1)] * s.W[2 * qn];
                    s.H[e] = h / nt;
                }
                __syncthreads();
                for (int e = tid; e < NC * ns * nt; e += TQ_THREADS) {
                    const int c = e / (ns * nt), rem = e % (ns * nt);
                    const int i = rem / nt, j = rem % nt;
                    s.EB[e] += wt * s.L[i] * s.H[c * nt + j];
                }
                __syncthreads();
            }
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
    p.rcnt = nullptr;
    p.rnlev = 0;

    AsyncAllocScope scope(s);
    std::vector<long long> cnt_off;
    std::vector<int> h_cnt, h_list;
    DevBuf d_geo, d_bad, d_cnt, d_off, d_list;
    if (ntube > 0 && ntarget > 0) {
        SBQ_TRY(d_geo.alloc(nelem * sizeof(ElemGeo)));
        SBQ_TRY(d_bad.alloc(sizeof(int)));
        SBQ_TRY(d_cnt.alloc(ntarget * sizeof(int)));
        SBQ_CUDA(cudaMemsetAsync(d_bad.p, 0, sizeof(int), s));
        const unsigned ge = static_cast<unsigned>((nelem + 63) / 64);
        k_elem_setup<<<ge, 64, 0, s>>>(nelem, p, src, nrm, d_geo.as<ElemGeo>(), d_bad.as<int>());
        SBQ_CUDA(cudaGetLastError());
        const unsigned gt = static_cast<unsigned>((ntarget + 127) / 128);
        k_near<<<gt, 128, 0, s>>>(ntarget, nelem, p, near_factor, src, trg, d_geo.as<ElemGeo>(),
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
        k_near<<<gt, 128, 0, s>>>(ntarget, nelem, p, near_factor, src, trg, d_geo.as<ElemGeo>(),
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

// Quadrature correction with compressed angular rules (see sbq.h): the same builder, the
// angular integrals of relative distance 2^-30 <= alpha < 1 taken with the caller's rule of
// level ceil(-log2 alpha) instead of the dyadic one.
extern "C" __attribute__((visibility("default"))) int tube_correction_rules(
    int64_t nelem, int ns, int nt, int64_t n_total, const double *src, const double *nrm,
    const double *w, int64_t ntrg, const double *trg, int laplace, double alpha, double beta,
    double near_factor, int nlev, const double *rule_phi, const double *rule_w,
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
    if (nlev < 1 || nlev > TQ_RULE_MAXLEV + 1 || !rule_phi || !rule_w || !rule_cnt)
        return bad("rules: nlev must be in 1..31 with non-null tables");
    for (int l = 0; l < nlev; ++l) {
        if (rule_cnt[l] < 0 || rule_cnt[l] > TQ_RULE_SLOT)
            return bad("rules: a level holds more than 64 nodes");
        for (int m = 0; m < rule_cnt[l]; ++m) {
            const double a = rule_phi[l * TQ_RULE_SLOT + m], b = rule_w[l * TQ_RULE_SLOT + m];
            if (!std::isfinite(a) || !std::isfinite(b) || std::fabs(a) > 3.14159265358979323846)
                return bad("rules: non-finite entry or offset outside [-pi, pi]");
        }
    }
    return build_tube_correction(nelem, ns, nt, n_total, src, nrm, w, trg ? ntrg : 0, trg,
                                 laplace, alpha, beta, near_factor, nnz_out, rowptr, col, val,
                                 static_cast<cudaStream_t>(stream), nlev, rule_phi, rule_w,
                                 rule_cnt);
}
