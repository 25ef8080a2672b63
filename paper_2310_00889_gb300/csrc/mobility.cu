// Stokes mobility problem, slender combined-field formulation (paper Sec. 4.2,
// Eqs. new-mobility-rep, new-mobility-bie, recover-rigidbody-motion):
//   (K (I - L) + L) sigma = u_s - S nu,    V = -L sigma,
// with K = I/2 + D + eta S (+ E) the operator of the handle, L the orthogonal projector onto
// the rigid-body motions of each body in the quadrature-weighted L^2 inner product
// <f, g> = sum_j w_j f_j . g_j, and nu the completion-flow density: the rigid motion of each
// body whose force and torque moments are the given (F_b, T_b).
//
// On body b with weights w_j, nodes x_j, area A_b = sum w_j, weighted centroid c_b and
// inertia I_b = sum w_j (|d_j|^2 I - d_j d_j^T), d_j = x_j - c_b, a rigid field
// r(x) = U + Omega x (x - c_b) has moments sum w r = A_b U and sum w d x r = I_b Omega (the
// first moment sum w d vanishes about the centroid).  Hence the projection of sigma is the
// rigid field with U = (sum w sigma) / A_b, Omega = I_b^-1 (sum w d x sigma), the completion
// flow has U = F_b / A_b, Omega = I_b^-1 T_b (torque about c_b), and the rigid velocity
// V = -L sigma.  The moments are reduced per body in a fixed order (blocks of one body,
// partials summed in block order), so results are deterministic.
#include "engine.h"

#include <cmath>

namespace sbq {

namespace {

constexpr int MB = 256;   // threads of the mobility kernels

// Per block: moments sum w sigma and sum w d x sigma over its node range of one body.
__global__ void k_mob_moments(const int4 *__restrict__ blk, const double *__restrict__ x,
                              const double *__restrict__ w, const double *__restrict__ cen,
                              const double *__restrict__ sigma, long long n, double *part)
{
    const int4 b = blk[blockIdx.x];
    const double cx = cen[3 * b.z], cy = cen[3 * b.z + 1], cz = cen[3 * b.z + 2];
    double m[6] = {0, 0, 0, 0, 0, 0};
    for (long long j = b.x + threadIdx.x; j < b.y; j += blockDim.x) {
        const double wj = w[j];
        const double sx = wj * sigma[j], sy = wj * sigma[n + j], sz = wj * sigma[2 * n + j];
        const double dx = x[j] - cx, dy = x[n + j] - cy, dz = x[2 * n + j] - cz;
        m[0] += sx;
        m[1] += sy;
        m[2] += sz;
        m[3] += dy * sz - dz * sy;
        m[4] += dz * sx - dx * sz;
        m[5] += dx * sy - dy * sx;
    }
    __shared__ double red[6][MB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k) {
        double v = m[k];
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int i = 0; i < MB / 32; ++i)
            v += red[threadIdx.x][i];
        part[6 * static_cast<size_t>(blockIdx.x) + threadIdx.x] = v;
    }
}

// Per body: rigid motion (U, Omega) = sign x (moments / A, I^-1 torque moment).
__global__ void k_mob_rigid(const int2 *__restrict__ bodyblk, const double *__restrict__ part,
                            const double *__restrict__ area, const double *__restrict__ iinv,
                            int nbody, double sign, double *rigid)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbody)
        return;
    double m[6] = {0, 0, 0, 0, 0, 0};
    const int2 bb = bodyblk[b];
    for (int i = 0; i < bb.y; ++i)
        for (int k = 0; k < 6; ++k)
            m[k] += part[6 * static_cast<size_t>(bb.x + i) + k];
    const double a = area[b];
    const double *J = iinv + 9 * b;
    for (int k = 0; k < 3; ++k) {
        rigid[6 * b + k] = a > 0.0 ? sign * m[k] / a : 0.0;
        rigid[6 * b + 3 + k] = sign * (J[3 * k] * m[3] + J[3 * k + 1] * m[4] + J[3 * k + 2] * m[5]);
    }
}

// out = base + s_r x r(x), r the rigid field of each node's body (base may be null: 0).
__global__ void k_mob_field(long long n, const int *__restrict__ body_of,
                            const double *__restrict__ x, const double *__restrict__ cen,
                            const double *__restrict__ rigid, const double *base, double s_r,
                            double *out)
{
    for (long long j = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int b = body_of[j];
        double r[3] = {0.0, 0.0, 0.0};
        if (b >= 0) {
            const double *R = rigid + 6 * b;
            const double dx = x[j] - cen[3 * b], dy = x[n + j] - cen[3 * b + 1],
                         dz = x[2 * n + j] - cen[3 * b + 2];
            r[0] = R[0] + R[4] * dz - R[5] * dy;
            r[1] = R[1] + R[5] * dx - R[3] * dz;
            r[2] = R[2] + R[3] * dy - R[4] * dx;
        }
        for (int c = 0; c < 3; ++c)
            out[c * n + j] = (base ? base[c * n + j] : 0.0) + s_r * r[c];
    }
}

unsigned field_grid(long long n)
{
    const long long b = (n + MB - 1) / MB;
    return static_cast<unsigned>(std::min<long long>(std::max<long long>(b, 1), 4096));
}

}  // namespace

int mob_setup(Op *op, int nbody, const int64_t *body_off, cudaStream_t s)
{
    const long long n = op->n;
    auto mob = std::make_unique<MobState>();
    mob->nbody = nbody;
    // geometry in the caller's order (the operator keeps it permuted)
    std::vector<double> hx(3 * n), hxi(3 * n), hw(n), hwi(n);
    std::vector<int> perm(n);
    SBQ_CUDA(cudaMemcpy(hxi.data(), op->src.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
    SBQ_CUDA(cudaMemcpy(hwi.data(), op->w.p, n * sizeof(double), cudaMemcpyDeviceToHost));
    SBQ_CUDA(cudaMemcpy(perm.data(), op->perm.p, n * sizeof(int), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < n; ++k) {
        const long long u = perm[k];
        for (int c = 0; c < 3; ++c)
            hx[c * n + u] = hxi[c * n + k];
        hw[u] = hwi[k];
    }
    std::vector<double> cen(3 * nbody), area(nbody), iinv(9 * nbody);
    std::vector<int> body_of(n, -1);
    std::vector<int4> blk;
    std::vector<int2> bodyblk(nbody);
    const long long chunk = 4096;
    for (int b = 0; b < nbody; ++b) {
        const long long a0 = body_off[b], a1 = body_off[b + 1];
        double A = 0.0, m[3] = {0, 0, 0};
        for (long long j = a0; j < a1; ++j) {
            A += hw[j];
            for (int c = 0; c < 3; ++c)
                m[c] += hw[j] * hx[c * n + j];
            body_of[j] = b;
        }
        for (int c = 0; c < 3; ++c)
            cen[3 * b + c] = A > 0.0 ? m[c] / A : 0.0;
        double I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (long long j = a0; j < a1; ++j) {
            const double d[3] = {hx[j] - cen[3 * b], hx[n + j] - cen[3 * b + 1],
                                 hx[2 * n + j] - cen[3 * b + 2]};
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                    I[p][q] += hw[j] * ((p == q ? d2 : 0.0) - d[p] * d[q]);
        }
        const double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                           I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                           I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
        if (a1 > a0 && !(std::fabs(det) > 0.0)) {
            set_error("body " + std::to_string(b) + " has a singular inertia tensor");
            return SBQ_EINVAL;
        }
        double *J = iinv.data() + 9 * b;
        if (a1 > a0) {
            J[0] = (I[1][1] * I[2][2] - I[1][2] * I[2][1]) / det;
            J[1] = (I[0][2] * I[2][1] - I[0][1] * I[2][2]) / det;
            J[2] = (I[0][1] * I[1][2] - I[0][2] * I[1][1]) / det;
            J[3] = (I[1][2] * I[2][0] - I[1][0] * I[2][2]) / det;
            J[4] = (I[0][0] * I[2][2] - I[0][2] * I[2][0]) / det;
            J[5] = (I[0][2] * I[1][0] - I[0][0] * I[1][2]) / det;
            J[6] = (I[1][0] * I[2][1] - I[1][1] * I[2][0]) / det;
            J[7] = (I[0][1] * I[2][0] - I[0][0] * I[2][1]) / det;
            J[8] = (I[0][0] * I[1][1] - I[0][1] * I[1][0]) / det;
        }
        area[b] = A;
        bodyblk[b].x = static_cast<int>(blk.size());
        for (long long j = a0; j < a1; j += chunk)
            blk.push_back(make_int4(static_cast<int>(j), static_cast<int>(std::min(a1, j + chunk)), b, 0));
        bodyblk[b].y = static_cast<int>(blk.size()) - bodyblk[b].x;
    }
    mob->h_area = area;
    mob->h_iinv = iinv;
    mob->h_cen = cen;
    mob->nblk = static_cast<int>(blk.size());
    SBQ_TRY(mob->x.alloc(3 * n * sizeof(double)));
    SBQ_TRY(mob->w.alloc(n * sizeof(double)));
    SBQ_TRY(mob->body_of.alloc(n * sizeof(int)));
    SBQ_TRY(mob->blk.alloc(std::max<size_t>(1, blk.size()) * sizeof(int4)));
    SBQ_TRY(mob->bodyblk.alloc(nbody * sizeof(int2)));
    SBQ_TRY(mob->cen.alloc(3 * nbody * sizeof(double)));
    SBQ_TRY(mob->area.alloc(nbody * sizeof(double)));
    SBQ_TRY(mob->iinv.alloc(9 * nbody * sizeof(double)));
    SBQ_TRY(mob->part.alloc(std::max<size_t>(1, blk.size()) * 6 * sizeof(double)));
    SBQ_TRY(mob->rigid.alloc(6 * nbody * sizeof(double)));
    SBQ_TRY(mob->y.alloc(3 * n * sizeof(double)));
    SBQ_TRY(mob->r.alloc(3 * n * sizeof(double)));
    SBQ_CUDA(cudaMemcpy(mob->x.p, hx.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->w.p, hw.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->body_of.p, body_of.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    if (!blk.empty())
        SBQ_CUDA(cudaMemcpy(mob->blk.p, blk.data(), blk.size() * sizeof(int4), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->bodyblk.p, bodyblk.data(), nbody * sizeof(int2), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->cen.p, cen.data(), 3 * nbody * sizeof(double), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->area.p, area.data(), nbody * sizeof(double), cudaMemcpyHostToDevice));
    SBQ_CUDA(cudaMemcpy(mob->iinv.p, iinv.data(), 9 * nbody * sizeof(double), cudaMemcpyHostToDevice));
    (void)s;
    op->mob = std::move(mob);
    if (op->gm) {   // captured solver graphs hold the old operator
        gmres_destroy(op->gm);
        op->gm = nullptr;
    }
    return SBQ_OK;
}

// rigid[] = sign x (L sigma)'s rigid motions, per body.
int mob_project(const Op *op, const double *sigma, double sign, cudaStream_t s)
{
    const MobState &m = *op->mob;
    if (m.nblk > 0)
        k_mob_moments<<<m.nblk, MB, 0, s>>>(m.blk.as<int4>(), m.x.as<double>(), m.w.as<double>(),
                                            m.cen.as<double>(), sigma, op->n, m.part.as<double>());
    k_mob_rigid<<<(m.nbody + 127) / 128, 128, 0, s>>>(m.bodyblk.as<int2>(), m.part.as<double>(),
                                                      m.area.as<double>(), m.iinv.as<double>(),
                                                      m.nbody, sign, m.rigid.as<double>());
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

// out = base + s_r x (the rigid field in mob->rigid).
int mob_field(const Op *op, const double *base, double s_r, double *out, cudaStream_t s)
{
    const MobState &m = *op->mob;
    k_mob_field<<<field_grid(op->n), MB, 0, s>>>(op->n, m.body_of.as<int>(), m.x.as<double>(),
                                                 m.cen.as<double>(), m.rigid.as<double>(), base,
                                                 s_r, out);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

int mob_rhs(Op *op, const double *FT, const double *us, double *rhs, int prec, cudaStream_t s)
{
    MobState &m = *op->mob;
    std::vector<double> rig(6 * m.nbody);
    for (int b = 0; b < m.nbody; ++b) {
        const double *J = m.h_iinv.data() + 9 * b;
        const double *T = FT + 6 * b + 3;
        for (int k = 0; k < 3; ++k) {
            rig[6 * b + k] = m.h_area[b] > 0.0 ? FT[6 * b + k] / m.h_area[b] : 0.0;
            rig[6 * b + 3 + k] = J[3 * k] * T[0] + J[3 * k + 1] * T[1] + J[3 * k + 2] * T[2];
        }
    }
    SBQ_CUDA(cudaMemcpyAsync(m.rigid.p, rig.data(), rig.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    // nu on the nodes, then S nu with the operator's packs (single-layer kind)
    SBQ_TRY(mob_field(op, nullptr, 1.0, m.r.as<double>(), s));
    SBQ_TRY(op_ensure_tuned(op, prec, s));
    int kind;
    double scale, kappa;
    kind_and_scale(1.0, 0.0, &kind, &scale, &kappa);
    const SrcPack &sp = (prec == SBQ_FP64) ? op->sp64 : (prec == SBQ_DF32 ? op->spdf : op->sp32);
    SBQ_TRY(run_pairsum(kind, prec, sp, *op->ts[prec], op->w.as<double>(), m.r.as<double>(),
                        op->n, op->src.as<double>(), op->n, m.y.as<double>(), scale, kappa, 0.0,
                        nullptr, s, nullptr, op->perm.as<int>()));
    // the accurate single layer: the punctured sum plus its correction, when one is set
    if (op->sl_nnz > 0)
        SBQ_CUDA(launch_csr_apply(3 * op->n, op->sl_rowptr.as<int64_t>(), op->sl_col.as<int64_t>(),
                                  op->sl_val.as<double>(), m.r.as<double>(), m.y.as<double>(), s));
    // rhs = u_s - S nu
    SBQ_CUDA(cudaMemsetAsync(rhs, 0, 3 * op->n * sizeof(double), s));
    if (us)
        SBQ_CUDA(cudaMemcpyAsync(rhs, us, 3 * op->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SBQ_TRY(mob_axpy(op->n, -1.0, m.y.as<double>(), rhs, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

int mob_velocity(Op *op, const double *sigma, double *UW, cudaStream_t s)
{
    MobState &m = *op->mob;
    SBQ_TRY(mob_project(op, sigma, -1.0, s));
    SBQ_CUDA(cudaMemcpyAsync(UW, m.rigid.p, 6 * m.nbody * sizeof(double), cudaMemcpyDeviceToHost, s));
    SBQ_CUDA(cudaStreamSynchronize(s));
    return SBQ_OK;
}

namespace {
__global__ void k_axpy(long long N, double a, const double *__restrict__ x, double *y)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}
}  // namespace

int mob_axpy(long long n, double a, const double *x, double *y, cudaStream_t s)
{
    k_axpy<<<field_grid(3 * n), MB, 0, s>>>(3 * n, a, x, y);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

}  // namespace sbq
