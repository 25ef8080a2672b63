// Double-layer singularity subtraction as a sparse correction E (paper Eq.
// nystrom-correction supplies the singular part of each node's own integral through a
// sparse E; this builds the classical local form of it for the double layer).
//
// On a closed surface the double layer of a constant density is -e/2 on the surface
// (Gauss-type identity of the double layer, the pv value between -e inside and 0
// outside).  Writing D[sigma](x_i) = D[sigma - sigma_i](x_i) + D[sigma_i](x_i) and
// replacing the second term by its exact value -sigma_i / 2 gives, per node i of body b,
//   E_ii = -R_i - I/2,   R_i = sum over j in b, j != i, of D(x_i, y_j; n_j) w_j  (3 x 3).
// With diag = 1/2 the operator then applies sum_j D_ij (sigma_j - sigma_i) over the
// node's own body, whose summand is bounded at r -> 0, plus the plain sums over the
// other bodies (their double layer is smooth at x_i).
// R is formed by three batched double-layer applies (one per unit density e_b) with one
// segment per body, so only the node's own body enters its row sum.
#include "engine.h"

namespace sbq {

namespace {

__global__ void k_unit_density(double *sig, long long n, int comp)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < 3 * n)
        sig[i] = (i / n == comp) ? 1.0 : 0.0;
}

// R: [b][a][i] = component a at node i of D[e_b].  Row (a, i) of E holds the three
// entries (a, i) x (b, i), b = 0..2, in column order.
__global__ void k_gauss_csr(long long n, const double *__restrict__ R, int64_t *rowptr,
                            int64_t *col, double *val)
{
    const long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (r >= 3 * n)
        return;
    const int a = static_cast<int>(r / n);
    const long long i = r - a * n;
    rowptr[r] = 3 * r;
    if (r == 0)
        rowptr[3 * n] = 9 * n;
    for (int b = 0; b < 3; ++b) {
        col[3 * r + b] = b * n + i;
        val[3 * r + b] = -R[(static_cast<long long>(b) * 3 + a) * n + i] - (a == b ? 0.5 : 0.0);
    }
}

}  // namespace

int dl_gauss_correction(int nbody, const int64_t *body_off, const double *src, const double *nrm,
                        const double *w, int prec, int64_t *rowptr, int64_t *col, double *val,
                        cudaStream_t s)
{
    const long long n = body_off[nbody];
    if (n == 0) {
        SBQ_CUDA(cudaMemsetAsync(rowptr, 0, sizeof(int64_t), s));
        return SBQ_OK;
    }
    int kind;
    double scale, kappa;
    kind_and_scale(0.0, 1.0, &kind, &scale, &kappa);
    const int layout = (prec == SBQ_FP64 || prec == SBQ_DF32) ? prec : SBQ_FP32;
    AsyncAllocScope scope(s);
    const std::vector<int64_t> off(body_off, body_off + nbody + 1);
    SrcPack sp;
    TrgSet ts;
    SBQ_TRY(build_src_pack(sp, layout, off, src, nrm, 1.0, n, s));
    SBQ_TRY(build_trg_set(ts, kind, prec, default_tune(prec, n), sp, off, src, n, off, s));
    DevBuf sig, R;
    SBQ_TRY(sig.alloc(3 * static_cast<size_t>(n) * sizeof(double)));
    SBQ_TRY(R.alloc(9 * static_cast<size_t>(n) * sizeof(double)));
    const int T = 256;
    const unsigned g3 = static_cast<unsigned>((3 * n + T - 1) / T);
    for (int b = 0; b < 3; ++b) {
        k_unit_density<<<g3, T, 0, s>>>(sig.as<double>(), n, b);
        SBQ_CUDA(cudaGetLastError());
        SBQ_TRY(run_pairsum(kind, prec, sp, ts, w, sig.as<double>(), n, src, n,
                            R.as<double>() + static_cast<size_t>(b) * 3 * n, scale, kappa, 0.0,
                            nullptr, s));
    }
    k_gauss_csr<<<g3, T, 0, s>>>(n, R.as<double>(), rowptr, col, val);
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}

}  // namespace sbq
