/*
 * CPU FP64 oracle for the Stokes boundary-integral pair sums.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plainly written reference
 * that the CUDA path is checked against.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * What it computes (all arrays are structure-of-arrays, FP64):
 *   points  p[0..n) = x, p[n..2n) = y, p[2n..3n) = z   (same for normals,
 *   densities and outputs).
 *
 *   Uncorrected Nystrom sum, paper Sec. 3.2.1, Eq. (nystrom-no-correction):
 *     u(x_t) = sum_{s : y_s != x_t} G(x_t, y_s) w_s sigma_s
 *   with G = alpha * S + beta * D, where
 *     S(r)      = (1/(8 pi)) (I/|r| + r r^T/|r|^3)                 paper Eq. (stokes-sl)
 *     D(r; n)   = (3/(4 pi)) (r . n) r r^T / |r|^5,   r = x - y    paper Eq. (stokes-dl)
 *   The paper prints D with a leading minus sign for r = x - y and outward n.
 *   That sign gives  int D[e] = +e  inside a closed surface, which contradicts
 *   the paper's own exterior limit I/2 + D (Eq. stokes-bie-new), its null-space
 *   statement (I/2 + D) v = 0 for rigid motions (Prop. p:null) and the interior
 *   Green's representation u = S[T] - D[u] (Appendix A).  All three hold with
 *   the sign used here, which equals the printed formula with r = y - x.
 *   A source whose position equals the target (the target's own node when the
 *   target lies on the surface) is skipped: the punctured Nystrom sum, to which
 *   the paper's local correction E (Eq. nystrom-correction) is later added.
 *
 * Each function below builds the 3x3 kernel tensor of every pair explicitly and
 * multiplies it with w_s sigma_s, in source order, one target per OpenMP
 * iteration.  No blocking, no reordering, no tricks.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

/* Stokeslet tensor S(r) = (1/8pi)(I/|r| + r r^T / |r|^3), paper Eq. (stokes-sl). */
static void stokeslet_tensor(const double r[3], double S[3][3])
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rl = sqrt(r2);
    double r3 = rl * r2;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = ((i == j ? 1.0 / rl : 0.0) + r[i] * r[j] / r3) / (8.0 * ORACLE_PI);
}

/* Stresslet (double-layer velocity) tensor D(r; n) = (3/4pi)(r.n) r r^T / |r|^5,
 * r = x - y, n = outward unit normal at the source y (sign reading: see header). */
static void stresslet_tensor(const double r[3], const double n[3], double D[3][3])
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rl = sqrt(r2);
    double r5 = r2 * r2 * rl;
    double rdn = r[0] * n[0] + r[1] * n[1] + r[2] * n[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            D[i][j] = 3.0 / (4.0 * ORACLE_PI) * rdn * r[i] * r[j] / r5;
}

/*
 * u = sum_s [alpha S(x_t - y_s) + beta D(x_t - y_s; n_s)] w_s sigma_s, skipping y_s == x_t.
 * nrm may be NULL when beta == 0.  u is overwritten.
 */
void oracle_stokes_combined(int64_t ns, const double *src, const double *nrm, const double *w,
                            const double *sigma, int64_t nt, const double *trg,
                            double alpha, double beta, double *u)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        double x[3] = {trg[t], trg[nt + t], trg[2 * nt + t]};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t s = 0; s < ns; ++s) {
            double y[3] = {src[s], src[ns + s], src[2 * ns + s]};
            if (y[0] == x[0] && y[1] == x[1] && y[2] == x[2])
                continue;                                   /* punctured sum */
            double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
            double f[3] = {w[s] * sigma[s], w[s] * sigma[ns + s], w[s] * sigma[2 * ns + s]};
            if (alpha != 0.0) {
                double S[3][3];
                stokeslet_tensor(r, S);
                for (int i = 0; i < 3; ++i)
                    acc[i] += alpha * (S[i][0] * f[0] + S[i][1] * f[1] + S[i][2] * f[2]);
            }
            if (beta != 0.0) {
                double n[3] = {nrm[s], nrm[ns + s], nrm[2 * ns + s]};
                double D[3][3];
                stresslet_tensor(r, n, D);
                for (int i = 0; i < 3; ++i)
                    acc[i] += beta * (D[i][0] * f[0] + D[i][1] * f[1] + D[i][2] * f[2]);
            }
        }
        u[t] = acc[0];
        u[nt + t] = acc[1];
        u[2 * nt + t] = acc[2];
    }
}

/* Single-layer velocity potential S[sigma] at the targets (paper Eq. stokes-sl). */
void oracle_stokes_sl(int64_t ns, const double *src, const double *w, const double *sigma,
                      int64_t nt, const double *trg, double *u)
{
    oracle_stokes_combined(ns, src, NULL, w, sigma, nt, trg, 1.0, 0.0, u);
}

/* Double-layer velocity potential D[sigma] at the targets (paper Eq. stokes-dl). */
void oracle_stokes_dl(int64_t ns, const double *src, const double *nrm, const double *w,
                      const double *sigma, int64_t nt, const double *trg, double *u)
{
    oracle_stokes_combined(ns, src, nrm, w, sigma, nt, trg, 0.0, 1.0, u);
}

/*
 * y += E x for a CSR matrix E (rows/cols are component-major SoA indices,
 * c * n + node), the sparse local correction of paper Eq. (nystrom-correction).
 */
void oracle_csr_apply(int64_t nrows, const int64_t *rowptr, const int64_t *col,
                      const double *val, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nrows; ++i) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += val[k] * x[col[k]];
        y[i] += acc;
    }
}

/*
 * Combined-field operator on the surface nodes (targets = sources):
 *   out = diag * sigma + (D + eta S)[sigma] + E sigma,
 * the discretised K = I/2 + D + eta S of paper Eq. (stokes-bie-new) with
 * diag = 1/2, the uncorrected sum plus the optional sparse correction E.
 */
void oracle_stokes_matvec(int64_t n, const double *src, const double *nrm, const double *w,
                          double eta, double diag, int64_t nnz, const int64_t *rowptr,
                          const int64_t *col, const double *val, const double *sigma,
                          double *out)
{
    oracle_stokes_combined(n, src, nrm, w, sigma, n, src, eta, 1.0, out);
    for (int64_t i = 0; i < 3 * n; ++i)
        out[i] += diag * sigma[i];
    if (nnz > 0)
        oracle_csr_apply(3 * n, rowptr, col, val, sigma, out);
}

/*
 * Laplace (paper Sec. 4.1): single layer G(r) = 1/(4 pi |r|), double layer
 * dG/dn_y = ((x - y) . n_y) / (4 pi |x - y|^3) (the double layer of a constant is -1
 * inside a closed surface with outward normals, 0 outside: consistent with the interior
 * Green's representation u = S[du/dn] - D[u] of Eq. greens-rep).
 *   u(x_t) = sum_{s : y_s != x_t} (alpha G + beta dG/dn_y) w_s sigma_s,  scalar sigma and u.
 */
void oracle_laplace_combined(int64_t ns, const double *src, const double *nrm, const double *w,
                             const double *sigma, int64_t nt, const double *trg, double alpha,
                             double beta, double *u)
{
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < nt; ++t) {
        const double x[3] = {trg[t], trg[nt + t], trg[2 * nt + t]};
        double acc = 0.0;
        for (int64_t s = 0; s < ns; ++s) {
            const double r[3] = {x[0] - src[s], x[1] - src[ns + s], x[2] - src[2 * ns + s]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0)
                continue;
            const double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double g = 0.0;
            if (alpha != 0.0)
                g += alpha / (4.0 * ORACLE_PI * rl);
            if (beta != 0.0) {
                const double rn = r[0] * nrm[s] + r[1] * nrm[ns + s] + r[2] * nrm[2 * ns + s];
                g += beta * rn / (4.0 * ORACLE_PI * rl * rl * rl);
            }
            acc += g * w[s] * sigma[s];
        }
        u[t] = acc;
    }
}

int oracle_num_threads(void)
{
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}
