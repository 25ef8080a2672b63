/*
 * sbq.h — C ABI of the GB300 (sm_103a) Stokes boundary-integral hot path.
 *
 * The library evaluates the uncorrected Nystrom sums of the Stokes single- and
 * double-layer velocity potentials between surface quadrature nodes and target
 * points (Malhotra & Barnett, arXiv 2310.00889, Sec. 3.2.1,
 * Eq. nystrom-no-correction), the combined-field operator
 * K = diag I + D + eta S (+ sparse correction E, Eq. nystrom-correction) of the
 * slender-body BIE (Sec. 4.1, Eq. stokes-bie-new), and solves K sigma = u0 with
 * GMRES (plain FP64 or double-float, or FP32 / compensated-FP32 inner solves with
 * FP64 or bound-certified double-float iterative refinement).  Also: the Laplace
 * layers and operator (Sec. 4.1), the Stokes mobility formulation (Sec. 4.2), the
 * paper's quadrature correction E of tube elements (Sec. 3.2.1-3.2.4, tube_correction)
 * and the double-layer singularity subtraction as a sparse correction.
 *
 * Kernels (viscosity 1, r = x - y, n = outward unit normal at the source y):
 *   S(r)    = (1/8pi) (I/|r| + r r^T / |r|^3)                     Eq. stokes-sl
 *   D(r; n) = (3/4pi) (r . n) r r^T / |r|^5                       Eq. stokes-dl
 * The double-layer sign is the one for which the paper's identities hold:
 * int D[e] = -e inside a closed surface, (I/2 + D) v = 0 for rigid motions
 * (Prop. p:null), u = S[T] - D[u] inside (Appendix A).  The formula printed in
 * Eq. stokes-dl carries the opposite sign for r = x - y.
 *
 * Conventions for every function:
 *  - Arrays are FP64, structure-of-arrays: a point set of n points is 3*n
 *    doubles x[0..n), y[0..n), z[0..n); densities and velocities likewise.
 *  - Pointers are DEVICE pointers unless a comment says otherwise.  Inputs are
 *    only read; outputs are overwritten.  The caller owns every buffer it passes.
 *  - Handles (plans, operators) are owned by the library: create them with the
 *    create calls and free them with sbq_destroy().
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All device work
 *    is enqueued on it; apply/matvec calls return without synchronising.
 *  - Every function returns an sbq_status; nothing is thrown across the ABI.  On
 *    failure sbq_last_error() (per host thread) describes the reason.
 *  - A source whose coordinates equal a target's exactly is skipped (the
 *    punctured sum; the correction E adds the true singular part).  The FP64
 *    path skips exactly those pairs.  The FP32 paths skip pairs closer than
 *    4e-6 times the sum of the radii of the two tiles (256 points) holding them,
 *    which catches every coincident pair whatever the FP32 rounding; they
 *    therefore require distinct points to be farther apart than that, and pair
 *    distances above ~1e-7 in the units of the input.  The double-float path
 *    uses 1e-10 of the radii of its 128-point tiles.
 *  - Operator handles may keep their nodes in an internal order (per segment, the
 *    caller's order or a recursive bisection of the nodes, whichever gives more
 *    compact tiles); every vector crossing the ABI is in the caller's order.
 */
#ifndef SBQ_H
#define SBQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBQ_API __attribute__((visibility("default")))

typedef enum {
    SBQ_OK = 0,
    SBQ_EINVAL = 1,       /* bad argument (null pointer, negative size, bad enum) */
    SBQ_ECUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    SBQ_ENOCONV = 3,      /* GMRES hit its iteration cap above the tolerance */
    SBQ_EBREAKDOWN = 4,   /* GMRES breakdown without convergence */
    SBQ_ENONFINITE = 5,   /* a NaN or Inf appeared (input or residual) */
    SBQ_ETIMEOUT = 6,     /* a device-side bounded wait expired (copy never landed) */
    SBQ_ENOMEM = 7        /* device allocation failed */
} sbq_status;

typedef enum {
    SBQ_FP64 = 0,         /* FP64 pair arithmetic and accumulation */
    SBQ_FP32 = 1,         /* FP32 pair arithmetic, plain FP32 accumulation per work item */
    SBQ_FP32_COMP = 2,    /* FP32 pair arithmetic, TwoSum-compensated (hi, lo) accumulation */
    SBQ_DF32 = 3          /* double-float: every value an unevaluated sum of two FP32 numbers,
                             error-free transformations throughout; about 1e-13 of the largest
                             term (FP64: 1e-15) at several times the FP64 pair rate */
} sbq_prec;

/* Tile shape of the pair-sum kernels.  targets per CTA = 32 * warps * r. */
typedef struct {
    int r;             /* targets per thread held in registers */
    int warps;         /* warps per CTA.  (r, warps): FP32 (1,4) (1,8) (2,4) (4,4) (8,4) (4,8) (4,2) (8,2);
                          FP64 (1,4) (2,4); DF32 (1,4) (2,4) (4,4) (2,8) */
    int chunk_tiles;   /* source tiles per work item; 0 = chosen from the SM count */
} sbq_tune;

/* GMRES options (Sec. 4: unpreconditioned GMRES; restart and orthogonalisation
 * are not specified by the paper: restarted GMRES(m), classical Gram-Schmidt
 * applied twice, Givens rotations, FP64 throughout except the inner operator). */
typedef struct {
    double tol;        /* stop when ||b - K x||_2 <= tol * ||b||_2 (FP64 true residual) */
    int restart;       /* Krylov vectors per cycle m, 1..256 */
    int max_iter;      /* cap on Arnoldi steps (summed over cycles and refinement steps) */
    int inner_prec;    /* SBQ_FP64 / SBQ_DF32: plain GMRES with K applied in that precision.
                          SBQ_FP32 / SBQ_FP32_COMP: the inner GMRES applies K in that
                          precision and a residual b - K x in resid_prec refines x
                          (iterative refinement) */
    double inner_tol;  /* relative tolerance of each inner solve (refinement only) */
    int max_outer;     /* cap on refinement steps */
    int use_graph;     /* 1: each Arnoldi step runs inside one CUDA graph whose while
                          node repeats it on the device until the cycle ends */
    int resid_prec;    /* refinement only: SBQ_FP64 (0, default) or SBQ_DF32, the precision of
                          the residuals b - K x that decide convergence.  A double-float
                          residual carries a bound on its rounding error; where the bound
                          exceeds tol/4 of a segment's ||b||, the residual is recomputed in
                          FP64 and the solve continues with FP64 residuals */
} sbq_gmres_opts;

#define SBQ_HIST 64
typedef struct {
    int status;               /* sbq_status of the solve */
    int iters;                /* Arnoldi steps in total */
    int outer_iters;          /* refinement steps (mixed) or restart cycles (FP64) */
    int matvecs_fp64;         /* operator applications in the high precision (SBQ_FP64 or
                                 SBQ_DF32: the plain solve's precision or resid_prec) */
    int matvecs_low;          /* FP32 / compensated-FP32 operator applications */
    int graph_used;           /* 1 if the Arnoldi steps ran inside a CUDA graph */
    int kernel_launches;      /* kernels of this library executed by the solve (graph
                                 replays included) */
    double rel_res;           /* final true relative residual ||b - K x|| / ||b||, computed in
                                 FP64, or in double-float plus its rounding-error bound (an
                                 upper bound); for an operator with a batch plan, the largest
                                 of the segments' ratios (each segment is solved to tol on its
                                 own norm) */
    int n_hist;               /* entries used in rel_res_hist */
    double rel_res_hist[SBQ_HIST]; /* the decisive relative residual (as rel_res) after each
                                      refinement step / restart cycle, starting with x0 */
    double time_ms;           /* wall time of the solve on the host clock */
    int resid_fallbacks;      /* double-float residuals whose error bound was too large to
                                 certify the tolerance, recomputed in FP64 (the solve then
                                 continued in FP64) */
} sbq_gmres_report;

/* Library version (major * 10000 + minor * 100 + patch). */
SBQ_API int sbq_version(void);

/* Description of the last error on this host thread ("" if none). */
SBQ_API const char *sbq_last_error(void);

/* Number of SMs of the current device and FP32 lanes per SM used for peaks. */
SBQ_API int sbq_device_info(int *num_sms, int *fp32_lanes_per_sm, int *cc_major, int *cc_minor);

/*
 * Single-layer velocity u(x_t) = sum_{s: y_s != x_t} S(x_t - y_s) w_s sigma_s
 * (Eq. stokes-sl discretised by Eq. nystrom-no-correction).
 *   ns, src[3*ns], w[ns], sigma[3*ns]  sources: positions, quadrature weights, density
 *   nt, trg[3*nt]                      targets
 *   u[3*nt]                            output velocity (overwritten)
 *   prec                               sbq_prec
 * Scratch memory is taken from the device's stream-ordered pool on `stream`.
 * Errors: SBQ_EINVAL for negative sizes, NULL pointers with a non-zero size or an
 * unknown prec; SBQ_ECUDA / SBQ_ENOMEM from the runtime.
 */
SBQ_API int stokes_sl_apply(int64_t ns, const double *src, const double *w, const double *sigma,
                            int64_t nt, const double *trg, double *u, int prec, void *stream);

/*
 * stokes_sl_apply without any allocation, for callers that cannot allocate GPU memory
 * when they need the sum (fixed memory budgets, pre-reserved pools, loops that must not
 * enter the allocator, hosts that forbid cudaMalloc / cudaFree or torch's allocator
 * after start-up).  The paper has no counterpart: this is a deployment variant of the
 * single-layer apply above, with the same arguments, meaning and result (up to the
 * summation grouping of its fixed tile shape).
 * Scratch: a 32 MiB array in device global memory declared by the library itself; every
 * GPU that loads the library holds it until the process exits.  Limits: ns <= 131072 and
 * nt <= 131072, else SBQ_EINVAL with a message naming the limit.
 * The first call on each device (with that device current) looks up the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call rewrites
 * what it reads): calls whose work may overlap on the GPU (unordered streams, several
 * host threads on one device) race and must be serialised by the caller.
 * On success the call performs no allocation of any kind; a rejected call records its
 * message for sbq_last_error() as every entry point does.
 * Like the other applies it returns before the kernels finish: a bounded wait that expired
 * inside them (SBQ_ETIMEOUT, output then incomplete) is recorded in a word of the fixed
 * array, kept across calls, and reported and cleared by the next sbq_check_device() on
 * that device.  Callers check it there after the apply.
 */
/* (prec: SBQ_FP64, SBQ_FP32 or SBQ_FP32_COMP; SBQ_DF32 is not offered here: SBQ_EINVAL.) */
SBQ_API int stokes_sl_apply_noalloc(int64_t ns, const double *src, const double *w,
                                    const double *sigma, int64_t nt, const double *trg, double *u,
                                    int prec, void *stream);

/*
 * Far-field acceleration of the layer sums (the paper's fast route for large N: an FMM for
 * the far field, Sec. 3.2; direct sums cost O(N^2), Sec. 3.4): a barycentric Lagrange
 * treecode for u = sum_s [alpha S + beta D](x_t - y_s) w_s sigma_s, the sum of
 * stokes_combined_apply, to a relative accuracy set by theta and order, in FP32 arithmetic
 * with FP64 sums of its list entries: about 2e-6 at theta = 0.5, order = 8.  Pairs closer
 * than 4e-6 times the sum of the radii of the source leaf and the target block holding
 * them are skipped (the FP32 paths' coincidence rule; on the surface it removes each
 * node's own term, and distinct points must be farther apart than that).
 *   stokes_tree_create: ns sources src[3*ns], unit normals nrm[3*ns] (may be NULL when
 *     beta == 0), weights w[ns], nt targets trg[3*nt] (DEVICE arrays; pass trg == src for
 *     the on-surface sum: one tree then serves both); alpha, beta as
 *     stokes_combined_apply.  theta in (0, 1): a cell of radius r acts through its proxy
 *     points on target blocks farther than r / theta; order in 2..10: Chebyshev points
 *     along the cell's longest side (fewer across thin sides).  Copies the geometry to the
 *     host, builds both octrees and the interaction lists there (the setup, once per
 *     geometry and coefficient pair) and uploads them; the handle owns its device memory
 *     (about 100 bytes per node plus 48 bytes per list entry and 16 (single layer) or 48
 *     bytes per proxy point).  *out receives the handle.
 *   stokes_tree_apply: u[3*nt] (DEVICE, overwritten) from sigma[3*ns] (DEVICE) on
 *     `stream`: source charges, proxy charges of the cells some list takes as far, one CTA
 *     per target block.
 *   stokes_tree_stats: *pairs = kernel evaluations per apply; counts[0..3] = cells, proxy
 *     points, list entries, target blocks.
 *   stokes_tree_destroy: frees the handle (NULL is accepted).
 * Errors: SBQ_EINVAL for sizes outside 0..2^30-1, null pointers, non-finite alpha or beta,
 * theta or order out of range, or a handle that is not a tree; SBQ_ECUDA / SBQ_ENOMEM from
 * the runtime.
 */
typedef struct sbq_tree_s sbq_tree;
SBQ_API int stokes_tree_create(int64_t ns, const double *src, const double *nrm, const double *w,
                               int64_t nt, const double *trg, double alpha, double beta,
                               double theta, int order, sbq_tree **out, void *stream);
SBQ_API int stokes_tree_apply(sbq_tree *tree, const double *sigma, double *u, void *stream);
SBQ_API int stokes_tree_stats(const sbq_tree *tree, double *pairs, int64_t *counts);
SBQ_API int stokes_tree_destroy(sbq_tree *tree);

/* Double-layer velocity u = sum D(x_t - y_s; n_s) w_s sigma_s (Eq. stokes-dl), nrm[3*ns]
 * unit outward normals.  Other arguments and errors as stokes_sl_apply. */
SBQ_API int stokes_dl_apply(int64_t ns, const double *src, const double *nrm, const double *w,
                            const double *sigma, int64_t nt, const double *trg, double *u,
                            int prec, void *stream);

/* Combined field u = sum [alpha S + beta D] w_s sigma_s in one pass (the representation
 * of Eq. stokes-bie-rep-new is alpha = eta, beta = 1).  nrm may be NULL if beta == 0. */
SBQ_API int stokes_combined_apply(int64_t ns, const double *src, const double *nrm,
                                  const double *w, const double *sigma, int64_t nt,
                                  const double *trg, double alpha, double beta, double *u,
                                  int prec, void *stream);

/*
 * Work-list plan for a batch of independent segments (surfaces).  Segment i owns
 * sources [seg_src_off[i], seg_src_off[i+1]) and targets [seg_trg_off[i],
 * seg_trg_off[i+1]) of the global arrays (HOST int64 arrays of nseg+1 prefix
 * offsets starting at 0).  Targets of a segment only see that segment's sources:
 * the operator is block-diagonal.  All pair sums of an operator built on the plan
 * run as ONE persistent launch over a (target tile, source-tile chunk) work-list
 * sorted by cost, followed by a fixed-order reduction of chunk partials.
 *   tune  HOST pointer or NULL; NULL lets stokes_op_create's autotuner choose.
 * Errors: SBQ_EINVAL for nseg < 1 or non-monotone offsets.
 */
SBQ_API int batch_plan(int nseg, const int64_t *seg_src_off, const int64_t *seg_trg_off,
                       const sbq_tune *tune, void **plan_out);

/*
 * Laplace layer potentials (Sec. 4.1; the scalar problem the paper studies first):
 *   laplace_sl_apply        u_t = sum_{y_s != x_t} G(x_t - y_s) w_s sigma_s,  G(r) = 1/(4 pi |r|)
 *   laplace_dl_apply        u_t = sum_{y_s != x_t} dG/dn_y w_s sigma_s
 *                                = sum ((x_t - y_s).n_s) / (4 pi |x_t - y_s|^3) w_s sigma_s
 *                           (the double layer of a constant density is -1 inside a closed
 *                           surface with outward normals, 0 outside)
 *   laplace_combined_apply  alpha S + beta D in one pass (Eq. laplace-bie-rep-new uses
 *                           alpha = 1/(2 eps log(1/eps)), beta = 1)
 * Same conventions as the Stokes applies, with SCALAR densities and outputs: sigma holds ns
 * doubles, u holds nt doubles (overwritten).  Precisions, coincident-pair skipping, errors:
 * as stokes_sl_apply.
 */
SBQ_API int laplace_sl_apply(int64_t ns, const double *src, const double *w, const double *sigma,
                             int64_t nt, const double *trg, double *u, int prec, void *stream);
SBQ_API int laplace_dl_apply(int64_t ns, const double *src, const double *nrm, const double *w,
                             const double *sigma, int64_t nt, const double *trg, double *u,
                             int prec, void *stream);
SBQ_API int laplace_combined_apply(int64_t ns, const double *src, const double *nrm,
                                   const double *w, const double *sigma, int64_t nt,
                                   const double *trg, double alpha, double beta, double *u,
                                   int prec, void *stream);

/*
 * Combined-field operator on the surface nodes (targets = sources):
 *   K sigma = diag sigma + (D + eta S)[sigma] + E sigma           Eq. stokes-bie-new
 * with the uncorrected pair sums and an optional sparse correction E (FP64 CSR over
 * component-major indices c*n + node; rowptr[3n+1], col[nnz], val[nnz] device
 * arrays; nnz = 0 and NULLs for none).  src, nrm, w: device arrays (copied into
 * library-owned packed tiles; the caller may free them after the call).  plan:
 * NULL for one segment, else a batch_plan handle (its offsets must cover n; the
 * operator keeps its own copy of the plan).  The tile shape is autotuned on first
 * use per precision unless the plan fixes it.  The operator owns all workspace of
 * matvec and gmres_solve, so neither allocates.
 */
SBQ_API int stokes_op_create(int64_t n, const double *src, const double *nrm, const double *w,
                             double eta, double diag, int64_t nnz, const int64_t *rowptr,
                             const int64_t *col, const double *val, const void *plan,
                             void **op_out);

/*
 * Double-layer singularity subtraction as a sparse correction E for stokes_op_create
 * (the local, classical form of the correction of Eq. nystrom-correction, Sec. 3.2.1).
 * The nodes are split into closed bodies: body b holds nodes body_off[b] ..
 * body_off[b+1]-1 (body_off: HOST array of nbody+1 non-decreasing offsets, body_off[0]
 * = 0, n = body_off[nbody]).  For node i of body b, with the 3 x 3 row sum
 *   R_i = sum over j in b, j != i, of D(x_i, y_j; n_j) w_j              (Eq. stokes-dl)
 * the correction is the diagonal block E_ii = -R_i - I/2.  Because the double layer
 * of a constant density is -e/2 on a closed surface, an operator with diag = 1/2 and
 * this E applies, at x_i, sum over the node's own body of D_ij (sigma_j - sigma_i)
 * (a summand bounded at r -> 0) plus the plain double-layer sums of the other bodies.
 * Rigid motions of one body are annihilated exactly by its own part.
 *   src, nrm, w  device arrays (SoA, 3n / 3n / n doubles), as for stokes_op_create.
 *   prec         precision of the three double-layer applies that form R (sbq_prec).
 *   rowptr       device, 3n+1 int64: written as 3 * row.
 *   col, val     device, 9n entries each: row c*n+i holds columns b*n+i, b = 0, 1, 2
 *                (component-major indices, ascending).
 * Caller owns every buffer; the call allocates its own temporary workspace on the
 * stream.  Errors: SBQ_EINVAL for bad offsets, sizes or null pointers.
 * Not a counterpart of the paper's quadrature (it builds E from modal and adaptive
 * rules); this local form is for inputs without such a correction.
 */
SBQ_API int stokes_dl_gauss_correction(int nbody, const int64_t *body_off, const double *src,
                                       const double *nrm, const double *w, int prec,
                                       int64_t *rowptr, int64_t *col, double *val,
                                       void *stream);

/*
 * Quadrature correction E of tube elements for stokes_op_create / laplace_op_create: the
 * paper's on-surface corrections (Eq. nystrom-correction; angular weights of Sec. 3.2.2,
 * Eqs. modal-greens-fn-coeff / modal-greens-fn-wts; near-singular rule of Sec. 3.2.3;
 * singular rule of Sec. 3.2.4, Eq. sing-nyst-correc).  Angular integrals, per s-node, the
 * rule with the fewest nodes among: the periodic trapezoidal rule on k N_theta angles (k <=
 * 8, k from its aliasing bound for the target's relative distance), the compiled-in
 * compressed rule of the distance's dyadic level (App. B; levels down to 2^-52, tables for
 * N_theta <= 32), and the dyadically refined Gauss-Legendre rule; the first two only where
 * the area element is resolved by a few modes beyond N_theta / 2 (a bound on the zeros of
 * |y_theta x y_t|^2).  Outer rule in the panel parameter: for a target on the element
 * itself, the compiled-in whole-element singular rule of Sec. 3.2.4 (App. B; ns = 8,
 * N_theta <= 16, element length / radius at the target in [1/4, 8192)), else dyadic panels
 * towards the target with a graded panel next to it; for other targets dyadic panels
 * towards the nearest parameter.
 *   nodes 0 .. nelem*ns*nt - 1 are tube elements: element k holds ns Gauss-Legendre nodes in
 *   its panel parameter times nt equispaced angles 2 pi j / nt, node k*ns*nt + i*nt + j, and
 *   every GL row of an element lies on a circle (a tube y = x_c(s) + rho(s)(e1 cos + e2
 *   sin), Eq. surface-coord).  n_total >= nelem*ns*nt is the operator's node count; nodes
 *   past the tubes (spheres, caps) get empty rows.
 *   src, nrm, w  device SoA arrays over n_total nodes, as for stokes_op_create.
 *   laplace      0: Stokes kernel alpha S + beta D (3 x 3 blocks, Eqs. stokes-sl /
 *                stokes-dl with the double-layer sign of stokes_dl_apply);
 *                1: Laplace alpha G + beta dG/dn_y (scalar).  An operator K = diag I + D +
 *                eta S takes alpha = eta, beta = 1.
 *   near_factor  element k corrects target x when x lies closer than radius_k + near_factor
 *                * max(length_k, 2 radius_k) to one of its centreline samples (its GL
 *                centres and the panel ends); its own element always.  0.5 .. 1 is typical;
 *                a negative value keeps the own element only.
 * For target node x and a near element k, row (a, x) gets the entries
 *   E_ij(x) = sum_m P_mi w_m h_j(x, t_m) - G(x, y_ij) w_ij     (G w of x's own node left out)
 * for every node (i, j) of k (times the three source components for Stokes): the
 * correction that turns the punctured sum over k into the accurate integral over k.
 * Layout: rows component-major (a * n_total + node), columns likewise; a target's row
 * lists its near elements in increasing order, each as (source component, node) blocks.
 * Two-phase use: with rowptr == NULL the call only runs the near search and stores the
 * entry count in *nnz_out (host); then allocate col/val of that size and rowptr of
 * (laplace ? 1 : 3) * n_total + 1 int64 and call again with the same arguments.
 * All CSR arrays are device memory; the call synchronises the stream before returning.
 * Errors: SBQ_EINVAL for sizes (ns in 2..16, nt even in 4..64), null pointers, or rows of
 * nodes that are not circles.  FP64 throughout.
 */
SBQ_API int tube_correction(int64_t nelem, int ns, int nt, int64_t n_total, const double *src,
                            const double *nrm, const double *w, int laplace, double alpha,
                            double beta, double near_factor, int64_t *nnz_out, int64_t *rowptr,
                            int64_t *col, double *val, void *stream);

/*
 * The same correction for off-surface targets near the tubes (Sec. 3.2.3, near-singular
 * quadrature): evaluating a layer potential at points close to a slender body.
 *   trg    device SoA array of ntrg target points (3 * ntrg doubles).  Targets must lie off
 *          the surface; a target on it takes the near-singular rule, which converges there
 *          only as fast as the dyadic refinement (60 levels at most) allows.
 *   Rows are component-major over the targets (a * ntrg + target), columns over the nodes
 *   (b * n_total + node), as for tube_correction; an element corrects a target when the
 *   target lies in its near region (near_factor as above; no element is the target's own).
 * Use: u(trg) = (alpha S + beta D)[sigma](trg) from stokes_combined_apply (or the Laplace
 * apply) plus this E times sigma.  Same two-phase use, ownership and errors as
 * tube_correction; rowptr holds (laplace ? 1 : 3) * ntrg + 1 entries.
 */
/*
 * tube_correction / tube_correction_targets with the caller's angular rules in place of the
 * compiled-in ones (Sec. 3.2.2 with the generalized Chebyshev rules of Appendix B).
 *   trg == NULL: on-surface targets (the tube nodes, as tube_correction; ntrg ignored);
 *   otherwise ntrg off-surface targets (as tube_correction_targets).
 *   nlev == 0: no compressed rules: neither the angular tables (every angular integral
 *   that the trapezoidal rule does not take goes to the dyadically refined Gauss-Legendre
 *   rule) nor the whole-element singular rules (own-element targets take dyadic panels and
 *   the graded panel next to t0); the table arguments are then ignored.
 *   nlev >= 1: HOST angular tables (the compiled-in singular rules stay on); level l
 *   (0 <= l < nlev <= 53) serves relative distances alpha
 *   in [2^-l, 2^(1-l)) and holds rule_cnt[l] <= 128 nodes: angle offsets
 *   rule_phi[l * 128 + m] from the circle point closest to the target, in [-pi, pi], and
 *   weights rule_w[l * 128 + m] (rule_cnt[l] = 0: that level keeps the dyadic rule).  The
 *   rules must integrate, for targets at relative distance alpha..2 alpha from the unit
 *   circle, the kernel components times e^{i l theta} for l <= rule_l0; rule_l0 must be at
 *   least nt/2 + 1 (paper_2310_00889_gb300/angular_rules.py writes such tables).
 * Otherwise the same arguments, layout, two-phase use and errors as tube_correction.
 */
SBQ_API int tube_correction_rules(int64_t nelem, int ns, int nt, int64_t n_total,
                                  const double *src, const double *nrm, const double *w,
                                  int64_t ntrg, const double *trg, int laplace, double alpha,
                                  double beta, double near_factor, int nlev, int rule_l0,
                                  const double *rule_phi, const double *rule_w,
                                  const int *rule_cnt, int64_t *nnz_out, int64_t *rowptr,
                                  int64_t *col, double *val, void *stream);

/*
 * Arithmetic-peak probe (measurement aid, not part of the method): times one launch of
 * long independent fused-multiply-add chains on every SM and returns the achieved rate.
 *   kind 0: FP32 FMA; 1: packed FP32x2 FMA (fma.rn.f32x2); 2: FP64 FMA.
 *   tflops, ms: HOST outputs (TFLOP/s with an FMA counted as 2 flops; kernel time).
 * Synchronises the stream.  Errors: SBQ_EINVAL for a bad kind or null outputs.
 */
SBQ_API int sbq_peak_probe(int kind, double *tflops, double *ms, void *stream);

SBQ_API int tube_correction_targets(int64_t nelem, int ns, int nt, int64_t n_total,
                                    const double *src, const double *nrm, const double *w,
                                    int64_t ntrg, const double *trg, int laplace, double alpha,
                                    double beta, double near_factor, int64_t *nnz_out,
                                    int64_t *rowptr, int64_t *col, double *val, void *stream);

/*
 * Laplace combined-field operator on the surface nodes (Eq. laplace-bie-new; eta = 1/(2 eps
 * log(1/eps)) for slender bodies):
 *   K sigma = diag sigma + (D + eta S)[sigma] + E sigma,  scalar sigma (n doubles)
 * with the Laplace layers of laplace_combined_apply.  Same arguments and ownership as
 * stokes_op_create, with the CSR correction over n rows (rowptr[n+1]).  stokes_matvec,
 * stokes_matvec_bounded, gmres_solve, sbq_autotune and sbq_destroy take the handle; their
 * vectors then hold n doubles.
 */
SBQ_API int laplace_op_create(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, int64_t nnz, const int64_t *rowptr,
                              const int64_t *col, const double *val, const void *plan,
                              void **op_out);

/*
 * Stokes mobility problem, slender combined-field formulation (Sec. 4.2, Eqs.
 * new-mobility-bie and recover-rigidbody-motion):
 *   (K (I - L) + L) sigma = u_s - S nu,     V = -L sigma
 * L: orthogonal projector onto the rigid-body motions of each body in the quadrature
 * L^2 inner product sum_j w_j f_j . g_j; nu: the completion-flow density, on each body the
 * rigid motion whose force sum w nu and torque sum w (x - c_b) x nu (about the body's
 * weighted centroid c_b) are the given F_b, T_b.
 * stokes_op_set_mobility turns a Stokes operator handle into the mobility operator for the
 *   bodies body_off[0] = 0 <= ... <= body_off[nbody] = n (HOST array): from then on
 *   stokes_matvec and gmres_solve apply K (I - L) + L.  Not reversible on the handle.
 * stokes_mobility_rhs: rhs = u_s - S nu for FT (HOST, 6 per body: F then T); us (device,
 *   3n, nullable for no slip); the single layer in precision prec.  Synchronises the stream.
 * stokes_mobility_velocity: V = -L sigma as the rigid motion of each body, UW (HOST, 6 per
 *   body: translational velocity of the centroid, then angular velocity).  Synchronises.
 * Errors: SBQ_EINVAL for bad offsets, a Laplace handle, a body with a singular inertia
 * tensor, or a handle without the mobility set-up.
 */
SBQ_API int stokes_op_set_mobility(void *op, int nbody, const int64_t *body_off, void *stream);
/* Far-field acceleration inside the operator: after stokes_op_set_tree(op, theta, order)
 * every apply of the operator in SBQ_FP32 (the plain FP32 pair sum; the inner solves of
 * gmres_solve with inner_prec = SBQ_FP32) evaluates eta S + D with the treecode of
 * stokes_tree_create (theta, order as there) and adds the correction E and the diagonal as
 * before; the other precisions keep the direct sums.  Builds the trees from the operator's
 * geometry (host set-up, once); theta <= 0 removes the treecode.  Synchronises the stream.
 * Errors: SBQ_EINVAL for a Laplace or batched operator, theta >= 1 or order outside
 * 2..10. */
SBQ_API int stokes_op_set_tree(void *op, double theta, int order, void *stream);
/* Correction of the single layer alone for stokes_mobility_rhs: S nu is then the punctured
 * sum plus this E times nu (Eq. nystrom-correction with the kernel S; e.g. tube_correction
 * with alpha = 1, beta = 0).  CSR over the operator's nodes as for stokes_op_create (device
 * arrays, rowptr of 3n + 1 entries, copied into the handle; nnz = 0 removes it).
 * Synchronises the stream.  Errors: SBQ_EINVAL for a Laplace handle or bad pointers. */
SBQ_API int stokes_op_set_sl_correction(void *op, int64_t nnz, const int64_t *rowptr,
                                        const int64_t *col, const double *val, void *stream);
SBQ_API int stokes_mobility_rhs(void *op, const double *FT, const double *us, double *rhs,
                                int prec, void *stream);
SBQ_API int stokes_mobility_velocity(void *op, const double *sigma, double *UW, void *stream);

/* out = K sigma (device arrays of 3*n doubles; n for a Laplace operator) in precision prec,
 * on `stream`. */
SBQ_API int stokes_matvec(const void *op, const double *sigma, double *out, int prec,
                          void *stream);

/*
 * out = K sigma in double-float (SBQ_DF32) together with bound[i] >= |error of out[i]|:
 * the kernel's sum of the magnitudes of the pair terms entering out[i] times the per-term
 * relative error bound of double-float (2^-40) and the prefactor (paper has no
 * counterpart; GMRES uses the bound to decide when a double-float residual can certify
 * the tolerance).  sigma, out, bound: device arrays of 3n doubles.
 */
SBQ_API int stokes_matvec_bounded(const void *op, const double *sigma, double *out, double *bound,
                                  void *stream);

/*
 * Kernel timing without a profiler (paper has no counterpart): runs `reps` >= 1 applies
 * out = K sigma as stokes_matvec does, records CUDA events on `stream` immediately before
 * and after each launch of the pair-sum kernel and around each whole apply, synchronises
 * the stream, and returns the mean durations in milliseconds (either pointer may be NULL).
 * Errors: SBQ_EINVAL for a bad handle or reps < 1; CUDA errors as SBQ_ECUDA.
 */
SBQ_API int sbq_op_time_pairsum(const void *op, const double *sigma, double *out, int prec,
                                int reps, void *stream, double *kernel_ms, double *apply_ms);

/*
 * Solve K x = rhs (device arrays of 3*n doubles).  x holds x0 on entry and the
 * solution on exit.  o and rep are HOST pointers (rep may be NULL).  Returns
 * SBQ_OK on convergence, SBQ_ENOCONV when max_iter / max_outer is reached first
 * (x then holds the best iterate), SBQ_ENONFINITE if a residual is not finite.
 * Synchronises `stream` (it reads residual norms back once per cycle).
 */
SBQ_API int gmres_solve(const void *op, const double *rhs, double *x, const sbq_gmres_opts *o,
                        sbq_gmres_report *rep, void *stream);

/* Autotune the tile shape of op for precision prec by timing candidate shapes on the
 * operator's own data; the winner is stored in op and in a process-wide cache keyed
 * by problem shape, and copied to *out if out is not NULL. */
SBQ_API int sbq_autotune(void *op, int prec, sbq_tune *out, void *stream);

/* Tile shape currently used by op for precision prec (HOST out pointer). */
SBQ_API int sbq_op_tune(const void *op, int prec, sbq_tune *out);

/* Launch statistics of the last matvec of op in precision prec: number of kernels
 * launched and the number of pair interactions evaluated (HOST out pointers). */
SBQ_API int sbq_op_stats(const void *op, int prec, int *kernels_per_matvec,
                         double *pairs_per_matvec);

/* Synchronise `stream` and report (then clear) the device error words set by bounded
 * waits inside kernels (the library's word of the current device and the word of
 * stokes_sl_apply_noalloc's fixed array): SBQ_ETIMEOUT if a wait expired since the last
 * check. */
SBQ_API int sbq_check_device(void *stream);

/* Failure-path self-test (no counterpart in the paper): launches one kernel on `stream`
 * that waits on an mbarrier phase no copy will complete, with the same bounded wait the
 * pair-sum kernels use and a limit of limit_ns nanoseconds (0 < limit_ns <= 2e9).  When
 * the wait expires the kernel sets the device error word and returns; a following
 * sbq_check_device() then reports SBQ_ETIMEOUT and clears the word.  Faults nothing. */
SBQ_API int sbq_selftest_bounded_wait(int64_t limit_ns, void *stream);

/*
 * Slender-body mixing parameter of the combined-field formulations (Sec. 4.1):
 *   eta = 1 / (2 eps log(1/eps)),  natural logarithm,
 * eps the slenderness (tube radius over length scale, or over centreline radius of
 * curvature).  eta: HOST output.  Errors: SBQ_EINVAL unless 0 < eps < 1.
 */
SBQ_API int sbq_slender_eta(double eps, double *eta);

/*
 * End-to-end calls on HOST buffers (paper has no counterpart: the same computation as the
 * device-pointer calls, with the host<->device copies done by the library on `stream`).
 * Every array argument is a HOST array (pinned memory makes the copies asynchronous DMA);
 * the library allocates, fills and frees its device copies inside the call, which returns
 * after synchronising the stream.  No tile shape is timed inside these calls: `tune`
 * (HOST, nullable) fixes the shape, else the process-wide tuning cache's entry for this
 * problem shape is used (filled by sbq_autotune or by the first apply of an operator of
 * the same shape), else the default shape.
 *
 * stokes_apply_host: out = diag sigma + (D + eta S)[sigma] on the n surface nodes
 *   (Eq. stokes-bie-new without a correction), precision prec.  src, nrm: 3n, w: n,
 *   sigma, out: 3n doubles (SoA).
 * stokes_solve_host: solves K x = rhs, K = diag I + D + eta S + E with GMRES (options and
 *   report as gmres_solve; o and rep HOST).  E: none when nbody == 0, else the double-layer
 *   singularity subtraction of stokes_dl_gauss_correction over the bodies body_off[0] = 0
 *   <= ... <= body_off[nbody] = n, its row sums in precision corr_prec.  x: in x0, out the
 *   solution (written back also for SBQ_ENOCONV).
 * Errors: as stokes_op_create / stokes_matvec / gmres_solve; SBQ_ENONFINITE for a
 * non-finite rhs.
 */
SBQ_API int stokes_apply_host(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, const double *sigma, double *out, int prec,
                              const sbq_tune *tune, void *stream);
SBQ_API int stokes_solve_host(int64_t n, const double *src, const double *nrm, const double *w,
                              double eta, double diag, int nbody, const int64_t *body_off,
                              int corr_prec, const double *rhs, double *x,
                              const sbq_gmres_opts *o, sbq_gmres_report *rep, void *stream);

/* Free a plan or operator handle (NULL is ignored). */
SBQ_API void sbq_destroy(void *handle);

#ifdef __cplusplus
}
#endif

#endif /* SBQ_H */
