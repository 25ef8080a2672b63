// Host-side engine of libsbq: tile tables, work lists, operator handles.
#pragma once

#include "sbq_common.cuh"

#include <memory>
#include <mutex>

namespace sbq {

constexpr uint32_t PLAN_MAGIC = 0x53425150u;   // "SBQP"
constexpr uint32_t OP_MAGIC = 0x5342514fu;     // "SBQO"

// Device buffer owned by the engine (cudaMalloc / cudaFree).
// Allocations made while an AsyncAllocScope is alive on this host thread are stream
// ordered (cudaMallocAsync / cudaFreeAsync on that stream); others use cudaMalloc.
struct AsyncAllocScope {
    explicit AsyncAllocScope(cudaStream_t s);
    ~AsyncAllocScope();
    cudaStream_t prev;
    bool prev_on;
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool async = false;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t n);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct PlanH {
    uint32_t magic = PLAN_MAGIC;
    int nseg = 0;
    std::vector<int64_t> src_off, trg_off;
    bool has_tune = false;
    sbq_tune tune{};
};

// Source tiles of one precision layout (FP32: packed pairs, FP64: TS_F64 doubles x9,
// double-float: TS_DF records of five float4).
struct SrcPack {
    int layout = -1;            // SBQ_FP32 (shared by FP32 and FP32_COMP), SBQ_FP64 or SBQ_DF32
    int TS = 0;
    int n_stiles = 0;
    std::vector<int> seg_tile_begin, seg_tile_count;
    DevBuf stiles, spack;
};

// Target tiles + work list for one tile shape.
struct TrgSet {
    sbq_tune tune{};
    int TT = 0;
    int n_ttiles = 0;
    int n_items = 0;
    int grid = 0;
    bool needs_reduce = false;
    double pairs = 0.0;         // pair interactions per apply (valid members only)
    std::vector<double> item_pairs;   // host: pair interactions of each work item, list order
    DevBuf ttiles, tpack, tpack_lo, tpack_l2, items, partial, counter;
};

// Mobility formulation state of an operator (mobility.cu): bodies, their areas, centroids
// and inverse inertia tensors, per-body reduction blocks and scratch.
struct MobState {
    int nbody = 0;
    int nblk = 0;
    std::vector<double> h_area, h_iinv, h_cen;
    DevBuf x, w, body_of, blk, bodyblk, cen, area, iinv, part, rigid, y, r;
};

// treecode (tree.cu) attached to an operator: replaces its plain FP32 pair sum
int tree_op_attach(struct Op *op, double theta, int order, cudaStream_t s);
int tree_op_apply(struct Op *op, const double *y, double *out, cudaStream_t s);
void tree_op_free(struct Op *op);

struct Op {
    uint32_t magic = OP_MAGIC;
    int device = 0;
    long long n = 0;
    double eta = 0.0, diag = 0.5;
    bool laplace = false;              // Laplace operator (scalar densities)
    int ncomp = 3;                     // components per node: 3 (Stokes) or 1 (Laplace)
    long long nnz = 0;
    DevBuf src, nrm, w;                // library copies (SoA), in the internal node order
    DevBuf perm;                       // int: caller's index of each internal node
    DevBuf rowptr, col, val;           // CSR correction
    long long sl_nnz = 0;              // correction of the single layer alone (mobility S nu)
    DevBuf sl_rowptr, sl_col, sl_val;
    PlanH plan;                        // segments (one segment if none given)
    SrcPack sp32, sp64, spdf;          // FP32 (plain and compensated), FP64, double-float
    std::unique_ptr<TrgSet> ts[4];     // per sbq_prec
    bool tuned[4] = {false, false, false, false};
    std::mutex mu;
    struct GmresWS *gm = nullptr;      // solver workspace (gmres.cu)
    std::unique_ptr<MobState> mob;     // set: the operator is K (I - L) + L (mobility)
    void *tree = nullptr;              // treecode (tree.cu) for applies in SBQ_FP32, or null
    ~Op();
};

// Segment layout helpers.
int build_src_pack(SrcPack &sp, int layout, const std::vector<int64_t> &src_off, const double *src,
                   const double *nrm, double nscale, long long ns, cudaStream_t s);
int build_trg_set(TrgSet &ts, int kind, int prec, const sbq_tune &tune, const SrcPack &sp,
                  const std::vector<int64_t> &trg_off, const double *trg, long long nt,
                  const std::vector<int64_t> &src_off, cudaStream_t s);

// Events recorded on the launching stream immediately before and after each pair-sum
// kernel launch of this host thread while set (kernel timing without a profiler).
struct PairsumTiming {
    cudaEvent_t before = nullptr, after = nullptr;
};
PairsumTiming *&pairsum_timing();

// One pair-sum apply: out = scale * sum(...) [+ diag * diag_sigma].
// bound (double-float only, nullable): per output entry, a bound on its rounding error.
// perm (nullable): the sources and targets are the same nodes in an internal order, perm
// gives each internal node's index in the caller's order (sigma, diag_sigma, out and bound
// are in the caller's order).
int run_pairsum(int kind, int prec, const SrcPack &sp, const TrgSet &ts, const double *w,
                const double *sigma, long long ns, const double *trg, long long nt, double *out,
                double scale, double kappa, double diag, const double *diag_sigma, cudaStream_t s,
                double *bound = nullptr, const int *perm = nullptr);

// Operator pieces used by the solver.
int op_matvec(Op *op, const double *sigma, double *out, int prec, cudaStream_t s,
              double *bound = nullptr);
int op_ensure_tuned(Op *op, int prec, cudaStream_t s);
// Work list of op for prec without timing anything: the given shape, else the tuning
// cache's entry for this problem shape, else the default shape.
int op_prepare_untimed(Op *op, int prec, const sbq_tune *tune, cudaStream_t s);
int op_kernels_per_matvec(const Op *op, int prec);

// Kind and prefactors of alpha S + beta D (Stokes; Laplace).
void kind_and_scale(double alpha, double beta, int *kind, double *scale, double *kappa);
void laplace_kind_and_scale(double alpha, double beta, int *kind, double *scale, double *kappa);

sbq_tune default_tune(int prec, long long nt);

// mobility.cu
int mob_setup(Op *op, int nbody, const int64_t *body_off, cudaStream_t s);
int mob_project(const Op *op, const double *sigma, double sign, cudaStream_t s);
int mob_field(const Op *op, const double *base, double s_r, double *out, cudaStream_t s);
int mob_rhs(Op *op, const double *FT, const double *us, double *rhs, int prec, cudaStream_t s);
int mob_velocity(Op *op, const double *sigma, double *UW, cudaStream_t s);
int mob_axpy(long long n, double a, const double *x, double *y, cudaStream_t s);

// correction.cu: E = -R_i - I/2 per node from per-body double-layer row sums.
int dl_gauss_correction(int nbody, const int64_t *body_off, const double *src, const double *nrm,
                        const double *w, int prec, int64_t *rowptr, int64_t *col, double *val,
                        cudaStream_t s);
// tube_quad.cu: quadrature correction of tube elements (on-surface targets).
// trg == nullptr: targets are the tube nodes (rows over all ntot nodes); else ntrg
// off-surface points.
// rules_*: optional compressed angular rules (HOST arrays, rules_nlev levels of 64 slots).
int build_tube_correction(long long nelem, int ns, int nt, long long ntot, const double *src,
                          const double *nrm, const double *w, long long ntrg, const double *trg,
                          int laplace, double alpha, double beta, double near_factor,
                          int64_t *nnz_out, int64_t *rowptr, int64_t *col, double *val,
                          cudaStream_t s, int rules_nlev = 0, const double *rules_phi = nullptr,
                          const double *rules_w = nullptr, const int *rules_cnt = nullptr);
int gmres_destroy(struct GmresWS *ws);

}  // namespace sbq
