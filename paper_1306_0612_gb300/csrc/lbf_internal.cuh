// Internal declarations of liblbfmm (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/lbfmm.h"

#define LBF_PI 3.14159265358979323846
#define LBF_MAX_TERMS 64  // expansion terms p + 1 supported by the kernels
#define LBF_MAX_LEVELS 31
#define LBF_ANC_STRIDE 32

// Per-process launch counter (lbf_launch_count).
extern std::atomic<int64_t> g_lbf_launches;

#define LBF_LAUNCH(kernel, grid, block, smem, stream, ...)                 \
    do {                                                                   \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
        g_lbf_launches.fetch_add(1, std::memory_order_relaxed);            \
    } while (0)

// Tracing: event pair around a launch when lbf_profile_enable(1) is on.
void lbf_prof_mark(int id, int begin, cudaStream_t s);
void lbf_prof_capture(bool on);  // this thread is capturing a CUDA graph: no marks
#define LBF_LAUNCH_P(id, kernel, grid, block, smem, stream, ...)           \
    do {                                                                   \
        lbf_prof_mark((id), 1, (stream));                                  \
        LBF_LAUNCH(kernel, grid, block, smem, stream, __VA_ARGS__);        \
        lbf_prof_mark((id), 0, (stream));                                  \
    } while (0)

#define LBF_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return LBF_ECUDA;                           \
    } while (0)

#define LBF_CHECK_LAUNCH() LBF_CUDA(cudaGetLastError())

// Device status word bits (lbf_sync_status).
#define LBF_DEV_POLE 1
#define LBF_DEV_TIMEOUT 2

__host__ __device__ static inline int64_t lbf_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Bump allocator over the caller's workspace (256-byte aligned slices).
struct Arena {
    char *base = nullptr;
    size_t cap = 0, off = 0;
    bool overflow = false;
    void *take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void *p = base ? base + off : nullptr;
        off += bytes;
        if (off > cap) overflow = true;
        return overflow ? nullptr : p;
    }
    template <class T> T *get(int64_t n) { return (T *)take(sizeof(T) * (size_t)(n > 0 ? n : 1)); }
};

// Adaptive quadtree (boxes numbered level by level, Morton order within a level).
struct Tree {
    int64_t cap = 0, nbox = 0, nleaf = 0;
    int nlev = 0;
    int64_t lev_start[LBF_MAX_LEVELS + 2] = {};
    double xmin = 0, ymin = 0, L = 1;  // bounding square
    int32_t *level, *ix, *iy, *parent, *child0, *nchild, *begin, *end;
    int32_t *leaves;                    // ids of the leaves, ascending
    // interaction lists
    int32_t *coll;                      // 9 colleagues per box (-1 = none)
    int32_t *vlist, *nv;                // V: up to 27 per box
    int32_t *coarse, *ncoarse;          // shallower leaves touching the box: up to 8
    int32_t *xlist, *nx;                // X: up to 16 per box
    int32_t *u_ptr, *u_idx;             // U (leaves only), CSR over boxes
    int32_t *w_ptr, *w_idx;             // W (leaves only), CSR over boxes
    int64_t u_cap = 0, w_cap = 0, u_len = 0, w_len = 0;
};

#define LBF_LN2 0.69314718055994530942

// Multiplier potential E y on the node quadtree, Schur complement from island
// moments (lbf_border.cu).
struct Border {
    int P = 0, P32 = 0;              // expansion terms (double, float) of the island moments,
                                     // the transposed and derivative potentials, the float E y
    int Pe = 0;                      // expansion terms of the accurate E y (P2L, L2L, L2P)
    int64_t pair_cap = 0, n_p2l = 0, n_near = 0;
    // direct centres in chunks of 32 per leaf, a warp each: chunk -> (leaf, chunk index),
    // per node the first of its partial sums (one per chunk of its leaf)
    int32_t *chunk_leaf = nullptr, *chunk_k = nullptr, *nodebase = nullptr;
    double *partial = nullptr;
    int64_t nchunks = 0, npartial = 0, partial_cap = 0;
    int32_t *leaf_of = nullptr;      // leaf box of each node (Morton order)
    double *ell = nullptr;           // log(1 + |xi_i|^2)
    double2 *xc = nullptr;           // planar centres
    int32_t *kind = nullptr;         // 0 pole, 1 inside the tree's square, 2 outside
    int32_t *live = nullptr;         // 1 unless at the pole (kind != 0, without the tree)
    int32_t *cell = nullptr;         // finest-level cell of each centre (2 per centre)
    double *lam = nullptr;           // log(1 + |xi_m|^2)
    int32_t *glob = nullptr, *nglob = nullptr;  // centres summed directly at every node
    int nglob_h = 0;
    int32_t *pairs_a = nullptr, *pairs_b = nullptr;  // staging of (box, centre) pairs
    int32_t *p2l_ptr = nullptr, *p2l_src = nullptr;  // P2L centres per box (CSR)
    int32_t *near_ptr = nullptr, *near_src = nullptr;  // direct centres per leaf (CSR)
    int32_t *cp2l = nullptr, *cnear = nullptr;  // per centre: offsets into pairs_a / pairs_b (M + 1)
    double2 *loc = nullptr;          // local expansions of the log potential, box x P
    float2 *loc32 = nullptr;         // box x P32
    double2 *zc = nullptr;           // island node means
    double *Rk = nullptr, *rk = nullptr, *slog = nullptr, *sell = nullptr;
    double2 *mu = nullptr, *nu = nullptr;  // island moments, M x P
    double *sums = nullptr;          // Y, Lam
};

struct GmresState;  // device-side scalars (lbf_krylov.cu)

struct lbf_plan {
    int64_t N = 0;
    int M = 0;
    int64_t n = 0;  // unknowns of the bordered system, N + M
    lbf_options opt{};
    int P = 0;      // expansion terms p + 1
    Arena arena;
    int64_t *island_ptr_h = nullptr;  // host copy
    int64_t *island_ptr = nullptr;    // device copy
    // per node, sorted (Morton) order
    double2 *xi = nullptr, *w = nullptr;
    double *dself = nullptr, *beta = nullptr;
    int32_t *perm = nullptr;  // sorted -> caller index
    int32_t *rank = nullptr;  // caller index -> sorted
    double *centres = nullptr;  // M x 3 after rotation
    double rot[9];
    int has_rot = 0;
    double *rot_d = nullptr;  // device copy of rot
    // translation-operator tables (filled on the host at plan time)
    double *tab_binom = nullptr;   // C(n, k), n < 2*LBF_MAX_TERMS, k < LBF_MAX_TERMS
    double2 *tab_dshift = nullptr; // d^k and (2d)^-k for the 4 child offsets, 8 x (LBF_MAX_TERMS + 1)
    double2 *tab_tpow = nullptr;   // 49 same-level offsets x (LBF_MAX_TERMS + 1) powers
    Tree tree;
    // FMM work
    double2 *q = nullptr, *mpole = nullptr, *local = nullptr;
    // float FMM (precision FP32_REFINE)
    int P32 = 0;
    float2 *q32 = nullptr, *mpole32 = nullptr, *local32 = nullptr;
    float2 *u32 = nullptr;  // per node: (xi - c)/r about the centre c, half-width r of its leaf
    int32_t *anc = nullptr;  // per leaf b: anc[b * LBF_ANC_STRIDE + s] = its ancestor s levels up
                             // (levels >= 2 only), for the float operator's ancestor walk
    int32_t *isl = nullptr;  // per node (sorted order): its island
    // the float forward pass's island split: per island its mean density (M), then
    // [M] 1 if the split is on, [M+1] the island whose planar curve encloses the others
    // (-1: none), [M+2] twice its winding number there; iacoef: the coefficient of an
    // island's own mean in its rows
    double *imean = nullptr, *iacoef = nullptr;
    // double-float operator (opt.fmm64): charges, leaf-local coordinates (pairs of
    // float pairs, 16 B), and the translation tables; expansions reuse mpole/local
    void *qdf = nullptr, *udf = nullptr;
    void *tabdf_binom = nullptr, *tabdf_tpow = nullptr, *tabdf_dshift = nullptr;
    float *tab32_binom = nullptr;
    float2 *tab32_tpow = nullptr, *tab32_dshift = nullptr;
    double *gr = nullptr, *gd = nullptr;  // refinement residual and correction
    // last solve: Arnoldi steps, FP64 applications, FP32 applications, refinement steps
    int64_t stats[4] = {0, 0, 0, 0};
    int32_t *upcnt = nullptr;   // per-box child arrival counters of the upward pass (kept at 0)
    // float downward pass: [0], [3] box counters of its two phases, [1] finished warps,
    // [2] epoch, then per box the epochs in which its M2L + P2L part and its full local
    // expansion were written (nbox each)
    uint32_t *pull = nullptr;
    int nsm = 0;                // streaming multiprocessors of the plan's device
    double *v = nullptr;        // (I + K - I) sigma = K sigma, doubled scaling
    double *bsig = nullptr;     // scalar beta . sigma
    double *red = nullptr;      // reduction partials
    unsigned int *red_count = nullptr;
    // border
    Border bd;                  // E y by island expansions (E itself is never formed)
    double *Sinv = nullptr;     // M x M inverse Schur complement, or (lu) its LU factors
    int lu = 0;                 // S^-1 by the double-float LU factors (lbf_schur_lu.cu)
    int *lu_piv = nullptr, *lu_perm = nullptr;  // row interchanges, final row order (M each)
    float2 *lu_z = nullptr;     // M-vector of the triangular solves (double-float)
    unsigned *lu_sync = nullptr;  // ticket, finished blocks, epoch, row-block flags
    float2 *lu_dinv = nullptr;    // inverses of the 64 x 64 diagonal blocks of L and U
    double *lu_S = nullptr;       // S itself (double), for the refinement step of accurate applies
    double *lu_r = nullptr;       // M: that step's residual
    float2 *lu_z2 = nullptr;      // M: its correction
    int lu_fast = 0;              // 1 while an FP64 Arnoldi step applies the operator: S^-1 from
                                  // the factors alone (every other application refines once)
    double *fvec = nullptr, *yvec = nullptr;  // M-vectors
    // generic N+M vectors for lbf_apply / gmres
    double *tin = nullptr, *tout = nullptr;
    // gmres
    double *V = nullptr, *H = nullptr, *gw = nullptr, *gx = nullptr, *gb = nullptr;
    double *gpart = nullptr;
    GmresState *gs = nullptr;
    int64_t ldv = 0;  // stride between basis vectors
    int mdot_blocks = 0;
    char *region = nullptr;      // GMRES basis, or plan-creation temporaries
    size_t region_bytes = 0;
    int *dev_status = nullptr;
    int *host_status = nullptr;  // pinned
    cudaEvent_t ev[2] = {nullptr, nullptr};  // GMRES chunk markers (no device memory)
    double *vstep = nullptr;                  // the Arnoldi input of a graph-replayed step
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [prec][transpose]
    int64_t gnodes[2][2] = {{0, 0}, {0, 0}};  // kernels per replay
    double *host_scalars = nullptr;  // pinned
    // plan creation only: the stream of the Schur complement and its inverse (beside the
    // tree build), and its fork and join events
    cudaStream_t side = nullptr;
    cudaEvent_t fork[2] = {nullptr, nullptr};
    // Right-hand sides advanced together (lbf_gmres_solve_many): a launch on a plan view
    // with nrhs > 1 covers all of them, blockIdx.y = the right-hand side, whose buffers
    // sit blockIdx.y * slab bytes after those the view points at (1 and 0 on a plan).
    int nrhs = 1;
    int64_t slab = 0;
    double *nearbuf = nullptr;  // views: the forward rows' near field of every right-hand side
};

// grid of a launch over the plan's right-hand sides
static inline dim3 lbf_grid(const lbf_plan *pl, int64_t gx)
{
    return dim3((unsigned)gx, (unsigned)pl->nrhs, 1u);
}

#ifdef __CUDACC__
// Moves each per-right-hand-side pointer of a kernel to right-hand side blockIdx.y
// (null pointers stay null; slab 0 leaves them as they are).
template <class... Ts> __device__ __forceinline__ void lbf_rhs(int64_t slab, Ts &...p)
{
    if (slab == 0) return;
    const int64_t o = (int64_t)blockIdx.y * slab;
    ((p = p ? (Ts)((const char *)p + o) : p), ...);
}
#endif

// ---- failure injection for tests (lbf_debug_inject) ------------------------------
// A barrier injection is consumed by the next plan creation on the calling thread:
// its poll limit goes into the plan's status block, and the grid barrier of the Schur
// complement's inverse or factorisation starts pre-arrived so that it never opens.
struct LbfInject {
    int barrier = 0;
    unsigned polls = 0;
};
LbfInject &lbf_inject_state();  // this thread's pending injection
// the barrier word of a grid barrier, to pre-arrive it when an injection is pending
void lbf_inject_barrier(unsigned *count, cudaStream_t s);

// ---- layout ------------------------------------------------------------------
void lbf_layout(lbf_plan *pl, int64_t N, int M, const lbf_options &opt, int64_t box_cap);

struct SortBufs {  // plan-time scratch of a pair sort (capacity max(N, pair capacity))
    uint64_t *key, *key_alt;
    int32_t *val_alt;
};

// ---- geometry (lbf_geometry.cu) ----------------------------------------------
int lbf_geometry_build(lbf_plan *pl, const double *x, const double *dx, const double *d2x,
                       const double *centres, int planar, cudaStream_t s, double2 *xi_o,
                       double2 *w_o, double *d_o, double *b_o);
int lbf_geometry_gather(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, const double2 *w_o,
                        const double *d_o, const double *b_o);
// S and S^-1 on the side stream (forked from s after the planar nodes exist)
int lbf_border_start(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, double *scratch);
// the tree-dependent part of the border on s, then s waits for S^-1
int lbf_border_build(lbf_plan *pl, cudaStream_t s, int32_t *work, int64_t work_len,
                     const SortBufs &sb);
void lbf_border_end(lbf_plan *pl);     // releases the side stream and events
size_t lbf_gj_scratch_doubles(int M);  // scratch of lbf_border_start
// ---- LU of the Schur complement (lbf_schur_lu.cu) ---------------------------------
size_t lbf_lu_scratch_bytes(int M);
int lbf_lu_sync_words(int M);
int64_t lbf_lu_dinv_entries(int M);
int lbf_schur_lu_factor(lbf_plan *pl, cudaStream_t s, void *scratch);
int lbf_schur_lu_apply(lbf_plan *pl, const double *f, double alpha, double *y, int trans,
                       const int *gate, cudaStream_t s, int accurate);
// ---- multiplier potential (lbf_border.cu) -------------------------------------
// S = D - F E into G (M x M) from the planar nodes and centres alone; work holds the
// list of entries summed directly
int lbf_schur_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, double *G, int32_t *work,
                    int64_t work_len);
int lbf_mp_build(lbf_plan *pl, cudaStream_t s, int32_t *work, int64_t work_len, const SortBufs &sb);
int lbf_mp_apply(lbf_plan *pl, const double *y, const double *x, const double *v, double sc,
                 double *out, const int *gate, cudaStream_t s, int prec);
// out = add + sc E^T tau (M-vectors, add nullable; tau sorted), FP64
int lbf_mp_apply_transpose(lbf_plan *pl, const double *tau, double sc, const double *add,
                           double *out, const int *gate, cudaStream_t s);
// out_i = gradient of (E y)_i with respect to (Re xi_i, Im xi_i), sorted order, FP64
int lbf_mp_gradient(lbf_plan *pl, const double *y, double2 *out, cudaStream_t s);
int lbf_geometry_out_impl(const lbf_plan *pl, double *xi, double *normal, double *weight,
                          double *arc, cudaStream_t s);

// ---- tree (lbf_tree.cu) --------------------------------------------------------
int lbf_tree_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, uint64_t *keys,
                   uint64_t *keys_alt, int32_t *perm_alt, int32_t *scratch, int64_t scratch_len,
                   int64_t *box_needed);
int lbf_lists_build(lbf_plan *pl, cudaStream_t s, int32_t *scratch, int64_t scratch_len,
                    int64_t *box_needed);
int lbf_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *scratch, int64_t scratch_len,
                 cudaStream_t s);  // exclusive scan, out may alias in
// stable LSD radix sort of (keys, vals) on the low `bits` bits of the keys; the
// result is in keys/vals, the *_alt arrays are scratch of the same length
int lbf_radix_sort(uint64_t *keys, uint64_t *keys_alt, int32_t *vals, int32_t *vals_alt, int64_t n,
                   int bits, int32_t *scratch, int64_t scratch_len, cudaStream_t s);

// ---- FMM / direct operator (lbf_fmm.cu) -----------------------------------------
// v = 2 [ (1/2pi) Im sum_{j!=i} q_j/(xi_j - xi_i) + d_i sigma_i + beta.sigma ]   (sorted order)
#define LBF_PREC_FP64 0
#define LBF_PREC_FP32 1
int lbf_apply_K(lbf_plan *pl, const double *sigma, double *v, const int *gate, cudaStream_t s,
                int prec);
int lbf_fmm_prepare(lbf_plan *pl, cudaStream_t s);  // plan time, after the tree and the gather
// v = 2 [ (1/2pi) Im(w_i sum_{j!=i} tau_j/(xi_i - xi_j)) + d_i tau_i + beta_i sum_j tau_j ]:
// the transposed rows (K^T tau)_i, doubled (sorted order)
int lbf_apply_KT(lbf_plan *pl, const double *tau, double *v, const int *gate, cudaStream_t s,
                 int prec);
// out_i = Phi'(xi_i) = -sum_{j!=i} q_j/(xi_i - xi_j)^2, q = w x (weighted) or (x, 0), FP64
int lbf_cauchy_deriv(lbf_plan *pl, const double *x, bool weighted, double2 *out, cudaStream_t s);
// scaled multipoles a_k = sum_j x_j ((xi_j - c)/r)^k, k < P, of real charges x on every
// box (P2M + M2M); also writes q = (x, 0) and *bsig = sum_j x_j
int lbf_multipoles(lbf_plan *pl, const double *x, int P, double2 *mp, const int *gate,
                   cudaStream_t s);
int lbf_evaluate_impl(lbf_plan *pl, const double *sigma_sorted, const double *a, int64_t T,
                      const double *t, double *u, cudaStream_t s);
int lbf_green_sum_impl(int64_t T, const double *t, int64_t S, const double *p,
                       const double *gamma, double *out, cudaStream_t s);

// ---- border / krylov (lbf_krylov.cu) -----------------------------------------------
int lbf_apply_op_sorted(lbf_plan *pl, int op, const double *in, double *out, const int *gate,
                        cudaStream_t s, int prec = LBF_PREC_FP64);
int lbf_precondition_rhs(lbf_plan *pl, const double *g2_sorted, double *out, cudaStream_t s);
int lbf_precondition_rhs_t(lbf_plan *pl, const double *r_sorted, double *out, cudaStream_t s);
int lbf_gmres_impl(lbf_plan *pl, const double *g, double *sigma, double *a, const double *x0,
                   int *iters, double *rel_res, cudaStream_t s, int transpose);
// lockstep right-hand sides (lbf_gmres_solve_many)
#define LBF_LOCKSTEP_MAX 16  // right-hand sides of one lockstep group
int lbf_many_view(const lbf_plan *pl, int R, void *work, size_t bytes, lbf_plan *view,
                  size_t *need);
lbf_plan lbf_view_at(const lbf_plan &v, int r);
int lbf_gmres_many_impl(lbf_plan *pl, int nrhs, const double *g, double *sigma, double *a,
                        int *iters, double *rel_res, void *work, size_t bytes, cudaStream_t s);
int lbf_dot(lbf_plan *pl, const double *a, const double *b, int64_t n, double *out, cudaStream_t s);
// ---- adjoint (lbf_adjoint.cu) ---------------------------------------------------------
int lbf_evaluate_transpose_impl(lbf_plan *pl, int64_t T, const double *t, const double *ub,
                                double *sbar, double *abar, cudaStream_t s);
int lbf_gradient_nodes_impl(lbf_plan *pl, const double *sigma, const double *a, const double *lam,
                            int64_t T, const double *t, const double *ub, double *grad,
                            cudaStream_t s);
int lbf_gradient_data_impl(lbf_plan *pl, const double *lam, double *grad_g, cudaStream_t s);
int lbf_permute_in(lbf_plan *pl, const double *in_caller, double *out_sorted, int with_a,
                   cudaStream_t s);
int lbf_permute_out(lbf_plan *pl, const double *in_sorted, double *out_caller, int with_a,
                    cudaStream_t s);
