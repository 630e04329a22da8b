// C ABI of liblbfmm (include/lbfmm.h): options, workspace layout, plan life
// cycle and the public calls.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "lbf_internal.cuh"

std::atomic<int64_t> g_lbf_launches{0};

int lbf_gmres_kernels_smem(int m);
int lbf_gmres_blocks();
int lbf_fmm_init_attrs();
int lbf_border_init_attrs();

namespace {

struct GmresStateBytes {
    char b[128];
};

int64_t box_capacity_estimate(int64_t N, const lbf_options &o)
{
    if (o.box_capacity > 0) return o.box_capacity;
    return 8 * N / std::max(1, o.leaf_size) + 64 * o.max_depth + 1024;
}

bool valid(const lbf_options &o)
{
    return o.tol > 0 && o.restart >= 1 && o.restart <= 200 && o.maxit >= 1 && o.p >= 4 &&
           o.p + 1 <= LBF_MAX_TERMS && o.leaf_size >= 1 && o.leaf_size <= 1024 &&
           o.max_depth >= 1 && o.max_depth <= 30 &&
           (o.matvec == LBF_MATVEC_FMM || o.matvec == LBF_MATVEC_DIRECT) &&
           (o.border == 0 || o.border == 1) &&
           (o.precision == LBF_PRECISION_FP64 || o.precision == LBF_PRECISION_FP32_REFINE) &&
           o.p32 >= 4 && o.p32 + 1 <= 32 && o.inner_tol > 0 && o.inner_tol < 1 &&
           o.max_refine >= 1 && o.graphs >= -1 && o.graphs <= 1 && (o.fmm64 == 0 || o.fmm64 == 1) &&
           o.schur >= LBF_SCHUR_AUTO && o.schur <= LBF_SCHUR_LU && o.p2p_warps >= 0 &&
           o.p2p_warps <= 8 && (o.precond == 0 || o.precond == 1);
}

// host tables of the translation operators (scaled expansions, see lbf_fmm.cu)
void make_tables(std::vector<double> &binom, std::vector<double2> &dshift,
                 std::vector<double2> &tpow)
{
    const int T = LBF_MAX_TERMS;
    binom.assign(2 * T * T, 0.0);
    // Pascal rows n = 0 .. 2T-1, kept for k < T
    std::vector<double> row(2 * T + 1, 0.0), nxt(2 * T + 1, 0.0);
    row[0] = 1.0;
    for (int n = 0; n < 2 * T; n++) {
        for (int k = 0; k < T; k++) binom[n * T + k] = k <= n ? row[k] : 0.0;
        nxt[0] = 1.0;
        for (int k = 1; k <= n + 1; k++) nxt[k] = row[k - 1] + (k <= n ? row[k] : 0.0);
        row.swap(nxt);
    }
    // child offsets d = ((2dx-1) + i (2dy-1))/2 over the parent half-width:
    // dshift[c][k] = d^k, dshift[4 + c][k] = (2d)^-k
    dshift.assign(8 * (T + 1), make_double2(0, 0));
    for (int c = 0; c < 4; c++) {
        std::complex<double> d(((c & 1) ? 0.5 : -0.5), ((c >> 1) ? 0.5 : -0.5));
        std::complex<double> p = 1.0, pinv = 1.0, inv2d = 1.0 / (2.0 * d);
        for (int k = 0; k <= T; k++) {
            dshift[c * (T + 1) + k] = make_double2(p.real(), p.imag());
            dshift[(4 + c) * (T + 1) + k] = make_double2(pinv.real(), pinv.imag());
            p *= d;
            pinv *= inv2d;
        }
    }
    tpow.assign(49 * (T + 1), make_double2(0, 0));
    for (int dx = -3; dx <= 3; dx++)
        for (int dy = -3; dy <= 3; dy++) {
            if (std::abs(dx) <= 1 && std::abs(dy) <= 1) continue;
            std::complex<double> t = 1.0 / (2.0 * std::complex<double>(dx, dy));
            std::complex<double> p = 1.0;
            int o = (dx + 3) * 7 + (dy + 3);
            for (int k = 0; k <= T; k++) {
                tpow[o * (T + 1) + k] = make_double2(p.real(), p.imag());
                p *= t;
            }
        }
}

}  // namespace

// Lay out every array of a plan over the arena (base == nullptr only sizes it).
void lbf_layout(lbf_plan *pl, int64_t N, int M, const lbf_options &o, int64_t cap)
{
    Arena &A = pl->arena;
    const int T = LBF_MAX_TERMS;
    int P = o.p + 1;
    int64_t n = N + M;
    pl->island_ptr = A.get<int64_t>(M + 1);
    pl->xi = A.get<double2>(N);
    pl->w = A.get<double2>(N);
    pl->dself = A.get<double>(N);
    pl->beta = A.get<double>(N);
    pl->perm = A.get<int32_t>(N);
    pl->rank = A.get<int32_t>(N);
    pl->centres = A.get<double>(3 * (int64_t)M);
    pl->rot_d = A.get<double>(9);
    pl->tab_binom = A.get<double>(2 * T * T);
    pl->tab_dshift = A.get<double2>(8 * (T + 1));
    pl->tab_tpow = A.get<double2>(49 * (T + 1));
    Tree &t = pl->tree;
    t.cap = cap;
    t.level = A.get<int32_t>(cap);
    t.ix = A.get<int32_t>(cap);
    t.iy = A.get<int32_t>(cap);
    t.parent = A.get<int32_t>(cap);
    t.child0 = A.get<int32_t>(cap);
    t.nchild = A.get<int32_t>(cap);
    t.begin = A.get<int32_t>(cap);
    t.end = A.get<int32_t>(cap);
    t.leaves = A.get<int32_t>(cap);
    t.coll = A.get<int32_t>(9 * cap);
    t.vlist = A.get<int32_t>(27 * cap);
    t.nv = A.get<int32_t>(cap);
    t.coarse = A.get<int32_t>(8 * cap);
    t.ncoarse = A.get<int32_t>(cap);
    t.xlist = A.get<int32_t>(16 * cap);
    t.nx = A.get<int32_t>(cap);
    t.u_cap = 24 * cap;
    t.w_cap = 16 * cap;
    t.u_ptr = A.get<int32_t>(cap + 1);
    t.u_idx = A.get<int32_t>(t.u_cap);
    t.w_ptr = A.get<int32_t>(cap + 1);
    t.w_idx = A.get<int32_t>(t.w_cap);
    pl->q = A.get<double2>(N);
    if (o.matvec == LBF_MATVEC_FMM) {
        pl->mpole = A.get<double2>(cap * P);
        pl->local = A.get<double2>(cap * P);
    }
    if (o.matvec == LBF_MATVEC_FMM || o.border) {
        pl->upcnt = A.get<int32_t>(cap);
        pl->pull = A.get<uint32_t>(2 * cap + 4);
    }
    if (o.matvec == LBF_MATVEC_FMM && o.fmm64) {
        pl->qdf = A.get<double2>(N);   // cx<df64>: 16 B per node
        pl->udf = A.get<double2>(N);
        pl->tabdf_binom = A.get<double>(2 * T * T);
        pl->tabdf_tpow = A.get<double2>(49 * (T + 1));
        pl->tabdf_dshift = A.get<double2>(8 * (T + 1));
    }
    if (o.precision == LBF_PRECISION_FP32_REFINE) {
        int P32 = o.p32 + 1;
        pl->P32 = P32;
        pl->q32 = A.get<float2>(N);
        pl->u32 = A.get<float2>(N);
        pl->anc = A.get<int32_t>(cap * LBF_ANC_STRIDE);
        pl->isl = A.get<int32_t>(N);
        pl->imean = A.get<double>((int64_t)M + 8);
        pl->iacoef = A.get<double>(M);
        if (o.matvec == LBF_MATVEC_FMM) {
            pl->mpole32 = A.get<float2>(cap * P32);
            pl->local32 = A.get<float2>(cap * P32);
        }
        pl->tab32_binom = A.get<float>(2 * T * T);
        pl->tab32_tpow = A.get<float2>(49 * (T + 1));
        pl->tab32_dshift = A.get<float2>(8 * (T + 1));
        if (o.border) {
            pl->gr = A.get<double>(n);
            pl->gd = A.get<double>(n);
        }
    }
    pl->v = A.get<double>(N);
    pl->bsig = A.get<double>(4);
    pl->red = A.get<double>(1024);
    pl->red_count = A.get<unsigned>(4);
    pl->dev_status = A.get<int>(2);  // [0] error bits, [1] poll limit of device waits (0: default)
    pl->fvec = A.get<double>(M);
    pl->yvec = A.get<double>(M);
    pl->tin = A.get<double>(n);
    pl->tout = A.get<double>(n);
    if (o.border) pl->vstep = A.get<double>(n);
    if (o.border) {
        Border &B = pl->bd;
        B.P = 36;   // (sqrt2/3)^36 / 36 ~ 1e-13 worst-case truncation of P2L + L2P
        B.Pe = 32;  // the accurate E y: (sqrt2/3)^32 / 32 ~ 1e-12, one coefficient per lane
        B.P32 = 16;
        B.pair_cap = (int64_t)M * 27 * (o.max_depth + 1);
        B.leaf_of = A.get<int32_t>(N);
        B.ell = A.get<double>(N);
        B.xc = A.get<double2>(M);
        B.kind = A.get<int32_t>(M);
        B.live = A.get<int32_t>(M);
        B.cell = A.get<int32_t>(2 * (int64_t)M);
        B.lam = A.get<double>(M);
        B.glob = A.get<int32_t>(M);
        B.nglob = A.get<int32_t>(1);
        B.pairs_a = A.get<int32_t>(B.pair_cap);
        B.pairs_b = A.get<int32_t>(B.pair_cap);
        B.p2l_ptr = A.get<int32_t>(cap + 1);
        B.p2l_src = A.get<int32_t>(B.pair_cap);
        B.near_ptr = A.get<int32_t>(cap + 1);
        B.near_src = A.get<int32_t>(B.pair_cap);
        B.chunk_leaf = A.get<int32_t>(B.pair_cap);
        B.chunk_k = A.get<int32_t>(B.pair_cap);
        B.nodebase = A.get<int32_t>(N + 1);
        // partial sums: sum over leaves of nodes x ceil(direct centres / 32) <= N + 2 pair_cap
        B.partial_cap = N + 2 * B.pair_cap;
        B.partial = A.get<double>(B.partial_cap);
        B.cp2l = A.get<int32_t>((int64_t)M + 1);
        B.cnear = A.get<int32_t>((int64_t)M + 1);
        B.loc = A.get<double2>(cap * B.P);
        if (o.precision == LBF_PRECISION_FP32_REFINE) B.loc32 = A.get<float2>(cap * B.P32);
        B.zc = A.get<double2>(M);
        B.Rk = A.get<double>(M);
        B.rk = A.get<double>(M);
        B.slog = A.get<double>(M);
        B.sell = A.get<double>(M);
        B.mu = A.get<double2>((int64_t)M * B.P);
        B.nu = A.get<double2>((int64_t)M * B.P);
        B.sums = A.get<double>(4);
        pl->Sinv = A.get<double>((int64_t)M * M);
        pl->lu = o.schur == LBF_SCHUR_LU || (o.schur == LBF_SCHUR_AUTO && M > 1024);
        if (pl->lu) {
            pl->lu_piv = A.get<int>(M);
            pl->lu_perm = A.get<int>(M);
            pl->lu_z = A.get<float2>(M);
            pl->lu_sync = A.get<unsigned>(lbf_lu_sync_words(M));
            pl->lu_dinv = A.get<float2>(lbf_lu_dinv_entries(M));
            pl->lu_S = A.get<double>((int64_t)M * M);
            pl->lu_r = A.get<double>(M);
            pl->lu_z2 = A.get<float2>(M);
        }
    }
    int m = o.restart;
    pl->ldv = (n + 31) / 32 * 32;
    // blocks of the Arnoldi reductions: about 2048 unknowns each, at most 2 per SM (a
    // small system's steps would otherwise pay for hundreds of near-empty blocks)
    pl->mdot_blocks = (int)std::min<int64_t>(lbf_gmres_blocks(), std::max<int64_t>(1, lbf_cdiv(n, 2048)));
    if (o.border) {
        pl->H = A.get<double>((int64_t)(m + 1) * m + 2 * (m + 1) + 2 * m + 2 * (m + 1) + m);
        pl->gw = A.get<double>(n);
        pl->gx = A.get<double>(n);
        pl->gb = A.get<double>(n);
        pl->gpart = A.get<double>((int64_t)pl->mdot_blocks * (m + 2));
        pl->gs = (GmresState *)A.take(sizeof(GmresStateBytes));
    }
    // Region shared by the basis V (solves) and the plan-creation temporaries.
    size_t vbytes = o.border ? sizeof(double) * (size_t)pl->ldv * (m + 1) : 0;
    int64_t nunits = lbf_cdiv(N, 1024);
    size_t tmp = 0;
    auto add = [&](size_t b) { tmp = ((tmp + 255) & ~size_t(255)) + b; };
    add(sizeof(double2) * N);      // xi_o
    add(sizeof(double2) * N);      // w_o
    add(sizeof(double) * N);       // d_o
    add(sizeof(double) * N);       // b_o
    const int64_t nk = std::max<int64_t>(N, o.border ? pl->bd.pair_cap : 0);  // tree and pair sorts
    add(sizeof(uint64_t) * nk);    // keys
    add(sizeof(uint64_t) * nk);    // keys_alt
    add(sizeof(int32_t) * nk);     // perm_alt
    int64_t iscr = std::max<int64_t>(256 * nunits + 4096, 4 * cap + 4096) + 6 * (int64_t)M + N / 512 + 8192;
    add(sizeof(int32_t) * iscr);   // integer scratch (scans, histograms, flags)
    add(std::max(sizeof(double) * lbf_gj_scratch_doubles(M), lbf_lu_scratch_bytes(M)));  // the inverse's or the factorisation's
    size_t big = std::max(vbytes, tmp);
    pl->region = (char *)A.take(big);
    pl->region_bytes = big;
    pl->V = o.border ? (double *)pl->region : nullptr;
}

// The buffers one right-hand side's solve writes, in the sizes lbf_layout gives them
// (which of them exist follows the options, as there), carved from A for a plan view of
// lbf_gmres_solve_many: each right-hand side has its own copy, while the geometry, the
// tree, the lists, the tables and S^-1 stay the plan's.  pl needs only the sizes that
// lbf_layout sets (it may have been laid out without memory).
static void layout_rhs(const lbf_plan *pl, lbf_plan *v, Arena &A)
{
    const lbf_options &o = pl->opt;
    const int64_t N = pl->N, n = pl->n, cap = pl->tree.cap;
    const int M = pl->M, P = pl->P, m = o.restart;
    const Border &B = pl->bd;
    const bool fmm = o.matvec == LBF_MATVEC_FMM, f32 = o.precision == LBF_PRECISION_FP32_REFINE;
    v->q = A.get<double2>(N);
    v->mpole = fmm ? A.get<double2>(cap * P) : nullptr;
    v->local = fmm ? A.get<double2>(cap * P) : nullptr;
    v->upcnt = fmm || o.border ? A.get<int32_t>(cap) : nullptr;
    v->pull = fmm || o.border ? A.get<uint32_t>(2 * cap + 4) : nullptr;
    v->qdf = fmm && o.fmm64 ? (void *)A.get<double2>(N) : nullptr;
    v->q32 = f32 ? A.get<float2>(N) : nullptr;
    v->mpole32 = f32 && fmm ? A.get<float2>(cap * (o.p32 + 1)) : nullptr;
    v->local32 = f32 && fmm ? A.get<float2>(cap * (o.p32 + 1)) : nullptr;
    v->imean = f32 ? A.get<double>((int64_t)M + 8) : nullptr;
    v->gr = f32 && o.border ? A.get<double>(n) : nullptr;
    v->gd = f32 && o.border ? A.get<double>(n) : nullptr;
    v->v = A.get<double>(N);
    v->bsig = A.get<double>(4);
    v->red = A.get<double>(1024);
    v->red_count = A.get<unsigned>(4);
    v->fvec = A.get<double>(M);
    v->yvec = A.get<double>(M);
    v->tin = A.get<double>(n);
    v->tout = A.get<double>(n);
    v->vstep = o.border ? A.get<double>(n) : nullptr;
    v->bd.partial = o.border ? A.get<double>(B.partial_cap) : nullptr;
    v->bd.loc = o.border ? A.get<double2>(cap * B.P) : nullptr;
    v->bd.loc32 = o.border && f32 ? A.get<float2>(cap * B.P32) : nullptr;
    v->bd.sums = o.border ? A.get<double>(4) : nullptr;
    v->H = A.get<double>((int64_t)(m + 1) * m + 2 * (m + 1) + 2 * m + 2 * (m + 1) + m);
    v->gw = A.get<double>(n);
    v->gx = A.get<double>(n);
    v->gb = A.get<double>(n);
    v->gpart = A.get<double>((int64_t)pl->mdot_blocks * (m + 2));
    v->gs = (GmresState *)A.take(sizeof(GmresStateBytes));
    v->nearbuf = A.get<double>(N);
    v->V = A.get<double>(pl->ldv * (m + 1));
    v->region = (char *)v->V;
    v->region_bytes = sizeof(double) * (size_t)pl->ldv * (m + 1);
}

// A view of plan pl over R right-hand sides whose buffers fill work (R slabs of equal
// size, then 3 R device states for the host's reads); *need = the bytes it takes.
// work == nullptr only sizes it.
int lbf_many_view(const lbf_plan *pl, int R, void *work, size_t bytes, lbf_plan *view,
                  size_t *need)
{
    lbf_plan v = *pl;
    Arena A;
    layout_rhs(pl, &v, A);  // sizes only
    const size_t slab = (A.off + 255) & ~size_t(255);
    const size_t total = slab * (size_t)R + 3 * (size_t)R * sizeof(GmresStateBytes);
    if (need) *need = total;
    if (!work || !view) return LBF_OK;
    if (bytes < total) return LBF_EWORKSPACE;
    Arena W;
    W.base = (char *)work;
    W.cap = slab;
    layout_rhs(pl, &v, W);
    if (W.overflow) return LBF_EWORKSPACE;
    v.nrhs = R;
    v.slab = (int64_t)slab;
    for (auto &row : v.gexec)
        for (auto &g : row) g = nullptr;  // the view captures its own step graph
    *view = v;
    return LBF_OK;
}

// The view's right-hand side r alone (one right-hand side, its own buffers)
lbf_plan lbf_view_at(const lbf_plan &v, int r)
{
    lbf_plan o = v;
    const int64_t off = (int64_t)r * v.slab;
    auto mv = [&](auto *&p) {
        using P = std::remove_reference_t<decltype(p)>;
        if (p) p = (P)((char *)p + off);
    };
    mv(o.q); mv(o.mpole); mv(o.local); mv(o.upcnt); mv(o.pull); mv(o.qdf); mv(o.q32);
    mv(o.mpole32); mv(o.local32); mv(o.imean); mv(o.gr); mv(o.gd); mv(o.v); mv(o.bsig);
    mv(o.red); mv(o.red_count); mv(o.fvec); mv(o.yvec); mv(o.tin); mv(o.tout); mv(o.vstep);
    mv(o.bd.partial); mv(o.bd.loc); mv(o.bd.loc32); mv(o.bd.sums); mv(o.H); mv(o.gw);
    mv(o.gx); mv(o.gb); mv(o.gpart); mv(o.gs); mv(o.V); mv(o.region); mv(o.nearbuf);
    o.nrhs = 1;
    o.slab = 0;
    return o;
}

namespace {
struct Temps {
    double2 *xi_o, *w_o;
    double *d_o, *b_o;
    uint64_t *keys, *keys_alt;
    int32_t *perm_alt, *iscr;
    int64_t iscr_len;
    double *gj;
};

Temps temps(lbf_plan *pl, char *region, int64_t N, int M, int64_t cap)
{
    Temps t;
    size_t off = 0;
    auto take = [&](size_t b) {
        off = (off + 255) & ~size_t(255);
        void *p = region + off;
        off += b;
        return p;
    };
    t.xi_o = (double2 *)take(sizeof(double2) * N);
    t.w_o = (double2 *)take(sizeof(double2) * N);
    t.d_o = (double *)take(sizeof(double) * N);
    t.b_o = (double *)take(sizeof(double) * N);
    const int64_t nk = std::max<int64_t>(N, pl->opt.border ? pl->bd.pair_cap : 0);
    t.keys = (uint64_t *)take(sizeof(uint64_t) * nk);
    t.keys_alt = (uint64_t *)take(sizeof(uint64_t) * nk);
    t.perm_alt = (int32_t *)take(sizeof(int32_t) * nk);
    int64_t nunits = lbf_cdiv(N, 1024);
    t.iscr_len = std::max<int64_t>(256 * nunits + 4096, 4 * cap + 4096) + 6 * (int64_t)M + N / 512 + 8192;
    t.iscr = (int32_t *)take(sizeof(int32_t) * t.iscr_len);
    t.gj = (double *)take(std::max(sizeof(double) * lbf_gj_scratch_doubles(M), lbf_lu_scratch_bytes(M)));
    return t;
}
}  // namespace

LbfInject &lbf_inject_state()
{
    static thread_local LbfInject st;
    return st;
}

void lbf_inject_barrier(unsigned *count, cudaStream_t s)
{
    if (lbf_inject_state().barrier) cudaMemsetAsync(count, 0xff, sizeof(unsigned), s);
}

extern "C" {

int lbf_default_options(lbf_options *o)
{
    if (!o) return LBF_EINVAL;
    o->tol = 1e-12;
    o->restart = 50;
    o->maxit = 2000;
    o->p = 26;
    o->leaf_size = 48;
    o->max_depth = 30;
    o->matvec = LBF_MATVEC_FMM;
    o->border = 1;
    o->box_capacity = 0;
    o->precision = LBF_PRECISION_FP64;
    o->p32 = 12;
    o->inner_tol = 3e-4;
    o->max_refine = 20;
    o->graphs = -1;
    o->fmm64 = 1;
    o->schur = LBF_SCHUR_AUTO;
    o->p2p_warps = 0;
    o->precond = 1;
    return LBF_OK;
}

const char *lbf_status_string(int s)
{
    switch (s) {
    case LBF_OK: return "ok";
    case LBF_NOCONV: return "GMRES reached maxit before tol";
    case LBF_EINVAL: return "invalid argument";
    case LBF_EPOLE: return "a node lies at the projection pole";
    case LBF_EDEPTH: return "quadtree deeper than supported";
    case LBF_EWORKSPACE: return "workspace too small";
    case LBF_ECUDA: return "CUDA runtime error";
    case LBF_ETIMEOUT: return "a bounded device wait gave up";
    case LBF_ENOTBUILT: return "the plan was created without the parts this call needs";
    case LBF_ESINGULAR: return "the Schur complement of the border is singular";
    default: return "unknown status";
    }
}

static int check_islands(int M, const int64_t *ptr, int64_t *N)
{
    if (M < 1 || !ptr || ptr[0] != 0) return LBF_EINVAL;
    for (int k = 0; k < M; k++)
        if (ptr[k + 1] - ptr[k] < 3) return LBF_EINVAL;
    if (ptr[M] >= (int64_t)1 << 31) return LBF_EINVAL;
    *N = ptr[M];
    return LBF_OK;
}

int lbf_workspace_size(int M, const int64_t *island_ptr, const lbf_options *opt, size_t *bytes)
{
    if (!opt || !bytes || !valid(*opt)) return LBF_EINVAL;
    int64_t N;
    int rc = check_islands(M, island_ptr, &N);
    if (rc) return rc;
    lbf_plan tmp;
    tmp.arena.base = nullptr;
    tmp.arena.cap = ~size_t(0);
    lbf_layout(&tmp, N, M, *opt, box_capacity_estimate(N, *opt));
    *bytes = tmp.arena.off + 256;
    return LBF_OK;
}

int lbf_batch_workspace_size(int M, const int64_t *island_ptr, const lbf_options *opt, int nrhs,
                             size_t *bytes)
{
    if (nrhs < 0 || !bytes) return LBF_EINVAL;
    size_t pb = 0;
    int rc = lbf_workspace_size(M, island_ptr, opt, &pb);
    if (rc) return rc;
    *bytes = pb;
    const bool lu = opt->schur == LBF_SCHUR_LU || (opt->schur == LBF_SCHUR_AUTO && M > 1024);
    if (nrhs < 2 || !opt->border || lu) return LBF_OK;
    const int64_t N = island_ptr[M];
    lbf_plan tmp;
    tmp.N = N;
    tmp.M = M;
    tmp.n = N + M;
    tmp.opt = *opt;
    tmp.P = opt->p + 1;
    tmp.arena.base = nullptr;
    tmp.arena.cap = ~size_t(0);
    lbf_layout(&tmp, N, M, *opt, box_capacity_estimate(N, *opt));
    size_t need = 0;
    if ((rc = lbf_many_view(&tmp, std::min(nrhs, LBF_LOCKSTEP_MAX), nullptr, 0, nullptr, &need)))
        return rc;
    *bytes = ((pb + 255) & ~size_t(255)) + need;
    return LBF_OK;
}

static int plan_create(lbf_plan **plan, int M, const int64_t *island_ptr, const double *x,
                       const double *dx, const double *d2x, const double *centres,
                       const double *pole_rotation, int planar, const lbf_options *opt,
                       void *workspace, size_t bytes, int64_t *box_needed, lbf_stream_t stream)
{
    if (!plan || !x || !dx || !d2x || !centres || !opt || !workspace || !valid(*opt))
        return LBF_EINVAL;
    *plan = nullptr;
    int64_t N;
    int rc = check_islands(M, island_ptr, &N);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = lbf_fmm_init_attrs()) || (rc = lbf_border_init_attrs())) return rc;
    lbf_plan *pl = new (std::nothrow) lbf_plan();
    if (!pl) return LBF_EINVAL;
    pl->N = N;
    pl->M = M;
    pl->n = N + M;
    pl->opt = *opt;
    pl->P = opt->p + 1;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&pl->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            delete pl;
            return LBF_ECUDA;
        }
    }
    int64_t cap = box_capacity_estimate(N, *opt);
    pl->arena.base = (char *)workspace;
    pl->arena.cap = bytes;
    lbf_layout(pl, N, M, *opt, cap);
    if (pl->arena.overflow) {
        delete pl;
        if (box_needed) *box_needed = cap;
        return LBF_EWORKSPACE;
    }
    auto fail = [&](int code) {
        lbf_border_end(pl);  // waits for the side stream's work first
        for (auto &e : pl->ev)
            if (e) cudaEventDestroy(e);
        if (pl->host_status) cudaFreeHost(pl->host_status);
        if (pl->host_scalars) cudaFreeHost(pl->host_scalars);
        delete[] pl->island_ptr_h;
        delete pl;
        return code;
    };
    if (cudaHostAlloc((void **)&pl->host_status, 64, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&pl->host_scalars, 64 * (4 + 3 * LBF_LOCKSTEP_MAX), cudaHostAllocDefault) != cudaSuccess)
        return fail(LBF_ECUDA);
    for (auto &e : pl->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LBF_ECUDA);
    pl->island_ptr_h = new int64_t[M + 1];
    memcpy(pl->island_ptr_h, island_ptr, sizeof(int64_t) * (M + 1));
    if (pole_rotation) {
        pl->has_rot = 1;
        memcpy(pl->rot, pole_rotation, sizeof(pl->rot));
    } else {
        pl->has_rot = 0;
        for (int i = 0; i < 9; i++) pl->rot[i] = (i % 4 == 0) ? 1.0 : 0.0;
    }
    std::vector<double> binom;
    std::vector<double2> dshift, tpow;
    make_tables(binom, dshift, tpow);
#define CK(call) do { if ((call) != cudaSuccess) return fail(LBF_ECUDA); } while (0)
    CK(cudaMemcpyAsync(pl->island_ptr, island_ptr, sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl->rot_d, pl->rot, sizeof(pl->rot), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl->tab_binom, binom.data(), sizeof(double) * binom.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl->tab_dshift, dshift.data(), sizeof(double2) * dshift.size(), cudaMemcpyHostToDevice, s));
    if (pl->tab32_binom) {  // the same tables rounded to float
        std::vector<float> b32(binom.begin(), binom.end());
        std::vector<float2> t32(tpow.size()), d32(dshift.size());
        for (size_t i = 0; i < tpow.size(); i++) t32[i] = make_float2((float)tpow[i].x, (float)tpow[i].y);
        for (size_t i = 0; i < dshift.size(); i++) d32[i] = make_float2((float)dshift[i].x, (float)dshift[i].y);
        CK(cudaMemcpyAsync(pl->tab32_binom, b32.data(), sizeof(float) * b32.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(pl->tab32_tpow, t32.data(), sizeof(float2) * t32.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(pl->tab32_dshift, d32.data(), sizeof(float2) * d32.size(), cudaMemcpyHostToDevice, s));
    }
    if (pl->tabdf_binom) {  // the same tables as double-floats (hi, lo per real)
        std::vector<float> b2(2 * binom.size()), t2(4 * tpow.size()), d2(4 * dshift.size());
        auto split = [](double v, float *o) {
            o[0] = (float)v;
            o[1] = (float)(v - (double)o[0]);
        };
        for (size_t i = 0; i < binom.size(); i++) split(binom[i], &b2[2 * i]);
        for (size_t i = 0; i < tpow.size(); i++) {
            split(tpow[i].x, &t2[4 * i]);
            split(tpow[i].y, &t2[4 * i + 2]);
        }
        for (size_t i = 0; i < dshift.size(); i++) {
            split(dshift[i].x, &d2[4 * i]);
            split(dshift[i].y, &d2[4 * i + 2]);
        }
        CK(cudaMemcpyAsync(pl->tabdf_binom, b2.data(), sizeof(float) * b2.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(pl->tabdf_tpow, t2.data(), sizeof(float) * t2.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(pl->tabdf_dshift, d2.data(), sizeof(float) * d2.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // the host vectors end with this scope
    }
    if (pl->upcnt) CK(cudaMemsetAsync(pl->upcnt, 0, sizeof(int32_t) * cap, s));
    if (pl->pull) CK(cudaMemsetAsync(pl->pull, 0, sizeof(uint32_t) * (2 * cap + 4), s));
    CK(cudaMemcpyAsync(pl->tab_tpow, tpow.data(), sizeof(double2) * tpow.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(pl->dev_status, 0, 2 * sizeof(int), s));
    if (lbf_inject_state().barrier) {  // a test's injection: this plan's poll limit
        const int lim = (int)lbf_inject_state().polls;
        CK(cudaMemcpyAsync(pl->dev_status + 1, &lim, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    CK(cudaMemsetAsync(pl->red_count, 0, 4 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(pl->bsig, 0, 4 * sizeof(double), s));
    // plan-creation temporaries overlay the region of the GMRES basis
    Temps tt = temps(pl, pl->region, N, M, cap);
    lbf_prof_mark(LBF_STAGE_GEOMETRY, 1, s);
    rc = lbf_geometry_build(pl, x, dx, d2x, centres, planar, s, tt.xi_o, tt.w_o, tt.d_o, tt.b_o);
    if (rc) return fail(rc);
    // S and its inverse need only the planar nodes and the centres: they run on a side
    // stream while this one builds the tree
    if (opt->border && (rc = lbf_border_start(pl, s, tt.xi_o, tt.gj))) return fail(rc);
    {
        int64_t need = 0;
        rc = lbf_tree_build(pl, s, tt.xi_o, tt.keys, tt.keys_alt, tt.perm_alt, tt.iscr, tt.iscr_len, &need);
        if (rc == LBF_OK && opt->matvec == LBF_MATVEC_FMM)
            rc = lbf_lists_build(pl, s, tt.iscr, tt.iscr_len, &need);
        if (rc == LBF_EWORKSPACE && box_needed) *box_needed = need;
        if (rc) return fail(rc);
    }
    rc = lbf_geometry_gather(pl, s, tt.xi_o, tt.w_o, tt.d_o, tt.b_o);
    if (rc) return fail(rc);
    if ((rc = lbf_fmm_prepare(pl, s))) return fail(rc);
    lbf_prof_mark(LBF_STAGE_GEOMETRY, 0, s);
    if (opt->border) {
        SortBufs sb{tt.keys, tt.keys_alt, tt.perm_alt};
        rc = lbf_border_build(pl, s, tt.iscr, tt.iscr_len, sb);
        if (rc) return fail(rc);
    }
    CK(cudaMemcpyAsync(pl->host_status, pl->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    lbf_border_end(pl);
#undef CK
    int st = *pl->host_status;
    if (st & LBF_DEV_POLE) return fail(LBF_EPOLE);
    if (st & LBF_DEV_TIMEOUT) return fail(LBF_ETIMEOUT);  // a grid barrier of the inverse gave up
    if (st & 4) return fail(LBF_ESINGULAR);   // singular Schur complement
    if (st & 8) return fail(LBF_EDEPTH);      // list overflow
    if (st & 16) return fail(LBF_EWORKSPACE); // more near centres per island than the border holds
    *plan = pl;
    return LBF_OK;
}

int lbf_plan_create(lbf_plan **plan, int M, const int64_t *island_ptr, const double *x,
                    const double *dx, const double *d2x, const double *centres,
                    const double *pole_rotation, const lbf_options *opt, void *workspace,
                    size_t bytes, int64_t *box_needed, lbf_stream_t stream)
{
    const int rc = plan_create(plan, M, island_ptr, x, dx, d2x, centres, pole_rotation, 0, opt,
                               workspace, bytes, box_needed, stream);
    lbf_inject_state() = LbfInject{};  // a pending injection applies to one plan creation
    return rc;
}

int lbf_plan_create_planar(lbf_plan **plan, int M, const int64_t *island_ptr, const double *xi,
                           const double *dxi, const double *d2xi, const double *centres,
                           const lbf_options *opt, void *workspace, size_t bytes,
                           int64_t *box_needed, lbf_stream_t stream)
{
    const int rc = plan_create(plan, M, island_ptr, xi, dxi, d2xi, centres, nullptr, 1, opt,
                               workspace, bytes, box_needed, stream);
    lbf_inject_state() = LbfInject{};
    return rc;
}

int lbf_plan_destroy(lbf_plan *pl)
{
    if (!pl) return LBF_EINVAL;
    for (auto &row : pl->gexec)
        for (auto &g : row)
            if (g) cudaGraphExecDestroy(g);
    for (auto &e : pl->ev)
        if (e) cudaEventDestroy(e);
    if (pl->host_status) cudaFreeHost(pl->host_status);
    if (pl->host_scalars) cudaFreeHost(pl->host_scalars);
    delete[] pl->island_ptr_h;
    delete pl;
    return LBF_OK;
}

int lbf_plan_info(const lbf_plan *pl, int64_t *N, int *M, int64_t *nbox, int64_t *nleaf, int *depth,
                  int *p)
{
    if (!pl) return LBF_EINVAL;
    if (N) *N = pl->N;
    if (M) *M = pl->M;
    if (nbox) *nbox = pl->tree.nbox;
    if (nleaf) *nleaf = pl->tree.nleaf;
    if (depth) *depth = pl->tree.nlev - 1;
    if (p) *p = pl->P - 1;
    return LBF_OK;
}

int lbf_geometry_out(const lbf_plan *pl, double *xi, double *normal, double *weight,
                     double *arc_weight, lbf_stream_t stream)
{
    if (!pl) return LBF_EINVAL;
    return lbf_geometry_out_impl(pl, xi, normal, weight, arc_weight, (cudaStream_t)stream);
}

int lbf_apply(lbf_plan *pl, int op, const double *in, double *out, lbf_stream_t stream)
{
    int prec = (op & LBF_OP_FP32) ? LBF_PREC_FP32 : LBF_PREC_FP64;
    const int tr = op & LBF_OP_TRANSPOSE;
    op &= ~(LBF_OP_FP32 | LBF_OP_TRANSPOSE);
    if (!pl || !in || !out || op < 0 || op > 2) return LBF_EINVAL;
    if (op != LBF_OP_K_ONLY && !pl->opt.border) return LBF_ENOTBUILT;
    if (prec == LBF_PREC_FP32 && !pl->q32) return LBF_ENOTBUILT;
    cudaStream_t s = (cudaStream_t)stream;
    int with_a = op != LBF_OP_K_ONLY;
    int rc = lbf_permute_in(pl, in, pl->tin, with_a, s);
    if (rc) return rc;
    rc = lbf_apply_op_sorted(pl, op | tr, pl->tin, pl->tout, nullptr, s, prec);
    if (rc) return rc;
    return lbf_permute_out(pl, pl->tout, out, with_a, s);
}

int lbf_gmres_solve(lbf_plan *pl, const double *g, double *sigma, double *a, const double *x0,
                    int *iters, double *rel_res, lbf_stream_t stream)
{
    if (!pl || !g || !sigma) return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    return lbf_gmres_impl(pl, g, sigma, a, x0, iters, rel_res, (cudaStream_t)stream, 0);
}

int lbf_gmres_workspace_many(const lbf_plan *pl, int nrhs, size_t *bytes)
{
    if (!pl || nrhs < 1 || !bytes) return LBF_EINVAL;
    *bytes = 0;
    if (pl->lu || !pl->opt.border) return LBF_OK;
    return lbf_many_view(pl, std::min(nrhs, LBF_LOCKSTEP_MAX), nullptr, 0, nullptr, bytes);
}

int lbf_gmres_solve_many(lbf_plan *pl, int nrhs, const double *g, double *sigma, double *a,
                         int *iters, double *rel_res, void *work, size_t bytes, lbf_stream_t stream)
{
    if (!pl || nrhs < 1 || !g || !sigma) return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    size_t need = 0;
    int rc = lbf_gmres_workspace_many(pl, nrhs, &need);
    if (rc) return rc;
    if (need > 0 && (!work || bytes < need || ((uintptr_t)work & 255))) return LBF_EWORKSPACE;
    return lbf_gmres_many_impl(pl, nrhs, g, sigma, a, iters, rel_res, work, bytes,
                               (cudaStream_t)stream);
}

int lbf_gmres_solve_transpose(lbf_plan *pl, const double *r, double *lam, const double *x0,
                              int *iters, double *rel_res, lbf_stream_t stream)
{
    if (!pl || !r || !lam) return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    return lbf_gmres_impl(pl, r, lam, nullptr, x0, iters, rel_res, (cudaStream_t)stream, 1);
}

int lbf_evaluate_transpose(lbf_plan *pl, int64_t T, const double *targets, const double *ubar,
                           double *sbar, double *abar, lbf_stream_t stream)
{
    if (!pl || T < 0 || !sbar || (T > 0 && (!targets || !ubar))) return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    if (pl->region_bytes < sizeof(double) * (4 * (size_t)pl->N + 8)) return LBF_EWORKSPACE;
    return lbf_evaluate_transpose_impl(pl, T, targets, ubar, sbar, abar, (cudaStream_t)stream);
}

int lbf_gradient_nodes(lbf_plan *pl, const double *sigma, const double *a, const double *lam,
                       int64_t T, const double *targets, const double *ubar, double *grad,
                       lbf_stream_t stream)
{
    if (!pl || !sigma || !a || !lam || !grad || T < 0 || (T > 0 && (!targets || !ubar)))
        return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    if (pl->region_bytes < sizeof(double) * (12 * (size_t)pl->N + 8)) return LBF_EWORKSPACE;
    return lbf_gradient_nodes_impl(pl, sigma, a, lam, T, targets, ubar, grad, (cudaStream_t)stream);
}

int lbf_gradient_data(lbf_plan *pl, const double *lam, double *grad_g, lbf_stream_t stream)
{
    if (!pl || !lam || !grad_g) return LBF_EINVAL;
    return lbf_gradient_data_impl(pl, lam, grad_g, (cudaStream_t)stream);
}

int lbf_solve_stats(const lbf_plan *pl, int64_t stats[4])
{
    if (!pl || !stats) return LBF_EINVAL;
    for (int k = 0; k < 4; k++) stats[k] = pl->stats[k];
    return LBF_OK;
}

int lbf_evaluate(lbf_plan *pl, const double *sigma, const double *a, int64_t T,
                 const double *targets, double *u, lbf_stream_t stream)
{
    if (!pl || !sigma || T < 0 || (T > 0 && (!targets || !u))) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = lbf_permute_in(pl, sigma, pl->tin, 0, s);
    if (rc) return rc;
    return lbf_evaluate_impl(pl, pl->tin, a, T, targets, u, s);
}

int lbf_green_sum(int64_t T, const double *t, int64_t S, const double *p, const double *gamma,
                  double *out, lbf_stream_t stream)
{
    if (T < 0 || S < 0 || (T > 0 && (!t || !out)) || (S > 0 && (!p || !gamma))) return LBF_EINVAL;
    return lbf_green_sum_impl(T, t, S, p, gamma, out, (cudaStream_t)stream);
}

int lbf_sync_status(lbf_plan *pl, lbf_stream_t stream)
{
    if (!pl) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(pl->host_status, pl->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LBF_ECUDA;
    int st = *pl->host_status;
    if (st & LBF_DEV_POLE) return LBF_EPOLE;
    if (st & LBF_DEV_TIMEOUT) return LBF_ETIMEOUT;
    if (st & 8) return LBF_EDEPTH;
    return LBF_OK;
}

int64_t lbf_launch_count(void) { return g_lbf_launches.load(); }

int lbf_debug_inject(lbf_plan *pl, int what, unsigned polls, lbf_stream_t stream)
{
    if (polls == 0 || polls > (1u << 30)) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (what == LBF_INJECT_BARRIER) {
        if (pl) return LBF_EINVAL;
        lbf_inject_state() = LbfInject{1, polls};
        return LBF_OK;
    }
    if (what != LBF_INJECT_CHAIN || !pl) return LBF_EINVAL;
    if (!pl->pull || pl->opt.matvec != LBF_MATVEC_FMM || pl->tree.nlev <= 3) return LBF_ENOTBUILT;
    // the poll limit, and the second phase of the next chain starting at the first box of
    // level 3: levels 0..2 are never marked done in that epoch, so their children's
    // parent waits run out; the chain's last warp resets the counters as always
    const int lim = (int)polls;
    const unsigned first = (unsigned)pl->tree.lev_start[3];
    LBF_CUDA(cudaMemcpyAsync(pl->dev_status + 1, &lim, sizeof(int), cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(pl->pull + 3, &first, sizeof(unsigned), cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

int lbf_debug_clear(lbf_plan *pl, lbf_stream_t stream)
{
    if (!pl) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    LBF_CUDA(cudaMemsetAsync(pl->dev_status, 0, 2 * sizeof(int), s));
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

}  // extern "C"
