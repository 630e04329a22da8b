// The multiplier potential of the bordered system (Sec. 4.1, Eq. u_multi;
// Sec. 5, Eq. matrix_eqns): (E y)_i = sum_m y_m 2 G(x_i, c_m) at every node, and
// the Schur complement S = D - F E of the block preconditioner (Eq. matrix_eqns_c),
// without forming the N x M block E (the paper notes E a could be evaluated by
// the FMM, Sec. 5).
//
// In the stereographic plane (Sec. 3, Eq. fundC), for a centre with finite image
// xi_m and for the centre at the pole,
//   2 G(x, c_m)   = (1/2pi) [ l(x) - log 2 + lam_m - 2 log|xi - xi_m| ],
//   2 G(x, pole)  = (1/2pi) [ l(x) - log 2 ],
// with l(x) = log(1 + |xi|^2), lam_m = log(1 + |xi_m|^2).  So
//   (E y)_i = (1/2pi) [ (l_i - log 2) Y + Lam - 2 sum_{m finite} y_m log|xi_i - xi_m| ],
// Y = sum_m y_m, Lam = sum_{m finite} y_m lam_m.
//
// The log sum runs on the nodes' quadtree: every finite centre is a point source
// that, level by level, enters the local expansion of each box that first
// becomes well separated from the centre's cell (P2L into boxes whose parent
// touches the cell of the parent level but which do not touch the centre's own
// cell); local expansions are shifted down (L2L) and evaluated at the nodes
// (L2P); a leaf that still touches the centre's cell at its own level sums that
// centre directly.  Every (node, centre) pair is counted exactly once.
//
// S needs sum_j log|xi_j - xi_m| over the nodes j of island k for every (k, m);
// it uses moments of the island's nodes about their mean z_k (radius R_k, inner
// radius rho_k): the multipole of the island where |xi_m - z_k| >= 3 R_k, its
// inner expansion where |xi_m - z_k| <= rho_k / 3, and a direct sum otherwise.
#include <algorithm>
#include <type_traits>

#include "lbf_df64.cuh"
#include "lbf_internal.cuh"
#include "lbf_sync.cuh"

namespace {

constexpr double kEta = 3.0;
constexpr int kMaxLevelsWalk = LBF_MAX_LEVELS + 1;

template <typename R> struct __align__(2 * sizeof(R)) cz {
    R x, y;
};
__device__ __forceinline__ double fmr(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmr(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ df64 fmr(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }
template <typename R> __device__ __forceinline__ cz<R> zmul(cz<R> a, cz<R> b)
{
    return cz<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __device__ __forceinline__ cz<R> zfma(cz<R> a, cz<R> b, cz<R> c)
{
    return cz<R>{fmr(a.x, b.x, fmr(-a.y, b.y, c.x)), fmr(a.x, b.y, fmr(a.y, b.x, c.y))};
}
__device__ __forceinline__ cz<double> zinv(cz<double> a)
{
    double d = 1.0 / (a.x * a.x + a.y * a.y);
    return cz<double>{a.x * d, -a.y * d};
}

// an expansion coefficient written by another warp of the same launch (through L2)
__device__ __forceinline__ cz<float> ldcg_cz(const cz<float> *p)
{
    const float2 v = __ldcg((const float2 *)p);
    return cz<float>{v.x, v.y};
}
__device__ __forceinline__ cz<double> ldcg_cz(const cz<double> *p)
{
    const double2 v = __ldcg((const double2 *)p);
    return cz<double>{v.x, v.y};
}
__device__ __forceinline__ cz<df64> ldcg_cz(const cz<df64> *p)
{
    const float4 v = __ldcg((const float4 *)p);
    return cz<df64>{df64(v.x, v.y, 0), df64(v.z, v.w, 0)};
}

template <typename R> __device__ __forceinline__ R wsum(R v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Geo {
    double xmin, ymin, L;
};
__device__ __forceinline__ void centre_of(const Geo &g, int l, int ix, int iy, double &cx,
                                          double &cy, double &r)
{
    double w = ldexp(g.L, -l);
    r = 0.5 * w;
    cx = g.xmin + (ix + 0.5) * w;
    cy = g.ymin + (iy + 0.5) * w;
}

// ---- plan time ------------------------------------------------------------------------

__global__ void k_mp_nodes(int64_t N, const double2 *__restrict__ xi, double *__restrict__ ell)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 z = xi[i];
    ell[i] = log1p(z.x * z.x + z.y * z.y);
}

__global__ void k_mp_leaf_of(int64_t nleaf, const int32_t *__restrict__ leaves,
                             const int32_t *__restrict__ bg, const int32_t *__restrict__ en,
                             int32_t *__restrict__ leaf_of)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int b = leaves[t];
    for (int i = bg[b]; i < en[b]; i++) leaf_of[i] = b;
}

// per centre: planar image and lam_m (live 0 at the pole)
__global__ void k_mp_centres_plane(int M, const double *__restrict__ c, double2 *__restrict__ xc,
                                   double *__restrict__ lam, int32_t *__restrict__ live)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double w = 1.0 - c[3 * m + 2];
    if (w < 1e-12) {
        live[m] = 0;
        xc[m] = make_double2(0, 0);
        lam[m] = 0;
        return;
    }
    double2 z = make_double2(c[3 * m] / w, c[3 * m + 1] / w);
    xc[m] = z;
    lam[m] = log1p(z.x * z.x + z.y * z.y);
    live[m] = 1;
}

// per centre: its cell at the finest level of the tree (kind 0: at the pole; 1: inside
// the tree's square; 2: outside it -> summed directly); the planar image as above
__global__ void k_mp_centres(int M, const double *__restrict__ c, Geo g, int D,
                             int32_t *__restrict__ kind, int32_t *__restrict__ cell)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double w = 1.0 - c[3 * m + 2];
    if (w < 1e-12) {
        kind[m] = 0;
        cell[2 * m] = cell[2 * m + 1] = 0;
        return;
    }
    double2 z = make_double2(c[3 * m] / w, c[3 * m + 1] / w);
    double fx = floor((z.x - g.xmin) / g.L * ldexp(1.0, D));
    double fy = floor((z.y - g.ymin) / g.L * ldexp(1.0, D));
    double cmax = ldexp(1.0, D) - 1.0;
    bool in = fx >= 0 && fy >= 0 && fx <= cmax && fy <= cmax;
    kind[m] = in ? 1 : 2;
    cell[2 * m] = in ? (int32_t)fx : 0;
    cell[2 * m + 1] = in ? (int32_t)fy : 0;
}

struct TView {
    const int32_t *level, *ix, *iy, *child0, *nchild;
};

// Walk one centre down the tree.  A holds the boxes of the current level that
// touch the centre's cell there (at most 9; every box of level 1 touches it).
// Children of A that do not touch the centre's cell at their level get a P2L;
// leaves that touch it sum the centre directly.  fill == 0 counts, fill == 1
// writes (box, centre) pairs at the centre's offsets.
__global__ void k_mp_walk(int M, const int32_t *__restrict__ kind, const int32_t *__restrict__ cell,
                          int D, TView T, int fill, int32_t *__restrict__ np2l,
                          int32_t *__restrict__ nnear, const int32_t *__restrict__ op2l,
                          const int32_t *__restrict__ onear, int32_t *__restrict__ p2l_box,
                          int32_t *__restrict__ near_box, int *__restrict__ status)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int cp = 0, cn = 0;
    int32_t *pb = fill ? p2l_box + op2l[m] : nullptr;
    int32_t *nb = fill ? near_box + onear[m] : nullptr;
    if (kind[m] == 1) {
        int cx = cell[2 * m], cy = cell[2 * m + 1];
        int A[9], nA = 0, An[9];
        if (T.nchild[0] == 0) {
            if (fill) nb[cn] = 0;
            cn++;
        } else {
            for (int c = T.child0[0]; c < T.child0[0] + T.nchild[0]; c++) A[nA++] = c;
        }
        for (int l = 1; nA > 0 && l < kMaxLevelsWalk; l++) {
            int nn = 0;
            for (int q = 0; q < nA; q++) {
                int b = A[q];
                if (T.nchild[b] == 0) {  // a leaf touching the centre's cell: direct
                    if (fill) nb[cn] = b;
                    cn++;
                    continue;
                }
                int lx = cx >> (D - l - 1), ly = cy >> (D - l - 1);
                for (int c = T.child0[b]; c < T.child0[b] + T.nchild[b]; c++) {
                    if (abs(T.ix[c] - lx) <= 1 && abs(T.iy[c] - ly) <= 1) {
                        if (nn < 9) An[nn] = c;
                        nn++;
                    } else {
                        if (fill) pb[cp] = c;
                        cp++;
                    }
                }
            }
            if (nn > 9) atomicOr(status, 8);
            nA = nn < 9 ? nn : 9;
            for (int q = 0; q < nA; q++) A[q] = An[q];
        }
    }
    if (!fill) {
        np2l[m] = cp;
        nnear[m] = cn;
    }
}

// transpose (box, centre) pairs, generated centre by centre, into lists per box
__global__ void k_pairs_count(int M, const int32_t *__restrict__ off, const int32_t *__restrict__ cnt,
                              const int32_t *__restrict__ box, int32_t *__restrict__ per_box)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int q = off[m]; q < off[m] + cnt[m]; q++) atomicAdd(&per_box[box[q]], 1);
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = wsum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
    __syncthreads();
    return t;
}
__device__ __forceinline__ double block_max(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) t = fmax(t, sh[k]);
    __syncthreads();
    return t;
}

// Per island (block of 256): node mean z_k, radii R_k (max) and rho_k (min),
// sum of log|xi_j - z_k|, sum of (l_j - log 2), and the scaled moments
//   mu_l = (1/l) sum_j ((xi_j - z_k)/R_k)^l,   nu_l = (1/l) sum_j (rho_k/(xi_j - z_k))^l,
// l = 1..P-1 (the 1/l of the log expansions applied once here), mu_0 = nu_0 = N_k.
__global__ void k_mp_islands(int M, int P, const int64_t *__restrict__ ptr,
                             const double2 *__restrict__ xi_o, double2 *__restrict__ zc,
                             double *__restrict__ Rk, double *__restrict__ rk,
                             double *__restrict__ slog, double *__restrict__ sell,
                             double2 *__restrict__ mu, double2 *__restrict__ nu)
{
    __shared__ double sh[32];
    __shared__ double2 smu[8][LBF_MAX_TERMS], snu[8][LBF_MAX_TERMS];
    int k = blockIdx.x;
    int64_t b = ptr[k], e = ptr[k + 1];
    double sx = 0, sy = 0;
    for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) { sx += xi_o[j].x; sy += xi_o[j].y; }
    double n = (double)(e - b);
    double cx = block_sum(sx, sh) / n, cy = block_sum(sy, sh) / n;
    double dmax = 0, dmin = -INFINITY, sl = 0, se = 0;
    for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        double dx = xi_o[j].x - cx, dy = xi_o[j].y - cy;
        double d2 = dx * dx + dy * dy;
        dmax = fmax(dmax, d2);
        dmin = fmax(dmin, -d2);
        sl += 0.5 * log(d2);
        double2 z = xi_o[j];
        se += log1p(z.x * z.x + z.y * z.y) - LBF_LN2;
    }
    double R = sqrt(block_max(dmax, sh));
    double rho = sqrt(-block_max(dmin, sh));
    double slv = block_sum(sl, sh), sev = block_sum(se, sh);
    if (threadIdx.x == 0) {
        zc[k] = make_double2(cx, cy);
        Rk[k] = R;
        rk[k] = rho;
        slog[k] = slv;
        sell[k] = sev;
    }
    // the moments sum_j u_j^l and sum_j v_j^l in double-float (pairs of floats, ~48 bits):
    // this GPU issues float arithmetic 64 times faster than double, and the powers and
    // warp sums are the whole cost of this kernel
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    using D = df64;
    const D zero(0.0f);
    cz<D> am0{zero, zero}, am1 = am0, an0 = am0, an1 = am0;
    const double iR = 1.0 / R;
    for (int64_t base = b + wid * 32; base < e; base += blockDim.x) {
        int64_t j = base + lane;
        cz<D> u{zero, zero}, v{zero, zero};
        if (j < e) {
            cz<double> d{xi_o[j].x - cx, xi_o[j].y - cy};
            cz<double> vd = zinv(cz<double>{d.x / rho, d.y / rho});
            u = cz<D>{D(d.x * iR), D(d.y * iR)};
            v = cz<D>{D(vd.x), D(vd.y)};
        }
        cz<D> pu = u, pv = v;
        for (int l = 1; l < P; l++) {
            D mx = wsum(pu.x), my = wsum(pu.y), nx = wsum(pv.x), ny = wsum(pv.y);
            if (lane == (l & 31)) {
                if (l < 32) { am0.x += mx; am0.y += my; an0.x += nx; an0.y += ny; }
                else { am1.x += mx; am1.y += my; an1.x += nx; an1.y += ny; }
            }
            pu = zmul(pu, u);
            pv = zmul(pv, v);
        }
    }
    auto dd = [](cz<D> a) { return make_double2((double)a.x, (double)a.y); };
    smu[wid][lane] = dd(am0);
    snu[wid][lane] = dd(an0);
    smu[wid][lane + 32] = dd(am1);
    snu[wid][lane + 32] = dd(an1);
    __syncthreads();
    for (int l = threadIdx.x; l < P; l += blockDim.x) {
        double2 a = make_double2(0, 0), c = a;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a.x += smu[w][l].x; a.y += smu[w][l].y;
            c.x += snu[w][l].x; c.y += snu[w][l].y;
        }
        const double il = l ? 1.0 / l : 0.0;
        mu[(int64_t)k * P + l] = l ? make_double2(a.x * il, a.y * il) : make_double2(n, 0);
        nu[(int64_t)k * P + l] = l ? make_double2(c.x * il, c.y * il) : make_double2(n, 0);
    }
}

// sum_j log|xi_j - xi_m| over the nodes j of island k by the island's expansions;
// false where xi_m is neither far from nor deep inside the island (direct sum needed)
__device__ bool island_logsum(int k, int P, double2 xm, double2 z, double R, double rho,
                              const double2 *mu, const double2 *nu, double slog, double &out)
{
    cz<double> d{xm.x - z.x, xm.y - z.y};
    double dd = sqrt(d.x * d.x + d.y * d.y);
    // Re sum_{l>=1} c_l t^l by Horner's rule (c = the moments with their 1/l)
    auto series = [&](const double2 *c, cz<double> t) {
        cz<double> a{c[P - 1].x, c[P - 1].y};
        for (int l = P - 2; l >= 1; l--) {
            const double2 cl = c[l];
            a = cz<double>{fma(a.x, t.x, fma(-a.y, t.y, cl.x)), fma(a.x, t.y, fma(a.y, t.x, cl.y))};
        }
        return a.x * t.x - a.y * t.y;
    };
    if (dd >= kEta * R) {
        // N_k log|xi_m - z_k| - Re sum_l mu_l (R/(xi_m - z_k))^l
        const cz<double> t = zinv(cz<double>{d.x / R, d.y / R});
        out = mu[(int64_t)k * P].x * log(dd) - series(mu + (int64_t)k * P, t);
        return true;
    }
    if (dd * kEta <= rho) {
        // sum_j log|xi_j - z_k| - Re sum_l nu_l ((xi_m - z_k)/rho)^l
        const cz<double> t{d.x / rho, d.y / rho};
        out = slog - series(nu + (int64_t)k * P, t);
        return true;
    }
    return false;
}

__device__ __forceinline__ double schur_entry(int M, int r, int m, const int64_t *ptr,
                                              const int32_t *live, const double *lam,
                                              const double *sell, double ls)
{
    if (r == M - 1) return 1.0;
    const int k = r + 1;
    double fe = sell[k];  // sum_j (l_j - log 2)
    if (live[m] != 0) fe += (double)(ptr[k + 1] - ptr[k]) * lam[m] - 2.0 * ls;
    return -fe / (2.0 * LBF_PI);
}

// S = D - F E into G (M x M, row-major): row r < M-1 is minus the sum
// of E over island r+1 (Eq. disc_constr), the last row is D's row of ones (Eq. sum_ak).
// Entries that need a direct sum over the island's nodes are listed for
// k_mp_schur_direct (a warp per entry) instead of looping in one lane.
__global__ void k_mp_schur(int M, int P, const int64_t *__restrict__ ptr,
                           const double2 *__restrict__ xi_o, const double2 *__restrict__ xc,
                           const int32_t *__restrict__ live, const double *__restrict__ lam,
                           const double2 *__restrict__ zc, const double *__restrict__ Rk,
                           const double *__restrict__ rk, const double *__restrict__ slog,
                           const double *__restrict__ sell, const double2 *__restrict__ mu,
                           const double2 *__restrict__ nu, double *__restrict__ G,
                           int32_t *__restrict__ dcount, int32_t *__restrict__ dlist, int dcap)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)M * M) return;
    int r = (int)(id / M), m = (int)(id % M);
    double ls = 0.0;
    bool listed = false;
    if (r < M - 1 && live[m] != 0) {
        const int k = r + 1;
        if (!island_logsum(k, P, xc[m], zc[k], Rk[k], rk[k], mu, nu, slog[k], ls)) {
            int q = atomicAdd(dcount, 1);
            if (q < dcap) {
                dlist[q] = (int32_t)id;
                listed = true;
            } else {  // list full: sum here
                ls = 0.0;
                for (int64_t j = ptr[k]; j < ptr[k + 1]; j++) {
                    double dx = xi_o[j].x - xc[m].x, dy = xi_o[j].y - xc[m].y;
                    ls += 0.5 * log(dx * dx + dy * dy);
                }
            }
        }
    }
    if (!listed) G[(int64_t)r * M + m] = schur_entry(M, r, m, ptr, live, lam, sell, ls);
}

__global__ void k_mp_schur_direct(int M, const int64_t *__restrict__ ptr,
                                  const double2 *__restrict__ xi_o, const double2 *__restrict__ xc,
                                  const int32_t *__restrict__ live, const double *__restrict__ lam,
                                  const double *__restrict__ sell, const int32_t *__restrict__ dcount,
                                  const int32_t *__restrict__ dlist, int dcap, double *__restrict__ G)
{
    const int n = min(*dcount, dcap);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < n; q += nwarps) {
        const int64_t id = dlist[q];
        const int r = (int)(id / M), m = (int)(id % M), k = r + 1;
        const double2 xm = xc[m];
        double ls = 0.0;
        for (int64_t j = ptr[k] + lane; j < ptr[k + 1]; j += 32) {
            double dx = xi_o[j].x - xm.x, dy = xi_o[j].y - xm.y;
            ls += 0.5 * log(dx * dx + dy * dy);
        }
        ls = wsum(ls);
        if (lane == 0) G[(int64_t)r * M + m] = schur_entry(M, r, m, ptr, live, lam, sell, ls);
    }
}

// direct centres of each leaf in chunks of 32 (a warp each at application time)
__global__ void k_chunk_count(int64_t nbox, const int32_t *__restrict__ nptr, int32_t *__restrict__ nch)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nbox) nch[b] = (nptr[b + 1] - nptr[b] + 31) / 32;
}

__global__ void k_chunk_fill(int64_t nbox, const int32_t *__restrict__ nch,
                             const int32_t *__restrict__ base, int32_t *__restrict__ cleaf,
                             int32_t *__restrict__ ck)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    for (int k = 0; k < nch[b]; k++) {
        cleaf[base[b] + k] = (int32_t)b;
        ck[base[b] + k] = k;
    }
}

__global__ void k_node_chunks(int64_t N, const int32_t *__restrict__ leaf_of,
                              const int32_t *__restrict__ nch, int32_t *__restrict__ cnt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) cnt[i] = nch[leaf_of[i]];
    if (i == N) cnt[i] = 0;
}

// ---- per application ---------------------------------------------------------------

// P2L of the log sources into every box (warp per box; lanes take centres, terms pass
// through shared memory, lanes then take coefficients and sum in centre order):
//   b_0 = sum y_m log|c - xi_m|,  b_l = sum y_m (-1)^(l+1) tau_m^l / l,  tau_m = r/(c - xi_m).
// The warp of box 0 also forms Y = sum_m y_m and Lam = sum_{m finite} y_m lam_m.
template <typename R>
__global__ void k_mp_p2l(int64_t nbox, int P, int M, const int32_t *__restrict__ ptr,
                         const int32_t *__restrict__ src, const int32_t *__restrict__ level,
                         const int32_t *__restrict__ ix, const int32_t *__restrict__ iy, Geo g,
                         const double2 *__restrict__ xc, const int32_t *__restrict__ kind,
                         const double *__restrict__ lam, const double *__restrict__ y,
                         cz<R> *__restrict__ loc, double *__restrict__ sums, const int *gate,
                         int64_t slab)
{
    lbf_rhs(slab, y, loc, sums, gate);
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smr[];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cz<R> *T = (cz<R> *)smr + (size_t)wid * P * 32;
    int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + wid;
    if (b >= nbox) return;
    if (b == 0) {
        double Y = 0.0, Lam = 0.0;
        for (int m = lane; m < M; m += 32) {
            Y += y[m];
            if (kind[m]) Lam += y[m] * lam[m];
        }
        Y = wsum(Y);
        Lam = wsum(Lam);
        if (lane == 0) { sums[0] = Y; sums[1] = Lam; }
    }
    if (ptr[b] == ptr[b + 1] && b != 0) {  // no centres: a zero expansion
        for (int l = lane; l < P; l += 32) loc[b * P + l] = cz<R>{R(0), R(0)};
        return;
    }
    double cx, cy, r;
    centre_of(g, level[b], ix[b], iy[b], cx, cy, r);
    const double ir = 1.0 / r;
    double b0 = 0.0;
    cz<R> a0{R(0), R(0)}, a1{R(0), R(0)};
    for (int base = ptr[b]; base < ptr[b + 1]; base += 32) {
        int q = base + lane;
        cz<R> tau{R(0), R(0)};
        R ym = R(0);
        if (q < ptr[b + 1]) {
            int m = src[q];
            double2 xm = xc[m];
            double dx = cx - xm.x, dy = cy - xm.y;
            if constexpr (std::is_same<R, float>::value) {
                // the float operator: the difference in double, the rest in float
                const float fx = (float)(dx * ir), fy = (float)(dy * ir);
                const float d2 = fx * fx + fy * fy, id = __fdividef(1.0f, d2);
                b0 += y[m] * (double)(0.5f * __logf(d2 * (float)(r * r)));
                tau = cz<R>{fx * id, -fy * id};
            } else {
                b0 += y[m] * 0.5 * log(dx * dx + dy * dy);
                cz<double> t = zinv(cz<double>{dx * ir, dy * ir});
                tau = cz<R>{(R)t.x, (R)t.y};
            }
            ym = (R)y[m];
        }
        const int nin = min(32, ptr[b + 1] - base);  // the chunk's centres (often a few)
        bool grouped = false;
        if constexpr (std::is_same<R, double>::value) grouped = nin <= 16 && P <= 33;
        if (grouped) {
            // few centres (most boxes): G lanes per centre (the largest power of two with
            // nin G <= 32), lane g of a centre forming the powers l = g L + 1 .. (g + 1) L,
            // L = 32 / G.  Its first power comes from tau^L (log2 L squarings) and an
            // exclusive product of tau^L over the group's lanes below it (log2 G steps):
            // about 7 + L complex products a lane instead of P - 1 with most lanes idle.
            int G = 2;
            while (G * 2 * nin <= 32) G *= 2;
            const int L = 32 / G, c = lane / G, g = lane % G, cl = c < nin ? c : 0;
            const cz<R> tc{__shfl_sync(0xffffffffu, tau.x, cl), __shfl_sync(0xffffffffu, tau.y, cl)};
            const R yc = __shfl_sync(0xffffffffu, ym, cl);
            cz<R> tl = tc;
            for (int q = 1; q < L; q <<= 1) tl = zmul(tl, tl);
            cz<R> x = g == 0 ? cz<R>{(R)1, (R)0} : tl;  // tau^(g L) after the scan
            if constexpr (std::is_same<R, double>::value) {
                for (int d = 1; d < G; d <<= 1) {
                    const cz<R> y2{__shfl_up_sync(0xffffffffu, x.x, d, G),
                                   __shfl_up_sync(0xffffffffu, x.y, d, G)};
                    if (g >= d) x = zmul(x, y2);
                }
            }
            cz<R> pw = zmul(x, cz<R>{yc * tc.x, yc * tc.y});  // y tau^(g L + 1)
            for (int q = 0; q < L; q++) {
                const int l = g * L + 1 + q;
                if (l < P && c < nin) T[l * 32 + c] = pw;
                pw = zmul(pw, tc);
            }
        } else {
            cz<R> pw{ym * tau.x, ym * tau.y};  // y tau^l, l = 1
            for (int l = 1; l < P; l++) {
                T[l * 32 + lane] = pw;
                pw = zmul(pw, tau);
            }
        }
        __syncwarp();
        for (int l = lane; l < P; l += 32) {
            if (l == 0) continue;
            cz<R> s{0, 0};
            for (int k = 0; k < nin; k++) { s.x += T[l * 32 + k].x; s.y += T[l * 32 + k].y; }
            if (l < 32) { a0.x += s.x; a0.y += s.y; }
            else { a1.x += s.x; a1.y += s.y; }
        }
        __syncwarp();
    }
    b0 = wsum(b0);
    for (int l = lane; l < P; l += 32) {
        cz<R> a = l < 32 ? a0 : a1;
        R f = ((l & 1) ? (R)1 : (R)-1) / (R)l;
        loc[b * P + l] = l == 0 ? cz<R>{(R)b0, 0} : cz<R>{a.x * f, a.y * f};
    }
}

// L2L into the boxes of one level: b'_l += (2d)^-l sum_{k>=l} C(k,l) d^k b_k
template <typename R>
__global__ void k_mp_l2l(int64_t ls, int64_t le, int P, const int32_t *__restrict__ parent,
                         const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                         const R *__restrict__ binom, const cz<R> *__restrict__ dtab,
                         cz<R> *__restrict__ loc, const int *gate, int64_t slab)
{
    lbf_rhs(slab, loc, gate);
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smr[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = (P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cd = (R *)smr;  // Cd[k*P + l] = C(k, l) (0 for k < l)
    cz<R> *A = (cz<R> *)(smr + tl) + (size_t)wid * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cd[e] = k >= l ? binom[k * LBF_MAX_TERMS + l] : R(0);
    }
    __syncthreads();
    int64_t b = ls + blockIdx.x * (int64_t)nw + wid;
    if (b >= le) return;
    int p = parent[b];
    int d = (ix[b] & 1) + 2 * (iy[b] & 1);
    const cz<R> *dp = dtab + (size_t)d * (LBF_MAX_TERMS + 1);
    const cz<R> *inv = dtab + (size_t)(4 + d) * (LBF_MAX_TERMS + 1);
    for (int k = lane; k < P; k += 32) A[k] = zmul(loc[(int64_t)p * P + k], dp[k]);
    __syncwarp();
    const int l0 = lane, l1 = lane + 32;
    const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
    cz<R> s0{0, 0}, s1{0, 0};
    // the second coefficient's sum only when P > 32: a test inside the loop leaves
    // predicated-off multiply-adds that still occupy the double pipe
    if (P > 32) {
        for (int k = 0; k < P; k++) {
            const cz<R> a = A[k];
            const R c0 = Cd[k * P + lc0], c1 = Cd[k * P + lc1];
            s0.x = fmr(c0, a.x, s0.x);
            s0.y = fmr(c0, a.y, s0.y);
            s1.x = fmr(c1, a.x, s1.x);
            s1.y = fmr(c1, a.y, s1.y);
        }
    } else {
        for (int k = 0; k < P; k++) {
            const cz<R> a = A[k];
            const R c0 = Cd[k * P + lc0];
            s0.x = fmr(c0, a.x, s0.x);
            s0.y = fmr(c0, a.y, s0.y);
        }
    }
    if (l0 < P) {
        cz<R> o = loc[b * P + l0], t = zmul(inv[l0], s0);
        loc[b * P + l0] = cz<R>{o.x + t.x, o.y + t.y};
    }
    if (l1 < P) {
        cz<R> o = loc[b * P + l1], t = zmul(inv[l1], s1);
        loc[b * P + l1] = cz<R>{o.x + t.x, o.y + t.y};
    }
}

// The float operator's L2L chain in one launch: warps take the boxes in index order
// (level by level) from a counter and add the parent's full expansion shifted down once
// the parent is marked done (a per-box epoch word; the parent was taken earlier by a
// running warp, so every wait ends; each wait is bounded and reports a time-out).  The
// last warp to finish resets the counters and advances the epoch.  pull: [1] finished
// warps, [2] epoch, [3] box counter, then nbox words unused here and nbox done epochs.
constexpr unsigned kChainSpins = 1u << 24;

template <typename R>
__global__ void k_mp_chain(int64_t nbox, int P, const int32_t *__restrict__ parent,
                           const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                           const int32_t *__restrict__ iy, const R *__restrict__ binom,
                           const cz<R> *__restrict__ dtab, cz<R> *loc, unsigned *pull, int *status,
                           const int *gate, int64_t slab)
{
    lbf_rhs(slab, loc, pull, gate);
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smr[];
    const int nw = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = (P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cd = (R *)smr;  // Cd[k*P + l] = C(k, l) (0 for k < l)
    cz<R> *A = (cz<R> *)(smr + tl) + (size_t)wid * 2 * P;  // two boxes a warp (below)
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int k = e / P, l = e % P;
        Cd[e] = k >= l ? binom[k * LBF_MAX_TERMS + l] : R(0);
    }
    __syncthreads();
    unsigned *done = pull + 4 + nbox;
    unsigned epoch = 0;
    if (lane == 0) epoch = *(volatile unsigned *)&pull[2];
    epoch = __shfl_sync(0xffffffffu, epoch, 0);
    if (P <= 32) {
        // Two boxes a warp, one per half-warp.  The shift matrix C(k, l) (k >= l) is
        // triangular: lane j of a half sums the rows l = j and l = P - 1 - j, P + 1 terms in
        // one loop (it moves to the second row inside the loop), so a half-warp does a box's
        // shift in P + 1 steps where a warp with a row per lane would take P steps for one box
        // with half of its terms zero.  Each half waits for its own box's parent; when that
        // parent is the other half's box, the other half marks it done first.
        const int hf = lane >> 4, j = lane & 15;
        const unsigned hmask = hf ? 0xffff0000u : 0x0000ffffu;
        const int nr = (P + 1) / 2;  // lanes of a half with rows
        const int r1 = j < nr ? j : 0, r2 = P - 1 - r1, n1 = P - r1;
        cz<R> *Ah = A + hf * P;
        for (;;) {
            unsigned bi = 0;
            if (lane == 0) bi = atomicAdd(&pull[3], 2u);
            const int64_t b0 = (int64_t)__shfl_sync(0xffffffffu, bi, 0);
            if (b0 >= nbox) break;
            const int64_t b = b0 + hf;
            if (b < nbox) {
                if (level[b] >= 3) {
                    const int p = parent[b];
                    if (j == 0) {
                        unsigned spins = 0;
                        const unsigned lim = wait_limit(status, kChainSpins);
                        while (*(volatile unsigned *)&done[p] != epoch + 1u)
                            if (++spins > lim) {
                                atomicOr(status, LBF_DEV_TIMEOUT);
                                break;
                            }
                    }
                    __syncwarp(hmask);
                    __threadfence();
                    const int d = (ix[b] & 1) + 2 * (iy[b] & 1);
                    const cz<R> *dp = dtab + (size_t)d * (LBF_MAX_TERMS + 1);
                    const cz<R> *inv = dtab + (size_t)(4 + d) * (LBF_MAX_TERMS + 1);
                    for (int k = j; k < P; k += 16) {
                        const cz<R> pk = ldcg_cz(&loc[(int64_t)p * P + k]);
                        Ah[k] = zmul(pk, dp[k]);
                    }
                    __syncwarp(hmask);
                    cz<R> acc{0, 0}, s1{0, 0};
                    for (int it = 0; it <= P; it++) {
                        const bool first = it < n1;
                        if (it == n1) {
                            s1 = acc;
                            acc = cz<R>{0, 0};
                        }
                        const int k = first ? r1 + it : r2 + (it - n1), l = first ? r1 : r2;
                        const cz<R> a = Ah[k];
                        const R c = Cd[k * P + l];
                        acc.x = fmr(c, a.x, acc.x);
                        acc.y = fmr(c, a.y, acc.y);
                    }
                    if (j < nr) {
                        const cz<R> o = loc[b * P + r1], t = zmul(inv[r1], s1);
                        loc[b * P + r1] = cz<R>{o.x + t.x, o.y + t.y};
                        if (r2 != r1) {
                            const cz<R> o2 = loc[b * P + r2], t2 = zmul(inv[r2], acc);
                            loc[b * P + r2] = cz<R>{o2.x + t2.x, o2.y + t2.y};
                        }
                    }
                    __threadfence();
                    __syncwarp(hmask);
                }
                if (j == 0) atomicExch(&done[b], epoch + 1u);
            }
        }
    } else {
        const int l0 = lane, l1 = lane + 32;
        const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
        for (;;) {
            unsigned bi = 0;
            if (lane == 0) bi = atomicAdd(&pull[3], 1u);
            const int64_t b = (int64_t)__shfl_sync(0xffffffffu, bi, 0);
            if (b >= nbox) break;
            if (level[b] >= 3) {
                const int p = parent[b];
                if (lane == 0) {
                    unsigned spins = 0;
                    const unsigned lim = wait_limit(status, kChainSpins);
                    while (*(volatile unsigned *)&done[p] != epoch + 1u)
                        if (++spins > lim) {
                            atomicOr(status, LBF_DEV_TIMEOUT);
                            break;
                        }
                }
                __syncwarp();
                __threadfence();
                const int d = (ix[b] & 1) + 2 * (iy[b] & 1);
                const cz<R> *dp = dtab + (size_t)d * (LBF_MAX_TERMS + 1);
                const cz<R> *inv = dtab + (size_t)(4 + d) * (LBF_MAX_TERMS + 1);
                for (int k = lane; k < P; k += 32) {
                    const cz<R> pk = ldcg_cz(&loc[(int64_t)p * P + k]);
                    A[k] = zmul(pk, dp[k]);
                }
                __syncwarp();
                cz<R> s0{0, 0}, s1{0, 0};
                // the second coefficient's sum only when P > 32: a test inside the loop leaves
                // predicated-off multiply-adds that still occupy the double pipe
                if (P > 32) {
                    for (int k = 0; k < P; k++) {
                        const cz<R> a = A[k];
                        const R c0 = Cd[k * P + lc0], c1 = Cd[k * P + lc1];
                        s0.x = fmr(c0, a.x, s0.x);
                        s0.y = fmr(c0, a.y, s0.y);
                        s1.x = fmr(c1, a.x, s1.x);
                        s1.y = fmr(c1, a.y, s1.y);
                    }
                } else {
                    for (int k = 0; k < P; k++) {
                        const cz<R> a = A[k];
                        const R c0 = Cd[k * P + lc0];
                        s0.x = fmr(c0, a.x, s0.x);
                        s0.y = fmr(c0, a.y, s0.y);
                    }
                }
                if (l0 < P) {
                    const cz<R> o = loc[b * P + l0], t = zmul(inv[l0], s0);
                    loc[b * P + l0] = cz<R>{o.x + t.x, o.y + t.y};
                }
                if (l1 < P) {
                    const cz<R> o = loc[b * P + l1], t = zmul(inv[l1], s1);
                    loc[b * P + l1] = cz<R>{o.x + t.x, o.y + t.y};
                }
                __threadfence();
                __syncwarp();
            }
            if (lane == 0) atomicExch(&done[b], epoch + 1u);
        }
    }
    if (lane == 0) {
        const unsigned total = gridDim.x * (unsigned)nw;
        if (atomicAdd(&pull[1], 1u) == total - 1u) {
            pull[1] = 0u;
            pull[3] = 0u;
            __threadfence();
            atomicExch(&pull[2], epoch + 1u);
        }
    }
}

// The centres a leaf sums directly, 32 per warp: for every node i of the leaf,
// partial[nodebase[i] + k] = sum over chunk k of y_m log|xi_i - xi_m| (in double; the
// float operator takes the log in float).  Spreading a long list over many warps keeps
// one leaf from holding the whole launch.
template <typename R>
__global__ void k_mp_near(int64_t nchunks, const int32_t *__restrict__ cleaf,
                          const int32_t *__restrict__ ck, const int32_t *__restrict__ nptr,
                          const int32_t *__restrict__ nsrc, const int32_t *__restrict__ bg,
                          const int32_t *__restrict__ en, const double2 *__restrict__ xi,
                          const double2 *__restrict__ xc, const double *__restrict__ y,
                          const int32_t *__restrict__ nodebase, double *__restrict__ partial,
                          const int *gate, int64_t slab)
{
    lbf_rhs(slab, y, partial, gate);
    if (gate && *gate == 0) return;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nchunks) return;
    const int b = cleaf[w], k = ck[w];
    const int q0 = nptr[b] + 32 * k, q1 = min(nptr[b + 1], q0 + 32);
    for (int i = bg[b] + lane; i < en[b]; i += 32) {
        const double2 zi = xi[i];
        double acc = 0.0;
        for (int q = q0; q < q1; q++) {
            const int m = nsrc[q];
            const double ex = zi.x - xc[m].x, ey = zi.y - xc[m].y;
            if constexpr (std::is_same<R, float>::value)
                acc += y[m] * (double)(0.5f * __logf((float)(ex * ex + ey * ey)));
            else
                acc += y[m] * 0.5 * log(ex * ex + ey * ey);
        }
        partial[nodebase[i] + k] = acc;
    }
}

// out_i = x_i + v_i + s (E y)_i at every node (Morton order), v nullable: L2P of the
// node's leaf, its direct centres, and the centres summed directly everywhere.
template <typename R>
__global__ void k_mp_eval(int64_t N, int P, const double2 *__restrict__ xi,
                          const int32_t *__restrict__ leaf_of, const int32_t *__restrict__ level,
                          const int32_t *__restrict__ ix, const int32_t *__restrict__ iy, Geo g,
                          const cz<R> *__restrict__ loc, const int32_t *__restrict__ nptr,
                          const int32_t *__restrict__ nsrc, const int32_t *__restrict__ glob,
                          int nglob, const double2 *__restrict__ xc, const double *__restrict__ y,
                          const double *__restrict__ ell, const double *__restrict__ sums,
                          const double *__restrict__ x, const double *__restrict__ v, double s,
                          double *__restrict__ out, const int *gate,
                          const int32_t *__restrict__ parent, const float2 *__restrict__ u32,
                          int walk, const cz<R> *__restrict__ uloc,
                          const int32_t *__restrict__ nodebase, const double *__restrict__ partial,
                          int64_t slab)
{
    lbf_rhs(slab, loc, y, sums, x, v, out, gate, partial);
    if (gate && *gate == 0) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int b = leaf_of[i];
    double2 zi = xi[i];
    double lsum = 0.0;
    if (!walk) {
        cz<R> u;
        if (uloc) {  // the leaf-local coordinate of the double-float operator
            u = uloc[i];
        } else {
            double cx, cy, r;
            centre_of(g, level[b], ix[b], iy[b], cx, cy, r);
            const double ir = 1.0 / r;
            u = cz<R>{(R)((zi.x - cx) * ir), (R)((zi.y - cy) * ir)};
        }
        const cz<R> *lb = loc + (int64_t)b * P;
        cz<R> acc = lb[P - 1];
        for (int l = P - 2; l >= 0; l--) acc = zfma(acc, u, lb[l]);
        lsum = (double)acc.x;
    } else {
        // float: every ancestor's own expansion at the node (no L2L chain), from the
        // node's leaf-local coordinate u: (z - c_a)/r_a = 2((ix_b - 2^s ix_a + 1/2) 2^-s - 1/2) + u 2^-s
        const float2 uu = u32[i];
        const int lv = level[b], bx = ix[b], by = iy[b];
        const int32_t *ab = parent + (int64_t)b * LBF_ANC_STRIDE;  // the ancestor table
        auto at = [&](int sh) {
            const R sc = (R)__int_as_float((127 - sh) << 23);  // 2^-sh
            const int dxi = bx & ((1 << sh) - 1), dyi = by & ((1 << sh) - 1);
            return cz<R>{(R)2 * (((R)dxi + (R)0.5) * sc - (R)0.5) + (R)uu.x * sc,
                         (R)2 * (((R)dyi + (R)0.5) * sc - (R)0.5) + (R)uu.y * sc};
        };
        // two ancestors at a time: two independent Horner chains
        R acc = 0;
        const int na = lv - 1;
        int sh = 0;
        for (; sh + 1 < na; sh += 2) {
            const cz<R> *la = loc + (int64_t)ab[sh] * P, *lb = loc + (int64_t)ab[sh + 1] * P;
            const cz<R> ua = at(sh), ub = at(sh + 1);
            cz<R> ta = la[P - 1], tb = lb[P - 1];
            for (int l = P - 2; l >= 0; l--) {
                ta = zfma(ta, ua, la[l]);
                tb = zfma(tb, ub, lb[l]);
            }
            acc += ta.x + tb.x;
        }
        if (sh < na) {
            const cz<R> *la = loc + (int64_t)ab[sh] * P;
            const cz<R> ua = at(sh);
            cz<R> t = la[P - 1];
            for (int l = P - 2; l >= 0; l--) t = zfma(t, ua, la[l]);
            acc += t.x;
        }
        lsum = (double)acc;
    }
    for (int q = nodebase[i]; q < nodebase[i + 1]; q++) lsum += partial[q];  // direct centres
    for (int q = 0; q < nglob; q++) {
        int m = glob[q];
        double ex = zi.x - xc[m].x, ey = zi.y - xc[m].y;
        lsum += y[m] * 0.5 * log(ex * ex + ey * ey);
    }
    double phi = ((ell[i] - LBF_LN2) * sums[0] + sums[1] - 2.0 * lsum) * (1.0 / (2.0 * LBF_PI));
    out[i] = x[i] + (v ? v[i] : 0.0) + s * phi;
}

__global__ void k_mp_glob(int M, const int32_t *__restrict__ kind, int32_t *__restrict__ glob,
                          int32_t *__restrict__ nglob)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int n = 0;
    for (int m = 0; m < M; m++)
        if (kind[m] == 2) glob[n++] = m;
    *nglob = n;
}

__global__ void k_zero_i32(int32_t *p, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

template <typename R> size_t l2l_smem(int P, int wpb)
{
    return (P * P * sizeof(R) + 15) / 16 * 16 + sizeof(cz<R>) * (size_t)wpb * 2 * P;
}

}  // namespace

int lbf_border_init_attrs()
{
    const int cap = 200 * 1024;
    LBF_CUDA(cudaFuncSetAttribute(k_mp_p2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    LBF_CUDA(cudaFuncSetAttribute(k_mp_p2l<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    LBF_CUDA(cudaFuncSetAttribute(k_mp_l2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    LBF_CUDA(cudaFuncSetAttribute(k_mp_l2l<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    LBF_CUDA(cudaFuncSetAttribute(k_mp_p2l<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    LBF_CUDA(cudaFuncSetAttribute(k_mp_l2l<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    return LBF_OK;
}

static int read_i32(const int32_t *d, int32_t *h, cudaStream_t s)
{
    LBF_CUDA(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

// (box, centre) pairs of one kind -> per-box lists in ascending centre order
// per pair of a centre-major list: sort key = the box, value = the centre
__global__ void k_pair_keys(int M, const int32_t *__restrict__ off, const int32_t *__restrict__ cnt,
                            const int32_t *__restrict__ box, uint64_t *__restrict__ key,
                            int32_t *__restrict__ centre)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int q = off[m]; q < off[m] + cnt[m]; q++) {
        key[q] = (uint64_t)box[q];
        centre[q] = m;
    }
}

// (box, centre) pairs generated centre by centre -> per-box lists in ascending
// centre order (CSR ptr/src): a stable radix sort by box of the centre-major
// pairs keeps every box's centres in generation (= centre) order.
static int pairs_to_boxes(lbf_plan *pl, cudaStream_t s, const int32_t *off, const int32_t *cnt,
                          const int32_t *box, int64_t npairs, int32_t *ptr, int32_t *src,
                          const SortBufs &sb, int32_t *work, int64_t work_len)
{
    int64_t nb = pl->tree.nbox;
    int M = pl->M;
    LBF_LAUNCH(k_zero_i32, lbf_cdiv(nb, 256), 256, 0, s, work, nb);
    LBF_LAUNCH(k_pairs_count, lbf_cdiv(M, 128), 128, 0, s, M, off, cnt, box, work);
    LBF_CHECK_LAUNCH();
    int rc = lbf_scan_i32(work, ptr, nb, work + nb, work_len - nb, s);
    if (rc) return rc;
    int32_t tot = (int32_t)npairs;
    LBF_CUDA(cudaMemcpyAsync(ptr + nb, &tot, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaStreamSynchronize(s));  // tot is a host local
    if (npairs == 0) return LBF_OK;
    LBF_LAUNCH(k_pair_keys, lbf_cdiv(M, 128), 128, 0, s, M, off, cnt, box, sb.key, src);
    LBF_CHECK_LAUNCH();
    int bits = 1;
    while (((int64_t)1 << bits) < nb) bits++;
    return lbf_radix_sort(sb.key, sb.key_alt, src, sb.val_alt, npairs, bits, work, work_len, s);
}

// Plan time, without the tree: the centres' planar images, the island moments and
// S = D - F E into G (M x M).  work holds a counter and the entries summed directly.
int lbf_schur_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, double *G, int32_t *work,
                    int64_t work_len)
{
    const int M = pl->M;
    Border &B = pl->bd;
    LBF_LAUNCH(k_mp_centres_plane, lbf_cdiv(M, 128), 128, 0, s, M, pl->centres, B.xc, B.lam, B.live);
    LBF_LAUNCH(k_mp_islands, M, 256, 0, s, M, B.P, pl->island_ptr, xi_o, B.zc, B.Rk, B.rk, B.slog,
               B.sell, B.mu, B.nu);
    int32_t *dcount = work, *dlist = work + 1;
    const int dcap = (int)std::min<int64_t>(work_len - 1, INT32_MAX);
    LBF_CUDA(cudaMemsetAsync(dcount, 0, sizeof(int32_t), s));
    LBF_LAUNCH(k_mp_schur, lbf_cdiv((int64_t)M * M, 128), 128, 0, s, M, B.P, pl->island_ptr, xi_o,
               B.xc, B.live, B.lam, B.zc, B.Rk, B.rk, B.slog, B.sell, B.mu, B.nu, G, dcount, dlist,
               dcap);
    LBF_LAUNCH(k_mp_schur_direct, 152 * 4, 256, 0, s, M, pl->island_ptr, xi_o, B.xc, B.live, B.lam,
               B.sell, dcount, dlist, dcap, G);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// Plan time, with the tree: node data, the centres' cells and walks down the tree (P2L
// and direct lists per box).
int lbf_mp_build(lbf_plan *pl, cudaStream_t s, int32_t *work, int64_t work_len, const SortBufs &sb)
{
    int64_t N = pl->N;
    int M = pl->M;
    Border &B = pl->bd;
    Tree &T = pl->tree;
    Geo g{T.xmin, T.ymin, T.L};
    int D = pl->opt.max_depth;
    LBF_LAUNCH(k_mp_nodes, lbf_cdiv(N, 256), 256, 0, s, N, pl->xi, B.ell);
    LBF_LAUNCH(k_mp_leaf_of, lbf_cdiv(T.nleaf, 128), 128, 0, s, T.nleaf, T.leaves, T.begin, T.end,
               B.leaf_of);
    LBF_LAUNCH(k_mp_centres, lbf_cdiv(M, 128), 128, 0, s, M, pl->centres, g, D, B.kind, B.cell);
    LBF_LAUNCH(k_mp_glob, 1, 32, 0, s, M, B.kind, B.glob, B.nglob);
    LBF_CHECK_LAUNCH();
    LBF_CUDA(cudaMemcpyAsync(&B.nglob_h, B.nglob, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    // walks: count, offsets, fill
    TView tv{T.level, T.ix, T.iy, T.child0, T.nchild};
    int32_t *np2l = work, *nnear = work + M, *op2l = work + 2 * M, *onear = work + 3 * M;
    int32_t *w2 = work + 4 * M;
    int64_t w2_len = work_len - 4 * M;
    LBF_LAUNCH(k_mp_walk, lbf_cdiv(M, 128), 128, 0, s, M, B.kind, B.cell, D, tv, 0, np2l, nnear,
               (const int32_t *)nullptr, (const int32_t *)nullptr, (int32_t *)nullptr,
               (int32_t *)nullptr, pl->dev_status);
    LBF_CHECK_LAUNCH();
    int rc = lbf_scan_i32(np2l, op2l, M, w2, w2_len, s);
    if (!rc) rc = lbf_scan_i32(nnear, onear, M, w2, w2_len, s);
    if (rc) return rc;
    int32_t a = 0, b = 0, c = 0, d = 0;
    if ((rc = read_i32(op2l + M - 1, &a, s)) || (rc = read_i32(np2l + M - 1, &b, s)) ||
        (rc = read_i32(onear + M - 1, &c, s)) || (rc = read_i32(nnear + M - 1, &d, s)))
        return rc;
    int64_t n_p2l = (int64_t)a + b, n_near = (int64_t)c + d;
    if (n_p2l > B.pair_cap || n_near > B.pair_cap) return LBF_EWORKSPACE;
    LBF_LAUNCH(k_mp_walk, lbf_cdiv(M, 128), 128, 0, s, M, B.kind, B.cell, D, tv, 1, np2l, nnear,
               op2l, onear, B.pairs_a, B.pairs_b, pl->dev_status);
    LBF_CHECK_LAUNCH();
    if ((rc = pairs_to_boxes(pl, s, op2l, np2l, B.pairs_a, n_p2l, B.p2l_ptr, B.p2l_src, sb, w2,
                             w2_len)))
        return rc;
    if ((rc = pairs_to_boxes(pl, s, onear, nnear, B.pairs_b, n_near, B.near_ptr, B.near_src, sb, w2,
                             w2_len)))
        return rc;
    // the centre-major lists stay: offsets per centre for the transposed potential
    LBF_CUDA(cudaMemcpyAsync(B.cp2l, op2l, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(B.cnear, onear, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, s));
    {
        int32_t tail[2] = {(int32_t)n_p2l, (int32_t)n_near};
        LBF_CUDA(cudaMemcpyAsync(B.cp2l + M, &tail[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
        LBF_CUDA(cudaMemcpyAsync(B.cnear + M, &tail[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
        LBF_CUDA(cudaStreamSynchronize(s));  // tail is a host local
    }
    B.n_p2l = n_p2l;
    B.n_near = n_near;
    {
        // the direct centres in chunks of 32 per leaf, and per node its partial-sum slots
        const int64_t nb = T.nbox;
        int32_t *nch = w2, *cbase = w2 + nb + 1, *sc = w2 + 2 * (nb + 1);
        const int64_t sc_len = w2_len - 2 * (nb + 1);
        LBF_LAUNCH(k_chunk_count, lbf_cdiv(nb, 256), 256, 0, s, nb, B.near_ptr, nch);
        LBF_CHECK_LAUNCH();
        if ((rc = lbf_scan_i32(nch, cbase, nb, sc, sc_len, s))) return rc;
        int32_t lastb = 0, lastn = 0;
        if ((rc = read_i32(cbase + nb - 1, &lastb, s)) || (rc = read_i32(nch + nb - 1, &lastn, s)))
            return rc;
        B.nchunks = (int64_t)lastb + lastn;
        if (B.nchunks > B.pair_cap) return LBF_EWORKSPACE;
        LBF_LAUNCH(k_chunk_fill, lbf_cdiv(nb, 256), 256, 0, s, nb, nch, cbase, B.chunk_leaf, B.chunk_k);
        LBF_LAUNCH(k_node_chunks, lbf_cdiv(N + 1, 256), 256, 0, s, N, B.leaf_of, nch, B.nodebase);
        LBF_CHECK_LAUNCH();
        if ((rc = lbf_scan_i32(B.nodebase, B.nodebase, N + 1, sc, sc_len, s))) return rc;
        int32_t np = 0;
        if ((rc = read_i32(B.nodebase + N, &np, s))) return rc;
        B.npartial = np;
        if (B.npartial > B.partial_cap) return LBF_EWORKSPACE;
    }
    return LBF_OK;
}

// out = x + v + s E y (Morton order; v nullable) in precision prec.
int lbf_mp_apply(lbf_plan *pl, const double *y, const double *x, const double *v, double sc,
                 double *out, const int *gate, cudaStream_t s, int prec)
{
    Border &B = pl->bd;
    Tree &T = pl->tree;
    Geo g{T.xmin, T.ymin, T.L};
    int M = pl->M;
    const int wpb = 4;
    bool f32 = prec == LBF_PREC_FP32 && B.loc32;
    if (f32) {
        int P = B.P32;
        size_t smem = sizeof(cz<float>) * (size_t)wpb * P * 32;
        LBF_LAUNCH(k_mp_p2l<float>, lbf_grid(pl, lbf_cdiv(T.nbox, wpb)), 32 * wpb, smem, s, T.nbox,
                   P, M, B.p2l_ptr, B.p2l_src, T.level, T.ix, T.iy, g, B.xc, B.kind, B.lam, y,
                   (cz<float> *)B.loc32, B.sums, gate, pl->slab);
        // float: the evaluation walks each node's ancestors (cheaper here than the L2L
        // chain, which is serial along each path while the walk is parallel over nodes)
        const bool chain = false;
        if (chain) {
            const int cw = 8;
            const int64_t grid = std::min<int64_t>(lbf_cdiv(T.nbox, cw), 4 * (int64_t)std::max(pl->nsm, 1));
            LBF_LAUNCH_P(LBF_KERNEL_ESUM32, k_mp_chain<float>, lbf_grid(pl, grid), 32 * cw,
                         l2l_smem<float>(P, cw), s, T.nbox, P, T.parent, T.level, T.ix, T.iy,
                         pl->tab32_binom, (const cz<float> *)pl->tab32_dshift, (cz<float> *)B.loc32,
                         pl->pull, pl->dev_status, gate, pl->slab);
        }
        if (B.nchunks)
            LBF_LAUNCH(k_mp_near<float>, lbf_grid(pl, lbf_cdiv(B.nchunks, 8)), 256, 0, s, B.nchunks,
                       B.chunk_leaf, B.chunk_k, B.near_ptr, B.near_src, T.begin, T.end, pl->xi,
                       B.xc, y, B.nodebase, B.partial, gate, pl->slab);
        LBF_LAUNCH_P(LBF_KERNEL_ESUM32, k_mp_eval<float>, lbf_grid(pl, lbf_cdiv(pl->N, 256)), 256,
                     0, s, pl->N, P, pl->xi, B.leaf_of, T.level, T.ix, T.iy, g,
                     (const cz<float> *)B.loc32, B.near_ptr, B.near_src, B.glob, B.nglob_h, B.xc, y,
                     B.ell, B.sums, x, v, sc, out, gate, pl->anc, pl->u32, chain ? 0 : 1,
                     chain ? (const cz<float> *)pl->u32 : (const cz<float> *)nullptr, B.nodebase,
                     B.partial, pl->slab);
    } else if (pl->udf) {
        // the accurate operator in double-float (P2L terms formed in double)
        int P = B.Pe;
        size_t smem = sizeof(cz<df64>) * (size_t)wpb * P * 32;
        LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_p2l<df64>, lbf_grid(pl, lbf_cdiv(T.nbox, wpb)), 32 * wpb,
                     smem, s, T.nbox, P, M, B.p2l_ptr, B.p2l_src, T.level, T.ix, T.iy, g, B.xc,
                     B.kind, B.lam, y, (cz<df64> *)B.loc, B.sums, gate, pl->slab);
        if (pl->pull) {  // the L2L chain in one launch
            const int cw = 8;
            const int64_t grid = std::min<int64_t>(lbf_cdiv(T.nbox, cw), 4 * (int64_t)std::max(pl->nsm, 1));
            LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_chain<df64>, lbf_grid(pl, grid), 32 * cw,
                         l2l_smem<df64>(P, cw), s, T.nbox, P, T.parent, T.level, T.ix, T.iy,
                         (const df64 *)pl->tabdf_binom, (const cz<df64> *)pl->tabdf_dshift,
                         (cz<df64> *)B.loc, pl->pull, pl->dev_status, gate, pl->slab);
        } else {
            for (int l = 3; l < T.nlev; l++) {
                int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
                if (le <= ls) continue;
                LBF_LAUNCH(k_mp_l2l<df64>, lbf_grid(pl, lbf_cdiv(le - ls, 8)), 256,
                           l2l_smem<df64>(P, 8), s, ls, le, P, T.parent, T.ix, T.iy,
                           (const df64 *)pl->tabdf_binom, (const cz<df64> *)pl->tabdf_dshift,
                           (cz<df64> *)B.loc, gate, pl->slab);
            }
        }
        if (B.nchunks)
            LBF_LAUNCH(k_mp_near<double>, lbf_grid(pl, lbf_cdiv(B.nchunks, 8)), 256, 0, s, B.nchunks,
                       B.chunk_leaf, B.chunk_k, B.near_ptr, B.near_src, T.begin, T.end, pl->xi,
                       B.xc, y, B.nodebase, B.partial, gate, pl->slab);
        LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_eval<df64>, lbf_grid(pl, lbf_cdiv(pl->N, 256)), 256, 0,
                     s, pl->N, P, pl->xi, B.leaf_of, T.level, T.ix, T.iy, g,
                     (const cz<df64> *)B.loc, B.near_ptr, B.near_src, B.glob, B.nglob_h, B.xc, y,
                     B.ell, B.sums, x, v, sc, out, gate, T.parent, (const float2 *)nullptr, 0,
                     (const cz<df64> *)pl->udf, B.nodebase, B.partial, pl->slab);
    } else {
        int P = B.Pe;
        size_t smem = sizeof(cz<double>) * (size_t)wpb * P * 32;
        LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_p2l<double>, lbf_grid(pl, lbf_cdiv(T.nbox, wpb)),
                     32 * wpb, smem, s, T.nbox, P, M, B.p2l_ptr, B.p2l_src, T.level, T.ix, T.iy, g,
                     B.xc, B.kind, B.lam, y, (cz<double> *)B.loc, B.sums, gate, pl->slab);
        if (pl->pull) {  // the L2L chain in one launch
            const int cw = 8;
            const int64_t grid = std::min<int64_t>(lbf_cdiv(T.nbox, cw), 4 * (int64_t)std::max(pl->nsm, 1));
            LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_chain<double>, lbf_grid(pl, grid), 32 * cw,
                         l2l_smem<double>(P, cw), s, T.nbox, P, T.parent, T.level, T.ix, T.iy,
                         pl->tab_binom, (const cz<double> *)pl->tab_dshift, (cz<double> *)B.loc,
                         pl->pull, pl->dev_status, gate, pl->slab);
        } else {
            for (int l = 3; l < T.nlev; l++) {
                int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
                if (le <= ls) continue;
                LBF_LAUNCH(k_mp_l2l<double>, lbf_grid(pl, lbf_cdiv(le - ls, 8)), 256,
                           l2l_smem<double>(P, 8), s, ls, le, P, T.parent, T.ix, T.iy,
                           pl->tab_binom, (const cz<double> *)pl->tab_dshift, (cz<double> *)B.loc,
                           gate, pl->slab);
            }
        }
        if (B.nchunks)
            LBF_LAUNCH(k_mp_near<double>, lbf_grid(pl, lbf_cdiv(B.nchunks, 8)), 256, 0, s, B.nchunks,
                       B.chunk_leaf, B.chunk_k, B.near_ptr, B.near_src, T.begin, T.end, pl->xi,
                       B.xc, y, B.nodebase, B.partial, gate, pl->slab);
        LBF_LAUNCH_P(LBF_KERNEL_ESUM, k_mp_eval<double>, lbf_grid(pl, lbf_cdiv(pl->N, 256)), 256, 0,
                     s, pl->N, P, pl->xi, B.leaf_of, T.level, T.ix, T.iy, g,
                     (const cz<double> *)B.loc, B.near_ptr, B.near_src, B.glob, B.nglob_h, B.xc, y,
                     B.ell, B.sums, x, v, sc, out, gate, T.parent, (const float2 *)nullptr, 0,
                     (const cz<double> *)nullptr, B.nodebase, B.partial, pl->slab);
    }
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

namespace {
__global__ void k_mp_counts(int64_t nleaf, const int32_t *__restrict__ leaves,
                            const int32_t *__restrict__ level, const int32_t *__restrict__ bg,
                            const int32_t *__restrict__ en, const int32_t *__restrict__ nptr,
                            unsigned long long *__restrict__ c)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int b = leaves[t];
    unsigned long long nb = (unsigned long long)(en[b] - bg[b]);
    atomicAdd(&c[0], nb * (unsigned long long)(nptr[b + 1] - nptr[b]));
    if (level[b] >= 2) atomicAdd(&c[1], nb * (unsigned long long)(level[b] - 1));
}
}  // namespace

extern "C" int lbf_border_counts(const lbf_plan *pl, int64_t counts[6], lbf_stream_t stream)
{
    if (!pl || !counts) return LBF_EINVAL;
    for (int k = 0; k < 6; k++) counts[k] = 0;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    cudaStream_t s = (cudaStream_t)stream;
    const Tree &T = pl->tree;
    const Border &B = pl->bd;
    unsigned long long *c = (unsigned long long *)pl->red;  // counters in the reduction scratch
    LBF_CUDA(cudaMemsetAsync(c, 0, 2 * sizeof(unsigned long long), s));
    LBF_LAUNCH(k_mp_counts, lbf_cdiv(T.nleaf, 256), 256, 0, s, T.nleaf, T.leaves, T.level, T.begin,
               T.end, B.near_ptr, c);
    LBF_CHECK_LAUNCH();
    unsigned long long h[2];
    LBF_CUDA(cudaMemcpyAsync(h, c, sizeof(h), cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    counts[0] = B.n_p2l;
    counts[1] = (int64_t)h[0];
    counts[2] = B.nglob_h;
    counts[3] = (int64_t)h[1];
    counts[4] = B.Pe;
    counts[5] = B.P32;
    return LBF_OK;
}

// ---- transposed and differentiated multiplier potential (adjoint) -----------------------
namespace {

// sums[2] = sum_i tau_i (l_i - log 2), one block, fixed order
__global__ void k_mp_tsum(int64_t N, const double *__restrict__ tau, const double *__restrict__ ell,
                          double *__restrict__ sums, const int *gate)
{
    if (gate && *gate == 0) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) a = fma(tau[i], ell[i] - LBF_LN2, a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) sums[2] = a;
}

// out_m = add_m + sc (E^T tau)_m, warp per centre (Sec. 4.1, Eq. u_multi, transposed):
//   (E^T tau)_m = (1/2pi) [ sum_i tau_i (l_i - log 2) + lam_m T - 2 sum_i tau_i log|xi_i - xi_m| ]
// (no lam and log terms for the centre at the pole), T = sum_i tau_i.  The log sum
// takes the same (box, centre) pairs as E y, transposed: the multipoles of the
// boxes the centre's walk entered by P2L (M2P at the centre), the leaves it sums
// directly, and every node for a centre outside the tree's square.
__global__ void k_mp_transpose(int M, int P, Geo g, const int32_t *__restrict__ level,
                               const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                               const int32_t *__restrict__ bg, const int32_t *__restrict__ en,
                               const int32_t *__restrict__ cp2l, const int32_t *__restrict__ pa,
                               const int32_t *__restrict__ cnear, const int32_t *__restrict__ pb,
                               const int32_t *__restrict__ kind, const double2 *__restrict__ xc,
                               const double *__restrict__ lam, int64_t N,
                               const double2 *__restrict__ xi, const double *__restrict__ tau,
                               const cz<double> *__restrict__ mp, const double *__restrict__ bsig,
                               const double *__restrict__ sums, double sc,
                               const double *__restrict__ add, double *__restrict__ out,
                               const int *gate)
{
    if (gate && *gate == 0) return;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (m >= M) return;
    double L = 0.0;
    if (kind[m] != 0) {
        const double2 xm = xc[m];
        for (int q = cp2l[m] + lane; q < cp2l[m + 1]; q += 32) {
            const int b = pa[q];
            double cx, cy, r;
            centre_of(g, level[b], ix[b], iy[b], cx, cy, r);
            const double dx = xm.x - cx, dy = xm.y - cy;
            const cz<double> rho = zinv(cz<double>{dx / r, dy / r});  // r / (xi_m - c)
            const cz<double> *a = mp + (int64_t)b * P;
            // A_0 log|xi_m - c| - Re sum_{l>=1} A_l rho^l / l
            cz<double> pw = rho;
            double s = 0.0;
            for (int l = 1; l < P; l++) {
                s += (a[l].x * pw.x - a[l].y * pw.y) / l;
                pw = zmul(pw, rho);
            }
            L += a[0].x * 0.5 * log(dx * dx + dy * dy) - s;
        }
        for (int q = cnear[m]; q < cnear[m + 1]; q++) {
            const int b = pb[q];
            for (int i = bg[b] + lane; i < en[b]; i += 32) {
                const double ex = xi[i].x - xm.x, ey = xi[i].y - xm.y;
                L += tau[i] * 0.5 * log(ex * ex + ey * ey);
            }
        }
        if (kind[m] == 2)
            for (int64_t i = lane; i < N; i += 32) {
                const double ex = xi[i].x - xm.x, ey = xi[i].y - xm.y;
                L += tau[i] * 0.5 * log(ex * ex + ey * ey);
            }
    }
    L = wsum(L);
    if (lane == 0) {
        const double e = kind[m] != 0 ? sums[2] + lam[m] * *bsig - 2.0 * L : sums[2];
        out[m] = (add ? add[m] : 0.0) + sc * e * (1.0 / (2.0 * LBF_PI));
    }
}

// grad_i (E y)_i as a 2-vector (d/dRe xi_i, d/dIm xi_i):
//   (1/2pi) [ Y 2 xi_i/(1 + |xi_i|^2) - 2 (Re Psi', -Im Psi') ],  Psi'(z) = sum_{m finite} y_m/(z - xi_m),
// Psi' from the derivative of the leaf's local expansion plus the direct centres.
__global__ void k_mp_grad(int64_t N, int P, const double2 *__restrict__ xi,
                          const int32_t *__restrict__ leaf_of, const int32_t *__restrict__ level,
                          const int32_t *__restrict__ ix, const int32_t *__restrict__ iy, Geo g,
                          const cz<double> *__restrict__ loc, const int32_t *__restrict__ nptr,
                          const int32_t *__restrict__ nsrc, const int32_t *__restrict__ glob,
                          int nglob, const double2 *__restrict__ xc, const double *__restrict__ y,
                          const double *__restrict__ sums, double2 *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = leaf_of[i];
    const double2 zi = xi[i];
    double cx, cy, r;
    centre_of(g, level[b], ix[b], iy[b], cx, cy, r);
    const cz<double> u{(zi.x - cx) / r, (zi.y - cy) / r};
    const cz<double> *lb = loc + (int64_t)b * P;
    cz<double> d{(P - 1) * lb[P - 1].x, (P - 1) * lb[P - 1].y};
    for (int l = P - 2; l >= 1; l--) d = zfma(d, u, cz<double>{l * lb[l].x, l * lb[l].y});
    double pr = d.x / r, pi = d.y / r;
    auto direct = [&](int m) {
        const double ex = zi.x - xc[m].x, ey = zi.y - xc[m].y;
        const double s = y[m] / (ex * ex + ey * ey);
        pr += s * ex;
        pi -= s * ey;
    };
    for (int q = nptr[b]; q < nptr[b + 1]; q++) direct(nsrc[q]);
    for (int q = 0; q < nglob; q++) direct(glob[q]);
    const double Y = sums[0], den = 1.0 + zi.x * zi.x + zi.y * zi.y;
    const double k = 1.0 / (2.0 * LBF_PI);
    out[i] = make_double2(k * (Y * 2.0 * zi.x / den - 2.0 * pr), k * (Y * 2.0 * zi.y / den + 2.0 * pi));
}

}  // namespace

// out = add + sc E^T tau (M-vectors; tau sorted, N), FP64.  Uses the plan's q, bsig and
// the double expansion buffer of the multiplier potential as scratch.
int lbf_mp_apply_transpose(lbf_plan *pl, const double *tau, double sc, const double *add,
                           double *out, const int *gate, cudaStream_t s)
{
    Border &B = pl->bd;
    Tree &T = pl->tree;
    Geo g{T.xmin, T.ymin, T.L};
    int rc = lbf_multipoles(pl, tau, B.P, B.loc, gate, s);
    if (rc) return rc;
    LBF_LAUNCH(k_mp_tsum, 1, 1024, 0, s, pl->N, tau, B.ell, B.sums, gate);
    LBF_LAUNCH(k_mp_transpose, lbf_cdiv(pl->M, 8), 256, 0, s, pl->M, B.P, g, T.level, T.ix, T.iy,
               T.begin, T.end, B.cp2l, B.pairs_a, B.cnear, B.pairs_b, B.kind, B.xc, B.lam, pl->N,
               pl->xi, tau, (const cz<double> *)B.loc, pl->bsig, B.sums, sc, add, out, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// out_i = grad_i (E y)_i (sorted order, N double2), FP64
int lbf_mp_gradient(lbf_plan *pl, const double *y, double2 *out, cudaStream_t s)
{
    Border &B = pl->bd;
    Tree &T = pl->tree;
    Geo g{T.xmin, T.ymin, T.L};
    int M = pl->M;
    int P = B.P;
    const int wpb = 4;
    size_t smem = sizeof(cz<double>) * (size_t)wpb * P * 32;
    LBF_LAUNCH(k_mp_p2l<double>, lbf_cdiv(T.nbox, wpb), 32 * wpb, smem, s, T.nbox, P, M, B.p2l_ptr,
               B.p2l_src, T.level, T.ix, T.iy, g, B.xc, B.kind, B.lam, y, (cz<double> *)B.loc,
               B.sums, (const int *)nullptr, (int64_t)0);
    for (int l = 3; l < T.nlev; l++) {
        int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
        if (le <= ls) continue;
        LBF_LAUNCH(k_mp_l2l<double>, lbf_cdiv(le - ls, 8), 256, l2l_smem<double>(P, 8), s, ls, le,
                   P, T.parent, T.ix, T.iy, pl->tab_binom, (const cz<double> *)pl->tab_dshift,
                   (cz<double> *)B.loc, (const int *)nullptr, (int64_t)0);
    }
    LBF_LAUNCH(k_mp_grad, lbf_cdiv(pl->N, 256), 256, 0, s, pl->N, P, pl->xi, B.leaf_of, T.level,
               T.ix, T.iy, g, (const cz<double> *)B.loc, B.near_ptr, B.near_src, B.glob,
               B.nglob_h, B.xc, y, B.sums, out);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
