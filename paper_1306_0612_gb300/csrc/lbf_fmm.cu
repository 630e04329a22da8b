// The density block of the operator, K sigma in the paper's doubled scaling
// (Sec. 5, Eq. disc_sphere; Cauchy term signed as derived from Eq. fundC and
// Eq. grad3):
//
//   v_i = 2 [ (1/2pi) c_i + dself_i sigma_i + sum_j beta_j sigma_j ],
//   c_i = Im sum_{j != i} q_j / (xi_j - xi_i),   q_j = sigma_j w_j,
//
// with the Cauchy sum c evaluated by a 2D fast multipole method on the adaptive
// quadtree (Sec. 5: "the two dimensional FMM based on the Coulomb potential"),
// or by a direct O(N^2) sum.  Expansions are of the Cauchy potential
// phi(z) = sum_j q_j/(z - xi_j), so c_i = -Im phi(xi_i) (self excluded).
//
// Scaled expansions about a box centre c with half-width r (level-independent
// translation operators, no overflow in deep trees):
//   multipole  phi(z) = sum_k a_k r^k / (z - c)^(k+1),  a_k = sum_j q_j ((xi_j - c)/r)^k
//   local      phi(z) = sum_l b_l ((z - c)/r)^l
#include <algorithm>

#include "lbf_internal.cuh"

namespace {

struct BoxGeo {
    double xmin, ymin, L;
};

__device__ __forceinline__ void box_centre(const BoxGeo &g, int l, int ix, int iy, double &cx,
                                           double &cy, double &r)
{
    double w = ldexp(g.L, -l);
    r = 0.5 * w;
    cx = g.xmin + (ix + 0.5) * w;
    cy = g.ymin + (iy + 0.5) * w;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)  // a*b + c
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 crcp(double2 a)
{
    double d = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}

// Reciprocal by Newton-Raphson iteration x_{n+1} = x_n (2 - a x_n) (Newton's
// method for 1/a), seeded by the single-precision reciprocal; two steps take
// the 2^-23 seed error below double rounding.  Outside the float range it falls
// back to the division operator.
__device__ __forceinline__ double rcp_nr(double a)
{
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / a;
    double x = (double)__frcp_rn((float)a);
    double e = fma(-a, x, 1.0);
    x = fma(x, e, x);
    e = fma(-a, x, 1.0);
    return fma(x, e, x);
}

__device__ __forceinline__ bool gate_closed(const int *gate) { return gate && *gate == 0; }

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// q = sigma w and beta . sigma (fixed-order two-level reduction; the last block
// to finish sums the block partials in block order).
__global__ void k_prep(int64_t N, const double *__restrict__ sigma, const double2 *__restrict__ w,
                       const double *__restrict__ beta, double2 *__restrict__ q,
                       double *__restrict__ part, unsigned *__restrict__ count,
                       double *__restrict__ out, const int *gate)
{
    if (gate_closed(gate)) return;
    __shared__ double sh[32];
    __shared__ bool last;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = sigma[i];
        double2 ww = w[i];
        q[i] = make_double2(s * ww.x, s * ww.y);
        acc = fma(beta[i], s, acc);
    }
    acc = warp_sum(acc);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
        part[blockIdx.x] = t;
        __threadfence();
        unsigned c = atomicAdd(count, 1u);
        last = (c == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) t += ((volatile double *)part)[b];
        *out = t;
        *count = 0u;
    }
}

// Shift tables of the scaled expansions for the four child positions c = dx + 2 dy,
// d = ((2dx-1) + i (2dy-1))/2 (child centre minus parent centre over the parent
// half-width): dtab[c][k] = d^k and dtab[4 + c][k] = (2d)^-k, k <= LBF_MAX_TERMS.
__device__ __forceinline__ const double2 *dpow(const double2 *dtab, int c)
{
    return dtab + (size_t)c * (LBF_MAX_TERMS + 1);
}
__device__ __forceinline__ const double2 *d2inv(const double2 *dtab, int c)
{
    return dtab + (size_t)(4 + c) * (LBF_MAX_TERMS + 1);
}

// Upward pass in one launch.  Every warp takes a leaf and forms its multipole
// (P2M, a_k = sum_j q_j ((xi_j - c)/r)^k: lanes take nodes, terms go through
// shared memory, lanes then take coefficients and sum in node order).  Then the
// warp that completes the last child of a box (a per-box arrival counter) forms
// that box's multipole from all its children, in child order, and climbs on:
//   M2M  a_l = d^l sum_{k<=l} C(l,k) (2d)^-k a'_k   (= sum_k C(l,k) d^(l-k) 2^-k a'_k).
// No warp waits for another; the summation order does not depend on arrival order.
__global__ void k_up(int64_t nleaf, const int32_t *__restrict__ leaves,
                     const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                     const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                     const int32_t *__restrict__ en, const int32_t *__restrict__ parent,
                     const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                     BoxGeo g, int P, const double *__restrict__ binom,
                     const double2 *__restrict__ dtab, const double2 *__restrict__ xi,
                     const double2 *__restrict__ q, double2 *mp, int *cnt, const int *gate)
{
    if (gate_closed(gate)) return;
    extern __shared__ double sm_up[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl_len = (P * P + 1) & ~1;                  // keep the double2 region 16-byte aligned
    double *Cl = sm_up;                                   // P x P, Cl[k*P + l] = C(l, k) (0 for k > l)
    double2 *T = (double2 *)(sm_up + cl_len) + (size_t)wid * P * 32;
    double2 *A = (double2 *)(sm_up + cl_len) + (size_t)nw * P * 32 + (size_t)wid * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cl[e] = k <= l ? binom[l * LBF_MAX_TERMS + k] : 0.0;
    }
    __syncthreads();
    int64_t t = blockIdx.x * (int64_t)nw + wid;
    if (t >= nleaf) return;
    int b = leaves[t];
    {
        double cx, cy, r;
        box_centre(g, level[b], ix[b], iy[b], cx, cy, r);
        double ir = 1.0 / r;
        double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
        for (int base = bg[b]; base < en[b]; base += 32) {
            int j = base + lane;
            double2 z = make_double2(0, 0), term = make_double2(0, 0);
            if (j < en[b]) {
                double2 x = xi[j];
                z = make_double2((x.x - cx) * ir, (x.y - cy) * ir);
                term = q[j];
            }
            for (int k = 0; k < P; k++) {
                T[k * 32 + lane] = term;
                term = cmul(term, z);
            }
            __syncwarp();
            for (int k = lane; k < P; k += 32) {
                double2 s = make_double2(0, 0);
                for (int m = 0; m < 32; m++) {
                    double2 v = T[k * 32 + m];
                    s.x += v.x;
                    s.y += v.y;
                }
                if (k < 32) { acc0.x += s.x; acc0.y += s.y; }
                else { acc1.x += s.x; acc1.y += s.y; }
            }
            __syncwarp();
        }
        if (lane < P) mp[(int64_t)b * P + lane] = acc0;
        if (lane + 32 < P) mp[(int64_t)b * P + lane + 32] = acc1;
    }
    int cur = b;
    for (;;) {
        int p = parent[cur];
        if (p < 0) break;
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            int old = atomicAdd(&cnt[p], 1);
            last = old == nchild[p] - 1;
            if (last) cnt[p] = 0;  // ready for the next application
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) break;
        __threadfence();
        int l0 = lane, l1 = lane + 32;
        double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
        for (int c = child0[p]; c < child0[p] + nchild[p]; c++) {
            int d = (ix[c] & 1) + 2 * (iy[c] & 1);
            const double2 *inv = d2inv(dtab, d);
            for (int k = lane; k < P; k += 32) A[k] = cmul(__ldcg(&mp[(int64_t)c * P + k]), inv[k]);
            __syncwarp();
            double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
            for (int k = 0; k < P; k++) {
                double2 a = A[k];
                double c0 = Cl[k * P + (l0 < P ? l0 : 0)];
                s0.x = fma(c0, a.x, s0.x);
                s0.y = fma(c0, a.y, s0.y);
                if (l1 < P) {
                    double c1 = Cl[k * P + l1];
                    s1.x = fma(c1, a.x, s1.x);
                    s1.y = fma(c1, a.y, s1.y);
                }
            }
            const double2 *dp = dpow(dtab, d);
            acc0 = cfma(dp[l0], s0, acc0);
            if (l1 < P) acc1 = cfma(dp[l1], s1, acc1);
            __syncwarp();
        }
        if (l0 < P) mp[(int64_t)p * P + l0] = acc0;
        if (l1 < P) mp[(int64_t)p * P + l1] = acc1;
        cur = p;
    }
}

__device__ __forceinline__ double2 warp_sum2(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Downward pass for the boxes of one level: the local expansion of box b is
//   L2L from its parent:  b'_l = (2d)^-l sum_{k>=l} C(k,l) d^k b_k
// plus, scaled by 1/r,
//   M2L over V(b):  (-1)^l t^(l+1) sum_k C(k+l, l) t^k a_k,  t = 1/(2 (dx + i dy))
//   P2L over X(b):  (-1)^l sum_j q_j tau_j^(l+1),  tau_j = r / (c - xi_j).
// Warp per box, lane per coefficient; the binomial tables sit in shared memory
// with lanes on consecutive entries.  For P2L the lanes take source nodes and
// run the power recurrence; each coefficient is summed across the warp.
__global__ void k_down(int64_t ls, int64_t le, const int32_t *__restrict__ level,
                       const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                       const int32_t *__restrict__ parent, const int32_t *__restrict__ vlist,
                       const int32_t *__restrict__ nv, const int32_t *__restrict__ xlist,
                       const int32_t *__restrict__ nx, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, BoxGeo g, int P,
                       const double *__restrict__ binom, const double2 *__restrict__ tpow,
                       const double2 *__restrict__ dtab, const double2 *__restrict__ xi,
                       const double2 *__restrict__ q, const double2 *__restrict__ mp,
                       double2 *__restrict__ loc, const int *gate)
{
    if (gate_closed(gate)) return;
    extern __shared__ double sm_dn[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *Cm = sm_dn;             // Cm[k*P + l] = C(k+l, l)
    double *Cd = sm_dn + P * P;     // Cd[k*P + l] = C(k, l) (0 for k < l)
    double2 *A = (double2 *)(sm_dn + 2 * P * P) + (size_t)wid * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cm[e] = binom[(k + l) * LBF_MAX_TERMS + l];
        Cd[e] = k >= l ? binom[k * LBF_MAX_TERMS + l] : 0.0;
    }
    __syncthreads();
    int64_t b = ls + blockIdx.x * (int64_t)nw + wid;
    if (b >= le) return;
    const int l0 = lane, l1 = lane + 32;
    const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
    int bx = ix[b], by = iy[b];
    double2 accL0 = make_double2(0, 0), accL1 = make_double2(0, 0);
    // L2L (the parent's local is complete: it belongs to the previous level's launch)
    if (level[b] >= 3) {
        int p = parent[b];
        int d = (bx & 1) + 2 * (by & 1);
        const double2 *dp = dpow(dtab, d);
        for (int k = lane; k < P; k += 32) A[k] = cmul(loc[(int64_t)p * P + k], dp[k]);
        __syncwarp();
        double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
        for (int k = 0; k < P; k++) {
            double2 a = A[k];
            double c0 = Cd[k * P + lc0];
            s0.x = fma(c0, a.x, s0.x);
            s0.y = fma(c0, a.y, s0.y);
            if (l1 < P) {
                double c1 = Cd[k * P + lc1];
                s1.x = fma(c1, a.x, s1.x);
                s1.y = fma(c1, a.y, s1.y);
            }
        }
        const double2 *inv = d2inv(dtab, d);
        accL0 = cmul(inv[l0], s0);
        if (l1 < P) accL1 = cmul(inv[l1], s1);
        __syncwarp();
    }
    double2 accF0 = make_double2(0, 0), accF1 = make_double2(0, 0);
    for (int vq = 0; vq < nv[b]; vq++) {
        int s = vlist[b * 27 + vq];
        int o = (bx - ix[s] + 3) * 7 + (by - iy[s] + 3);
        const double2 *tp = tpow + (size_t)o * (LBF_MAX_TERMS + 1);
        for (int k = lane; k < P; k += 32) A[k] = cmul(mp[(int64_t)s * P + k], tp[k]);
        __syncwarp();
        double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
        for (int k = 0; k < P; k++) {
            double2 a = A[k];
            double c0 = Cm[k * P + lc0];
            s0.x = fma(c0, a.x, s0.x);
            s0.y = fma(c0, a.y, s0.y);
            if (l1 < P) {
                double c1 = Cm[k * P + lc1];
                s1.x = fma(c1, a.x, s1.x);
                s1.y = fma(c1, a.y, s1.y);
            }
        }
        double2 f0 = tp[l0 + 1];
        if (l0 & 1) { f0.x = -f0.x; f0.y = -f0.y; }
        accF0 = cfma(f0, s0, accF0);
        if (l1 < P) {
            double2 f1 = tp[l1 + 1];
            if (l1 & 1) { f1.x = -f1.x; f1.y = -f1.y; }
            accF1 = cfma(f1, s1, accF1);
        }
        __syncwarp();
    }
    double cx, cy, r;
    box_centre(g, level[b], bx, by, cx, cy, r);
    double ir = 1.0 / r;
    for (int xq = 0; xq < nx[b]; xq++) {
        int s = xlist[b * 16 + xq];
        for (int base = bg[s]; base < en[s]; base += 32) {
            int j = base + lane;
            double2 tau = make_double2(0, 0), term = make_double2(0, 0);
            if (j < en[s]) {
                double2 z = xi[j];
                tau = crcp(make_double2((cx - z.x) * ir, (cy - z.y) * ir));
                term = cmul(q[j], tau);  // q tau^(l+1) at l = 0
            }
            for (int l = 0; l < P; l++) {
                double2 v = warp_sum2(term);
                if (l & 1) { v.x = -v.x; v.y = -v.y; }
                if (lane == (l & 31)) {
                    if (l < 32) { accF0.x += v.x; accF0.y += v.y; }
                    else { accF1.x += v.x; accF1.y += v.y; }
                }
                term = cmul(term, tau);
            }
        }
    }
    if (l0 < P)
        loc[b * P + l0] = make_double2(accL0.x + accF0.x * ir, accL0.y + accF0.y * ir);
    if (l1 < P)
        loc[b * P + l1] = make_double2(accL1.x + accF1.x * ir, accL1.y + accF1.y * ir);
}

constexpr int kLeafWarps = 4;
constexpr int kSrcChunk = 256;

// Per leaf: far field (L2P of the leaf's local expansion plus M2P from W(b)),
// near field (P2P over U(b), self excluded), and the combine into v.
__global__ void k_leaf(int64_t nleaf, const int32_t *__restrict__ leaves,
                       const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                       const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, const int32_t *__restrict__ uptr,
                       const int32_t *__restrict__ uidx, const int32_t *__restrict__ wptr,
                       const int32_t *__restrict__ widx, BoxGeo g, int P,
                       const double2 *__restrict__ xi, const double2 *__restrict__ q,
                       const double2 *__restrict__ mp, const double2 *__restrict__ loc,
                       const double *__restrict__ sigma, const double *__restrict__ dself,
                       const double *__restrict__ bsig, double *__restrict__ v, const int *gate)
{
    if (gate_closed(gate)) return;
    __shared__ double2 sx[kLeafWarps][kSrcChunk];
    __shared__ double2 sq[kLeafWarps][kSrcChunk];
    __shared__ int32_t sj[kLeafWarps][kSrcChunk];
    __shared__ double cn[kLeafWarps][32];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t t = blockIdx.x * (int64_t)kLeafWarps + wid;
    if (t >= nleaf) return;
    int b = leaves[t];
    double cx, cy, r;
    box_centre(g, level[b], ix[b], iy[b], cx, cy, r);
    double ir = 1.0 / r;
    const double2 *lb = loc + (int64_t)b * P;
    double bs = *bsig;
    for (int tb = bg[b]; tb < en[b]; tb += 32) {
        int nt = min(32, en[b] - tb);
        // ---- far field, lane = target
        double cfar = 0.0;
        int i = tb + lane;
        double2 zi = make_double2(0, 0);
        if (lane < nt) {
            zi = xi[i];
            double2 u = make_double2((zi.x - cx) * ir, (zi.y - cy) * ir);
            double2 phi = lb[P - 1];
            for (int l = P - 2; l >= 0; l--) phi = cfma(phi, u, lb[l]);
            for (int wq = wptr[b]; wq < wptr[b + 1]; wq++) {
                int s = widx[wq];
                double sx_, sy_, sr;
                box_centre(g, level[s], ix[s], iy[s], sx_, sy_, sr);
                double2 rho = crcp(make_double2((zi.x - sx_) / sr, (zi.y - sy_) / sr));
                const double2 *a = mp + (int64_t)s * P;
                double2 ps = a[P - 1];
                for (int k = P - 2; k >= 0; k--) ps = cfma(ps, rho, a[k]);
                ps = cmul(ps, rho);
                phi.x += ps.x / sr;
                phi.y += ps.y / sr;
            }
            cfar = -phi.y;
        }
        cn[wid][lane] = 0.0;
        __syncwarp();
        // ---- near field, lane = source, loop over the chunk's targets
        int fill = 0;
        auto process = [&]() {
            __syncwarp();
            for (int tt = 0; tt < nt; tt++) {
                int ti = tb + tt;
                double2 z = xi[ti];
                double acc = 0.0;
                for (int m = lane; m < fill; m += 32) {
                    if (sj[wid][m] == ti) continue;
                    double dr = sx[wid][m].x - z.x, di = sx[wid][m].y - z.y;
                    double2 qq = sq[wid][m];
                    double num = fma(qq.y, dr, -qq.x * di);
                    double den = fma(dr, dr, di * di);
                    acc = fma(num, rcp_nr(den), acc);
                }
                acc = warp_sum(acc);
                if (lane == tt) cn[wid][tt] += acc;
            }
            __syncwarp();
            fill = 0;
        };
        for (int uq = uptr[b]; uq < uptr[b + 1]; uq++) {
            int s = uidx[uq];
            int sb = bg[s], se = en[s];
            while (sb < se) {
                int take = min(se - sb, kSrcChunk - fill);
                for (int m = lane; m < take; m += 32) {
                    sx[wid][fill + m] = xi[sb + m];
                    sq[wid][fill + m] = q[sb + m];
                    sj[wid][fill + m] = sb + m;
                }
                fill += take;
                sb += take;
                if (fill == kSrcChunk) process();
            }
        }
        if (fill > 0) process();
        __syncwarp();
        if (lane < nt) {
            double c = cfar + cn[wid][lane];
            v[i] = 2.0 * (c * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + bs);
        }
        __syncwarp();
    }
}

// Direct O(N^2) Cauchy sum with the same combine (tiled through shared memory).
__global__ void k_direct(int64_t N, const double2 *__restrict__ xi, const double2 *__restrict__ q,
                         const double *__restrict__ sigma, const double *__restrict__ dself,
                         const double *__restrict__ bsig, double *__restrict__ v, const int *gate)
{
    if (gate_closed(gate)) return;
    __shared__ double2 sx[256], sq[256];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double2 z = i < N ? xi[i] : make_double2(0, 0);
    double acc = 0.0;
    for (int64_t base = 0; base < N; base += 256) {
        int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < N) { sx[threadIdx.x] = xi[j]; sq[threadIdx.x] = q[j]; }
        __syncthreads();
        int n = (int)(N - base < 256 ? N - base : 256);
        for (int m = 0; m < n; m++) {
            if (base + m == i) continue;
            double dr = sx[m].x - z.x, di = sx[m].y - z.y;
            double num = fma(sq[m].y, dr, -sq[m].x * di);
            double den = fma(dr, dr, di * di);
            acc = fma(num, rcp_nr(den), acc);
        }
    }
    if (i < N) v[i] = 2.0 * (acc * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + *bsig);
}

// u(t) at off-curve targets: (1/2pi) Im sum_j q_j/(xi_j - xi_t) + beta.sigma
// + sum_m a_m G(t, c_m)  (Eq. u_multi, planar form of the double layer, Eq. dlpC).
__global__ void k_evaluate(int64_t N, int M, const double2 *__restrict__ xi,
                           const double2 *__restrict__ q, const double *__restrict__ bsig,
                           const double *__restrict__ a, const double *__restrict__ c,
                           int64_t T, const double *__restrict__ t, int rot_on, const double *rot,
                           double *__restrict__ u)
{
    // one block per target; threads stride over the nodes, fixed-order block reduction
    __shared__ double red[32];
    int64_t wid = blockIdx.x;
    int lane = threadIdx.x & 31;
    if (wid >= T) return;
    double p[3] = {t[3 * wid], t[3 * wid + 1], t[3 * wid + 2]};
    if (rot_on) {
        double r0 = rot[0] * p[0] + rot[1] * p[1] + rot[2] * p[2];
        double r1 = rot[3] * p[0] + rot[4] * p[1] + rot[5] * p[2];
        double r2 = rot[6] * p[0] + rot[7] * p[1] + rot[8] * p[2];
        p[0] = r0; p[1] = r1; p[2] = r2;
    }
    double w = 1.0 - p[2];
    double acc = 0.0;
    if (w > 0.0) {  // a target at the pole sees no Cauchy term (xi = infinity)
        double zx = p[0] / w, zy = p[1] / w;
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
            double dr = xi[j].x - zx, di = xi[j].y - zy;
            double2 qq = q[j];
            acc = fma(fma(qq.y, dr, -qq.x * di), rcp_nr(fma(dr, dr, di * di)), acc);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        acc = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) acc += red[k];
        acc *= 1.0 / (2.0 * LBF_PI);
        double s = acc + *bsig;
        if (a) {
            for (int m = 0; m < M; m++) {
                double d0 = p[0] - c[3 * m], d1 = p[1] - c[3 * m + 1], d2 = p[2] - c[3 * m + 2];
                s += a[m] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
            }
        }
        u[wid] = s;
    }
}

__global__ void k_green_sum(int64_t T, const double *__restrict__ t, int64_t S,
                            const double *__restrict__ p, const double *__restrict__ gm,
                            double *__restrict__ out)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    double x0 = t[3 * q], x1 = t[3 * q + 1], x2 = t[3 * q + 2];
    double s = 0.0;
    for (int64_t k = 0; k < S; k++) {
        double d0 = x0 - p[3 * k], d1 = x1 - p[3 * k + 1], d2 = x2 - p[3 * k + 2];
        // G = -(1/2pi) log|x - p| + (1/4pi) log 2 = (1/4pi) log(2/|x - p|^2)
        s += gm[k] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
    }
    out[q] = s;
}

}  // namespace

int lbf_fmm_init_attrs()
{
    LBF_CUDA(cudaFuncSetAttribute(k_up, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    LBF_CUDA(cudaFuncSetAttribute(k_down, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return LBF_OK;
}

static int prep(lbf_plan *pl, const double *sigma, const int *gate, cudaStream_t s)
{
    int nb = (int)std::min<int64_t>(lbf_cdiv(pl->N, 256), 1024);
    LBF_LAUNCH(k_prep, nb, 256, 0, s, pl->N, sigma, pl->w, pl->beta, pl->q, pl->red,
               pl->red_count, pl->bsig, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_apply_K(lbf_plan *pl, const double *sigma, double *v, const int *gate, cudaStream_t s)
{
    int rc = prep(pl, sigma, gate, s);
    if (rc) return rc;
    int64_t N = pl->N;
    if (pl->opt.matvec == LBF_MATVEC_DIRECT) {
        LBF_LAUNCH_P(LBF_KERNEL_DIRECT, k_direct, lbf_cdiv(N, 256), 256, 0, s, N, pl->xi, pl->q, sigma, pl->dself,
                   pl->bsig, v, gate);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    Tree &T = pl->tree;
    BoxGeo g{T.xmin, T.ymin, T.L};
    int P = pl->P;
    {   // upward pass: P2M and every M2M level in one launch
        const int wpb = 2;
        size_t smem = sizeof(double) * ((P * P + 1) & ~1) + sizeof(double2) * (size_t)wpb * P * 33;
        LBF_LAUNCH_P(LBF_KERNEL_UP, k_up, lbf_cdiv(T.nleaf, wpb), 32 * wpb, smem, s, T.nleaf,
                     T.leaves, T.level, T.ix, T.iy, T.begin, T.end, T.parent, T.child0, T.nchild,
                     g, P, pl->tab_binom, pl->tab_dshift, pl->xi, pl->q, pl->mpole, pl->upcnt,
                     gate);
        LBF_CHECK_LAUNCH();
    }
    {   // downward pass, level by level: L2L + M2L + P2L into the local expansions
        const int wpb = 8;
        size_t smem = sizeof(double) * 2 * P * P + sizeof(double2) * (size_t)wpb * P;
        for (int l = 0; l < T.nlev; l++) {
            int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
            if (le <= ls) continue;
            LBF_LAUNCH_P(LBF_KERNEL_DOWN, k_down, lbf_cdiv(le - ls, wpb), 32 * wpb, smem, s, ls, le,
                         T.level, T.ix, T.iy, T.parent, T.vlist, T.nv, T.xlist, T.nx, T.begin,
                         T.end, g, P, pl->tab_binom, pl->tab_tpow, pl->tab_dshift, pl->xi, pl->q,
                         pl->mpole, pl->local, gate);
            LBF_CHECK_LAUNCH();
        }
    }
    LBF_LAUNCH_P(LBF_KERNEL_LEAF, k_leaf, lbf_cdiv(T.nleaf, kLeafWarps), 32 * kLeafWarps, 0, s, T.nleaf, T.leaves,
               T.level, T.ix, T.iy, T.begin, T.end, T.u_ptr, T.u_idx, T.w_ptr, T.w_idx, g, P,
               pl->xi, pl->q, pl->mpole, pl->local, sigma, pl->dself, pl->bsig, v, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_evaluate_impl(lbf_plan *pl, const double *sigma_sorted, const double *a, int64_t T,
                      const double *t, double *u, cudaStream_t s)
{
    int rc = prep(pl, sigma_sorted, nullptr, s);
    if (rc) return rc;
    if (T <= 0) return LBF_OK;
    LBF_LAUNCH(k_evaluate, T, 256, 0, s, pl->N, pl->M, pl->xi, pl->q,
               pl->bsig, a, pl->centres, T, t, pl->has_rot, pl->rot_d, u);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_green_sum_impl(int64_t T, const double *t, int64_t S, const double *p, const double *gamma,
                       double *out, cudaStream_t s)
{
    if (T <= 0) return LBF_OK;
    LBF_LAUNCH(k_green_sum, lbf_cdiv(T, 128), 128, 0, s, T, t, S, p, gamma, out);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
