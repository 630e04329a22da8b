// FMM kernels templated on the real type R (double: the accurate operator;
// float: the inner operator of iterative refinement).  Box geometry, node
// offsets from box centres and the final combine are formed in double; the
// expansions, translations and near-field pair sums run in R.
//
// Scaled expansions about a box centre c with half-width r:
//   multipole  phi(z) = sum_k a_k r^k / (z - c)^(k+1),  a_k = sum_j q_j ((xi_j - c)/r)^k
//   local      phi(z) = sum_l b_l ((z - c)/r)^l
// of the Cauchy potential phi(z) = sum_j q_j / (z - xi_j); the operator needs
// c_i = Im sum_{j != i} q_j / (xi_j - xi_i) = -Im phi(xi_i).
#pragma once

#include "lbf_internal.cuh"

namespace fmm {

template <typename R> struct __align__(2 * sizeof(R)) cx {
    R x, y;
};

__device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename R> __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return cx<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c)  // a*b + c
{
    return cx<R>{fm(a.x, b.x, fm(-a.y, b.y, c.x)), fm(a.x, b.y, fm(a.y, b.x, c.y))};
}

// Reciprocal: in double by Newton-Raphson iteration x <- x (2 - a x) seeded by the
// single-precision reciprocal (two steps reach double rounding; outside the float
// range it falls back to the division operator); in float the hardware
// approximation (the inner operator only needs single precision).
__device__ __forceinline__ double rcp(double a)
{
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / a;
    double x = (double)__frcp_rn((float)a);
    double e = fma(-a, x, 1.0);
    x = fma(x, e, x);
    e = fma(-a, x, 1.0);
    return fma(x, e, x);
}
__device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }

template <typename R> __device__ __forceinline__ cx<R> crcp(cx<R> a)
{
    R d = rcp(a.x * a.x + a.y * a.y);
    return cx<R>{a.x * d, -a.y * d};
}

__device__ __forceinline__ bool gate_closed(const int *gate) { return gate && *gate == 0; }

template <typename R> __device__ __forceinline__ R wsum(R v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct BoxGeo {
    double xmin, ymin, L;
};

__device__ __forceinline__ void box_centre(const BoxGeo &g, int l, int ix, int iy, double &cx_,
                                           double &cy_, double &r)
{
    double w = ldexp(g.L, -l);
    r = 0.5 * w;
    cx_ = g.xmin + (ix + 0.5) * w;
    cy_ = g.ymin + (iy + 0.5) * w;
}

// shift tables for the four child positions: d^k and (2d)^-k, k <= LBF_MAX_TERMS
template <typename R> __device__ __forceinline__ const cx<R> *dpow(const cx<R> *dtab, int c)
{
    return dtab + (size_t)c * (LBF_MAX_TERMS + 1);
}
template <typename R> __device__ __forceinline__ const cx<R> *d2inv(const cx<R> *dtab, int c)
{
    return dtab + (size_t)(4 + c) * (LBF_MAX_TERMS + 1);
}

// Upward pass in one launch (see lbf_fmm.cu): P2M per leaf, then M2M by the warp
// that completes a box's last child:  a_l = d^l sum_{k<=l} C(l,k) (2d)^-k a'_k.
template <typename R>
__global__ void k_up(int64_t nleaf, const int32_t *__restrict__ leaves,
                     const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                     const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                     const int32_t *__restrict__ en, const int32_t *__restrict__ parent,
                     const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                     BoxGeo g, int P, const R *__restrict__ binom, const cx<R> *__restrict__ dtab,
                     const double2 *__restrict__ xi, const cx<R> *__restrict__ q, cx<R> *mp,
                     int *cnt, const int *gate)
{
    if (gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl_len = (P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cl = (R *)sm_raw;  // Cl[k*P + l] = C(l, k) (0 for k > l)
    cx<R> *T = (cx<R> *)(sm_raw + cl_len) + (size_t)wid * P * 32;
    cx<R> *A = (cx<R> *)(sm_raw + cl_len) + (size_t)nw * P * 32 + (size_t)wid * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cl[e] = k <= l ? binom[l * LBF_MAX_TERMS + k] : R(0);
    }
    __syncthreads();
    int64_t t = blockIdx.x * (int64_t)nw + wid;
    if (t >= nleaf) return;
    int b = leaves[t];
    {
        double cxd, cyd, r;
        box_centre(g, level[b], ix[b], iy[b], cxd, cyd, r);
        double ir = 1.0 / r;
        cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
        for (int base = bg[b]; base < en[b]; base += 32) {
            int j = base + lane;
            cx<R> z = mk<R>(0, 0), term = mk<R>(0, 0);
            if (j < en[b]) {
                double2 x = xi[j];
                z = mk<R>((R)((x.x - cxd) * ir), (R)((x.y - cyd) * ir));
                term = q[j];
            }
            for (int k = 0; k < P; k++) {
                T[k * 32 + lane] = term;
                term = cmul(term, z);
            }
            __syncwarp();
            for (int k = lane; k < P; k += 32) {
                cx<R> s = mk<R>(0, 0);
                for (int m = 0; m < 32; m++) {
                    cx<R> v = T[k * 32 + m];
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
        const int l0 = lane, l1 = lane + 32;
        const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
        cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
        for (int c = child0[p]; c < child0[p] + nchild[p]; c++) {
            int d = (ix[c] & 1) + 2 * (iy[c] & 1);
            const cx<R> *inv = d2inv(dtab, d);
            for (int k = lane; k < P; k += 32) {
                cx<R> a;
                const cx<R> *src = &mp[(int64_t)c * P + k];
                // written by other warps in this launch: read through L2
                if (sizeof(R) == 8) {
                    double2 v = __ldcg((const double2 *)src);
                    a = mk<R>((R)v.x, (R)v.y);
                } else {
                    float2 v = __ldcg((const float2 *)src);
                    a = mk<R>((R)v.x, (R)v.y);
                }
                A[k] = cmul(a, inv[k]);
            }
            __syncwarp();
            cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
            for (int k = 0; k < P; k++) {
                cx<R> a = A[k];
                R c0 = Cl[k * P + lc0];
                s0.x = fm(c0, a.x, s0.x);
                s0.y = fm(c0, a.y, s0.y);
                if (l1 < P) {
                    R c1 = Cl[k * P + lc1];
                    s1.x = fm(c1, a.x, s1.x);
                    s1.y = fm(c1, a.y, s1.y);
                }
            }
            const cx<R> *dp = dpow(dtab, d);
            acc0 = cfma(dp[l0], s0, acc0);
            if (l1 < P) acc1 = cfma(dp[l1], s1, acc1);
            __syncwarp();
        }
        if (l0 < P) mp[(int64_t)p * P + l0] = acc0;
        if (l1 < P) mp[(int64_t)p * P + l1] = acc1;
        cur = p;
    }
}

// Downward pass for one level (see lbf_fmm.cu): L2L + M2L (V) + P2L (X).
// P2L lanes take source nodes and run the power recurrence; their terms go
// through shared memory and lanes then take coefficients and sum in node order.
template <typename R>
__global__ void k_down(int64_t ls, int64_t le, const int32_t *__restrict__ level,
                       const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                       const int32_t *__restrict__ parent, const int32_t *__restrict__ vlist,
                       const int32_t *__restrict__ nv, const int32_t *__restrict__ xlist,
                       const int32_t *__restrict__ nx, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, BoxGeo g, int P,
                       const R *__restrict__ binom, const cx<R> *__restrict__ tpow,
                       const cx<R> *__restrict__ dtab, const double2 *__restrict__ xi,
                       const cx<R> *__restrict__ q, const cx<R> *__restrict__ mp,
                       cx<R> *__restrict__ loc, const int *gate, int with_l2l)
{
    if (gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = (2 * P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cm = (R *)sm_raw;          // Cm[k*P + l] = C(k+l, l)
    R *Cd = Cm + P * P;           // Cd[k*P + l] = C(k, l) (0 for k < l)
    cx<R> *A = (cx<R> *)(sm_raw + tl) + (size_t)wid * P;
    cx<R> *T = (cx<R> *)(sm_raw + tl) + (size_t)nw * P + (size_t)wid * P * 32;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cm[e] = binom[(k + l) * LBF_MAX_TERMS + l];
        Cd[e] = k >= l ? binom[k * LBF_MAX_TERMS + l] : R(0);
    }
    __syncthreads();
    int64_t b = ls + blockIdx.x * (int64_t)nw + wid;
    if (b >= le) return;
    const int l0 = lane, l1 = lane + 32;
    const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
    int bx = ix[b], by = iy[b];
    cx<R> accL0 = mk<R>(0, 0), accL1 = mk<R>(0, 0);
    // L2L: b'_l = (2d)^-l sum_{k>=l} C(k,l) d^k b_k (the parent belongs to the previous launch);
    // skipped when the leaf kernel evaluates every ancestor's expansion itself (with_l2l == 0)
    if (with_l2l && level[b] >= 3) {
        int p = parent[b];
        int d = (bx & 1) + 2 * (by & 1);
        const cx<R> *dp = dpow(dtab, d);
        for (int k = lane; k < P; k += 32) A[k] = cmul(loc[(int64_t)p * P + k], dp[k]);
        __syncwarp();
        cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
        for (int k = 0; k < P; k++) {
            cx<R> a = A[k];
            R c0 = Cd[k * P + lc0];
            s0.x = fm(c0, a.x, s0.x);
            s0.y = fm(c0, a.y, s0.y);
            if (l1 < P) {
                R c1 = Cd[k * P + lc1];
                s1.x = fm(c1, a.x, s1.x);
                s1.y = fm(c1, a.y, s1.y);
            }
        }
        const cx<R> *inv = d2inv(dtab, d);
        accL0 = cmul(inv[l0], s0);
        if (l1 < P) accL1 = cmul(inv[l1], s1);
        __syncwarp();
    }
    // M2L: (-1)^l t^(l+1) sum_k C(k+l, l) t^k a_k,  t = 1/(2 (dx + i dy))  (times 1/r below)
    cx<R> accF0 = mk<R>(0, 0), accF1 = mk<R>(0, 0);
    for (int vq = 0; vq < nv[b]; vq++) {
        int s = vlist[b * 27 + vq];
        int o = (bx - ix[s] + 3) * 7 + (by - iy[s] + 3);
        const cx<R> *tp = tpow + (size_t)o * (LBF_MAX_TERMS + 1);
        for (int k = lane; k < P; k += 32) A[k] = cmul(mp[(int64_t)s * P + k], tp[k]);
        __syncwarp();
        cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
        for (int k = 0; k < P; k++) {
            cx<R> a = A[k];
            R c0 = Cm[k * P + lc0];
            s0.x = fm(c0, a.x, s0.x);
            s0.y = fm(c0, a.y, s0.y);
            if (l1 < P) {
                R c1 = Cm[k * P + lc1];
                s1.x = fm(c1, a.x, s1.x);
                s1.y = fm(c1, a.y, s1.y);
            }
        }
        cx<R> f0 = tp[l0 + 1];
        if (l0 & 1) { f0.x = -f0.x; f0.y = -f0.y; }
        accF0 = cfma(f0, s0, accF0);
        if (l1 < P) {
            cx<R> f1 = tp[l1 + 1];
            if (l1 & 1) { f1.x = -f1.x; f1.y = -f1.y; }
            accF1 = cfma(f1, s1, accF1);
        }
        __syncwarp();
    }
    // P2L: (-1)^l sum_j q_j tau_j^(l+1), tau_j = r / (c - xi_j)  (times 1/r below)
    double cxd, cyd, r;
    box_centre(g, level[b], bx, by, cxd, cyd, r);
    double ir = 1.0 / r;
    for (int xq = 0; xq < nx[b]; xq++) {
        int s = xlist[b * 16 + xq];
        for (int base = bg[s]; base < en[s]; base += 32) {
            int j = base + lane;
            cx<R> tau = mk<R>(0, 0), term = mk<R>(0, 0);
            if (j < en[s]) {
                double2 z = xi[j];
                tau = crcp(mk<R>((R)((cxd - z.x) * ir), (R)((cyd - z.y) * ir)));
                term = cmul(q[j], tau);  // l = 0
            }
            for (int l = 0; l < P; l++) {
                T[l * 32 + lane] = (l & 1) ? mk<R>(-term.x, -term.y) : term;
                term = cmul(term, tau);
            }
            __syncwarp();
            for (int l = lane; l < P; l += 32) {
                cx<R> sm = mk<R>(0, 0);
                for (int m = 0; m < 32; m++) {
                    cx<R> v = T[l * 32 + m];
                    sm.x += v.x;
                    sm.y += v.y;
                }
                if (l < 32) { accF0.x += sm.x; accF0.y += sm.y; }
                else { accF1.x += sm.x; accF1.y += sm.y; }
            }
            __syncwarp();
        }
    }
    const R irr = (R)ir;
    if (l0 < P) loc[b * P + l0] = mk<R>(accL0.x + accF0.x * irr, accL0.y + accF0.y * irr);
    if (l1 < P) loc[b * P + l1] = mk<R>(accL1.x + accF1.x * irr, accL1.y + accF1.y * irr);
}

constexpr int kLeafWarps = 4;
constexpr int kSrcChunk = 256;

// Per leaf: far field (L2P of the leaf's local expansion and M2P from W(b)),
// near field (P2P over U(b), self excluded) in coordinates relative to the leaf
// centre (formed in double, so the cancellation of close nodes happens before
// any rounding to R), and the combine into v in double:
//   v_i = 2 [ (1/2pi) c_i + dself_i sigma_i + beta.sigma ].
template <typename R>
__global__ void k_leaf(int64_t nleaf, const int32_t *__restrict__ leaves,
                       const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                       const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, const int32_t *__restrict__ uptr,
                       const int32_t *__restrict__ uidx, const int32_t *__restrict__ wptr,
                       const int32_t *__restrict__ widx, BoxGeo g, int P,
                       const double2 *__restrict__ xi, const cx<R> *__restrict__ q,
                       const cx<R> *__restrict__ mp, const cx<R> *__restrict__ loc,
                       const double *__restrict__ sigma, const double *__restrict__ dself,
                       const double *__restrict__ bsig, double *__restrict__ v, const int *gate,
                       const int32_t *__restrict__ parent, int walk)
{
    if (gate_closed(gate)) return;
    __shared__ cx<R> sx[kLeafWarps][kSrcChunk];
    __shared__ cx<R> sq[kLeafWarps][kSrcChunk];
    __shared__ int32_t sj[kLeafWarps][kSrcChunk];
    __shared__ R cn[kLeafWarps][32];
    __shared__ cx<R> sz[kLeafWarps][32];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t t = blockIdx.x * (int64_t)kLeafWarps + wid;
    if (t >= nleaf) return;
    int b = leaves[t];
    double cxd, cyd, r;
    box_centre(g, level[b], ix[b], iy[b], cxd, cyd, r);
    double ir = 1.0 / r;
    const cx<R> *lb = loc + (int64_t)b * P;
    double bs = *bsig;
    for (int tb = bg[b]; tb < en[b]; tb += 32) {
        int nt = min(32, en[b] - tb);
        int i = tb + lane;
        R cfar = 0;
        if (lane < nt) {
            double2 zi = xi[i];
            sz[wid][lane] = mk<R>((R)(zi.x - cxd), (R)(zi.y - cyd));
            cx<R> u = mk<R>((R)((zi.x - cxd) * ir), (R)((zi.y - cyd) * ir));
            cx<R> phi = mk<R>(0, 0);
            if (!walk) {
                phi = lb[P - 1];
                for (int l = P - 2; l >= 0; l--) phi = cfma(phi, u, lb[l]);
            } else {
                // every ancestor's own local expansion at the target (no L2L chain):
                // (z - c_a)/r_a = 2((ix_b - 2^s ix_a + 1/2) 2^-s - 1/2) + u 2^-s, s = depth gap
                const int lv = level[b];
                for (int a = b; a >= 0 && level[a] >= 2; a = parent[a]) {
                    const int sh = lv - level[a];
                    const R sc = (R)ldexp(1.0, -sh);
                    const int dxi = ix[b] - (ix[a] << sh), dyi = iy[b] - (iy[a] << sh);
                    cx<R> ua = mk<R>((R)2 * (((R)dxi + (R)0.5) * sc - (R)0.5) + u.x * sc,
                                     (R)2 * (((R)dyi + (R)0.5) * sc - (R)0.5) + u.y * sc);
                    const cx<R> *la = loc + (int64_t)a * P;
                    cx<R> t = la[P - 1];
                    for (int l = P - 2; l >= 0; l--) t = cfma(t, ua, la[l]);
                    phi.x += t.x;
                    phi.y += t.y;
                }
            }
            for (int wq = wptr[b]; wq < wptr[b + 1]; wq++) {
                int s = widx[wq];
                double sxd, syd, sr;
                box_centre(g, level[s], ix[s], iy[s], sxd, syd, sr);
                double isr = 1.0 / sr;
                cx<R> rho = crcp(mk<R>((R)((zi.x - sxd) * isr), (R)((zi.y - syd) * isr)));
                const cx<R> *a = mp + (int64_t)s * P;
                cx<R> ps = a[P - 1];
                for (int k = P - 2; k >= 0; k--) ps = cfma(ps, rho, a[k]);
                ps = cmul(ps, rho);
                phi.x += ps.x * (R)isr;
                phi.y += ps.y * (R)isr;
            }
            cfar = -phi.y;
        }
        cn[wid][lane] = 0;
        __syncwarp();
        int fill = 0;
        auto process = [&]() {
            __syncwarp();
            for (int tt = 0; tt < nt; tt++) {
                int ti = tb + tt;
                cx<R> z = sz[wid][tt];
                R acc = 0;
                for (int m = lane; m < fill; m += 32) {
                    if (sj[wid][m] == ti) continue;
                    R dr = sx[wid][m].x - z.x, di = sx[wid][m].y - z.y;
                    cx<R> qq = sq[wid][m];
                    R num = fm(qq.y, dr, -qq.x * di);
                    R den = fm(dr, dr, di * di);
                    acc = fm(num, rcp(den), acc);
                }
                acc = wsum(acc);
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
                    double2 zs = xi[sb + m];
                    sx[wid][fill + m] = mk<R>((R)(zs.x - cxd), (R)(zs.y - cyd));
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
            double c = (double)cfar + (double)cn[wid][lane];
            v[i] = 2.0 * (c * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + bs);
        }
        __syncwarp();
    }
}

}  // namespace fmm
