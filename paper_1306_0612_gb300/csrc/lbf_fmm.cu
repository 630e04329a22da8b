// The density block of the operator, K sigma in the paper's doubled scaling
// (Sec. 5, Eq. disc_sphere; Cauchy term signed as derived from Eq. fundC and
// Eq. grad3):
//
//   v_i = 2 [ (1/2pi) c_i + dself_i sigma_i + sum_j beta_j sigma_j ],
//   c_i = Im sum_{j != i} q_j / (xi_j - xi_i),   q_j = sigma_j w_j,
//
// with the Cauchy sum c evaluated by a 2D fast multipole method on the adaptive
// quadtree (Sec. 5: "the two dimensional FMM based on the Coulomb potential")
// in double (the accurate operator) or in float (the inner operator of
// iterative refinement), or by a direct O(N^2) sum.  The self terms and the
// rank-one sphere correction are always formed in double.
//
// Launch structure of one FMM application: prep (q, beta.sigma); the upward
// pass in one launch (P2M, then M2M by the warp that completes a box's last
// child: no warp waits for another); the downward pass one launch per level
// (L2L + M2L + P2L); the leaf kernel (L2P + M2P + P2P + combine).
#include <algorithm>

#include "lbf_fmm_tpl.cuh"

using fmm::BoxGeo;
using fmm::cx;

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Charges and one scalar for an FMM pass: q = sigma w (w given) or q = (sigma, 0)
// (w null), in double and/or float, and sum_i beta_i sigma_i (beta given) or
// sum_i sigma_i (beta null), by a fixed-order two-level reduction (the last block
// sums the block partials in order).
__global__ void k_prep(int64_t N, const double *__restrict__ sigma, const double2 *__restrict__ w,
                       const double *__restrict__ beta, double2 *__restrict__ q,
                       float2 *__restrict__ q32, cx<df64> *__restrict__ qdf,
                       double *__restrict__ part, unsigned *__restrict__ count,
                       double *__restrict__ out, const int *gate,
                       const int32_t *__restrict__ isl, const double *__restrict__ mean,
                       int64_t slab)
{
    lbf_rhs(slab, sigma, q, q32, qdf, part, count, out, gate, mean);
    if (fmm::gate_closed(gate)) return;
    __shared__ double sh[32];
    __shared__ bool last;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = sigma[i];
        const double sc = isl ? s - mean[isl[i]] : s;  // the charges of sigma less its island means
        double2 qq = make_double2(sc, 0.0);
        if (w) {
            double2 ww = w[i];
            qq = make_double2(sc * ww.x, sc * ww.y);
        }
        if (q) q[i] = qq;
        if (q32) q32[i] = make_float2((float)qq.x, (float)qq.y);
        if (qdf) qdf[i] = cx<df64>{df64(qq.x), df64(qq.y)};
        acc = beta ? fma(beta[i], s, acc) : acc + s;
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
    if (!last) return;
    // the last block sums the block partials in a fixed order (strided, then by warps)
    __threadfence();
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(&part[b]);
    t = warp_sum(t);
    if (lane == 0) sh[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) u += sh[k];
        *out = u;
        *count = 0u;
    }
}

// island of each node (sorted order), a warp per island
__global__ void k_island_ids(int M, const int64_t *__restrict__ ptr, const int32_t *__restrict__ rank,
                             int32_t *__restrict__ isl)
{
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= M) return;
    for (int64_t j = ptr[wg] + lane; j < ptr[wg + 1]; j += 32) isl[rank[j]] = (int32_t)wg;
}

// The rows of a density constant on one island.  With the planar double layer
// P(u)_i = (1/2pi) Im sum_{j != i} w_j u_j/(xi_j - xi_i) + dself_i u_i, the discrete form
// of Gauss' theorem (Sec. 3) gives, for the indicator 1_k of island k's nodes,
//   P(1_k) = (o_k/2) 1_k + n_k (1 - 1_k)
// with o_k = +-1 the curve's orientation and n_k its winding number about the other
// islands (0, or +-1 for the one island whose planar image encloses all the others).
// So 2 K 1_k = 2 P(1_k) + 2 (beta . 1_k) 1 = (o_k - 2 n_k) 1_k + (2 n_k + 2 beta . 1_k) 1.
// A warp per island evaluates o_k/2 at its first node and n_k at two nodes of the next
// island, rounds them, and flags the split off if a value is not near its rounding or
// more than one island encloses others.
__global__ void k_island_modes(int M, const int64_t *__restrict__ ptr, const int32_t *__restrict__ rank,
                               const double2 *__restrict__ xi, const double2 *__restrict__ w,
                               const double *__restrict__ dself, double *__restrict__ acoef,
                               double *__restrict__ scal, unsigned *__restrict__ flags)
{
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= M) return;
    const int64_t b = ptr[k], e = ptr[k + 1];
    const int64_t k1 = (k + 1) % M;
    const double2 z0 = xi[rank[b]];
    const double2 z1 = xi[rank[ptr[k1]]], z2 = xi[rank[(ptr[k1] + ptr[k1 + 1]) / 2]];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    auto term = [](double2 wj, double2 zj, double2 z) {  // Im(w_j / (xi_j - z))
        const double dx = zj.x - z.x, dy = zj.y - z.y;
        return (wj.y * dx - wj.x * dy) / (dx * dx + dy * dy);
    };
    for (int64_t j = b + lane; j < e; j += 32) {
        const int32_t r = rank[j];
        const double2 wj = w[r], zj = xi[r];
        if (j != b) s0 += term(wj, zj, z0);
        if (M > 1) {
            s1 += term(wj, zj, z1);
            s2 += term(wj, zj, z2);
        }
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane != 0) return;
    const double on = s0 / (2.0 * LBF_PI) + dself[rank[b]];
    const double n1 = s1 / (2.0 * LBF_PI), n2 = s2 / (2.0 * LBF_PI);
    const double o = on > 0.0 ? 1.0 : -1.0, n = rint(n1);
    const bool good = fabs(2.0 * on - o) < 0.02 && fabs(n1 - n) < 0.01 && fabs(n2 - n) < 0.01 &&
                      fabs(n) <= 1.0;
    acoef[k] = good ? o - 2.0 * n : 0.0;  // finite even where a sum was not (the split is off then)
    if (!good) atomicOr(&flags[0], 1u);
    if (n != 0.0) {
        atomicAdd(&flags[1], 1u);
        scal[1] = (double)k;
        scal[2] = 2.0 * n;
    }
}

__global__ void k_island_modes_end(double *__restrict__ scal, unsigned *__restrict__ flags)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const bool ok = flags[0] == 0u && flags[1] <= 1u;
    scal[0] = ok ? 1.0 : 0.0;
    if (!ok || flags[1] == 0u) {
        scal[1] = -1.0;
        scal[2] = 0.0;
    }
}

// mean of sigma (sorted order) over each island's nodes, a warp per island, fixed order
// (0 where the split is off)
__global__ void k_island_means(int M, const int64_t *__restrict__ ptr, const int32_t *__restrict__ rank,
                               const double *__restrict__ sigma, double *__restrict__ mean,
                               const int *gate, int64_t slab)
{
    lbf_rhs(slab, sigma, mean, gate);
    if (fmm::gate_closed(gate)) return;
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= M) return;
    const int64_t b = ptr[wg], e = ptr[wg + 1];
    double acc = 0.0;
    for (int64_t j = b + lane; j < e; j += 32) acc += sigma[rank[j]];
    acc = warp_sum(acc);
    if (lane == 0) mean[wg] = (e > b && mean[M] != 0.0) ? acc / (double)(e - b) : 0.0;
}

// Direct O(N^2) Cauchy sums with the same outputs as the leaf kernel's modes
// (tiled through shared memory).
template <int MODE>
__global__ void k_direct(int64_t N, const double2 *__restrict__ xi, const double2 *__restrict__ q,
                         const double *__restrict__ sigma, const double *__restrict__ dself,
                         const double2 *__restrict__ w, const double *__restrict__ beta,
                         const double *__restrict__ bsig, double *__restrict__ v, const int *gate,
                         int64_t slab)
{
    lbf_rhs(slab, q, sigma, bsig, v, gate);
    if (fmm::gate_closed(gate)) return;
    __shared__ double2 sx[256], sq[256];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double2 z = i < N ? xi[i] : make_double2(0, 0);
    double accI = 0.0, ar = 0.0, ai = 0.0;
    for (int64_t base = 0; base < N; base += 256) {
        int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < N) { sx[threadIdx.x] = xi[j]; sq[threadIdx.x] = q[j]; }
        __syncthreads();
        int n = (int)(N - base < 256 ? N - base : 256);
        for (int m = 0; m < n; m++) {
            if (base + m == i) continue;
            double dr = sx[m].x - z.x, di = sx[m].y - z.y;
            double2 qq = sq[m];
            double ir2 = fmm::rcp(fma(dr, dr, di * di));
            if (MODE == fmm::kLeafForward) {
                accI = fma(fma(qq.y, dr, -qq.x * di), ir2, accI);
            } else if (MODE == fmm::kLeafTranspose) {
                ar = fma(fma(qq.x, dr, qq.y * di), ir2, ar);
                ai = fma(fma(qq.y, dr, -qq.x * di), ir2, ai);
            } else {
                double er = (dr * dr - di * di) * ir2 * ir2, ei = -2 * dr * di * ir2 * ir2;
                ar = fma(qq.x, er, fma(-qq.y, ei, ar));
                ai = fma(qq.x, ei, fma(qq.y, er, ai));
            }
        }
    }
    if (i >= N) return;
    if (MODE == fmm::kLeafForward) {
        v[i] = 2.0 * (accI * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + *bsig);
    } else if (MODE == fmm::kLeafTranspose) {
        double2 ww = w[i];
        double im = -(ww.x * ai + ww.y * ar);
        v[i] = 2.0 * (im * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + beta[i] * *bsig);
    } else {
        ((double2 *)v)[i] = make_double2(-ar, -ai);
    }
}

// u(t) at off-curve targets: (1/2pi) Im sum_j q_j/(xi_j - xi_t) + beta.sigma
// + sum_m a_m G(t, c_m)  (Eq. u_multi, planar form of the double layer, Eq. dlpC).
// One block per target; threads stride over the nodes, fixed-order block reduction.
__global__ void k_evaluate(int64_t N, int M, const double2 *__restrict__ xi,
                           const double2 *__restrict__ q, const double *__restrict__ bsig,
                           const double *__restrict__ a, const double *__restrict__ c,
                           int64_t T, const double *__restrict__ t, int rot_on, const double *rot,
                           double *__restrict__ u)
{
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
            acc = fma(fma(qq.y, dr, -qq.x * di), fmm::rcp(fma(dr, dr, di * di)), acc);
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

// u(t) with the far field from the quadtree: the same representation formula as
// k_evaluate, but boxes at least kEvalSep half-widths from the target enter through
// their multipole expansion (M2P: every node of the box is within sqrt(2) r of its
// centre, so the series ratio is at most 1/3 and the truncation after P terms is below
// 3^-P relative), leaves closer than that by the direct sum, other boxes are opened.
// One warp per target; each level's frontier is written in a fixed order (warp prefix
// sums), so the sum is reproducible.
constexpr double kEvalSep = 4.25;  // >= 3 sqrt(2): |(xi - c)/(t - c)| <= 1/3 in the box
constexpr int kEvalFront = 2048;   // frontier capacity per warp (per level)
constexpr int kEvalWarps = 4;

template <typename R>
__global__ void k_evaluate_tree(int64_t N, int M, const double2 *__restrict__ xi,
                                const double2 *__restrict__ q, const cx<R> *__restrict__ mp,
                                int P, const int32_t *__restrict__ level,
                                const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                                const int32_t *__restrict__ child0,
                                const int32_t *__restrict__ nchild, const int32_t *__restrict__ bg,
                                const int32_t *__restrict__ en, BoxGeo g,
                                const double *__restrict__ bsig, const double *__restrict__ a,
                                const double *__restrict__ c, int64_t T,
                                const double *__restrict__ t, int rot_on,
                                const double *__restrict__ rot, double *__restrict__ u,
                                int *__restrict__ status)
{
    extern __shared__ int32_t front[];  // [warp][2][kEvalFront]
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tq = blockIdx.x * (int64_t)kEvalWarps + wid;
    if (tq >= T) return;
    int32_t *fr[2] = {front + (size_t)wid * 2 * kEvalFront, front + (size_t)wid * 2 * kEvalFront + kEvalFront};
    double p[3] = {t[3 * tq], t[3 * tq + 1], t[3 * tq + 2]};
    if (rot_on) {
        double r0 = rot[0] * p[0] + rot[1] * p[1] + rot[2] * p[2];
        double r1 = rot[3] * p[0] + rot[4] * p[1] + rot[5] * p[2];
        double r2 = rot[6] * p[0] + rot[7] * p[1] + rot[8] * p[2];
        p[0] = r0; p[1] = r1; p[2] = r2;
    }
    const double w = 1.0 - p[2];
    double accr = 0.0, acci = 0.0;  // sum over sources of q/(xi - t)
    if (w > 0.0) {                  // a target at the pole sees no Cauchy term
        const double zx = p[0] / w, zy = p[1] / w;
        int cur = 0, n = 1;
        if (lane == 0) fr[0][0] = 0;
        __syncwarp();
        while (n > 0) {
            int nn = 0;
            for (int base = 0; base < n; base += 32) {
                const int e = base + lane;
                int kids = 0, b = -1;
                if (e < n) {
                    b = fr[cur][e];
                    double cxd, cyd, r;
                    box_centre(g, level[b], ix[b], iy[b], cxd, cyd, r);
                    const double dx = zx - cxd, dy = zy - cyd;
                    if (b != 0 && dx * dx + dy * dy >= kEvalSep * kEvalSep * r * r) {
                        // M2P: Phi(t) = (1/r) sum_k a_k rho^(k+1), rho = r/(t - c); q/(xi - t) = -Phi
                        const double id = fmm::rcp_near(dx * dx + dy * dy);
                        const cx<R> rho{R(r * dx * id), R(-r * dy * id)};
                        const cx<R> *ak = mp + (int64_t)b * P;
                        cx<R> ps = ak[P - 1];
                        for (int k = P - 2; k >= 0; k--) ps = fmm::cfma(ps, rho, ak[k]);
                        ps = fmm::cmul(ps, rho);
                        const double ir = 1.0 / r;
                        accr -= (double)ps.x * ir;
                        acci -= (double)ps.y * ir;
                    } else if (nchild[b] == 0) {
                        for (int j = bg[b]; j < en[b]; j++) {
                            const double dr = xi[j].x - zx, di = xi[j].y - zy;
                            const double2 qq = q[j];
                            const double d2 = fma(dr, dr, di * di);
                            const double id = d2 > 0x1p-120 ? fmm::rcp_near(d2) : 1.0 / d2;
                            accr += (qq.x * dr + qq.y * di) * id;
                            acci += (qq.y * dr - qq.x * di) * id;
                        }
                    } else {
                        kids = nchild[b];
                    }
                }
                // children in frontier order: exclusive prefix sum of the lanes' counts
                int incl = kids;
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                int pos = nn + incl - kids;
                for (int k = 0; k < kids; k++, pos++) {
                    if (pos < kEvalFront) fr[1 - cur][pos] = child0[b] + k;
                }
                nn += total;
            }
            if (nn > kEvalFront) {
                if (lane == 0) atomicOr(status, 8);
                nn = 0;
            }
            __syncwarp();
            cur = 1 - cur;
            n = nn;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        accr += __shfl_xor_sync(0xffffffffu, accr, o);
        acci += __shfl_xor_sync(0xffffffffu, acci, o);
    }
    double sa = 0.0;
    if (a) {
        for (int m = lane; m < M; m += 32) {
            double d0 = p[0] - c[3 * m], d1 = p[1] - c[3 * m + 1], d2 = p[2] - c[3 * m + 2];
            sa += a[m] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
        }
        for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    if (lane == 0) u[tq] = acci * (1.0 / (2.0 * LBF_PI)) + *bsig + sa;
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

// per node: (xi - c)/r about its leaf's centre c and half-width r, rounded to
// float once per geometry (warp per leaf)
__global__ void k_local_coords(int64_t nleaf, const int32_t *__restrict__ leaves,
                               const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                               const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                               const int32_t *__restrict__ en, fmm::BoxGeo g,
                               const double2 *__restrict__ xi, float2 *__restrict__ u32,
                               cx<df64> *__restrict__ udf)
{
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= nleaf) return;
    int b = leaves[t];
    double cx_, cy_, r;
    fmm::box_centre(g, level[b], ix[b], iy[b], cx_, cy_, r);
    double ir = 1.0 / r;
    for (int i = bg[b] + lane; i < en[b]; i += 32) {
        double2 z = xi[i];
        const double ux = (z.x - cx_) * ir, uy = (z.y - cy_) * ir;
        if (u32) u32[i] = make_float2((float)ux, (float)uy);
        if (udf) udf[i] = cx<df64>{df64(ux), df64(uy)};
    }
}

// per leaf: its ancestors at levels >= 2, nearest first (the leaf itself at s = 0)
__global__ void k_ancestors(int64_t nleaf, const int32_t *__restrict__ leaves,
                            const int32_t *__restrict__ level, const int32_t *__restrict__ parent,
                            int32_t *__restrict__ anc)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    const int b = leaves[t];
    int s = 0;
    for (int a = b; a >= 0 && level[a] >= 2 && s < LBF_ANC_STRIDE; a = parent[a])
        anc[(int64_t)b * LBF_ANC_STRIDE + s++] = a;
}

// shared-memory bytes of the two FMM pass kernels
template <typename R> size_t up_smem(int P, int wpb)
{
    return (P * P * sizeof(R) + 15) / 16 * 16 + sizeof(cx<R>) * (size_t)wpb * P * 34;
}
template <typename R> size_t down_smem(int P, int wpb)
{
    return (2 * P * P * sizeof(R) + 15) / 16 * 16 + sizeof(cx<R>) * (size_t)wpb * P * 34;
}
constexpr size_t kSmemCap = 200 * 1024;

// warps per block of the downward pass: the most resident warps per SM that its
// shared memory allows (228 KB per SM, 1 KB of it reserved per block)
template <typename R> int down_warps(int P)
{
    int best = 1, most = 0;
    for (int w = 8; w >= 1; w--) {
        const size_t sm = down_smem<R>(P, w);
        if (sm > kSmemCap) continue;
        const int resident = w * (int)((228 * 1024) / (sm + 1024));
        if (resident > most) { most = resident; best = w; }
    }
    return best;
}

struct FmmArrays {
    int P;
    const void *q;
    void *mp, *loc;
    const void *binom, *tpow, *dshift;
    const void *uloc;  // leaf-local node coordinates (float, double-float), else null
};

// split (float forward rows): the passes see sigma less its island means m_k, and the
// leaf kernel adds the means' rows exactly (k_island_modes): for islands traversed with
// the land on one side, (I + 2K) 1_k is a constant vector, far smaller than 1_k, so the
// float passes never form the near-cancelling sum of a mean density, which is what the
// corrections of the refinement are made of.
template <typename R, int MODE>
int fmm_apply(lbf_plan *pl, const FmmArrays &a, const double *sigma, double *v, const int *gate,
              cudaStream_t s, bool split = false)
{
    Tree &T = pl->tree;
    BoxGeo g{T.xmin, T.ymin, T.L, (float)(1.0 / T.L), df64(1.0 / T.L), 1.0 / T.L};
    const int P = a.P;
    const cx<R> *q = (const cx<R> *)a.q;
    cx<R> *mp = (cx<R> *)a.mp, *loc = (cx<R> *)a.loc;
    const R *binom = (const R *)a.binom;
    const cx<R> *tpow = (const cx<R> *)a.tpow, *dsh = (const cx<R> *)a.dshift;
    const cx<R> *uloc = (const cx<R> *)a.uloc;
    // the float passes form coordinates across large level gaps in double-float
    const cx<df64> *udf = sizeof(R) == sizeof(float) ? (const cx<df64> *)pl->udf : nullptr;
    const bool dbl = sizeof(R) == sizeof(double);
    const int kid_up = dbl ? LBF_KERNEL_UP : LBF_KERNEL_UP32;
    const int kid_down = dbl ? LBF_KERNEL_DOWN : LBF_KERNEL_DOWN32;
    const int kid_leaf = dbl ? LBF_KERNEL_LEAF : LBF_KERNEL_LEAF32;
    {
        const int wpb = 2;
        LBF_LAUNCH_P(kid_up, fmm::k_up<R>, lbf_grid(pl, lbf_cdiv(T.nleaf, wpb)), 32 * wpb,
                     up_smem<R>(P, wpb), s, T.nleaf, T.leaves, T.level, T.ix, T.iy, T.begin,
                     T.end, T.parent, T.child0, T.nchild, g, P, binom, dsh, pl->xi, uloc, q,
                     mp, pl->upcnt, gate, pl->slab);
        LBF_CHECK_LAUNCH();
    }
    // float forward rows: no chain, the far field comes from the per-node walk below
    const bool walk = sizeof(R) == sizeof(float) && MODE == fmm::kLeafForward && pl->anc &&
                      pl->bd.leaf_of;
    // Every box runs in one launch, taking the boxes in index order and shifting its
    // parent's full expansion down once the parent is done, so the leaf kernel
    // evaluates one expansion per target (level by level only if the plan has no
    // counters for it).
    {
        const int wpb = down_warps<R>(P);
        const size_t smem = down_smem<R>(P, wpb);
        if (walk) {  // every box's own M2L + P2L, a warp per box, no chain
            LBF_LAUNCH_P(kid_down, fmm::k_down<R>, lbf_grid(pl, lbf_cdiv(T.nbox, wpb)), 32 * wpb,
                         smem, s, (int64_t)0, T.nbox, T.level, T.ix, T.iy, T.parent, T.vlist, T.nv,
                         T.xlist, T.nx, T.begin, T.end, g, P, binom, tpow, dsh, pl->xi, uloc, q, mp,
                         loc, gate, 0, (unsigned *)nullptr, pl->dev_status, udf, pl->slab);
            LBF_CHECK_LAUNCH();
        } else if (pl->pull) {
            const int64_t grid = std::min<int64_t>(lbf_cdiv(T.nbox, wpb), 4 * (int64_t)std::max(pl->nsm, 1));
            LBF_LAUNCH_P(kid_down, fmm::k_down<R>, lbf_grid(pl, grid), 32 * wpb, smem, s, (int64_t)0,
                         T.nbox, T.level, T.ix, T.iy, T.parent, T.vlist, T.nv, T.xlist, T.nx, T.begin,
                         T.end, g, P, binom, tpow, dsh, pl->xi, uloc, q, mp, loc, gate, 2, pl->pull,
                         pl->dev_status, udf, pl->slab);
            LBF_CHECK_LAUNCH();
        } else {
            for (int l = 0; l < T.nlev; l++) {
                int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
                if (le <= ls) continue;
                LBF_LAUNCH_P(kid_down, fmm::k_down<R>, lbf_grid(pl, lbf_cdiv(le - ls, wpb)), 32 * wpb,
                             smem, s, ls, le, T.level, T.ix, T.iy, T.parent, T.vlist, T.nv, T.xlist,
                             T.nx, T.begin, T.end, g, P, binom, tpow, dsh, pl->xi, uloc, q, mp, loc,
                             gate, 1, (unsigned *)nullptr, pl->dev_status, udf, pl->slab);
                LBF_CHECK_LAUNCH();
            }
        }
    }
    // Several right-hand sides in lockstep: the double forward rows' near field in one pass
    // that forms each pair's geometry once (k_near_multi), the leaf kernel adding it.  (The
    // float operator keeps a leaf pass per right-hand side: its pairs are cheap on the
    // float pipes, and one warp per leaf for all right-hand sides left too few warps to
    // hide the latency of a small system: measured slower.)
    const bool multi = MODE == fmm::kLeafForward && pl->nrhs > 1 && pl->nearbuf &&
                       std::is_same<R, double>::value;
    if constexpr (MODE == fmm::kLeafForward && std::is_same<R, double>::value) if (multi) {
        const int nr = pl->nrhs;
        const int64_t nb = lbf_cdiv(2 * T.nleaf, 4);  // two warps a leaf
        const int32_t *isl = split ? (const int32_t *)pl->isl : nullptr;
        const double *im = split ? (const double *)pl->imean : nullptr;
#define LBF_NEAR_MULTI(NR)                                                                       \
        LBF_LAUNCH_P(kid_leaf, (fmm::k_near_multi<R, NR>), nb, 128, (fmm::near_multi_smem<R, NR>(4)), \
                     s, T.nleaf, T.leaves, T.level, T.ix, T.iy, T.begin, T.end, T.u_ptr, T.u_idx, g,  \
                     pl->xi, uloc, udf, pl->w, sigma, isl, im, nr, pl->slab, pl->nearbuf, gate)
        if (nr <= 2) LBF_NEAR_MULTI(2);
        else if (nr <= 4) LBF_NEAR_MULTI(4);
        else if (nr <= 8) LBF_NEAR_MULTI(8);
        else LBF_NEAR_MULTI(16);
#undef LBF_NEAR_MULTI
        LBF_CHECK_LAUNCH();
    }
    const int lw = pl->opt.p2p_warps > 0 ? pl->opt.p2p_warps : fmm::kLeafWarps;
    LBF_LAUNCH_P(kid_leaf, (fmm::k_leaf<R, MODE>), lbf_grid(pl, lbf_cdiv(T.nleaf, lw)), 32 * lw,
                 (fmm::leaf_smem<R, MODE>(lw)), s, T.nleaf, T.leaves, T.level, T.ix, T.iy, T.begin,
                 T.end, T.u_ptr, T.u_idx, T.w_ptr, T.w_idx, g, P, pl->xi, uloc, q, mp, loc,
                 sigma, pl->dself, pl->w, pl->beta, pl->bsig, v, gate, udf, walk ? 0 : 1,
                 split ? (const int32_t *)pl->isl : (const int32_t *)nullptr,
                 split ? (const double *)pl->imean : (const double *)nullptr,
                 split ? (const double *)pl->iacoef : (const double *)nullptr, pl->M, pl->slab,
                 multi ? (const double *)pl->nearbuf : (const double *)nullptr);
    if (walk) {
        LBF_LAUNCH_P(kid_leaf, fmm::k_l2p_walk, lbf_grid(pl, lbf_cdiv(pl->N, 256)), 256, 0, s, pl->N,
                     P, pl->bd.leaf_of, T.level, T.ix, T.iy, pl->anc, (const float2 *)uloc,
                     (const cx<float> *)loc, v, gate, pl->slab);
    }
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

}  // namespace

int lbf_fmm_init_attrs()
{
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_up<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_up<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_down<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_down<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_up<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(k_evaluate_tree<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(int32_t) * 2 * kEvalFront * kEvalWarps)));
    LBF_CUDA(cudaFuncSetAttribute(k_evaluate_tree<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(int32_t) * 2 * kEvalFront * kEvalWarps)));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_down<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    // the leaf pass: up to 8 warps of staged near-field sources
    const int leaf_cap = (int)fmm::leaf_smem<double, fmm::kLeafForward>(8);
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<double, fmm::kLeafForward>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<double, fmm::kLeafTranspose>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<double, fmm::kLeafDeriv>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<df64, fmm::kLeafForward>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<df64, fmm::kLeafTranspose>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<df64, fmm::kLeafDeriv>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<float, fmm::kLeafForward>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<float, fmm::kLeafTranspose>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    LBF_CUDA(cudaFuncSetAttribute(fmm::k_leaf<float, fmm::kLeafDeriv>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_cap));
    return LBF_OK;
}

// charges and the scalar of one pass: forward q = w sigma with beta . sigma;
// transposed and real-charge passes q = (sigma, 0) with sum sigma
// arithmetic of one pass: float, double, or double-float
enum class Arith { F32, F64, DF64 };

// split: the charges of sigma less its island means (the float forward pass; the leaf
// kernel adds the means' part back exactly)
static int prep(lbf_plan *pl, const double *sigma, Arith ar, bool weighted, const int *gate,
                cudaStream_t s, bool split = false)
{
    int nb = (int)std::min<int64_t>(lbf_cdiv(pl->N, 256), 1024);
    if (split)
        LBF_LAUNCH(k_island_means, lbf_grid(pl, lbf_cdiv((int64_t)pl->M * 32, 256)), 256, 0, s,
                   pl->M, pl->island_ptr, pl->rank, sigma, pl->imean, gate, pl->slab);
    LBF_LAUNCH(k_prep, lbf_grid(pl, nb), 256, 0, s, pl->N, sigma,
               weighted ? pl->w : (const double2 *)nullptr,
               weighted ? pl->beta : (const double *)nullptr,
               ar == Arith::F64 ? pl->q : (double2 *)nullptr,
               ar == Arith::F32 ? pl->q32 : (float2 *)nullptr,
               ar == Arith::DF64 ? (cx<df64> *)pl->qdf : (cx<df64> *)nullptr, pl->red,
               pl->red_count, pl->bsig, gate,
               split ? (const int32_t *)pl->isl : (const int32_t *)nullptr,
               split ? (const double *)pl->imean : (const double *)nullptr, pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

template <int MODE>
static int apply_mode(lbf_plan *pl, const double *sigma, double *v, const int *gate, cudaStream_t s,
                      int prec, bool weighted)
{
    if (prec == LBF_PREC_FP32 && !pl->q32) return LBF_ENOTBUILT;
    if (pl->opt.matvec == LBF_MATVEC_DIRECT || MODE == fmm::kLeafDeriv) prec = LBF_PREC_FP64;
    const Arith ar = prec == LBF_PREC_FP32 ? Arith::F32
                     : (pl->qdf && MODE != fmm::kLeafDeriv && pl->opt.matvec == LBF_MATVEC_FMM)
                         ? Arith::DF64
                         : Arith::F64;
    // the float forward rows split off each island's mean density (see fmm_apply)
    const bool split = ar == Arith::F32 && MODE == fmm::kLeafForward && weighted && pl->isl;
    int rc = prep(pl, sigma, ar, weighted, gate, s, split);
    if (rc) return rc;
    int64_t N = pl->N;
    if (pl->opt.matvec == LBF_MATVEC_DIRECT) {
        LBF_LAUNCH_P(LBF_KERNEL_DIRECT, k_direct<MODE>, lbf_grid(pl, lbf_cdiv(N, 256)), 256, 0, s, N,
                     pl->xi, pl->q, sigma, pl->dself, pl->w, pl->beta, pl->bsig, v, gate, pl->slab);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if (ar == Arith::F32) {
        FmmArrays a{pl->P32, pl->q32, pl->mpole32, pl->local32, pl->tab32_binom, pl->tab32_tpow,
                    pl->tab32_dshift, pl->u32};
        return fmm_apply<float, MODE>(pl, a, sigma, v, gate, s, split);
    }
    if (ar == Arith::DF64) {
        FmmArrays a{pl->P, pl->qdf, pl->mpole, pl->local, pl->tabdf_binom, pl->tabdf_tpow,
                    pl->tabdf_dshift, pl->udf};
        return fmm_apply<df64, MODE>(pl, a, sigma, v, gate, s);
    }
    FmmArrays a{pl->P, pl->q, pl->mpole, pl->local, pl->tab_binom, pl->tab_tpow, pl->tab_dshift,
                nullptr};
    return fmm_apply<double, MODE>(pl, a, sigma, v, gate, s);
}

int lbf_apply_K(lbf_plan *pl, const double *sigma, double *v, const int *gate, cudaStream_t s,
                int prec)
{
    return apply_mode<fmm::kLeafForward>(pl, sigma, v, gate, s, prec, true);
}

int lbf_apply_KT(lbf_plan *pl, const double *tau, double *v, const int *gate, cudaStream_t s,
                 int prec)
{
    return apply_mode<fmm::kLeafTranspose>(pl, tau, v, gate, s, prec, false);
}

int lbf_cauchy_deriv(lbf_plan *pl, const double *x, bool weighted, double2 *out, cudaStream_t s)
{
    return apply_mode<fmm::kLeafDeriv>(pl, x, (double *)out, nullptr, s, LBF_PREC_FP64, weighted);
}

int lbf_multipoles(lbf_plan *pl, const double *x, int P, double2 *mp, const int *gate,
                   cudaStream_t s)
{
    if (P > LBF_MAX_TERMS) return LBF_EINVAL;
    int rc = prep(pl, x, Arith::F64, false, gate, s);
    if (rc) return rc;
    Tree &T = pl->tree;
    BoxGeo g{T.xmin, T.ymin, T.L, (float)(1.0 / T.L), df64(1.0 / T.L), 1.0 / T.L};
    const int wpb = 2;
    LBF_LAUNCH(fmm::k_up<double>, lbf_cdiv(T.nleaf, wpb), 32 * wpb, up_smem<double>(P, wpb), s,
               T.nleaf, T.leaves, T.level, T.ix, T.iy, T.begin, T.end, T.parent, T.child0,
               T.nchild, g, P, pl->tab_binom, (const cx<double> *)pl->tab_dshift, pl->xi,
               (const cx<double> *)nullptr, (const cx<double> *)pl->q, (cx<double> *)mp,
               pl->upcnt, gate, (int64_t)0);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_fmm_prepare(lbf_plan *pl, cudaStream_t s)
{
    if (pl->isl) {
        const int M = pl->M;
        unsigned *flags = (unsigned *)(pl->imean + M + 4);
        LBF_CUDA(cudaMemsetAsync(pl->imean, 0, sizeof(double) * ((size_t)M + 8), s));
        LBF_LAUNCH(k_island_ids, lbf_cdiv((int64_t)M * 32, 256), 256, 0, s, M, pl->island_ptr,
                   pl->rank, pl->isl);
        LBF_LAUNCH(k_island_modes, lbf_cdiv((int64_t)M * 32, 256), 256, 0, s, M, pl->island_ptr,
                   pl->rank, pl->xi, pl->w, pl->dself, pl->iacoef, pl->imean + M, flags);
        LBF_LAUNCH(k_island_modes_end, 1, 32, 0, s, pl->imean + M, flags);
    }
    if (!pl->u32 && !pl->udf) return LBF_OK;
    Tree &T = pl->tree;
    fmm::BoxGeo g{T.xmin, T.ymin, T.L, (float)(1.0 / T.L), df64(1.0 / T.L), 1.0 / T.L};
    LBF_LAUNCH(k_local_coords, lbf_cdiv(T.nleaf, 8), 256, 0, s, T.nleaf, T.leaves, T.level, T.ix,
               T.iy, T.begin, T.end, g, pl->xi, pl->u32, (cx<df64> *)pl->udf);
    if (pl->anc)
        LBF_LAUNCH(k_ancestors, lbf_cdiv(T.nleaf, 256), 256, 0, s, T.nleaf, T.leaves, T.level,
                   T.parent, pl->anc);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_evaluate_impl(lbf_plan *pl, const double *sigma_sorted, const double *a, int64_t T,
                      const double *t, double *u, cudaStream_t s)
{
    if (pl->opt.matvec == LBF_MATVEC_FMM && pl->qdf && T > 0) {
        // charges in double (direct part) and double-float (multipoles), beta . sigma
        int nb = (int)std::min<int64_t>(lbf_cdiv(pl->N, 256), 1024);
        LBF_LAUNCH(k_prep, nb, 256, 0, s, pl->N, sigma_sorted, pl->w, pl->beta, pl->q,
                   (float2 *)nullptr, (cx<df64> *)pl->qdf, pl->red, pl->red_count, pl->bsig,
                   (const int *)nullptr, (const int32_t *)nullptr, (const double *)nullptr, (int64_t)0);
        LBF_CHECK_LAUNCH();
        Tree &Tr = pl->tree;
        BoxGeo g{Tr.xmin, Tr.ymin, Tr.L, (float)(1.0 / Tr.L), df64(1.0 / Tr.L), 1.0 / Tr.L};
        const int P = pl->P, wpb = 2;
        LBF_LAUNCH(fmm::k_up<df64>, lbf_cdiv(Tr.nleaf, wpb), 32 * wpb, up_smem<df64>(P, wpb), s,
                   Tr.nleaf, Tr.leaves, Tr.level, Tr.ix, Tr.iy, Tr.begin, Tr.end, Tr.parent,
                   Tr.child0, Tr.nchild, g, P, (const df64 *)pl->tabdf_binom,
                   (const cx<df64> *)pl->tabdf_dshift, pl->xi, (const cx<df64> *)pl->udf,
                   (const cx<df64> *)pl->qdf, (cx<df64> *)pl->mpole, pl->upcnt,
                   (const int *)nullptr, (int64_t)0);
        LBF_LAUNCH(k_evaluate_tree<df64>, lbf_cdiv(T, kEvalWarps), 32 * kEvalWarps,
                   sizeof(int32_t) * 2 * kEvalFront * kEvalWarps, s, pl->N, pl->M, pl->xi, pl->q,
                   (const cx<df64> *)pl->mpole, P, Tr.level, Tr.ix, Tr.iy, Tr.child0, Tr.nchild,
                   Tr.begin, Tr.end, g, pl->bsig, a, pl->centres, T, t, pl->has_rot, pl->rot_d, u,
                   pl->dev_status);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if (pl->opt.matvec == LBF_MATVEC_FMM && T > 0) {
        // native double: double charges and multipoles, the same tree walk
        int rc = prep(pl, sigma_sorted, Arith::F64, true, nullptr, s);
        if (rc) return rc;
        Tree &Tr = pl->tree;
        BoxGeo g{Tr.xmin, Tr.ymin, Tr.L, (float)(1.0 / Tr.L), df64(1.0 / Tr.L), 1.0 / Tr.L};
        const int P = pl->P, wpb = 2;
        LBF_LAUNCH(fmm::k_up<double>, lbf_cdiv(Tr.nleaf, wpb), 32 * wpb, up_smem<double>(P, wpb), s,
                   Tr.nleaf, Tr.leaves, Tr.level, Tr.ix, Tr.iy, Tr.begin, Tr.end, Tr.parent,
                   Tr.child0, Tr.nchild, g, P, pl->tab_binom, (const cx<double> *)pl->tab_dshift,
                   pl->xi, (const cx<double> *)nullptr, (const cx<double> *)pl->q,
                   (cx<double> *)pl->mpole, pl->upcnt, (const int *)nullptr, (int64_t)0);
        LBF_LAUNCH(k_evaluate_tree<double>, lbf_cdiv(T, kEvalWarps), 32 * kEvalWarps,
                   sizeof(int32_t) * 2 * kEvalFront * kEvalWarps, s, pl->N, pl->M, pl->xi, pl->q,
                   (const cx<double> *)pl->mpole, P, Tr.level, Tr.ix, Tr.iy, Tr.child0, Tr.nchild,
                   Tr.begin, Tr.end, g, pl->bsig, a, pl->centres, T, t, pl->has_rot, pl->rot_d, u,
                   pl->dev_status);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    int rc = prep(pl, sigma_sorted, Arith::F64, true, nullptr, s);
    if (rc) return rc;
    if (T <= 0) return LBF_OK;
    LBF_LAUNCH(k_evaluate, T, 256, 0, s, pl->N, pl->M, pl->xi, pl->q, pl->bsig, a, pl->centres, T,
               t, pl->has_rot, pl->rot_d, u);
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

namespace {
// The Dirichlet data of point vortices in the ocean (Sec. 6, Example 2): the regular part
// psi* of psi = psi* + sum_s Gamma_s G(., v_s) takes g = -sum_s Gamma_s G(x_j, v_s) on the
// curves.  x_j comes back from its planar image in the plan's frame,
// x = (2 Re xi, 2 Im xi, |xi|^2 - 1) / (|xi|^2 + 1), and the vortices are rotated into
// that frame; g is written in the caller's node order.
__global__ void k_vortex_data(int64_t N, const double2 *__restrict__ xi,
                              const int32_t *__restrict__ perm, int64_t S,
                              const double *__restrict__ v, const double *__restrict__ gam,
                              int rot_on, const double *__restrict__ rot, double *__restrict__ g)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 z = xi[i];
    const double r2 = z.x * z.x + z.y * z.y, id = 1.0 / (r2 + 1.0);
    const double x0 = 2.0 * z.x * id, x1 = 2.0 * z.y * id, x2 = (r2 - 1.0) * id;
    double sum = 0.0;
    for (int64_t k = 0; k < S; k++) {
        double p0 = v[3 * k], p1 = v[3 * k + 1], p2 = v[3 * k + 2];
        if (rot_on) {
            const double a = rot[0] * p0 + rot[1] * p1 + rot[2] * p2;
            const double b = rot[3] * p0 + rot[4] * p1 + rot[5] * p2;
            const double c = rot[6] * p0 + rot[7] * p1 + rot[8] * p2;
            p0 = a; p1 = b; p2 = c;
        }
        const double d0 = x0 - p0, d1 = x1 - p1, d2 = x2 - p2;
        sum += gam[k] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
    }
    g[perm[i]] = -sum;
}

// u_t += sum_s Gamma_s G(t, v_s) (the singular part, in the caller's frame)
__global__ void k_green_add(int64_t T, const double *__restrict__ t, int64_t S,
                            const double *__restrict__ p, const double *__restrict__ gm,
                            double *__restrict__ u)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    const double x0 = t[3 * q], x1 = t[3 * q + 1], x2 = t[3 * q + 2];
    double sum = 0.0;
    for (int64_t k = 0; k < S; k++) {
        const double d0 = x0 - p[3 * k], d1 = x1 - p[3 * k + 1], d2 = x2 - p[3 * k + 2];
        sum += gm[k] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
    }
    u[q] += sum;
}

// out_q = (1/2) sum_s Re 1/(xi_q - xi_s), xi = (x1 + i x2)/(1 - x3); a source at the pole
// (1 - x3 <= 0) adds nothing
__global__ void k_dipole_sum(int64_t T, const double *__restrict__ t, int64_t S,
                             const double *__restrict__ p, double *__restrict__ out)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    const double w = 1.0 - t[3 * q + 2];
    const double zx = t[3 * q] / w, zy = t[3 * q + 1] / w;
    double sum = 0.0;
    for (int64_t k = 0; k < S; k++) {
        const double wk = 1.0 - p[3 * k + 2];
        if (!(wk > 0.0)) continue;
        const double dx = zx - p[3 * k] / wk, dy = zy - p[3 * k + 1] / wk;
        sum += dx / (dx * dx + dy * dy);
    }
    out[q] = 0.5 * sum;
}

__global__ void k_selftest_rcp(int64_t n, const double *__restrict__ a, double *__restrict__ out,
                               int variant)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = variant == 0 ? fmm::rcp(a[i]) : fmm::rcp_near(a[i]);
}
}  // namespace

extern "C" int lbf_selftest_rcp(int variant, int64_t n, const double *a, double *out,
                                lbf_stream_t stream)
{
    if ((variant != 0 && variant != 1) || n < 0 || (n > 0 && (!a || !out))) return LBF_EINVAL;
    if (n == 0) return LBF_OK;
    LBF_LAUNCH(k_selftest_rcp, lbf_cdiv(n, 256), 256, 0, (cudaStream_t)stream, n, a, out, variant);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

extern "C" int lbf_point_vortices(lbf_plan *pl, int64_t S, const double *vortices,
                                  const double *gamma, int64_t T, const double *targets, double *u,
                                  double *sigma, double *a, int *iters, double *rel_res,
                                  lbf_stream_t stream)
{
    if (!pl || S < 1 || !vortices || !gamma || T < 0 || (T > 0 && (!targets || !u)) || !sigma || !a)
        return LBF_EINVAL;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    cudaStream_t s = (cudaStream_t)stream;
    // the data into sigma (caller order), then the solve reads it before writing sigma
    LBF_LAUNCH(k_vortex_data, lbf_cdiv(pl->N, 256), 256, 0, s, pl->N, pl->xi, pl->perm, S, vortices,
               gamma, pl->has_rot, pl->rot_d, sigma);
    LBF_CHECK_LAUNCH();
    const int rc = lbf_gmres_impl(pl, sigma, sigma, a, nullptr, iters, rel_res, s, 0);
    if (rc < 0) return rc;
    if (T > 0) {
        const int re = lbf_evaluate(pl, sigma, a, T, targets, u, stream);
        if (re) return re;
        LBF_LAUNCH(k_green_add, lbf_cdiv(T, 128), 128, 0, s, T, targets, S, vortices, gamma, u);
        LBF_CHECK_LAUNCH();
    }
    return rc;
}

extern "C" int lbf_dipole_sum(int64_t T, const double *t, int64_t S, const double *p, double *out,
                              lbf_stream_t stream)
{
    if (T < 0 || S < 0 || (T > 0 && (!t || !out)) || (S > 0 && !p)) return LBF_EINVAL;
    if (T == 0) return LBF_OK;
    LBF_LAUNCH(k_dipole_sum, lbf_cdiv(T, 128), 128, 0, (cudaStream_t)stream, T, t, S, p, out);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
