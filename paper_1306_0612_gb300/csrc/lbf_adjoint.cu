// Adjoint of the solve-and-evaluate map (Sec. 4.1, Eq. u_multi; Sec. 5, Eq. disc_sphere):
// the transposed evaluation at off-curve targets and the gradient of a target
// functional with respect to the planar node positions xi_j (xi'_j, xi''_j fixed).
//
// With A z = b (z = [sigma; a], b = [2 g; 0]) and u = C z at the targets, a scalar
// L(u) with ubar = dL/du has dL/dg = 2 lam_sigma where A^T lam = C^T ubar, and
//   dL/dxi_j = d/dxi_j (ubar^T C z) - lam^T (dA/dxi_j) z.
// Every term is a Cauchy-type sum (the derivative FMM), a node-target sum, or the
// gradient of the multiplier potential; they are combined per node below.
#include "lbf_internal.cuh"

namespace {

__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Rot3 {
    double r[9];
    int on;
};

// target t on the sphere -> the plan's frame; xi_t, or w <= 0 at the pole
__device__ __forceinline__ void target_plane(const double *t, int64_t k, const Rot3 &R, double p[3],
                                             double &zx, double &zy, bool &finite)
{
    p[0] = t[3 * k];
    p[1] = t[3 * k + 1];
    p[2] = t[3 * k + 2];
    if (R.on) {
        double a = R.r[0] * p[0] + R.r[1] * p[1] + R.r[2] * p[2];
        double b = R.r[3] * p[0] + R.r[4] * p[1] + R.r[5] * p[2];
        double c = R.r[6] * p[0] + R.r[7] * p[1] + R.r[8] * p[2];
        p[0] = a; p[1] = b; p[2] = c;
    }
    double w = 1.0 - p[2];
    finite = w > 0.0;
    zx = finite ? p[0] / w : 0.0;
    zy = finite ? p[1] / w : 0.0;
}

// per node (sorted): S1 = sum_t ubar_t/(xi - xi_t), S2 = sum_t ubar_t/(xi - xi_t)^2
// (targets tiled through shared memory, projected by each block)
__global__ void k_node_target(int64_t N, const double2 *__restrict__ xi, int64_t T,
                              const double *__restrict__ t, Rot3 R, const double *__restrict__ ub,
                              double2 *__restrict__ S1, double2 *__restrict__ S2)
{
    __shared__ double2 tz[256];
    __shared__ double tu[256];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double2 z = i < N ? xi[i] : make_double2(0, 0);
    double a1r = 0, a1i = 0, a2r = 0, a2i = 0;
    for (int64_t base = 0; base < T; base += 256) {
        __syncthreads();
        int64_t k = base + threadIdx.x;
        if (k < T) {
            double p[3], zx, zy;
            bool fin;
            target_plane(t, k, R, p, zx, zy, fin);
            tz[threadIdx.x] = make_double2(zx, zy);
            tu[threadIdx.x] = fin ? ub[k] : 0.0;  // a target at the pole has no Cauchy term
        }
        __syncthreads();
        int n = (int)(T - base < 256 ? T - base : 256);
        for (int m = 0; m < n; m++) {
            const double dr = z.x - tz[m].x, di = z.y - tz[m].y;
            const double id = 1.0 / fma(dr, dr, di * di);
            // 1/d = conj(d)/|d|^2, 1/d^2 = conj(d)^2/|d|^4
            const double er = dr * id, ei = -di * id;
            a1r = fma(tu[m], er, a1r);
            a1i = fma(tu[m], ei, a1i);
            a2r = fma(tu[m], er * er - ei * ei, a2r);
            a2i = fma(tu[m], 2.0 * er * ei, a2i);
        }
    }
    if (i < N) {
        S1[i] = make_double2(a1r, a1i);
        S2[i] = make_double2(a2r, a2i);
    }
}

// s[0] = sum ubar, s[1] = sum lam_sigma (lam nullable), s[2] = sum a (a nullable); one block
__global__ void k_sums3(int64_t T, const double *__restrict__ ub, int64_t N,
                        const double *__restrict__ lam, int M, const double *__restrict__ a,
                        double *__restrict__ s)
{
    __shared__ double sh[3][32];
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t k = threadIdx.x; k < T; k += blockDim.x) v[0] += ub[k];
    if (lam)
        for (int64_t k = threadIdx.x; k < N; k += blockDim.x) v[1] += lam[k];
    if (a)
        for (int64_t k = threadIdx.x; k < M; k += blockDim.x) v[2] += a[k];
    for (int c = 0; c < 3; c++) {
        double x = wsum(v[c]);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += sh[threadIdx.x][w];
        s[threadIdx.x] = x;
    }
}

// sbar_i = (1/2pi) Im(w_i S1_i) + beta_i sum ubar  (sorted i -> caller perm[i])
__global__ void k_sbar(int64_t N, const int32_t *__restrict__ perm, const double2 *__restrict__ w,
                       const double *__restrict__ beta, const double2 *__restrict__ S1,
                       const double *__restrict__ s, double *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 ww = w[i], a = S1[i];
    out[perm[i]] = (ww.x * a.y + ww.y * a.x) * (1.0 / (2.0 * LBF_PI)) + beta[i] * s[0];
}

// abar_m = sum_t ubar_t G(t, c_m), G = (1/4pi) log(2 / |t - c|^2) (Eq. greens_func); warp per centre
__global__ void k_abar(int M, const double *__restrict__ c, int64_t T, const double *__restrict__ t,
                       Rot3 R, const double *__restrict__ ub, double *__restrict__ out)
{
    int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (m >= M) return;
    double acc = 0.0;
    for (int64_t k = lane; k < T; k += 32) {
        double p[3], zx, zy;
        bool fin;
        target_plane(t, k, R, p, zx, zy, fin);
        double d0 = p[0] - c[3 * m], d1 = p[1] - c[3 * m + 1], d2 = p[2] - c[3 * m + 2];
        acc += ub[k] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
    }
    acc = wsum(acc);
    if (lane == 0) out[m] = acc;
}

// gradient of beta_i = -(1/2pi) (X w_y - Y w_x) / (1 + X^2 + Y^2) in (X, Y) = xi_i
__device__ __forceinline__ double2 grad_beta(double2 z, double2 w)
{
    const double num = z.x * w.y - z.y * w.x, den = 1.0 + z.x * z.x + z.y * z.y;
    const double k = -1.0 / (2.0 * LBF_PI * den * den);
    return make_double2(k * (w.y * den - 2.0 * z.x * num), k * (-w.x * den - 2.0 * z.y * num));
}

// dL/dxi_i, sorted i -> caller perm[i] (N x 2):
//   (a)  Im/Re of  -(w_i sigma_i/2pi) S2_i        + U sigma_i grad beta_i        (evaluation)
//   (b1) -2 Im/Re of (w_i sigma_i/2pi) Dlam_i                                     (i as a source)
//   (b2) +2 lam_i Im/Re of (1/2pi) Dq_i                                           (i as a target)
//   (b3) -2 Lam sigma_i grad beta_i                                               (sphere correction)
//   (b4) -lam_i grad (E a)_i                                                      (multiplier potential)
// with Dlam = Phi'_lam, Dq = Phi'_(w sigma), U = sum ubar, Lam = sum lam_sigma.
__global__ void k_grad(int64_t N, const int32_t *__restrict__ perm, const double2 *__restrict__ xi,
                       const double2 *__restrict__ w, const double *__restrict__ sig,
                       const double *__restrict__ lam, const double2 *__restrict__ S2,
                       const double2 *__restrict__ Dl, const double2 *__restrict__ Dq,
                       const double2 *__restrict__ Eg, const double *__restrict__ s,
                       double *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double k = 1.0 / (2.0 * LBF_PI);
    const double2 ww = w[i], z = xi[i];
    const double sg = sig[i], lm = lam[i];
    // c = w_i sigma_i / 2pi
    const double cr = ww.x * sg * k, ci = ww.y * sg * k;
    auto cm = [](double ar, double ai, double br, double bi, double &rr, double &ri) {
        rr = ar * br - ai * bi;
        ri = ar * bi + ai * br;
    };
    double gr, gi;  // (Im F', Re F') convention: d/dX = Im F', d/dY = Re F'
    double gx = 0.0, gy = 0.0;
    cm(cr, ci, S2[i].x, S2[i].y, gr, gi);  // (a): F' = -c S2
    gx += -gi;
    gy += -gr;
    cm(cr, ci, Dl[i].x, Dl[i].y, gr, gi);  // (b1): H = c Dlam, contributes -2 (Im H, Re H)
    gx -= 2.0 * gi;
    gy -= 2.0 * gr;
    // (b2): Q = -(1/2pi) Dq, contributes -2 lam (Im Q, Re Q)
    gx += 2.0 * lm * k * Dq[i].y;
    gy += 2.0 * lm * k * Dq[i].x;
    const double2 gb = grad_beta(z, ww);
    const double fb = (s[0] - 2.0 * s[1]) * sg;  // (a) beta term and (b3)
    gx += fb * gb.x;
    gy += fb * gb.y;
    gx -= lm * Eg[i].x;  // (b4)
    gy -= lm * Eg[i].y;
    const int32_t j = perm[i];
    out[2 * j] = gx;
    out[2 * j + 1] = gy;
}

Rot3 plan_rot(const lbf_plan *pl)
{
    Rot3 R;
    R.on = pl->has_rot;
    for (int i = 0; i < 9; i++) R.r[i] = pl->rot[i];
    return R;
}

// dL/dg_j = 2 lam_j: the Dirichlet data enter the bordered system only through its
// doubled right-hand side [2 g; 0] (Eq. disc_sphere), so the adjoint of b -> z carries
// the factor 2 onto the node part of lam (caller order in and out)
__global__ void k_grad_data(int64_t N, const double *__restrict__ lam, double *__restrict__ gg)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < N) gg[j] = 2.0 * lam[j];
}

}  // namespace

int lbf_gradient_data_impl(lbf_plan *pl, const double *lam, double *grad_g, cudaStream_t s)
{
    if (pl->N > 0) LBF_LAUNCH(k_grad_data, lbf_cdiv(pl->N, 256), 256, 0, s, pl->N, lam, grad_g);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_evaluate_transpose_impl(lbf_plan *pl, int64_t T, const double *t, const double *ub,
                                double *sbar, double *abar, cudaStream_t s)
{
    int64_t N = pl->N;
    int M = pl->M;
    // scratch: the GMRES basis region (unused outside a solve)
    double2 *S1 = (double2 *)pl->region, *S2 = S1 + N;
    double *sums = (double *)(S2 + N);
    Rot3 R = plan_rot(pl);
    LBF_LAUNCH(k_sums3, 1, 1024, 0, s, T, ub, N, (const double *)nullptr, M,
               (const double *)nullptr, sums);
    LBF_LAUNCH(k_node_target, lbf_cdiv(N, 256), 256, 0, s, N, pl->xi, T, t, R, ub, S1, S2);
    LBF_LAUNCH(k_sbar, lbf_cdiv(N, 256), 256, 0, s, N, pl->perm, pl->w, pl->beta, S1, sums, sbar);
    if (abar) LBF_LAUNCH(k_abar, lbf_cdiv((int64_t)M * 32, 256), 256, 0, s, M, pl->centres, T, t, R, ub, abar);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_gradient_nodes_impl(lbf_plan *pl, const double *sigma, const double *a, const double *lam,
                            int64_t T, const double *t, const double *ub, double *grad,
                            cudaStream_t s)
{
    int64_t N = pl->N;
    int M = pl->M;
    double2 *S1 = (double2 *)pl->region, *S2 = S1 + N, *Dl = S2 + N, *Dq = Dl + N, *Eg = Dq + N;
    double *sg = (double *)(Eg + N), *lm = sg + N, *sums = lm + N;
    Rot3 R = plan_rot(pl);
    int rc;
    if ((rc = lbf_permute_in(pl, sigma, sg, 0, s)) || (rc = lbf_permute_in(pl, lam, lm, 0, s)))
        return rc;
    LBF_LAUNCH(k_sums3, 1, 1024, 0, s, T, ub, N, lm, M, a, sums);
    LBF_LAUNCH(k_node_target, lbf_cdiv(N, 256), 256, 0, s, N, pl->xi, T, t, R, ub, S1, S2);
    LBF_CHECK_LAUNCH();
    if ((rc = lbf_cauchy_deriv(pl, lm, false, Dl, s))) return rc;
    if ((rc = lbf_cauchy_deriv(pl, sg, true, Dq, s))) return rc;
    if ((rc = lbf_mp_gradient(pl, a, Eg, s))) return rc;
    LBF_LAUNCH(k_grad, lbf_cdiv(N, 256), 256, 0, s, N, pl->perm, pl->xi, pl->w, sg, lm, S2, Dl, Dq,
               Eg, sums, grad);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
