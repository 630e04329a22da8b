// Per-node precompute (Sec. 3 and Sec. 5) and the inverse Schur complement of
// the block preconditioner (Sec. 5).
#include "lbf_internal.cuh"

namespace {

__device__ __forceinline__ int island_of(const int64_t *ptr, int M, int64_t j)
{
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ptr[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Rot {
    double r[9];
    int on;
};

__device__ __forceinline__ void rotate(const Rot &R, double *v)
{
    if (!R.on) return;
    double a = R.r[0] * v[0] + R.r[1] * v[1] + R.r[2] * v[2];
    double b = R.r[3] * v[0] + R.r[4] * v[1] + R.r[5] * v[2];
    double c = R.r[6] * v[0] + R.r[7] * v[1] + R.r[8] * v[2];
    v[0] = a; v[1] = b; v[2] = c;
}

// Stereographic projection xi = (x1 + i x2)/(1 - x3) with its first two
// alpha-derivatives by the chain rule (Sec. 3), and the per-node Nystrom data
// (Sec. 5, Eq. disc_sphere with the Cauchy sign of Eq. dlpC corrected):
//   w_j    = h xi'_j                               (complex trapezoidal weight)
//   dself_j = (h/4pi) Im(xi''_j / xi'_j)           (diagonal limit, Eq. cont_kern)
//   beta_j = -(h/2pi) Im(conj(xi_j) xi'_j / (1 + |xi_j|^2))  (sphere correction)
__global__ void k_project(int64_t N, int M, const int64_t *__restrict__ ptr,
                          const double *__restrict__ x, const double *__restrict__ dx,
                          const double *__restrict__ d2x, Rot R, double2 *__restrict__ xi_o,
                          double *__restrict__ x3_o, double2 *__restrict__ w_o,
                          double *__restrict__ d_o, double *__restrict__ b_o,
                          int *__restrict__ status)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int k = island_of(ptr, M, j);
    double h = 2.0 * LBF_PI / (double)(ptr[k + 1] - ptr[k]);
    double p0[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
    double p1[3] = {dx[3 * j], dx[3 * j + 1], dx[3 * j + 2]};
    double p2[3] = {d2x[3 * j], d2x[3 * j + 1], d2x[3 * j + 2]};
    rotate(R, p0);
    rotate(R, p1);
    rotate(R, p2);
    x3_o[3 * j] = p0[0];
    x3_o[3 * j + 1] = p0[1];
    x3_o[3 * j + 2] = p0[2];
    double w = __dsub_rn(1.0, p0[2]);
    if (!(w >= 1e-12)) {
        atomicOr(status, LBF_DEV_POLE);
        w = 1e-12;
    }
    // xi itself is two correctly rounded quotients (the quadtree keys depend on its bits)
    double xr = __ddiv_rn(p0[0], w), xim = __ddiv_rn(p0[1], w);
    double wp = -p1[2], wpp = -p2[2];
    double iw = 1.0 / w, iw2 = iw * iw, iw3 = iw2 * iw;
    // xi' = z'/w - z w'/w^2
    double ar = p1[0] * iw - p0[0] * wp * iw2;
    double ai = p1[1] * iw - p0[1] * wp * iw2;
    // xi'' = z''/w - 2 z' w'/w^2 - z w''/w^2 + 2 z w'^2/w^3
    double br = p2[0] * iw - 2.0 * p1[0] * wp * iw2 - p0[0] * wpp * iw2 + 2.0 * p0[0] * wp * wp * iw3;
    double bi = p2[1] * iw - 2.0 * p1[1] * wp * iw2 - p0[1] * wpp * iw2 + 2.0 * p0[1] * wp * wp * iw3;
    xi_o[j] = make_double2(xr, xim);
    w_o[j] = make_double2(h * ar, h * ai);
    double a2 = ar * ar + ai * ai;
    // Im(xi''/xi') = Im(xi'' conj(xi'))/|xi'|^2
    d_o[j] = (h / (4.0 * LBF_PI)) * (bi * ar - br * ai) / a2;
    // Im(conj(xi) xi') = xr*ai - xim*ar
    b_o[j] = -(h / (2.0 * LBF_PI)) * (xr * ai - xim * ar) / (1.0 + xr * xr + xim * xim);
}

__global__ void k_gather_nodes(int64_t N, const int32_t *__restrict__ perm,
                               const double2 *__restrict__ xi_o, const double2 *__restrict__ w_o,
                               const double *__restrict__ d_o, const double *__restrict__ b_o,
                               double2 *__restrict__ xi, double2 *__restrict__ w,
                               double *__restrict__ d, double *__restrict__ b,
                               int32_t *__restrict__ rank)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t j = perm[i];
    xi[i] = xi_o[j];
    w[i] = w_o[j];
    d[i] = d_o[j];
    b[i] = b_o[j];
    rank[j] = (int32_t)i;
}

__global__ void k_rotate_centres(int M, const double *__restrict__ c, Rot R, double *__restrict__ out)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double v[3] = {c[3 * m], c[3 * m + 1], c[3 * m + 2]};
    rotate(R, v);
    out[3 * m] = v[0];
    out[3 * m + 1] = v[1];
    out[3 * m + 2] = v[2];
}

// Gauss-Jordan step k on [S | I] (M x 2M, row-major): partial pivoting on column
// k, swap, scale the pivot row.  One block.
__global__ void k_gj_pivot(int M, int k, double *__restrict__ G, int *__restrict__ status)
{
    __shared__ double sval[1024];
    __shared__ int sidx[1024];
    int t = threadIdx.x;
    double best = -1.0;
    int bi = M;
    for (int i = k + t; i < M; i += blockDim.x) {
        double a = fabs(G[(int64_t)i * 2 * M + k]);
        if (a > best || (a == best && i < bi)) { best = a; bi = i; }
    }
    sval[t] = best;
    sidx[t] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            double a = sval[t + o];
            int i = sidx[t + o];
            if (a > sval[t] || (a == sval[t] && i < sidx[t])) { sval[t] = a; sidx[t] = i; }
        }
        __syncthreads();
    }
    int p = sidx[0];
    double piv = G[(int64_t)p * 2 * M + k];
    if (t == 0 && !(fabs(piv) > 0.0)) atomicOr(status, 4);
    double inv = 1.0 / piv;
    for (int j = t; j < 2 * M; j += blockDim.x) {
        double a = G[(int64_t)k * 2 * M + j];
        double b = G[(int64_t)p * 2 * M + j];
        if (p != k) G[(int64_t)p * 2 * M + j] = a;
        G[(int64_t)k * 2 * M + j] = b * inv;
    }
}

__global__ void k_gj_elim(int M, int k, double *__restrict__ G)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t ncol = 2 * M - (k + 1);
    if (id >= (int64_t)M * ncol) return;
    int i = (int)(id / ncol);
    int j = k + 1 + (int)(id % ncol);
    if (i == k) return;
    double f = G[(int64_t)i * 2 * M + k];
    G[(int64_t)i * 2 * M + j] -= f * G[(int64_t)k * 2 * M + j];
}

__global__ void k_copy_inverse(int M, const double *__restrict__ G, double *__restrict__ Sinv)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)M * M) return;
    int i = (int)(id / M), j = (int)(id % M);
    Sinv[id] = G[(int64_t)i * 2 * M + M + j];
}

__global__ void k_geometry_out(int64_t N, const int32_t *__restrict__ rank,
                               const double2 *__restrict__ xi, const double2 *__restrict__ w,
                               double *__restrict__ xi_out, double *__restrict__ nrm,
                               double *__restrict__ wout, double *__restrict__ arc)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int32_t i = rank[j];
    double2 z = xi[i], ww = w[i];
    double a = sqrt(ww.x * ww.x + ww.y * ww.y);
    if (xi_out) { xi_out[2 * j] = z.x; xi_out[2 * j + 1] = z.y; }
    // -i w/|w|: the unit normal pointing into the island (it lies to the right of the curve)
    if (nrm) { nrm[2 * j] = ww.y / a; nrm[2 * j + 1] = -ww.x / a; }
    if (wout) { wout[2 * j] = ww.x; wout[2 * j + 1] = ww.y; }
    if (arc) arc[j] = a;
}

Rot make_rot(const lbf_plan *pl)
{
    Rot R;
    R.on = pl->has_rot;
    for (int i = 0; i < 9; i++) R.r[i] = pl->rot[i];
    return R;
}

}  // namespace

int lbf_geometry_build(lbf_plan *pl, const double *x, const double *dx, const double *d2x,
                       const double *centres, cudaStream_t s, double2 *xi_o, double *x3_o,
                       double2 *w_o, double *d_o, double *b_o)
{
    int64_t N = pl->N;
    Rot R = make_rot(pl);
    LBF_LAUNCH(k_project, lbf_cdiv(N, 256), 256, 0, s, N, pl->M, pl->island_ptr, x, dx, d2x, R,
               xi_o, x3_o, w_o, d_o, b_o, pl->dev_status);
    LBF_CHECK_LAUNCH();
    LBF_LAUNCH(k_rotate_centres, lbf_cdiv(pl->M, 128), 128, 0, s, pl->M, centres, R, pl->centres);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_geometry_gather(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, const double2 *w_o,
                        const double *d_o, const double *b_o)
{
    int64_t N = pl->N;
    LBF_LAUNCH(k_gather_nodes, lbf_cdiv(N, 256), 256, 0, s, N, pl->perm, xi_o, w_o, d_o, b_o,
               pl->xi, pl->w, pl->dself, pl->beta, pl->rank);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// S = D - F E from the island expansions of the multiplier potential, then its
// inverse by Gauss-Jordan elimination with partial pivoting.
int lbf_border_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, double *scratch,
                     int32_t *work, int64_t work_len)
{
    int M = pl->M;
    double *G = scratch;  // M x 2M
    lbf_prof_mark(LBF_STAGE_BORDER, 1, s);
    int rc = lbf_mp_build(pl, s, xi_o, G, work, work_len);
    lbf_prof_mark(LBF_STAGE_BORDER, 0, s);
    if (rc) return rc;
    lbf_prof_mark(LBF_STAGE_INVERSE, 1, s);
    for (int k = 0; k < M; k++) {
        LBF_LAUNCH(k_gj_pivot, 1, 1024, 0, s, M, k, G, pl->dev_status);
        int64_t work = (int64_t)M * (2 * M - (k + 1));
        if (work > 0) LBF_LAUNCH(k_gj_elim, lbf_cdiv(work, 256), 256, 0, s, M, k, G);
    }
    LBF_CHECK_LAUNCH();
    LBF_LAUNCH(k_copy_inverse, lbf_cdiv((int64_t)M * M, 256), 256, 0, s, M, G, pl->Sinv);
    LBF_CHECK_LAUNCH();
    lbf_prof_mark(LBF_STAGE_INVERSE, 0, s);
    return LBF_OK;
}

int lbf_geometry_out_impl(const lbf_plan *pl, double *xi, double *normal, double *weight,
                          double *arc, cudaStream_t s)
{
    int64_t N = pl->N;
    LBF_LAUNCH(k_geometry_out, lbf_cdiv(N, 256), 256, 0, s, N, pl->rank, pl->xi, pl->w, xi,
               normal, weight, arc);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
