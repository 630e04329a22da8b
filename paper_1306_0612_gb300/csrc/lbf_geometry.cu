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
                          double2 *__restrict__ w_o,
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

// The same per-node data from planar nodes xi, xi', xi'' (caller's plane)
__global__ void k_planar(int64_t N, int M, const int64_t *__restrict__ ptr,
                         const double *__restrict__ xi, const double *__restrict__ dxi,
                         const double *__restrict__ d2xi, double2 *__restrict__ xi_o,
                         double2 *__restrict__ w_o, double *__restrict__ d_o,
                         double *__restrict__ b_o)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int k = island_of(ptr, M, j);
    double h = 2.0 * LBF_PI / (double)(ptr[k + 1] - ptr[k]);
    double xr = xi[2 * j], xim = xi[2 * j + 1];
    double ar = dxi[2 * j], ai = dxi[2 * j + 1];
    double br = d2xi[2 * j], bi = d2xi[2 * j + 1];
    xi_o[j] = make_double2(xr, xim);
    w_o[j] = make_double2(h * ar, h * ai);
    d_o[j] = (h / (4.0 * LBF_PI)) * (bi * ar - br * ai) / (ar * ar + ai * ai);
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
// ---- inverse of the Schur complement ---------------------------------------------------
//
// Gauss-Jordan elimination with partial pivoting (row interchanges), all M steps in
// one cooperative launch.  Step k reads matrix A_k and writes A_(k+1) (two buffers
// in turn), so every block takes the pivot row p, row k and column k straight from
// A_k and one grid barrier per step suffices:
//   row k:       A'_kj = A_pj / A_pk                   (A'_kk = 1 / A_pk)
//   row i != k:  A'_ij = B_ij - B_ik A_pj / A_pk,  A'_ik = -B_ik / A_pk,
// B being A_k with rows k and p interchanged.  The same pass forms each block's
// partial maximum of |A'_i,k+1|, i > k (two sets of partials, by step parity, so a
// block never overwrites values another block is still reducing).  Every block
// reduces the partials the same way, so all agree on the next pivot.  The
// interchanges are undone at the end by swapping columns k and p, k = M-1, ..., 0.
//
// The grid barrier is a counter and a generation word; every block is resident
// (cooperative launch), and each wait gives up after kBarrierSpins polls, setting
// status bit LBF_DEV_TIMEOUT, so the kernel always ends.

constexpr unsigned kBarrierSpins = 1u << 22;
constexpr int kGjThreads = 512;
constexpr int kGjMaxBlocks = 1024;

struct GridBarrier {
    unsigned count, gen;
};

__device__ bool grid_barrier(GridBarrier *bar, unsigned nb, int *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = &bar->gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nb - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == g) {
                if (++it > kBarrierSpins) {
                    atomicOr(status, LBF_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int *)status & LBF_DEV_TIMEOUT) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// block-wide (max |value|, smallest index) reduction; result valid in every thread
__device__ void block_argmax(double &v, int &idx, double *sv, int *si)
{
    const int t = threadIdx.x;
    sv[t] = v;
    si[t] = idx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            double a = sv[t + o];
            int i = si[t + o];
            if (a > sv[t] || (a == sv[t] && i < si[t])) {
                sv[t] = a;
                si[t] = i;
            }
        }
        __syncthreads();
    }
    v = sv[0];
    idx = si[0];
    __syncthreads();
}

__global__ void __launch_bounds__(kGjThreads)
k_gj_coop(int M, double *A0, double *A1, double *pval, int *pidx, double *amax, int *pivrow,
          GridBarrier *bar, int *status)
{
    __shared__ double sv[kGjThreads];
    __shared__ int si[kGjThreads];
    const unsigned nb = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)nb * blockDim.x;
    const int64_t MM = (int64_t)M * M;
    const int i0 = (int)(tid / M), j0 = (int)(tid % M);
    const int di = (int)(nthr / M), dj = (int)(nthr % M);
    // partial maxima of column 0 (parity 0) and of every |S_ij|
    {
        double best = -1.0, big = 0.0;
        int bi = M, unused = 0;
        for (int64_t i = tid; i < M; i += nthr) {
            double a = fabs(A0[i * M]);
            if (a > best) { best = a; bi = (int)i; }
        }
        for (int64_t e = tid; e < MM; e += nthr) big = fmax(big, fabs(A0[e]));
        block_argmax(best, bi, sv, si);
        block_argmax(big, unused, sv, si);
        if (threadIdx.x == 0) {
            pval[blockIdx.x] = best;
            pidx[blockIdx.x] = bi;
            amax[blockIdx.x] = big;
        }
    }
    if (!grid_barrier(bar, nb, status)) return;
    // a pivot at or below M 2^-52 max|S_ij| counts as zero: S is singular to double precision
    double tiny = 0.0;
    for (unsigned q = 0; q < nb; q++) tiny = fmax(tiny, __ldcg(&amax[q]));
    tiny *= (double)M * 0x1p-52;
    for (int k = 0; k < M; k++) {
        const double *Ain = (k & 1) ? A1 : A0;
        double *Aout = (k & 1) ? A0 : A1;
        const double *pv = pval + (k & 1) * kGjMaxBlocks;
        const int *pi = pidx + (k & 1) * kGjMaxBlocks;
        double best = -1.0;
        int p = M;
        for (unsigned q = threadIdx.x; q < nb; q += blockDim.x) {
            double a = __ldcg(&pv[q]);
            int i = __ldcg(&pi[q]);
            if (a > best || (a == best && i < p)) { best = a; p = i; }
        }
        block_argmax(best, p, sv, si);
        if (!(best > tiny) || p >= M) {  // every block sees the same value: all stop here
            if (tid == 0) atomicOr(status, 4);
            return;
        }
        if (tid == 0) pivrow[k] = p;
        const double ipiv = 1.0 / __ldcg(&Ain[(int64_t)p * M + k]);
        const double *rowp = Ain + (int64_t)p * M;
        double nbest = -1.0;
        int ni = M;
        // four elements per pass, their loads issued before any is used (the loop is
        // bound by L2 latency); (i, j) of element e advanced without dividing
        int i = i0, j = j0;
        for (int64_t e = tid; e < MM; e += 4 * nthr) {
            int64_t ee[4];
            int ii[4], jj[4];
            double fa[4], aa[4], rp[4];
            for (int u = 0; u < 4; u++) {
                ee[u] = e + u * nthr;
                ii[u] = i;
                jj[u] = j;
                i += di;
                j += dj;
                if (j >= M) { j -= M; i++; }
            }
            for (int u = 0; u < 4; u++) {
                fa[u] = aa[u] = rp[u] = 0.0;
                if (ee[u] < MM && ii[u] != k) {
                    const int src = (ii[u] == p) ? k : ii[u];  // row i of B
                    fa[u] = __ldcg(&Ain[(int64_t)src * M + k]);
                    if (jj[u] != k) aa[u] = __ldcg(&Ain[(int64_t)src * M + jj[u]]);
                }
                if (ee[u] < MM && jj[u] != k) rp[u] = __ldcg(&rowp[jj[u]]);
            }
            for (int u = 0; u < 4; u++) {
                if (ee[u] >= MM) break;
                double val;
                if (ii[u] == k) val = (jj[u] == k) ? ipiv : rp[u] * ipiv;
                else if (jj[u] == k) val = -fa[u] * ipiv;
                else val = fma(-fa[u] * ipiv, rp[u], aa[u]);
                Aout[ee[u]] = val;
                if (jj[u] == k + 1 && ii[u] > k) {
                    double av = fabs(val);
                    if (av > nbest || (av == nbest && ii[u] < ni)) { nbest = av; ni = ii[u]; }
                }
            }
        }
        block_argmax(nbest, ni, sv, si);
        if (threadIdx.x == 0) {
            pval[((k + 1) & 1) * kGjMaxBlocks + blockIdx.x] = nbest;
            pidx[((k + 1) & 1) * kGjMaxBlocks + blockIdx.x] = ni;
        }
        if (!grid_barrier(bar, nb, status)) return;
    }
}

__global__ void k_gj_init(int M, int *__restrict__ pivrow)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) pivrow[k] = k;
}

// undo the row interchanges: swap columns k and pivrow[k] for k = M-1, ..., 0 (thread per
// row).  pivrow starts as the identity, so steps an early stop (a singular pivot or a
// barrier that gave up) never reached swap nothing.
__global__ void k_gj_unscramble(int M, double *__restrict__ A, const int *__restrict__ pivrow)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    double *row = A + i * M;
    for (int k = M - 1; k >= 0; k--) {
        int p = pivrow[k];
        if (p != k && p >= 0 && p < M) {
            double t = row[k];
            row[k] = row[p];
            row[p] = t;
        }
    }
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
                       const double *centres, int planar, cudaStream_t s, double2 *xi_o,
                       double2 *w_o, double *d_o, double *b_o)
{
    int64_t N = pl->N;
    Rot R = make_rot(pl);
    if (planar)
        LBF_LAUNCH(k_planar, lbf_cdiv(N, 256), 256, 0, s, N, pl->M, pl->island_ptr, x, dx, d2x,
                   xi_o, w_o, d_o, b_o);
    else
        LBF_LAUNCH(k_project, lbf_cdiv(N, 256), 256, 0, s, N, pl->M, pl->island_ptr, x, dx, d2x,
                   R, xi_o, w_o, d_o, b_o, pl->dev_status);
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
// inverse in place by Gauss-Jordan elimination with partial pivoting.
size_t lbf_gj_scratch_doubles(int M)
{
    return (size_t)M * M + 5 * (size_t)kGjMaxBlocks + (size_t)M + 64;
}

int lbf_border_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, double *scratch,
                     int32_t *work, int64_t work_len, const SortBufs &sb)
{
    int M = pl->M;
    double *S = pl->Sinv;
    lbf_prof_mark(LBF_STAGE_BORDER, 1, s);
    int rc = lbf_mp_build(pl, s, xi_o, S, work, work_len, sb);
    lbf_prof_mark(LBF_STAGE_BORDER, 0, s);
    if (rc) return rc;
    lbf_prof_mark(LBF_STAGE_INVERSE, 1, s);
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    LBF_CUDA(cudaGetDevice(&dev));
    LBF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    LBF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    LBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_coop, kGjThreads, 0));
    if (!coop || per_sm < 1) return LBF_ECUDA;
    // one block per SM: every SM's double pipe busy, one barrier arrival per SM
    int64_t want = lbf_cdiv((int64_t)M * M, (int64_t)kGjThreads);
    int nb = (int)std::min<int64_t>(std::min<int64_t>(nsm, kGjMaxBlocks), std::max<int64_t>(want, 1));
    double *S1 = scratch;                         // the second M x M buffer
    double *pval = scratch + (size_t)M * M;       // 2 x kGjMaxBlocks
    int *pidx = (int *)(pval + 2 * kGjMaxBlocks); // 2 x kGjMaxBlocks
    double *amax = (double *)(pidx + 2 * kGjMaxBlocks);  // kGjMaxBlocks
    int *pivrow = (int *)(amax + kGjMaxBlocks);   // M
    GridBarrier *bar = (GridBarrier *)(pivrow + M + (M & 1));
    LBF_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s));
    LBF_LAUNCH(k_gj_init, lbf_cdiv(M, 256), 256, 0, s, M, pivrow);
    int *status = pl->dev_status;
    void *args[] = {&M, &S, &S1, &pval, &pidx, &amax, &pivrow, &bar, &status};
    LBF_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_coop, dim3(nb), dim3(kGjThreads), args,
                                         0, s));
    g_lbf_launches.fetch_add(1, std::memory_order_relaxed);
    // after M steps the result is in the buffer step M wrote
    if (M & 1) LBF_CUDA(cudaMemcpyAsync(S, S1, sizeof(double) * (size_t)M * M, cudaMemcpyDeviceToDevice, s));
    LBF_LAUNCH(k_gj_unscramble, lbf_cdiv(M, 128), 128, 0, s, M, S, pivrow);
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
