// Bordered operator, block preconditioner and device-resident restarted GMRES
// (Sec. 5, Eq. matrix_eqns and matrix_eqns_c).
//
// Unknowns live in the plan's sorted (Morton) node order: x = [sigma (N); a (M)].
//   A x       = [sigma + v + E a ; F sigma + D a],   v = K sigma (lbf_apply_K)
//   P         = [[I, E], [F, D]],  S = D - F E
//   P^-1 r    : z_a = S^-1 (r_a - F r_sigma),  z_sigma = r_sigma - E z_a
// The preconditioned operator is applied in the algebraically equal form
//   P^-1 A x  = x + P^-1 [v; 0] = [sigma + v + E y ; a - y],  y = S^-1 F v,
// which needs one pass over E per matvec instead of two.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "lbf_internal.cuh"

struct GmresState {
    int go;         // 1 while Arnoldi steps of the current cycle may run (kernel gate)
    int j;          // Arnoldi columns completed in the current cycle
    int it;         // iterations completed in total
    int converged;  // 1 once the preconditioned residual reached tol
    int maxit, m;
    double tol, bnorm, beta, resid, inv;
};

namespace {

constexpr int kRowsPerChunk = 1024;
constexpr int kDotBlocks = 152 * 2;

__device__ __forceinline__ bool gate_closed(const int *gate) { return gate && *gate == 0; }

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_permute_in(int64_t N, int M, const int32_t *__restrict__ perm,
                             const double *__restrict__ in, double *__restrict__ out, int with_a)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) out[i] = in[perm[i]];
    else if (with_a && i < N + M) out[i] = in[i];
}

__global__ void k_permute_out(int64_t N, int M, const int32_t *__restrict__ perm,
                              const double *__restrict__ in, double *__restrict__ out, int with_a)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) out[perm[i]] = in[i];
    else if (with_a && i < N + M) out[i] = in[i];
}

// F u: the unweighted constraint sums over islands 1..M-1 (Eq. disc_constr), in a
// fixed order (caller order within the island).  Row M-1 of F is zero.
__global__ void k_island_sums(int M, const int64_t *__restrict__ ptr, const int32_t *__restrict__ rank,
                              const double *__restrict__ u, double scale, double *__restrict__ out,
                              const int *gate, int64_t slab)
{
    lbf_rhs(slab, u, out, gate);
    if (gate_closed(gate)) return;
    int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= M) return;
    double s = 0.0;
    if (r < M - 1)
        for (int64_t j = ptr[r + 1] + lane; j < ptr[r + 2]; j += 32) s += u[rank[j]];
    s = warp_sum(s);
    if (lane == 0) out[r] = scale * s;
}

// y = alpha S^-1 f (one warp per row)
__global__ void k_small_gemv(int M, const double *__restrict__ A, const double *__restrict__ f,
                             double alpha, double *__restrict__ y, const int *gate, int64_t slab)
{
    lbf_rhs(slab, f, y, gate);
    if (gate_closed(gate)) return;
    int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= M) return;
    double s = 0.0;
    for (int m = lane; m < M; m += 32) s = fma(A[(int64_t)r * M + m], f[m], s);
    s = warp_sum(s);
    if (lane == 0) y[r] = alpha * s;
}

__global__ void k_add(int64_t n, const double *__restrict__ x, const double *__restrict__ v,
                      double *__restrict__ out, const int *gate, int64_t slab)
{
    lbf_rhs(slab, x, v, out, gate);
    if (gate_closed(gate)) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i] + v[i];
}

// a-rows of the bordered operator.
//   mode 0 (A x):      out_r = f_r (r < M-1), out_{M-1} = sum_m a_m
//   mode 1 (P^-1 A x): out_m = a_m - y_m
__global__ void k_arows(int M, int mode, const double *__restrict__ a, const double *__restrict__ f,
                        double *__restrict__ out, const int *gate, int64_t slab)
{
    lbf_rhs(slab, a, f, out, gate);
    if (gate_closed(gate)) return;
    int m = threadIdx.x;
    if (mode == 0) {
        if (m < M - 1) {
            for (int r = m; r < M - 1; r += blockDim.x) out[r] = f[r];
        }
        if (m == 0) {
            double s = 0.0;
            for (int k = 0; k < M; k++) s += a[k];
            out[M - 1] = s;
        }
    } else {
        for (int r = m; r < M; r += blockDim.x) out[r] = a[r] - f[r];
    }
}

// out_i = x_i + sc mu_{k-1} for the nodes i of island k >= 1 (F^T mu, Eq. disc_constr
// transposed), out_i = x_i on island 0; thread per caller index, sorted outputs
__global__ void k_island_scatter(int64_t N, int M, const int64_t *__restrict__ ptr,
                                 const int32_t *__restrict__ rank, const double *__restrict__ x,
                                 const double *__restrict__ mu, double sc, double *__restrict__ out,
                                 const int *gate)
{
    if (gate_closed(gate)) return;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ptr[mid] <= j) lo = mid; else hi = mid - 1;
    }
    const int i = rank[j];
    out[i] = x[i] + (lo >= 1 ? sc * mu[lo - 1] : 0.0);
}

// y = alpha S^-T f (thread per output, coalesced over the rows of S^-1)
__global__ void k_small_gemv_t(int M, const double *__restrict__ A, const double *__restrict__ f,
                               double alpha, double *__restrict__ y, const int *gate)
{
    if (gate_closed(gate)) return;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    double s = 0.0;
    for (int m = 0; m < M; m++) s = fma(A[(int64_t)m * M + r], f[m], s);
    y[r] = alpha * s;
}

// out_m += c_{M-1} (D^T c: D is the row of ones of Eq. sum_ak, in row M-1)
__global__ void k_add_last(int M, const double *__restrict__ c, double *__restrict__ out,
                           const int *gate)
{
    if (gate_closed(gate)) return;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) out[m] += c[M - 1];
}

// the Arnoldi input v_j of the current step (j from the device state) into a fixed buffer
template <typename T>
__global__ void k_copy_vj(int64_t n, const T *__restrict__ V, int64_t ldv,
                          const GmresState *__restrict__ st, double *__restrict__ out, int64_t slab)
{
    lbf_rhs(slab, V, st, out);
    if (st->go == 0) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)V[(int64_t)st->j * ldv + i];
}

// ---- GMRES kernels --------------------------------------------------------------------

// Partial dot products of w with V[0..nv) over one block's row chunk; the last block
// to finish sums the partials in block order into h.
template <typename T>
__device__ void dots_phase(const T *V, int64_t ldv, int nv, const T *ws, int rows,
                           int64_t row0, double *acc)
{
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = wid; k < nv; k += nw) {
        const T *vk = V + (int64_t)k * ldv + row0;
        T s = T(0);
        for (int r = lane; r < rows; r += 32) s = fma(vk[r], ws[r], s);
        s = warp_sum(s);
        if (lane == 0) acc[k] += (double)s;
    }
}

__device__ bool finish_block(unsigned *count)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(count, 1u) == gridDim.x - 1);
    __syncthreads();
    return last;
}

// mode 0: h = V^T w (columns 0..j)
// mode 1: w -= V h;  h2 = V^T w
// mode 2: w -= V h2; ||w||^2 -> Hessenberg column j, Givens rotation, convergence test
// T: the storage and arithmetic of the basis.  double: w is both the operator's output
// and the working vector.  float (the inner solves of the refinement, whose operator is
// float too): mode 0 rounds the operator's output w into the float working vector wt;
// dot products accumulate in float per thread and in double across threads and blocks.
template <typename T>
__global__ void k_arnoldi(int64_t n, const T *__restrict__ V, int64_t ldv, const double *w,
                          T *wt, double *part, unsigned *count, double *hbuf, double *H,
                          double *cs, double *sn, double *gv, GmresState *st, int mode, int64_t slab)
{
    lbf_rhs(slab, V, w, wt, part, count, hbuf, H, cs, sn, gv, st);
    if (st->go == 0) return;
    extern __shared__ double sh[];
    int m = st->m;
    int j = st->j;
    int nv = j + 1;
    T *ws = (T *)sh;                   // kRowsPerChunk
    double *acc = sh + kRowsPerChunk;  // m + 2
    T *hc = (T *)(acc + (m + 2));      // m + 1 (coefficients for the update)
    for (int k = threadIdx.x; k < m + 2; k += blockDim.x) acc[k] = 0.0;
    const double *hin = (mode == 1) ? hbuf : hbuf + (m + 1);
    if (mode >= 1)
        for (int k = threadIdx.x; k < nv; k += blockDim.x) hc[k] = (T)hin[k];
    __syncthreads();
    int64_t per = lbf_cdiv(n, gridDim.x);
    int64_t r0 = blockIdx.x * per, r1 = std::min<int64_t>(n, r0 + per);
    T nrm = T(0);
    for (int64_t c0 = r0; c0 < r1; c0 += kRowsPerChunk) {
        int rows = (int)std::min<int64_t>(kRowsPerChunk, r1 - c0);
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            T x;
            if (mode == 0) {
                x = (T)w[c0 + r];
                if constexpr (!std::is_same<T, double>::value) wt[c0 + r] = x;
            } else {
                x = wt[c0 + r];
                for (int k = 0; k < nv; k++) x = fma(-hc[k], V[(int64_t)k * ldv + c0 + r], x);
                wt[c0 + r] = x;
            }
            ws[r] = x;
            nrm = fma(x, x, nrm);
        }
        __syncthreads();
        if (mode <= 1) dots_phase(V, ldv, nv, ws, rows, c0, acc);
        __syncthreads();
    }
    if (mode == 2) {
        nrm = warp_sum(nrm);
        __shared__ double wsum[32];
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = (double)nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += wsum[k];
            acc[0] = t;
        }
        __syncthreads();
    }
    int nout = (mode == 2) ? 1 : nv;
    for (int k = threadIdx.x; k < nout; k += blockDim.x) part[(int64_t)blockIdx.x * (m + 2) + k] = acc[k];
    if (!finish_block(count)) return;
    // last block: fixed-order reduction over blocks, a warp per output (lanes strided
    // over the blocks, then a warp sum)
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int k = wid; k < nout; k += nw) {
            double s = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(&part[(int64_t)b * (m + 2) + k]);
            s = warp_sum(s);
            if (lane == 0) {
                if (mode == 0) hbuf[k] = s;
                else if (mode == 1) hbuf[(m + 1) + k] = s;
                else acc[0] = s;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *count = 0u;
        if (mode == 2) {
            // Hessenberg column j: h = h1 + h2, H[j+1][j] = ||w||
            double *Hj = H + (int64_t)j * (m + 1);
            for (int k = 0; k <= j; k++) Hj[k] = hbuf[k] + hbuf[(m + 1) + k];
            double hn = sqrt(acc[0]);
            Hj[j + 1] = hn;
            // apply the previous Givens rotations, then a new one zeroing H[j+1][j]
            for (int k = 0; k < j; k++) {
                double a = Hj[k], b = Hj[k + 1];
                Hj[k] = cs[k] * a + sn[k] * b;
                Hj[k + 1] = -sn[k] * a + cs[k] * b;
            }
            double a = Hj[j], b = Hj[j + 1];
            double rr = hypot(a, b);
            double c = rr > 0.0 ? a / rr : 1.0, s = rr > 0.0 ? b / rr : 0.0;
            cs[j] = c;
            sn[j] = s;
            Hj[j] = rr;
            Hj[j + 1] = 0.0;
            gv[j + 1] = -s * gv[j];
            gv[j] = c * gv[j];
            st->resid = fabs(gv[j + 1]);
            st->it += 1;
            st->j = j + 1;
            st->inv = hn > 0.0 ? 1.0 / hn : 0.0;
            bool conv = st->resid <= st->tol * st->bnorm;
            if (conv) st->converged = 1;
            if (conv || st->it >= st->maxit || j + 1 >= m || !(hn > 0.0)) st->go = 0;
        }
    }
}

// V[j] = w * inv (j = st->j after the Arnoldi step)
template <typename T>
__global__ void k_scale_next(int64_t n, const T *__restrict__ w, T *V, int64_t ldv,
                             const GmresState *st, int64_t slab)
{
    lbf_rhs(slab, w, V, st);
    if (st->go == 0) return;
    int j = st->j;
    const T inv = (T)st->inv;
    T *vj = V + (int64_t)j * ldv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        vj[i] = w[i] * inv;
}

// end of a cycle: y = H^-1 g (upper triangular, j columns), x += V y
__global__ void k_solve_y(const double *H, const double *gv, double *y, GmresState *st, int64_t slab)
{
    lbf_rhs(slab, H, gv, y, st);
    if (threadIdx.x != 0) return;
    int m = st->m, j = st->j;
    for (int i = j - 1; i >= 0; i--) {
        double s = gv[i];
        for (int k = i + 1; k < j; k++) s -= H[(int64_t)k * (m + 1) + i] * y[k];
        y[i] = s / H[(int64_t)i * (m + 1) + i];
    }
}

template <typename T>
__global__ void k_xupdate(int64_t n, const T *__restrict__ V, int64_t ldv,
                          const double *__restrict__ y, const GmresState *st, double *x, int64_t slab)
{
    lbf_rhs(slab, V, y, st, x);
    int j = st->j;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int k = 0; k < j; k++) s = fma((T)y[k], V[(int64_t)k * ldv + i], s);
        x[i] += (double)s;
    }
}

// r = b - Ax (Ax nullable = 0) into V[0], ||r||^2 partials; the last block starts a
// new cycle: beta = ||r||, g = (beta, 0, ...), j = 0, go = (beta > tol ||b||).
// With init != 0 it also records ||b|| (the first call, x = 0 or the initial guess).
template <typename T>
__global__ void k_restart(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax,
                          T *V, double *part, unsigned *count, double *gv, GmresState *st,
                          int init, const double *__restrict__ bn, int64_t slab)
{
    lbf_rhs(slab, b, Ax, V, part, count, gv, st, bn);
    // a restart of a system that has finished (the others of a lockstep solve go on)
    // leaves it as it is, with no columns left to add to its solution
    if (!init && (st->converged || st->it >= st->maxit)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->j = 0;
        return;
    }
    __shared__ double wsum[32];
    double nrm = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r = b[i] - (Ax ? Ax[i] : 0.0);
        V[i] = (T)r;
        nrm = fma(r, r, nrm);
    }
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += wsum[k];
        part[blockIdx.x] = t;
    }
    if (!finish_block(count)) return;
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) s += __ldcg(&part[k]);
        s = warp_sum(s);
    }
    if (threadIdx.x == 0) {
        *count = 0u;
        double beta = sqrt(s);
        if (init) st->bnorm = *bn;
        st->beta = beta;
        st->resid = beta;
        st->j = 0;
        st->inv = beta > 0.0 ? 1.0 / beta : 0.0;
        for (int k = 0; k <= st->m; k++) gv[k] = 0.0;
        gv[0] = beta;
        bool conv = beta <= st->tol * st->bnorm;
        st->converged = conv ? 1 : 0;
        st->go = (!conv && st->it < st->maxit) ? 1 : 0;
    }
}

template <typename T>
__global__ void k_scale_first(int64_t n, T *V, const GmresState *st, int64_t slab)
{
    lbf_rhs(slab, V, st);
    const T inv = (T)st->inv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        V[i] *= inv;
}

// ||v|| with a fixed-order reduction: block partials, then the last block to finish
// sums them (strided, then by warps) and resets the counter
__global__ void k_norm2(int64_t n, const double *__restrict__ v, double *part, unsigned *count,
                        double *out, int64_t slab)
{
    lbf_rhs(slab, v, part, count, out);
    __shared__ double wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s = fma(v[i], v[i], s);
    s = warp_sum(s);
    if (lane == 0) wsum[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < nw; k++) t += wsum[k];
        part[blockIdx.x] = t;
    }
    if (!finish_block(count)) return;
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(&part[b]);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) wsum[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < nw; k++) u += wsum[k];
        *out = sqrt(u);
        *count = 0u;
    }
}

__global__ void k_init_state(GmresState *st, int m, int maxit, double tol, int64_t slab)
{
    lbf_rhs(slab, st);
    st->go = 0; st->j = 0; st->it = 0; st->converged = 0;
    st->m = m; st->maxit = maxit; st->tol = tol;
    st->bnorm = 0; st->beta = 0; st->resid = 0; st->inv = 0;
}

__global__ void k_scale(int64_t n, double alpha, double *p, int64_t slab)
{
    lbf_rhs(slab, p);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] *= alpha;
}

// out = alpha x + beta y (out may alias x or y)
__global__ void k_axpby(int64_t n, double alpha, const double *x, double beta, const double *y,
                        double *out, int64_t slab)
{
    lbf_rhs(slab, x, y, out);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = alpha * x[i] + beta * y[i];
}

__global__ void k_widen(int64_t n, const float *__restrict__ in, double *__restrict__ out, int64_t slab)
{
    lbf_rhs(slab, in, out);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

__global__ void k_fill(double *p, int64_t n, double v, int64_t slab)
{
    lbf_rhs(slab, p);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

int lbf_permute_in(lbf_plan *pl, const double *in_caller, double *out_sorted, int with_a,
                   cudaStream_t s)
{
    int64_t n = pl->N + (with_a ? pl->M : 0);
    LBF_LAUNCH(k_permute_in, lbf_cdiv(n, 256), 256, 0, s, pl->N, pl->M, pl->perm, in_caller,
               out_sorted, with_a);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_permute_out(lbf_plan *pl, const double *in_sorted, double *out_caller, int with_a,
                    cudaStream_t s)
{
    int64_t n = pl->N + (with_a ? pl->M : 0);
    LBF_LAUNCH(k_permute_out, lbf_cdiv(n, 256), 256, 0, s, pl->N, pl->M, pl->perm, in_sorted,
               out_caller, with_a);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// out = x + v + sc E c (the multiplier potential of the centres' strengths c)
static int esum(lbf_plan *pl, const double *x, const double *v, const double *c, double sc,
                double *out, const int *gate, cudaStream_t s, int prec = LBF_PREC_FP64)
{
    return lbf_mp_apply(pl, c, x, v, sc, out, gate, s, prec);
}

static int island_sums(lbf_plan *pl, const double *u, double scale, double *out, const int *gate,
                       cudaStream_t s)
{
    LBF_LAUNCH(k_island_sums, lbf_grid(pl, lbf_cdiv((int64_t)pl->M * 32, 256)), 256, 0, s, pl->M,
               pl->island_ptr, pl->rank, u, scale, out, gate, pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

static int small_gemv(lbf_plan *pl, const double *f, double alpha, double *y, const int *gate,
                      cudaStream_t s)
{
    if (pl->lu) return lbf_schur_lu_apply(pl, f, alpha, y, 0, gate, s, !pl->lu_fast);
    LBF_LAUNCH(k_small_gemv, lbf_grid(pl, lbf_cdiv((int64_t)pl->M * 32, 256)), 256, 0, s, pl->M,
               pl->Sinv, f, alpha, y, gate, pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

static int island_scatter(lbf_plan *pl, const double *x, const double *mu, double sc, double *out,
                          const int *gate, cudaStream_t s)
{
    LBF_LAUNCH(k_island_scatter, lbf_cdiv(pl->N, 256), 256, 0, s, pl->N, pl->M, pl->island_ptr,
               pl->rank, x, mu, sc, out, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

static int small_gemv_t(lbf_plan *pl, const double *f, double alpha, double *y, const int *gate,
                        cudaStream_t s)
{
    if (pl->lu) return lbf_schur_lu_apply(pl, f, alpha, y, 1, gate, s, !pl->lu_fast);
    LBF_LAUNCH(k_small_gemv_t, lbf_cdiv(pl->M, 128), 128, 0, s, pl->M, pl->Sinv, f, alpha, y, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// Transposed operators (sorted order), in = [tau; mu]:
//   K_ONLY:         tau + 2 K^T tau
//   FULL:           A^T in = [tau + 2 K^T tau + F^T mu ; E^T tau + D^T mu]
//   PRECONDITIONED: P^-T A^T in = in + [v - F^T y ; y],  v = 2 K^T tau,  y = -S^-T E^T v
// (A^T = P^T + [[2 K^T, 0], [0, 0]], P^T = [[I, F^T], [E^T, D^T]], Sec. 5, Eq. matrix_eqns_c)
static int apply_op_transposed(lbf_plan *pl, int op, const double *in, double *out,
                               const int *gate, cudaStream_t s, int prec)
{
    int64_t N = pl->N;
    int M = pl->M;
    int rc = lbf_apply_KT(pl, in, pl->v, gate, s, prec);
    if (rc) return rc;
    LBF_LAUNCH(k_add, lbf_grid(pl, lbf_cdiv(N, 256)), 256, 0, s, N, in, pl->v, out, gate, pl->slab);
    LBF_CHECK_LAUNCH();
    if (op == LBF_OP_K_ONLY) return LBF_OK;
    if (!pl->opt.border) return LBF_ENOTBUILT;
    if (op == LBF_OP_FULL) {
        if ((rc = island_scatter(pl, out, in + N, 1.0, out, gate, s))) return rc;
        if ((rc = lbf_mp_apply_transpose(pl, in, 1.0, nullptr, out + N, gate, s))) return rc;
        LBF_LAUNCH(k_add_last, lbf_cdiv(M, 128), 128, 0, s, M, in + N, out + N, gate);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if ((rc = lbf_mp_apply_transpose(pl, pl->v, 1.0, nullptr, pl->fvec, gate, s))) return rc;
    if ((rc = small_gemv_t(pl, pl->fvec, -1.0, pl->yvec, gate, s))) return rc;
    if ((rc = island_scatter(pl, out, pl->yvec, -1.0, out, gate, s))) return rc;
    LBF_LAUNCH(k_add, lbf_grid(pl, lbf_cdiv(M, 128)), 128, 0, s, M, in + N, pl->yvec, out + N, gate,
               pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// out = P^-T r:  z_a = S^-T (r_a - E^T r_sigma),  z_sigma = r_sigma - F^T z_a
int lbf_precondition_rhs_t(lbf_plan *pl, const double *r_sorted, double *out, cudaStream_t s)
{
    int64_t N = pl->N;
    int rc;
    if ((rc = lbf_mp_apply_transpose(pl, r_sorted, -1.0, r_sorted + N, pl->fvec, nullptr, s))) return rc;
    if ((rc = small_gemv_t(pl, pl->fvec, 1.0, out + N, nullptr, s))) return rc;
    return island_scatter(pl, r_sorted, out + N, -1.0, out, nullptr, s);
}

int lbf_apply_op_sorted(lbf_plan *pl, int op, const double *in, double *out, const int *gate,
                        cudaStream_t s, int prec)
{
    if (op & LBF_OP_TRANSPOSE) return apply_op_transposed(pl, op & ~LBF_OP_TRANSPOSE, in, out, gate, s, prec);
    int64_t N = pl->N;
    int M = pl->M;
    int rc = lbf_apply_K(pl, in, pl->v, gate, s, prec);
    if (rc) return rc;
    if (op == LBF_OP_K_ONLY) {
        LBF_LAUNCH(k_add, lbf_grid(pl, lbf_cdiv(N, 256)), 256, 0, s, N, in, pl->v, out, gate, pl->slab);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if (!pl->opt.border) return LBF_ENOTBUILT;
    if (op == LBF_OP_FULL) {
        if ((rc = island_sums(pl, in, 1.0, pl->fvec, gate, s))) return rc;
        if ((rc = esum(pl, in, pl->v, in + N, 1.0, out, gate, s))) return rc;
        LBF_LAUNCH(k_arows, lbf_grid(pl, 1), 256, 0, s, M, 0, in + N, pl->fvec, out + N, gate,
                   pl->slab);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    // preconditioned: y = S^-1 F v; out = [sigma + v + E y ; a - y]
    if ((rc = island_sums(pl, pl->v, 1.0, pl->fvec, gate, s))) return rc;
    if ((rc = small_gemv(pl, pl->fvec, 1.0, pl->yvec, gate, s))) return rc;
    if ((rc = esum(pl, in, pl->v, pl->yvec, 1.0, out, gate, s, prec))) return rc;
    LBF_LAUNCH(k_arows, lbf_grid(pl, 1), 256, 0, s, M, 1, in + N, pl->yvec, out + N, gate, pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// out = P^-1 [g2; 0]:  z_a = -S^-1 F g2,  z_sigma = g2 - E z_a
int lbf_precondition_rhs(lbf_plan *pl, const double *g2_sorted, double *out, cudaStream_t s)
{
    int rc;
    if ((rc = island_sums(pl, g2_sorted, 1.0, pl->fvec, nullptr, s))) return rc;
    if ((rc = small_gemv(pl, pl->fvec, -1.0, out + pl->N, nullptr, s))) return rc;
    if ((rc = esum(pl, g2_sorted, nullptr, out + pl->N, -1.0, out, nullptr, s))) return rc;
    return LBF_OK;
}

static int read_state(lbf_plan *pl, GmresState *h, cudaStream_t s)
{
    LBF_CUDA(cudaMemcpyAsync(pl->host_scalars, pl->gs, sizeof(GmresState), cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    memcpy(h, pl->host_scalars, sizeof(GmresState));
    return LBF_OK;
}

// Restarted GMRES on P^-1 A x = b (sorted order, n unknowns) from x (x_given) or
// from 0, with the operator in precision prec, stopping at ||b - P^-1 A x|| <=
// tol * (*bnorm_dev).  Counts operator applications in pl->stats.
// One Arnoldi step on stream s: w = op(v_j), CGS2 against V, Givens update, v_{j+1}.
// from_state: the input is copied from V by the device's j (graph-replayable);
// otherwise v_j is addressed from the host's k.
// The float basis of the inner solves of the refinement: the first (m + 1) ldv floats of
// the basis region, then the float working vector.
static float *basis32(lbf_plan *pl) { return (float *)pl->V; }
static float *work32(lbf_plan *pl) { return (float *)pl->V + (int64_t)(pl->opt.restart + 1) * pl->ldv; }

template <typename T>
static int arnoldi_step_t(lbf_plan *pl, int opc, int prec, int k, bool from_state, T *V, T *wt,
                          cudaStream_t s)
{
    int64_t n = pl->n;
    int m = pl->opt.restart;
    double *w = pl->gw;
    int64_t ldv = pl->ldv;
    int nblk = pl->mdot_blocks;
    double *hbuf = pl->H + (int64_t)(m + 1) * m;
    double *cs = hbuf + 2 * (m + 1), *sn = cs + m, *gv = sn + m;
    unsigned *count = pl->red_count + 1;
    size_t smem = sizeof(double) * (size_t)(kRowsPerChunk + 2 * (m + 2));
    const double *vj = std::is_same<T, double>::value ? (const double *)(V + (int64_t)k * ldv) : nullptr;
    if (from_state || !vj) {
        // the operator reads v_j in double: from the device's j (graph-replayable), or a
        // float basis vector widened
        if (from_state) {
            LBF_LAUNCH(k_copy_vj<T>, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n, V, ldv, pl->gs,
                       pl->vstep, pl->slab);
        } else {
            LBF_LAUNCH(k_widen, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n,
                       (const float *)(V + (int64_t)k * ldv), pl->vstep, pl->slab);
        }
        vj = pl->vstep;
    }
    // FP64 Arnoldi steps take S^-1 from the factors alone; the refinement's float inner
    // steps keep the refinement step, so that they approximate the same P^-1 A as the
    // FP64 residual (a coarser S^-1 there costs refinement steps when S is ill-conditioned)
    pl->lu_fast = prec == LBF_PREC_FP64 ? 1 : 0;
    int rc = lbf_apply_op_sorted(pl, opc, vj, w, &pl->gs->go, s, prec);
    pl->lu_fast = 0;
    if (rc) return rc;
    for (int mode = 0; mode < 3; mode++)
        LBF_LAUNCH_P(LBF_KERNEL_ARNOLDI, k_arnoldi<T>, lbf_grid(pl, nblk), 256, smem, s, n, V, ldv,
                     w, wt, pl->gpart, count, hbuf, pl->H, cs, sn, gv, pl->gs, mode, pl->slab);
    LBF_LAUNCH(k_scale_next<T>, lbf_grid(pl, nblk), 256, 0, s, n, wt, V, ldv, pl->gs, pl->slab);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// The float operator's solves keep their basis in float (the inner solves of the
// refinement need ~1e-4; the accurate operator's solves keep double).
static int arnoldi_step(lbf_plan *pl, int opc, int prec, int k, bool from_state, cudaStream_t s)
{
    if (prec == LBF_PREC_FP32)
        return arnoldi_step_t<float>(pl, opc, prec, k, from_state, basis32(pl), work32(pl), s);
    return arnoldi_step_t<double>(pl, opc, prec, k, from_state, pl->V, pl->gw, s);
}

// The captured step graph of (prec, transpose), built on first use; null when graphs
// are off for this plan or the stream cannot capture (the legacy default stream).
static cudaGraphExec_t step_graph(lbf_plan *pl, int opc, int prec, cudaStream_t s)
{
    const int g = pl->opt.graphs;
    if (g == 0 || (g < 0 && pl->N > (1 << 18)) || s == nullptr || !pl->vstep) return nullptr;
    if (!(opc & LBF_OP_PRECONDITIONED)) return nullptr;  // the graphs hold the preconditioned step
    const int pi = prec == LBF_PREC_FP32 ? 1 : 0, ti = (opc & LBF_OP_TRANSPOSE) ? 1 : 0;
    if (pl->gexec[pi][ti]) return pl->gexec[pi][ti];
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    lbf_prof_capture(true);
    const int64_t n0 = g_lbf_launches.load();
    int rc = arnoldi_step(pl, opc, prec, 0, true, s);
    // captured, not launched: count them at every replay instead
    pl->gnodes[pi][ti] = g_lbf_launches.load() - n0;
    g_lbf_launches.fetch_sub(pl->gnodes[pi][ti]);
    lbf_prof_capture(false);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == LBF_OK && e == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
        pl->gexec[pi][ti] = exec;
    else
        cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return pl->gexec[pi][ti];
}

static int gmres_core(lbf_plan *pl, int opc, const double *b, const double *bnorm_dev, double *x,
                      bool x_given, double tol, int maxit, int prec, cudaStream_t s,
                      GmresState *out)
{
    int64_t n = pl->n;
    int m = pl->opt.restart;
    int rc;
    double *w = pl->gw, *V = pl->V;
    int64_t ldv = pl->ldv;
    int nblk = pl->mdot_blocks;
    double *hbuf = pl->H + (int64_t)(m + 1) * m;   // 2 (m + 1)
    double *cs = hbuf + 2 * (m + 1), *sn = cs + m, *gv = sn + m, *y = gv + (m + 1);
    unsigned *count = pl->red_count + 1;
    int64_t *applies = prec == LBF_PREC_FP32 ? &pl->stats[2] : &pl->stats[1];
    LBF_LAUNCH(k_init_state, lbf_grid(pl, 1), 1, 0, s, pl->gs, m, maxit, tol, pl->slab);
    LBF_CHECK_LAUNCH();
    const double *Ax = nullptr;
    if (x_given) {
        if ((rc = lbf_apply_op_sorted(pl, opc, x, w, nullptr, s, prec))) return rc;
        (*applies)++;
        Ax = w;
    } else {
        LBF_LAUNCH(k_fill, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, x, n, 0.0, pl->slab);
        LBF_CHECK_LAUNCH();
    }
    const bool f32 = prec == LBF_PREC_FP32;
    float *V32 = basis32(pl);
    if (f32) {
        LBF_LAUNCH(k_restart<float>, lbf_grid(pl, nblk), 256, 0, s, n, b, Ax, V32, pl->gpart, count,
                   gv, pl->gs, 1, bnorm_dev, pl->slab);
        LBF_LAUNCH(k_scale_first<float>, lbf_grid(pl, nblk), 256, 0, s, n, V32, pl->gs, pl->slab);
    } else {
        LBF_LAUNCH(k_restart<double>, lbf_grid(pl, nblk), 256, 0, s, n, b, Ax, V, pl->gpart, count,
                   gv, pl->gs, 1, bnorm_dev, pl->slab);
        LBF_LAUNCH(k_scale_first<double>, lbf_grid(pl, nblk), 256, 0, s, n, V, pl->gs, pl->slab);
    }
    LBF_CHECK_LAUNCH();
    cudaGraphExec_t sg = step_graph(pl, opc, prec, s);
    const int64_t sg_nodes =
        pl->gnodes[prec == LBF_PREC_FP32 ? 1 : 0][(opc & LBF_OP_TRANSPOSE) ? 1 : 0];
    GmresState hs;
    for (;;) {
        if ((rc = read_state(pl, &hs, s))) return rc;
        if (hs.converged || hs.it >= hs.maxit || hs.go == 0) break;
        int steps = std::min(m, hs.maxit - hs.it);
        // Arnoldi steps are queued in chunks; before queueing a chunk the host looks
        // at the state copied after the chunk before last (double-buffered pinned
        // copy + event), so at most two chunks run past convergence, and those
        // return at once on the device gate.
        const int chunk = 4;
        for (int c = 0, k0 = 0; k0 < steps; c++) {
            const int slot = c & 1;
            if (c >= 2) {  // the state recorded after chunk c-2 (chunk c-1 keeps the GPU busy)
                LBF_CUDA(cudaEventSynchronize(pl->ev[slot]));
                GmresState chk;
                memcpy(&chk, (char *)pl->host_scalars + 64 * (1 + slot), sizeof(GmresState));
                if (chk.go == 0) break;
            }
            int k1 = std::min(steps, k0 + chunk);
            for (int k = k0; k < k1; k++) {
                // w = P^-1 A v_j: within a cycle the device's j equals the host's k
                if (sg) {
                    LBF_CUDA(cudaGraphLaunch(sg, s));
                    g_lbf_launches.fetch_add(sg_nodes, std::memory_order_relaxed);
                } else if ((rc = arnoldi_step(pl, opc, prec, k, false, s))) {
                    return rc;
                }
            }
            k0 = k1;
            LBF_CUDA(cudaMemcpyAsync((char *)pl->host_scalars + 64 * (1 + slot), pl->gs,
                                     sizeof(GmresState), cudaMemcpyDeviceToHost, s));
            LBF_CUDA(cudaEventRecord(pl->ev[slot], s));
        }
        // cycle end: x += V y
        LBF_LAUNCH(k_solve_y, lbf_grid(pl, 1), 32, 0, s, pl->H, gv, y, pl->gs, pl->slab);
        if (f32) LBF_LAUNCH(k_xupdate<float>, lbf_grid(pl, nblk), 256, 0, s, n, V32, ldv, y, pl->gs,
                            x, pl->slab);
        else LBF_LAUNCH(k_xupdate<double>, lbf_grid(pl, nblk), 256, 0, s, n, V, ldv, y, pl->gs, x,
                        pl->slab);
        LBF_CHECK_LAUNCH();
        if ((rc = read_state(pl, &hs, s))) return rc;
        if (hs.converged || hs.it >= hs.maxit) break;
        // restart from the true preconditioned residual
        if ((rc = lbf_apply_op_sorted(pl, opc, x, w, nullptr, s, prec))) return rc;
        (*applies)++;
        if (f32) {
            LBF_LAUNCH(k_restart<float>, lbf_grid(pl, nblk), 256, 0, s, n, b, w, V32, pl->gpart,
                       count, gv, pl->gs, 0, bnorm_dev, pl->slab);
            LBF_LAUNCH(k_scale_first<float>, lbf_grid(pl, nblk), 256, 0, s, n, V32, pl->gs, pl->slab);
        } else {
            LBF_LAUNCH(k_restart<double>, lbf_grid(pl, nblk), 256, 0, s, n, b, w, V, pl->gpart,
                       count, gv, pl->gs, 0, bnorm_dev, pl->slab);
            LBF_LAUNCH(k_scale_first<double>, lbf_grid(pl, nblk), 256, 0, s, n, V, pl->gs, pl->slab);
        }
        LBF_CHECK_LAUNCH();
    }
    if ((rc = read_state(pl, &hs, s))) return rc;
    *applies += hs.it;
    pl->stats[0] += hs.it;
    *out = hs;
    return LBF_OK;
}

// Forward (transpose == 0): A [sigma; a] = [2 g; 0] from g (N, caller order).
// Adjoint (transpose == 1): A^T lam = r from r = g (N + M, caller order), lam into
// sigma (N + M, caller order), a unused.  Left preconditioning by P (P^T).
int lbf_gmres_impl(lbf_plan *pl, const double *g, double *sigma, double *a, const double *x0,
                   int *iters, double *rel_res, cudaStream_t s, int transpose)
{
    if (!pl->opt.border) return LBF_ENOTBUILT;
    int64_t N = pl->N, n = pl->n;
    int rc;
    double *b = pl->gb, *x = pl->gx;
    const bool pc = pl->opt.precond != 0;
    const int opc = (pc ? LBF_OP_PRECONDITIONED : LBF_OP_FULL) | (transpose ? LBF_OP_TRANSPOSE : 0);
    for (auto &v : pl->stats) v = 0;
    if (!pc) {
        // without the preconditioner (the comparison of Sec. 6, Example 1): b = [2 g; 0]
        // (or r for the adjoint), in sorted order
        if ((rc = lbf_permute_in(pl, g, b, transpose ? 1 : 0, s))) return rc;
        if (!transpose) {
            LBF_LAUNCH(k_scale, lbf_grid(pl, lbf_cdiv(N, 256)), 256, 0, s, N, 2.0, b, pl->slab);
            LBF_CUDA(cudaMemsetAsync(b + N, 0, sizeof(double) * pl->M, s));
            LBF_CHECK_LAUNCH();
        }
    } else if (transpose) {
        // b = P^-T r
        if ((rc = lbf_permute_in(pl, g, pl->tin, 1, s))) return rc;
        if ((rc = lbf_precondition_rhs_t(pl, pl->tin, b, s))) return rc;
    } else {
        // b = P^-1 [2 g; 0] in sorted order (tin holds the permuted data), with the
        // doubled right-hand side 2 g of Eq. disc_sphere
        if ((rc = lbf_permute_in(pl, g, pl->tin, 0, s))) return rc;
        LBF_LAUNCH(k_scale, lbf_grid(pl, lbf_cdiv(N, 256)), 256, 0, s, N, 2.0, pl->tin, pl->slab);
        LBF_CHECK_LAUNCH();
        if ((rc = lbf_precondition_rhs(pl, pl->tin, b, s))) return rc;
    }
    double *bn = pl->bsig + 1, *rn = pl->bsig + 2;
    LBF_LAUNCH(k_norm2, lbf_grid(pl, pl->mdot_blocks), 256, 0, s, n, b, pl->gpart,
               pl->red_count + 2, bn, pl->slab);
    LBF_CHECK_LAUNCH();
    if (x0 && (rc = lbf_permute_in(pl, x0, x, 1, s))) return rc;
    GmresState hs{};
    bool converged = false;
    double rel = 0.0;
    int its = 0;
    if (pl->opt.precision == LBF_PRECISION_FP64 || !pl->q32) {
        if ((rc = gmres_core(pl, opc, b, bn, x, x0 != nullptr, pl->opt.tol, pl->opt.maxit, LBF_PREC_FP64, s,
                             &hs)))
            return rc;
        converged = hs.converged;
        its = hs.it;
        rel = hs.bnorm > 0 ? hs.resid / hs.bnorm : 0.0;
    } else {
        // iterative refinement: FP64 residual, FP32-operator GMRES correction
        double *r = pl->gr, *d = pl->gd;
        if (!x0) {
            LBF_LAUNCH(k_fill, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, x, n, 0.0, pl->slab);
            LBF_CHECK_LAUNCH();
        }
        double hb[3];
        for (int k = 0;; k++) {
            if (k == 0 && !x0) {
                LBF_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            } else {
                if ((rc = lbf_apply_op_sorted(pl, opc, x, pl->gw, nullptr, s,
                                              LBF_PREC_FP64)))
                    return rc;
                pl->stats[1]++;
                LBF_LAUNCH(k_axpby, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n, 1.0, b, -1.0,
                           pl->gw, r, pl->slab);
                LBF_CHECK_LAUNCH();
            }
            LBF_LAUNCH(k_norm2, lbf_grid(pl, pl->mdot_blocks), 256, 0, s, n, r, pl->gpart,
                       pl->red_count + 2, rn, pl->slab);
            LBF_CHECK_LAUNCH();
            LBF_CUDA(cudaMemcpyAsync(hb, pl->bsig, sizeof(hb), cudaMemcpyDeviceToHost, s));
            LBF_CUDA(cudaStreamSynchronize(s));
            rel = hb[1] > 0 ? hb[2] / hb[1] : 0.0;
            if (rel <= pl->opt.tol) { converged = true; break; }
            if (k >= pl->opt.max_refine || its >= pl->opt.maxit) break;
            pl->stats[3]++;
            if ((rc = gmres_core(pl, opc, r, rn, d, false, pl->opt.inner_tol, pl->opt.maxit - its,
                                 LBF_PREC_FP32, s, &hs)))
                return rc;
            its += hs.it;
            LBF_LAUNCH(k_axpby, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n, 1.0, x, 1.0, d, x,
                       pl->slab);
            LBF_CHECK_LAUNCH();
        }
    }
    // outputs in the caller's order
    LBF_LAUNCH(k_permute_out, lbf_cdiv(transpose ? n : N, 256), 256, 0, s, N, pl->M, pl->perm, x,
               sigma, transpose);
    LBF_CHECK_LAUNCH();
    if (a && !transpose)
        LBF_CUDA(cudaMemcpyAsync(a, x + N, sizeof(double) * pl->M, cudaMemcpyDeviceToDevice, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = its;
    if (rel_res) *rel_res = rel;
    return converged ? LBF_OK : LBF_NOCONV;
}

int lbf_gmres_kernels_smem(int m) { return (int)(sizeof(double) * (kRowsPerChunk + 2 * (m + 2))); }
int lbf_gmres_blocks() { return kDotBlocks; }

// ---- right-hand sides in lockstep -----------------------------------------------------

static_assert(sizeof(GmresState) <= 64, "GMRES state: 64-byte host slots");

namespace {

struct RhsInts {  // one value per right-hand side of a lockstep group, passed by value
    int v[LBF_LOCKSTEP_MAX];
};

// the states of the view's right-hand sides, packed (a thread each)
__global__ void k_gather_states(const GmresState *st, int64_t slab, int nrhs, GmresState *out)
{
    const int r = threadIdx.x;
    if (r < nrhs) out[r] = *(const GmresState *)((const char *)st + (int64_t)r * slab);
}

// k_init_state with each right-hand side's own iteration limit (0: it takes no step)
__global__ void k_init_states(GmresState *st, int m, RhsInts maxit, double tol, int64_t slab)
{
    const int mx = maxit.v[blockIdx.y];
    lbf_rhs(slab, st);
    st->go = 0; st->j = 0; st->it = 0; st->converged = 0;
    st->m = m; st->maxit = mx; st->tol = tol;
    st->bnorm = 0; st->beta = 0; st->resid = 0; st->inv = 0;
}

// the gates of the next launches: open for the right-hand sides marked in on
__global__ void k_set_gates(GmresState *st, RhsInts on, int64_t slab)
{
    const int g = on.v[blockIdx.y];
    lbf_rhs(slab, st);
    st->go = g;
}

// before a restart's operator application: the right-hand sides still iterating
// pass their gate again (the others stay closed)
__global__ void k_reopen(GmresState *st, int64_t slab)
{
    lbf_rhs(slab, st);
    if (!st->converged && st->it < st->maxit) st->go = 1;
}

inline bool finished(const GmresState &h) { return h.converged || h.it >= h.maxit; }

}  // namespace

// The view's states into pinned host slot k (0: read now; 1, 2: the chunk checks),
// staged in device slot k of dst (3 R states after the slabs).
static int stage_states(lbf_plan *v, GmresState *dst, int k, cudaStream_t s)
{
    const int R = v->nrhs;
    LBF_LAUNCH(k_gather_states, 1, 32, 0, s, v->gs, v->slab, R, dst + (int64_t)k * R);
    LBF_CHECK_LAUNCH();
    LBF_CUDA(cudaMemcpyAsync((char *)v->host_scalars + 256 + (size_t)64 * R * k, dst + (int64_t)k * R,
                             sizeof(GmresState) * R, cudaMemcpyDeviceToHost, s));
    return LBF_OK;
}
static const GmresState *host_states(lbf_plan *v, int k)
{
    return (const GmresState *)((char *)v->host_scalars + 256 + (size_t)64 * v->nrhs * k);
}

// gmres_core on every right-hand side of view v from x = 0: b, ||b|| (bn) and x are the
// first right-hand side's (the others' follow at the view's stride), maxit[r] the
// iteration limit of right-hand side r (0: none).  Each launch covers all right-hand
// sides and is gated per right-hand side by its own state; one that finishes stops (its
// gate closes, its restarts are skipped, and later cycle ends add nothing to its x), so
// its iterates are those of gmres_core on it alone (up to the rounding of the group's
// near field, when the native-double operator forms it in one pass).
static int gmres_core_many(lbf_plan *pl, int opc, int prec, const double *b, const double *bn,
                           double *x, double tol, const int *maxit, GmresState *dst,
                           cudaStream_t s, GmresState *out)
{
    const int R = pl->nrhs;
    int64_t n = pl->n;
    int m = pl->opt.restart;
    int rc;
    double *w = pl->gw, *V = pl->V;
    int64_t ldv = pl->ldv;
    int nblk = pl->mdot_blocks;
    double *hbuf = pl->H + (int64_t)(m + 1) * m;
    double *cs = hbuf + 2 * (m + 1), *sn = cs + m, *gv = sn + m, *y = gv + (m + 1);
    unsigned *count = pl->red_count + 1;
    const bool f32 = prec == LBF_PREC_FP32;
    float *V32 = basis32(pl);
    RhsInts mx{};
    int mmax = 0;
    for (int r = 0; r < R; r++) {
        mx.v[r] = maxit[r];
        mmax = std::max(mmax, maxit[r]);
    }
    LBF_LAUNCH(k_init_states, lbf_grid(pl, 1), 1, 0, s, pl->gs, m, mx, tol, pl->slab);
    LBF_LAUNCH(k_fill, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, x, n, 0.0, pl->slab);
    auto restart = [&](const double *Ax, int init) -> int {
        if (f32) {
            LBF_LAUNCH(k_restart<float>, lbf_grid(pl, nblk), 256, 0, s, n, b, Ax, V32, pl->gpart, count,
                       gv, pl->gs, init, bn, pl->slab);
            LBF_LAUNCH(k_scale_first<float>, lbf_grid(pl, nblk), 256, 0, s, n, V32, pl->gs, pl->slab);
        } else {
            LBF_LAUNCH(k_restart<double>, lbf_grid(pl, nblk), 256, 0, s, n, b, Ax, V, pl->gpart, count,
                       gv, pl->gs, init, bn, pl->slab);
            LBF_LAUNCH(k_scale_first<double>, lbf_grid(pl, nblk), 256, 0, s, n, V, pl->gs, pl->slab);
        }
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    };
    if ((rc = restart(nullptr, 1))) return rc;
    cudaGraphExec_t sg = step_graph(pl, opc, prec, s);
    const int64_t sg_nodes = pl->gnodes[f32 ? 1 : 0][0];
    auto read_all = [&]() -> int {
        int e = stage_states(pl, dst, 0, s);
        if (e) return e;
        LBF_CUDA(cudaStreamSynchronize(s));
        return LBF_OK;
    };
    int64_t restarts = 0;
    for (;;) {
        if ((rc = read_all())) return rc;
        const GmresState *hs = host_states(pl, 0);
        int it_act = -1;
        for (int r = 0; r < R; r++)
            if (hs[r].go) it_act = std::max(it_act, hs[r].it);
        if (it_act < 0) break;
        const int steps = std::min(m, mmax - it_act);
        const int chunk = 4;
        for (int c = 0, k0 = 0; k0 < steps; c++) {
            const int slot = 1 + (c & 1);
            if (c >= 2) {  // the states recorded after chunk c-2
                LBF_CUDA(cudaEventSynchronize(pl->ev[c & 1]));
                const GmresState *chk = host_states(pl, slot);
                bool any = false;
                for (int r = 0; r < R; r++) any = any || chk[r].go;
                if (!any) break;
            }
            const int k1 = std::min(steps, k0 + chunk);
            for (int k = k0; k < k1; k++) {
                if (sg) {
                    LBF_CUDA(cudaGraphLaunch(sg, s));
                    g_lbf_launches.fetch_add(sg_nodes, std::memory_order_relaxed);
                } else if ((rc = arnoldi_step(pl, opc, prec, k, false, s))) {
                    return rc;
                }
            }
            k0 = k1;
            if ((rc = stage_states(pl, dst, slot, s))) return rc;
            LBF_CUDA(cudaEventRecord(pl->ev[c & 1], s));
        }
        // cycle end: x += V y on every right-hand side (none for those finished earlier)
        LBF_LAUNCH(k_solve_y, lbf_grid(pl, 1), 32, 0, s, pl->H, gv, y, pl->gs, pl->slab);
        if (f32)
            LBF_LAUNCH(k_xupdate<float>, lbf_grid(pl, nblk), 256, 0, s, n, V32, ldv, y, pl->gs, x,
                       pl->slab);
        else
            LBF_LAUNCH(k_xupdate<double>, lbf_grid(pl, nblk), 256, 0, s, n, V, ldv, y, pl->gs, x,
                       pl->slab);
        LBF_CHECK_LAUNCH();
        if ((rc = read_all())) return rc;
        hs = host_states(pl, 0);
        int open = 0;
        for (int r = 0; r < R; r++) open += finished(hs[r]) ? 0 : 1;
        if (open == 0) break;
        // restart the unfinished ones from their true preconditioned residual
        LBF_LAUNCH(k_reopen, lbf_grid(pl, 1), 1, 0, s, pl->gs, pl->slab);
        LBF_CHECK_LAUNCH();
        if ((rc = lbf_apply_op_sorted(pl, opc, x, w, &pl->gs->go, s, prec))) return rc;
        restarts += open;
        if ((rc = restart(w, 0))) return rc;
    }
    if ((rc = read_all())) return rc;
    const GmresState *hs = host_states(pl, 0);
    int64_t its = 0;
    for (int r = 0; r < R; r++) {
        out[r] = hs[r];
        its += hs[r].it;
    }
    pl->stats[0] += its;
    pl->stats[f32 ? 2 : 1] += its + restarts;
    return LBF_OK;
}

// GMRES-IR of lbf_gmres_impl on every right-hand side of view v (b, ||b|| in the view's
// buffers): a refinement round forms the FP64 residuals of the right-hand sides still
// open, stops those that meet tol or their limits, and runs the float inner solves of
// the others together.
static int refine_many(lbf_plan *pl, int opc, GmresState *dst, cudaStream_t s, int *its_out,
                       double *rel_out, int *conv_out)
{
    const int R = pl->nrhs;
    const int64_t n = pl->n;
    double *x = pl->gx, *b = pl->gb, *r = pl->gr, *d = pl->gd;
    const double *bn = pl->bsig + 1;
    double *rn = pl->bsig + 2;
    int rc;
    int its[LBF_LOCKSTEP_MAX] = {0};
    bool open[LBF_LOCKSTEP_MAX];
    for (int q = 0; q < R; q++) {
        open[q] = true;
        conv_out[q] = 0;
        rel_out[q] = 0.0;
    }
    LBF_LAUNCH(k_fill, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, x, n, 0.0, pl->slab);
    LBF_CHECK_LAUNCH();
    double *hb = (double *)((char *)pl->host_scalars + 256);  // R x (||b||, ||r||) after the reads
    for (int k = 0;; k++) {
        RhsInts on{};
        int nopen = 0;
        for (int q = 0; q < R; q++) {
            on.v[q] = open[q] ? 1 : 0;
            nopen += on.v[q];
        }
        if (nopen == 0) break;
        if (k == 0) {
            for (int q = 0; q < R; q++)
                LBF_CUDA(cudaMemcpyAsync(r + q * (pl->slab / 8), b + q * (pl->slab / 8), sizeof(double) * n,
                                         cudaMemcpyDeviceToDevice, s));
        } else {
            LBF_LAUNCH(k_set_gates, lbf_grid(pl, 1), 1, 0, s, pl->gs, on, pl->slab);
            LBF_CHECK_LAUNCH();
            if ((rc = lbf_apply_op_sorted(pl, opc, x, pl->gw, &pl->gs->go, s, LBF_PREC_FP64))) return rc;
            pl->stats[1] += nopen;
            LBF_LAUNCH(k_axpby, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n, 1.0, b, -1.0, pl->gw, r,
                       pl->slab);
            LBF_CHECK_LAUNCH();
        }
        LBF_LAUNCH(k_norm2, lbf_grid(pl, pl->mdot_blocks), 256, 0, s, n, r, pl->gpart,
                   pl->red_count + 2, rn, pl->slab);
        LBF_CHECK_LAUNCH();
        for (int q = 0; q < R; q++)
            LBF_CUDA(cudaMemcpyAsync(hb + 2 * q, (const char *)bn + q * pl->slab, sizeof(double) * 2,
                                     cudaMemcpyDeviceToHost, s));
        LBF_CUDA(cudaStreamSynchronize(s));
        int lim[LBF_LOCKSTEP_MAX] = {0};
        int nin = 0;
        for (int q = 0; q < R; q++) {
            if (!open[q]) continue;
            const double rel = hb[2 * q] > 0 ? hb[2 * q + 1] / hb[2 * q] : 0.0;
            rel_out[q] = rel;
            if (rel <= pl->opt.tol) {
                conv_out[q] = 1;
                open[q] = false;
                continue;
            }
            if (k >= pl->opt.max_refine || its[q] >= pl->opt.maxit) {
                open[q] = false;
                continue;
            }
            lim[q] = pl->opt.maxit - its[q];
            nin++;
            pl->stats[3]++;
        }
        if (nin == 0) break;
        GmresState hs[LBF_LOCKSTEP_MAX];
        if ((rc = gmres_core_many(pl, opc, LBF_PREC_FP32, r, rn, d, pl->opt.inner_tol, lim, dst, s, hs)))
            return rc;
        for (int q = 0; q < R; q++) its[q] += lim[q] > 0 ? hs[q].it : 0;
        // x += d (d = 0 on the right-hand sides without an inner solve)
        LBF_LAUNCH(k_axpby, lbf_grid(pl, lbf_cdiv(n, 256)), 256, 0, s, n, 1.0, x, 1.0, d, x, pl->slab);
        LBF_CHECK_LAUNCH();
    }
    for (int q = 0; q < R; q++) its_out[q] = its[q];
    return LBF_OK;
}

// nrhs right-hand sides of one plan, in lockstep groups of up to LBF_LOCKSTEP_MAX; the
// plans whose S^-1 is applied by LU factors solve them one after another (lbf_gmres_impl).
int lbf_gmres_many_impl(lbf_plan *pl, int nrhs, const double *g, double *sigma, double *a,
                        int *iters, double *rel_res, void *work, size_t bytes, cudaStream_t s)
{
    const int64_t N = pl->N;
    const int M = pl->M;
    int worst = LBF_OK;
    for (auto &v : pl->stats) v = 0;
    if (pl->lu) {
        int64_t st[4] = {0, 0, 0, 0};
        for (int r = 0; r < nrhs; r++) {
            int its = 0;
            double rr = 0.0;
            int rc = lbf_gmres_impl(pl, g + r * N, sigma + r * N, a ? a + (int64_t)r * M : nullptr,
                                    nullptr, &its, &rr, s, 0);
            if (rc < 0) return rc;
            if (rc == LBF_NOCONV) worst = LBF_NOCONV;
            for (int k = 0; k < 4; k++) st[k] += pl->stats[k];
            if (iters) iters[r] = its;
            if (rel_res) rel_res[r] = rr;
        }
        for (int k = 0; k < 4; k++) pl->stats[k] = st[k];
        return worst;
    }
    const bool pc = pl->opt.precond != 0;
    const int opc = pc ? LBF_OP_PRECONDITIONED : LBF_OP_FULL;
    const bool ir = pl->opt.precision != LBF_PRECISION_FP64 && pl->q32;
    for (int r0 = 0; r0 < nrhs; r0 += LBF_LOCKSTEP_MAX) {
        const int R = std::min(LBF_LOCKSTEP_MAX, nrhs - r0);
        lbf_plan v;
        size_t need = 0;
        int rc = lbf_many_view(pl, R, work, bytes, &v, &need);
        if (rc) return rc;
        GmresState *dst = (GmresState *)((char *)work + (size_t)v.slab * R);
        LBF_CUDA(cudaMemsetAsync(work, 0, (size_t)v.slab * R, s));
        if (pl->imean)  // the island-mean constants of the float split, per right-hand side
            for (int r = 0; r < R; r++)
                LBF_CUDA(cudaMemcpyAsync(lbf_view_at(v, r).imean + M, pl->imean + M, sizeof(double) * 8,
                                         cudaMemcpyDeviceToDevice, s));
        // b = P^-1 [2 g; 0] (or [2 g; 0] without the preconditioner) and ||b||
        for (int r = 0; r < R; r++) {
            lbf_plan vr = lbf_view_at(v, r);
            if ((rc = lbf_permute_in(&vr, g + (int64_t)(r0 + r) * N, pc ? vr.tin : vr.gb, 0, s))) return rc;
        }
        LBF_LAUNCH(k_scale, lbf_grid(&v, lbf_cdiv(N, 256)), 256, 0, s, N, 2.0, pc ? v.tin : v.gb,
                   v.slab);
        LBF_CHECK_LAUNCH();
        if (pc) {
            if ((rc = lbf_precondition_rhs(&v, v.tin, v.gb, s))) return rc;
        } else {
            LBF_LAUNCH(k_fill, lbf_grid(&v, lbf_cdiv(M, 256)), 256, 0, s, v.gb + N, (int64_t)M, 0.0,
                       v.slab);
            LBF_CHECK_LAUNCH();
        }
        LBF_LAUNCH(k_norm2, lbf_grid(&v, v.mdot_blocks), 256, 0, s, v.n, v.gb, v.gpart, v.red_count + 2,
                   v.bsig + 1, v.slab);
        LBF_CHECK_LAUNCH();
        for (auto &k : v.stats) k = 0;
        int its[LBF_LOCKSTEP_MAX], conv[LBF_LOCKSTEP_MAX];
        double rel[LBF_LOCKSTEP_MAX];
        if (ir) {
            rc = refine_many(&v, opc, dst, s, its, rel, conv);
        } else {
            GmresState hs[LBF_LOCKSTEP_MAX];
            int lim[LBF_LOCKSTEP_MAX];
            for (int r = 0; r < R; r++) lim[r] = pl->opt.maxit;
            rc = gmres_core_many(&v, opc, LBF_PREC_FP64, v.gb, v.bsig + 1, v.gx, pl->opt.tol, lim, dst, s,
                                 hs);
            for (int r = 0; r < R; r++) {
                its[r] = hs[r].it;
                conv[r] = hs[r].converged;
                rel[r] = hs[r].bnorm > 0 ? hs[r].resid / hs[r].bnorm : 0.0;
            }
        }
        for (auto &row : v.gexec)
            for (auto &ge : row)
                if (ge) cudaGraphExecDestroy(ge);
        if (rc) return rc;
        for (int k = 0; k < 4; k++) pl->stats[k] += v.stats[k];
        for (int r = 0; r < R; r++) {
            lbf_plan vr = lbf_view_at(v, r);
            LBF_LAUNCH(k_permute_out, lbf_cdiv(N, 256), 256, 0, s, N, M, pl->perm, vr.gx,
                       sigma + (int64_t)(r0 + r) * N, 0);
            LBF_CHECK_LAUNCH();
            if (a)
                LBF_CUDA(cudaMemcpyAsync(a + (int64_t)(r0 + r) * M, vr.gx + N, sizeof(double) * M,
                                         cudaMemcpyDeviceToDevice, s));
            if (!conv[r]) worst = LBF_NOCONV;
            if (iters) iters[r0 + r] = its[r];
            if (rel_res) rel_res[r0 + r] = rel[r];
        }
        LBF_CUDA(cudaStreamSynchronize(s));
    }
    return worst;
}
