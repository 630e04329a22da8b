// Per-node precompute (Sec. 3 and Sec. 5) and the inverse Schur complement of
// the block preconditioner (Sec. 5).
#include <utility>

#include "lbf_internal.cuh"
#include "lbf_sync.cuh"

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

// ---- inverse of the Schur complement ---------------------------------------------------
//
// Gauss-Jordan elimination with partial pivoting (row interchanges), in place, all M
// steps in one cooperative launch.  Step k, with B = A after interchanging rows k and
// p (p the pivot row):
//   row k:       A'_kj = B_kj / B_kk                  (A'_kk = 1 / B_kk)
//   row i != k:  A'_ij = B_ij - B_ik A'_kj,   A'_ik = -B_ik / B_kk.
// The interchanges are undone at the end by swapping columns k and p, k = M-1, ..., 0.
// A singular S (a pivot at or below M 2^-52 max|S_ij|) sets status bit 4.
//
// The grid barrier is a counter and a generation word; every block is resident
// (cooperative launch), and each wait gives up after kBarrierSpins polls, setting
// status bit LBF_DEV_TIMEOUT, so the kernel always ends.

constexpr int kGjThreads = 512;
constexpr int kGjMaxBlocks = 1024;

// Magnitudes are compared as the bit patterns of |x| (for doubles that are not NaN the
// order of |x| is the unsigned order of its bits), so the pivot searches issue integer
// instructions only: the double pipe of this GPU is narrow.  A NaN sorts above every
// number, so a NaN pivot reads as a singular matrix.
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull, kInfBits = 0x7ff0000000000000ull;

__device__ __forceinline__ unsigned long long abs_key(double x)
{
    return (unsigned long long)__double_as_longlong(x) & kAbsMask;
}

// block-wide (max key, smallest index) reduction, result in every thread: warp
// shuffles, then one warp over the warps' results.  sk, si hold 33 entries.
__device__ void block_argmax(unsigned long long &key, int &idx, unsigned long long *sk, int *si)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, key, o);
        const int i = __shfl_xor_sync(0xffffffffu, idx, o);
        if (a > key || (a == key && i < idx)) { key = a; idx = i; }
    }
    if (lane == 0) { sk[wid] = key; si[wid] = idx; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        key = lane < nw ? sk[lane] : 0ull;
        idx = lane < nw ? si[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, key, o);
            const int i = __shfl_xor_sync(0xffffffffu, idx, o);
            if (a > key || (a == key && i < idx)) { key = a; idx = i; }
        }
        if (lane == 0) { sk[32] = key; si[32] = idx; }
    }
    __syncthreads();
    key = sk[32];
    idx = si[32];
}

// Blocked Gauss-Jordan: the same elimination, kGjPanel pivot steps per round q.
// Panel P = [k0, k0 + np).  Let B = Pi A_P (the panel's columns after its row
// interchanges Pi) and B_P its rows at the panel positions.  The panel's elementary
// transformations multiply to Q = I + (W - I_P) e_P^T with Q B = e_P, so W_P = B_P^-1
// and W_R = -B_R B_P^-1 on the other rows R.  Every other column j becomes
//   Q Pi A_j:   rows i in P:  G_j = B_P^-1 (Pi A_j)_P,   rows i in R:  (Pi A_j)_i - B_i G_j,
// and the panel's own columns become W.
//
// Round q reads matrix A_q and writes A_(q+1) (two buffers in turn), so any block may
// update any part of it.  Block 0 searches the pivots: it runs the panel's steps on
// rows >= k0 only (the rows above never take part in pivoting, and W on rows >= k0,
// B_P^-1 included, does not depend on them), in shared memory, and publishes the
// pivot rows and B_P^-1.  Look-ahead: while blocks 1.. apply panel q to the matrix,
// block 0 waits only for the columns of panel q + 1 (done first, in row chunks, each
// chunk signalling a counter) and then searches panel q + 1's pivots, so the serial
// pivot search overlaps the update and each round costs one grid barrier.
//
// Panel steps: a thread owns rows i = k0 + t, k0 + t + 512, ...; the previous step's
// update already reduced its rows to one pivot candidate, so a step is one block
// reduction, the new pivot row formed by one warp, and eight fused multiply-adds per
// row (the pivot column is updated as a column whose entry is zero, which gives
// -B_ik / B_kk).
constexpr int kGjPanel = 8;

template <bool STAGE>
__device__ __forceinline__ float gj_ldf(const float *P, int64_t idx)
{
    if constexpr (STAGE) return P[idx];
    else return __ldcg(P + idx);
}

// |x| of a float as the unsigned order of its bits; a NaN sorts above infinity
__device__ __forceinline__ unsigned fkey(float x) { return __float_as_uint(x) & 0x7fffffffu; }
constexpr unsigned kFInfBits = 0x7f800000u;

struct GjShared {
    unsigned long long sk[33];
    int si[33];
    float nk[kGjPanel], rk[kGjPanel];   // new pivot row, old row k (the search, in float)
    int rrow[2 * kGjPanel], rsrc[2 * kGjPanel], nR, pv[kGjPanel];
    int bsrc[kGjPanel], okB;             // source rows of B_P; its inverse succeeded
    double binv[kGjPanel][kGjPanel];    // B_P^-1 of the round's panel
    double V[kGjPanel][kGjPanel], G[kGjPanel][kGjPanel];
    double B[kGjPanel][kGjPanel];       // B_P, then B_P^-1 (block 0)
};

// Pivot search of the panel [k0, k0 + np) of A (one block), then B_P^-1 (row c at
// binv + c kGjPanel).  The search only chooses the pivot rows, so it runs the panel's
// steps in float (the narrow double pipe made it the serial part of every round):
// rows >= k0 of the panel columns, rounded to float, into Pw (column-major,
// Pw[c M + i]).  B_P (the chosen rows of the panel, in their order, from the double
// matrix) is then inverted in double by one warp without further pivoting -- the
// elimination the double search would have done on those rows -- and a pivot at or
// below tinykey there means S is singular.  Returns false if S is singular.
template <bool STAGE>
__device__ bool gj_panel(int M, const double *A, int k0, int np, unsigned long long tinykey,
                         float *Pw, int *pivrow, double *binv, GjShared &sh)
{
    for (int e = threadIdx.x; e < (M - k0) * np; e += blockDim.x) {
        const int i = k0 + e / np, c = e % np;
        Pw[c * M + i] = (float)__ldcg(&A[(int64_t)i * M + k0 + c]);
    }
    __syncthreads();
    unsigned long long ck = 0ull;
    int ci = M;
    for (int i = k0 + threadIdx.x; i < M; i += blockDim.x) {
        const unsigned long long a = fkey(gj_ldf<STAGE>(Pw, i));
        if (a > ck) { ck = a; ci = i; }
    }
    bool ok = true;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = 0; c < np; c++) {
        const int k = k0 + c;
        // pivot: the block's (max |B_ik|, smallest i) over i >= k; warp 0 then forms the
        // new pivot row and keeps the old row k, all before the second barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, ck, o);
            const int i = __shfl_xor_sync(0xffffffffu, ci, o);
            if (a > ck || (a == ck && i < ci)) { ck = a; ci = i; }
        }
        if (lane == 0) { sh.sk[wid] = ck; sh.si[wid] = ci; }
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            ck = lane < nw ? sh.sk[lane] : 0ull;
            ci = lane < nw ? sh.si[lane] : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, ck, o);
                const int i = __shfl_xor_sync(0xffffffffu, ci, o);
                if (a > ck || (a == ck && i < ci)) { ck = a; ci = i; }
            }
            if (lane == 0) { sh.sk[32] = ck; sh.si[32] = ci; }
            if (ck > 0ull && ck <= kFInfBits && ci < M && lane < np) {
                const int p = ci;
                const float ipiv = 1.0f / gj_ldf<STAGE>(Pw, c * M + p);
                sh.rk[lane] = gj_ldf<STAGE>(Pw, lane * M + k);
                sh.nk[lane] = lane == c ? ipiv : gj_ldf<STAGE>(Pw, lane * M + p) * ipiv;
                if (lane == 0) sh.pv[c] = p;
            }
        }
        __syncthreads();  // rows k and p read before any row is written
        ck = sh.sk[32];
        ci = sh.si[32];
        if (ck == 0ull || ck > kFInfBits || ci >= M) {  // same values in every thread
            ok = false;
            break;
        }
        const int p = ci;
        float nk[kGjPanel], rk[kGjPanel];
#pragma unroll
        for (int cc = 0; cc < kGjPanel; cc++) {
            nk[cc] = cc < np ? sh.nk[cc] : 0.0f;
            rk[cc] = cc < np ? sh.rk[cc] : 0.0f;
        }
        ck = 0ull;
        ci = M;
        for (int i = k0 + threadIdx.x; i < M; i += blockDim.x) {
            if (i == k) {
#pragma unroll
                for (int cc = 0; cc < kGjPanel; cc++)
                    if (cc < np) Pw[cc * M + k] = nk[cc];
                continue;
            }
            float b[kGjPanel], f = 0.0f;
#pragma unroll
            for (int cc = 0; cc < kGjPanel; cc++) {
                b[cc] = cc >= np ? 0.0f : (i == p ? rk[cc] : gj_ldf<STAGE>(Pw, cc * M + i));
                if (cc == c) { f = b[cc]; b[cc] = 0.0f; }
            }
#pragma unroll
            for (int cc = 0; cc < kGjPanel; cc++) {
                if (cc >= np) continue;
                const float v = fmaf(-f, nk[cc], b[cc]);
                Pw[cc * M + i] = v;
                if (cc == c + 1 && i > k) {
                    const unsigned long long a = fkey(v);
                    if (a > ck) { ck = a; ci = i; }  // rows ascending per thread: first wins ties
                }
            }
        }
    }
    __syncthreads();
    if (!ok) return false;
    // the rows that the interchanges bring to positions k0 .. k0 + np - 1
    if (threadIdx.x == 0) {
        int pos[2 * kGjPanel], src[2 * kGjPanel], n = 0;
        auto find = [&](int r) {
            for (int t = 0; t < n; t++)
                if (pos[t] == r) return t;
            pos[n] = r;
            src[n] = r;
            return n++;
        };
        for (int c = 0; c < np; c++) {
            pivrow[k0 + c] = sh.pv[c];
            const int ta = find(k0 + c), tb = find(sh.pv[c]);
            const int t = src[ta];
            src[ta] = src[tb];
            src[tb] = t;
        }
        for (int m = 0; m < np; m++) sh.bsrc[m] = src[find(k0 + m)];
    }
    __syncthreads();
    // B_P^-1 in double by warp 0: Gauss-Jordan in the chosen order (entries lane, lane + 32)
    if (wid == 0) {
        for (int e = lane; e < kGjPanel * kGjPanel; e += 32) {
            const int r = e / kGjPanel, c = e % kGjPanel;
            sh.B[r][c] = (r < np && c < np) ? __ldcg(&A[(int64_t)sh.bsrc[r] * M + k0 + c])
                                            : (r == c ? 1.0 : 0.0);
        }
        __syncwarp();
        bool good = true;
        for (int c = 0; c < np; c++) {
            const double piv = sh.B[c][c];
            const unsigned long long pk = abs_key(piv);
            if (pk <= tinykey || pk > kInfBits) { good = false; break; }  // same in every lane
            const double ip = 1.0 / piv;
            double nv[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int e = lane + 32 * h, r = e / kGjPanel, j = e % kGjPanel;
                const double bc = sh.B[c][j], f = sh.B[r][c];
                if (r == c) nv[h] = j == c ? ip : bc * ip;
                else nv[h] = j == c ? -f * ip : fma(-f, bc * ip, sh.B[r][j]);
            }
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int e = lane + 32 * h;
                sh.B[e / kGjPanel][e % kGjPanel] = nv[h];
            }
            __syncwarp();
        }
        if (lane == 0) sh.okB = good ? 1 : 0;
    }
    __syncthreads();
    if (!sh.okB) return false;
    for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e % np;
        binv[r * kGjPanel + c] = sh.B[r][c];
    }
    return true;
}

// The swap set of the panel [k0, k0 + np): the rows its interchanges move (rrow) and,
// for each, the row its value comes from (rsrc); slot[row] = entry or -1 (thread 0,
// from the pivot rows in sh.pv).
__device__ void gj_swapset(int k0, int np, int *slot, GjShared &sh)
{
    int n = 0;
    for (int k = k0; k < k0 + np; k++) {
        const int p = sh.pv[k - k0];
        int a = -1, b = -1;
        for (int t = 0; t < n; t++)
            if (sh.rrow[t] == k) a = t;
        if (a < 0) { sh.rrow[n] = k; sh.rsrc[n] = k; a = n++; }
        for (int t = 0; t < n; t++)
            if (sh.rrow[t] == p) b = t;
        if (b < 0) { sh.rrow[n] = p; sh.rsrc[n] = p; b = n++; }
        const int tmp = sh.rsrc[a];
        sh.rsrc[a] = sh.rsrc[b];
        sh.rsrc[b] = tmp;
    }
    sh.nR = n;
    for (int t = 0; t < n; t++) slot[sh.rrow[t]] = t;
}

// One work item of round q (one block): column tile `tile` (kGjPanel columns), rows
// [r0, r1), read from Aq and written to Aq1.  The panel's own tile gets W.
__device__ void gj_item(int M, const double *Aq, double *Aq1, int k0, int np, int tile, int r0, int r1,
                        const int *slot, GjShared &sh)
{
    const int jc = threadIdx.x % kGjPanel, rg = threadIdx.x / kGjPanel, nrg = blockDim.x / kGjPanel;
    const int j = tile * kGjPanel + jc;
    const bool wtile = tile * kGjPanel == k0;
    if (!wtile) {
        // (Pi A_j)_P and G_j = B_P^-1 (Pi A_j)_P for the tile's columns
        for (int e = threadIdx.x; e < np * kGjPanel; e += blockDim.x) {
            const int m = e / kGjPanel, c = e % kGjPanel, jj = tile * kGjPanel + c;
            const int src = sh.rsrc[slot[k0 + m]];
            sh.V[m][c] = jj < M ? __ldcg(&Aq[(int64_t)src * M + jj]) : 0.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < np * kGjPanel; e += blockDim.x) {
            const int m = e / kGjPanel, c = e % kGjPanel;
            double g = 0.0;
            for (int l = 0; l < np; l++) g = fma(sh.binv[m][l], sh.V[l][c], g);
            sh.G[m][c] = g;
        }
        __syncthreads();
    }
    if (j < M && (!wtile || jc < np)) {
        double g[kGjPanel];
#pragma unroll
        for (int m = 0; m < kGjPanel; m++) g[m] = m < np ? (wtile ? sh.binv[m][jc] : sh.G[m][jc]) : 0.0;
        for (int i0 = r0 + rg; i0 < r1; i0 += 4 * nrg) {
            double x[4], b[4][kGjPanel];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * nrg;
                x[u] = 0.0;
#pragma unroll
                for (int m = 0; m < kGjPanel; m++) b[u][m] = 0.0;
                if (i < r1 && (i < k0 || i >= k0 + np)) {
                    const int sl = slot[i];
                    const int64_t src = (int64_t)(sl >= 0 ? sh.rsrc[sl] : i) * M;
                    if (!wtile) x[u] = __ldcg(&Aq[src + j]);
#pragma unroll
                    for (int m = 0; m < kGjPanel; m++)
                        if (m < np) b[u][m] = __ldcg(&Aq[src + k0 + m]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * nrg;
                if (i >= r1) break;
                double out = x[u];
                if (i >= k0 && i < k0 + np) {
#pragma unroll
                    for (int m = 0; m < kGjPanel; m++)
                        if (i == k0 + m) out = wtile ? sh.binv[m][jc] : sh.G[m][jc];
                } else {
#pragma unroll
                    for (int m = 0; m < kGjPanel; m++) out = fma(-b[u][m], g[m], out);
                }
                Aq1[(int64_t)i * M + j] = out;
            }
        }
    }
    __syncthreads();  // V, G reused by the next item
}

// Bounded wait of block 0 for `target` finished chunks; false (status set) on time-out.
__device__ bool gj_wait(unsigned *done, unsigned target, int *status)
{
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned it = 0;
        const unsigned lim = wait_limit(status, kBarrierSpins);
        while (*(volatile unsigned *)done < target)
            if (++it > lim) {
                atomicOr(status, LBF_DEV_TIMEOUT);
                ok = 0;
                break;
            }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <bool STAGE>
__global__ void __launch_bounds__(kGjThreads)
k_gj_blocked(int M, double *A0, double *A1, double *amax, int *pivrow, double *binv, unsigned *done,
             GridBarrier *bar, int *status, double *Pg)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    int *slot = (int *)gsm;                                     // M: swap-set entry of a row, or -1
    float *Pw = STAGE ? (float *)(slot + M) : (float *)Pg;      // block 0's panel, Pw[c M + i]
    __shared__ GjShared sh;
    const unsigned nb = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)nb * blockDim.x;
    const int64_t MM = (int64_t)M * M;
    unsigned long long *akey = (unsigned long long *)amax;
    for (int i = threadIdx.x; i < M; i += blockDim.x) slot[i] = -1;
    {
        unsigned long long big = 0ull;
        int unused = 0;
        for (int64_t e = tid; e < MM; e += nthr) big = max(big, abs_key(A0[e]));
        block_argmax(big, unused, sh.sk, sh.si);
        if (threadIdx.x == 0) akey[blockIdx.x] = big;
    }
    if (!grid_barrier(bar, nb, status)) return;
    // a pivot at or below M 2^-52 max|S_ij| counts as zero: S is singular to double precision
    unsigned long long big = 0ull;
    for (unsigned q = 0; q < nb; q++) big = max(big, __ldcg(&akey[q]));
    const unsigned long long tinykey =
        big > kInfBits ? kInfBits : abs_key(__longlong_as_double((long long)big) * (double)M * 0x1p-52);
    const int ntile = (M + kGjPanel - 1) / kGjPanel;
    // row chunks of the next panel's tile and of the panel's own tile
    const int hc = max(64, (((M + 15) / 16 + 63) / 64) * 64), nch = (M + hc - 1) / hc;
    const bool lone = nb == 1;  // a single block does everything itself
    const int nwk = lone ? 1 : (int)nb - 1, wk = lone ? 0 : (int)blockIdx.x - 1;
    if (blockIdx.x == 0 &&
        !gj_panel<STAGE>(M, A0, 0, min(M, kGjPanel), tinykey, Pw, pivrow, binv, sh) && threadIdx.x == 0)
        atomicOr(status, 4);
    unsigned waited = 0;
    for (int k0 = 0, q = 0; k0 < M; k0 += kGjPanel, q++) {
        const int np = min(M - k0, kGjPanel), n0 = k0 + kGjPanel;
        const double *Aq = (q & 1) ? A1 : A0;
        double *Aq1 = (q & 1) ? A0 : A1;
        if (!grid_barrier(bar, nb, status)) return;
        if (*(volatile int *)status & 4) return;  // singular: every block stops here
        const bool worker = blockIdx.x != 0 || lone;
        if (worker) {
            for (int e = threadIdx.x; e < kGjPanel * kGjPanel; e += blockDim.x)
                sh.binv[e / kGjPanel][e % kGjPanel] = __ldcg(&binv[(q & 1) * kGjPanel * kGjPanel + e]);
            if (threadIdx.x < np) sh.pv[threadIdx.x] = __ldcg(&pivrow[k0 + threadIdx.x]);
            __syncthreads();
            if (threadIdx.x == 0) gj_swapset(k0, np, slot, sh);
            __syncthreads();
        }
        const int tp = k0 / kGjPanel, tn = n0 < M ? tp + 1 : -1;
        const int cn = tn >= 0 ? nch : 0;  // chunk items of the next panel's tile
        // the other tiles in R row parts when there are more tiles than blocks to take them
        const int nother = ntile - 1 - (tn >= 0 ? 1 : 0);
        const int R = (nwk < cn + nch + nother && M >= 256) ? 2 : 1, hr = (M + R - 1) / R;
        const int nitems = cn + nch + R * nother;
        double *binv1 = binv + ((q + 1) & 1) * kGjPanel * kGjPanel;
        if (blockIdx.x == 0 && !lone) {
            if (tn >= 0) {
                waited += cn;
                if (!gj_wait(done, waited, status)) return;
                if (!gj_panel<STAGE>(M, Aq1, n0, min(M - n0, kGjPanel), tinykey, Pw, pivrow, binv1, sh) &&
                    threadIdx.x == 0)
                    atomicOr(status, 4);
            }
        } else {
            for (int w = wk; w < nitems; w += nwk) {
                int tile, r0 = 0, r1 = M;
                if (w < cn) {
                    tile = tn;
                    r0 = w * hc;
                    r1 = min(M, r0 + hc);
                } else if (w < cn + nch) {
                    tile = tp;
                    r0 = (w - cn) * hc;
                    r1 = min(M, r0 + hc);
                } else {  // the other tiles in order, skipping tp and tn, in R row parts
                    const int t = w - cn - nch;
                    tile = t / R;
                    r0 = (t % R) * hr;
                    r1 = min(M, r0 + hr);
                    const int lo = tn >= 0 ? min(tp, tn) : tp, hi = tn >= 0 ? max(tp, tn) : INT_MAX;
                    if (tile >= lo) tile++;
                    if (tile >= hi) tile++;
                }
                gj_item(M, Aq, Aq1, k0, np, tile, r0, r1, slot, sh);
                if (w < cn) {  // the chunk's rows visible device-wide, then counted
                    __threadfence();
                    __syncthreads();
                    if (threadIdx.x == 0) atomicAdd(done, 1u);
                    if (lone && w == cn - 1 &&
                        !gj_panel<STAGE>(M, Aq1, n0, min(M - n0, kGjPanel), tinykey, Pw, pivrow, binv1, sh) &&
                        threadIdx.x == 0)
                        atomicOr(status, 4);
                }
            }
        }
        __syncthreads();
        if (worker && threadIdx.x == 0)
            for (int t = 0; t < sh.nR; t++) slot[sh.rrow[t]] = -1;
    }
}

__global__ void k_gj_init(int M, int *__restrict__ pivrow)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) pivrow[k] = k;
}

// Undo the row interchanges: swapping columns k and pivrow[k] for k = M-1, ..., 0 is
// the column permutation out_j = in_perm[j]; one thread composes it.  pivrow starts
// as the identity, so steps an early stop (a singular pivot or a barrier that gave up)
// never reached swap nothing.
__global__ void k_gj_perm(int M, const int *__restrict__ pivrow, int *__restrict__ perm)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int j = 0; j < M; j++) perm[j] = j;
    for (int k = M - 1; k >= 0; k--) {
        const int p = pivrow[k];
        if (p != k && p >= 0 && p < M) {
            const int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
        }
    }
}

// out[i][j] = in[i][perm[j]] (block per row)
__global__ void k_gj_gather(int M, const double *__restrict__ in, const int *__restrict__ perm,
                            double *__restrict__ out)
{
    const int64_t i = blockIdx.x;
    for (int j = threadIdx.x; j < M; j += blockDim.x) out[i * M + j] = __ldg(&in[i * M + perm[j]]);
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
constexpr size_t kGjSmemCap = 200 * 1024;

// scratch of lbf_border_start: the second matrix buffer, block 0's panel (when it
// does not fit in shared memory), the partial maxima, pivot rows, permutation, B_P^-1
// twice, the chunk counter and the grid barrier
size_t lbf_gj_scratch_doubles(int M)
{
    return (size_t)M * M + (size_t)M * kGjPanel + kGjMaxBlocks + (size_t)M + 2 * kGjPanel * kGjPanel + 64;
}

// S and S^-1 need the planar nodes and the centres only, not the tree: they run on a
// side stream (highest priority) that forks from s here, and the inverse takes part of
// the SMs so that the tree build on s proceeds beside it.
int lbf_border_start(lbf_plan *pl, cudaStream_t s0, const double2 *xi_o, double *scratch)
{
    int M = pl->M;
    double *S = pl->Sinv;
    int lo = 0, hi = 0;
    LBF_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    LBF_CUDA(cudaStreamCreateWithPriority(&pl->side, cudaStreamNonBlocking, hi));
    for (auto &e : pl->fork) LBF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    LBF_CUDA(cudaEventRecord(pl->fork[0], s0));
    const cudaStream_t s = pl->side;
    LBF_CUDA(cudaStreamWaitEvent(s, pl->fork[0], 0));
    lbf_prof_mark(LBF_STAGE_INVERSE, 1, s);
    // until the inverse starts, the first M^2 doubles of its scratch hold the list of
    // Schur entries summed directly (at most M^2 - M of them)
    int rc = lbf_schur_build(pl, s, xi_o, S, (int32_t *)scratch, 2 * (int64_t)M * M);
    if (rc) return rc;
    if (pl->lu) {  // many islands: LU factors in double-float instead of the inverse
        if ((rc = lbf_schur_lu_factor(pl, s, scratch))) return rc;
        lbf_prof_mark(LBF_STAGE_INVERSE, 0, s);
        LBF_CUDA(cudaEventRecord(pl->fork[1], s));
        return LBF_OK;
    }
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    LBF_CUDA(cudaGetDevice(&dev));
    LBF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    LBF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    // shared memory: the row slots (M), block 0's panel if it fits
    const size_t sm_base = sizeof(int) * (size_t)(M + 1);
    const size_t sm_w = sizeof(float) * (size_t)M * kGjPanel;
    const bool stage = sm_base + sm_w <= kGjSmemCap;
    const size_t smem = sm_base + (stage ? sm_w : 0);
    if (smem > kGjSmemCap) return LBF_EINVAL;  // M above ~51,000
    const void *fn = stage ? (const void *)k_gj_blocked<true> : (const void *)k_gj_blocked<false>;
    LBF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGjSmemCap));
    LBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGjThreads, smem));
    if (!coop || per_sm < 1) return LBF_ECUDA;
    // one block per SM, on two thirds of the SMs: the rest build the tree meanwhile
    // (measured at M = 1024: half, two thirds and four fifths within 1 % of each other
    // over the whole step; all SMs stall the tree build)
    // and no more blocks than a round has work items (block 0 and, per round, the chunks
    // of two tiles and the other tiles): each block holds a whole SM, so a small S must
    // not take the GPU from other streams' work
    const int ntile = (M + kGjPanel - 1) / kGjPanel;
    const int hc = std::max(64, (((M + 15) / 16 + 63) / 64) * 64), nch = (M + hc - 1) / hc;
    const int nb = (int)std::min<int64_t>(std::min(std::max(2, 2 * nsm / 3), 1 + 2 * nch + ntile),
                                          kGjMaxBlocks);
    double *S1 = scratch;                                        // M x M
    double *Pg = S1 + (size_t)M * M;                             // M x kGjPanel
    double *amax = Pg + (size_t)M * kGjPanel;                    // kGjMaxBlocks
    double *binv = amax + kGjMaxBlocks;                          // 2 x kGjPanel^2
    int *pivrow = (int *)(binv + 2 * kGjPanel * kGjPanel);       // M
    int *perm = pivrow + M;                                      // M
    unsigned *done = (unsigned *)(perm + M);                     // 1
    GridBarrier *bar = (GridBarrier *)(done + 2);
    LBF_CUDA(cudaMemsetAsync(done, 0, 2 * sizeof(unsigned) + sizeof(GridBarrier), s));
    lbf_inject_barrier(&bar->count, s);
    LBF_LAUNCH(k_gj_init, lbf_cdiv(M, 256), 256, 0, s, M, pivrow);
    // round q reads A_q and writes A_(q+1); start so that the result lands in S1
    const int rounds = (M + kGjPanel - 1) / kGjPanel;
    double *A0 = S, *A1 = S1;
    if (!(rounds & 1)) {
        LBF_CUDA(cudaMemcpyAsync(S1, S, sizeof(double) * (size_t)M * M, cudaMemcpyDeviceToDevice, s));
        std::swap(A0, A1);
    }
    int *status = pl->dev_status;
    void *args[] = {&M, &A0, &A1, &amax, &pivrow, &binv, &done, &bar, &status, &Pg};
    LBF_CUDA(cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kGjThreads), args, smem, s));
    g_lbf_launches.fetch_add(1, std::memory_order_relaxed);
    LBF_LAUNCH(k_gj_perm, 1, 32, 0, s, M, pivrow, perm);
    LBF_LAUNCH(k_gj_gather, M, 256, 0, s, M, S1, perm, S);
    LBF_CHECK_LAUNCH();
    lbf_prof_mark(LBF_STAGE_INVERSE, 0, s);
    LBF_CUDA(cudaEventRecord(pl->fork[1], s));
    return LBF_OK;
}

int lbf_border_build(lbf_plan *pl, cudaStream_t s, int32_t *work, int64_t work_len,
                     const SortBufs &sb)
{
    lbf_prof_mark(LBF_STAGE_BORDER, 1, s);
    int rc = lbf_mp_build(pl, s, work, work_len, sb);
    lbf_prof_mark(LBF_STAGE_BORDER, 0, s);
    if (rc) return rc;
    // join: later work on s sees S^-1
    LBF_CUDA(cudaStreamWaitEvent(s, pl->fork[1], 0));
    return LBF_OK;
}

void lbf_border_end(lbf_plan *pl)
{
    if (pl->side) {
        cudaStreamSynchronize(pl->side);
        cudaStreamDestroy(pl->side);
        pl->side = nullptr;
    }
    for (auto &e : pl->fork)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
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
