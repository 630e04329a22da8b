// The Schur complement S = D - F E of the border (Sec. 5, Eq. matrix_eqns_c) for many
// islands: LU factorisation with partial pivoting in double-float arithmetic, and the
// action of S^-1 (and S^-T) by triangular solves.
//
// Why not the inverse: the preconditioner needs S^-1 once per GMRES iteration, and
// the Gauss-Jordan inverse costs 2 M^3 flops on this GPU's narrow double pipe (11.5 s
// at M = 16384).  Why not float: S is a first-kind (log-kernel) system between the
// islands, and its condition number grows with M (about 4e5 at M = 256, 3e7 at
// M = 1024, 2e8 at M = 4096 for the star-cap family), beyond what a float
// factorisation can refine.  So the factorisation runs in double-float (pairs of
// floats, ~48-bit significands): the panels, the triangular solves and the combination
// of the trailing update's partial products on the float pipes, which issue 64 times
// faster than the double pipe, and the trailing update's products, almost all of its
// M^3 / 3 multiply-adds (the inverse would take M^3), on the tensor cores through an
// exact split of the operands into bf16 slices.  The
// preconditioner only has to be close to P^-1: GMRES solves the bordered system to
// its own tolerance whatever the rounding of S^-1 (which is about cond(S) 2^-46).
//
// Layout: the factors overwrite S in place, each entry stored as (hi, lo) floats in the
// 8 bytes of its double: L strictly below the diagonal (unit diagonal implied), U on
// and above it.  piv[k] = the row interchanged with row k at step k (row interchanges
// in the order of the steps, as in LAPACK's getrf); perm[i] = the original row that
// ends at position i, so P S = L U with (P f)_i = f_perm[i].
//
// Per panel of kLuNb columns [k0, k0 + w):
//   k_lu_panel (cooperative launch): the panel's elimination over the rows >= k0 with
//              the pivot search; each block keeps its share of the panel's rows in
//              shared memory; one grid barrier per column, at which every block
//              publishes its best candidate row (and the owner of row k its row), so
//              the interchange needs no second barrier;
//   k_lu_swap: the panel's interchanges applied to every column outside it;
//   k_lu_trsm: U12 = L11^-1 A12 (the panel's rows to the right of it);
//   k_oz_slice_rows, k_oz_slice_cols, k_lu_gemm_tc: A22 -= L21 U12 (the trailing
//              matrix) on the tensor cores, by an exact split of the double-float
//              operands into bf16 integer slices (below).
// A pivot at or below M 2^-50 max|S_ij| reports a singular S (status bit 4), a grid
// barrier that gave up a time-out; every later kernel of the factorisation then returns
// at once.
#include <algorithm>
#include <cuda_bf16.h>

#include "lbf_df64.cuh"
#include "lbf_internal.cuh"
#include "lbf_sync.cuh"

namespace {

constexpr int kLuNb = 64;          // panel width
constexpr int kLuThreads = 256;
constexpr int kLuTs = 64;          // row block of the triangular solves, GEMM tile
constexpr int kLuPad = 65;         // shared-memory row stride of 64-wide tiles
constexpr unsigned kLuSpins = 1u << 24;
constexpr int kLuMaxPanelBlocks = 1024;
constexpr size_t kLuSmemCap = 200 * 1024;

__device__ __forceinline__ df64 ld(float2 v) { return df64(v.x, v.y, 0); }
__device__ __forceinline__ float2 pk(df64 v) { return make_float2(v.hi, v.lo); }
__device__ __forceinline__ unsigned mag_key(float2 v) { return __float_as_uint(v.x) & 0x7fffffffu; }
constexpr unsigned kFInf = 0x7f800000u;

__device__ __forceinline__ bool lu_failed(const int *status)
{
    return (*(const volatile int *)status & (4 | LBF_DEV_TIMEOUT)) != 0;
}

// S (double) -> (hi, lo) floats in the same 8 bytes, and max |S_ij| as a bit key
__global__ void k_lu_convert(int64_t n, double *S, unsigned *amax)
{
    unsigned best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = S[i];
        const float hi = (float)d;
        const float lo = (float)(d - (double)hi);
        ((float2 *)S)[i] = make_float2(hi, lo);
        best = max(best, __float_as_uint(hi) & 0x7fffffffu);
    }
    __shared__ unsigned wb[32];
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) best = max(best, wb[k]);
        atomicMax(amax, best);
    }
}

// The panel [k0, k0 + w) over rows [k0, M).  Block b owns rows [k0 + b rpb, ...).
__global__ void __launch_bounds__(kLuThreads)
k_lu_panel(int M, int k0, int w, int rpb, float2 *A, int *piv, const unsigned *amax,
           unsigned *ckey, int *crow, float2 *cval, float2 *rjval, GridBarrier *bar, int *status)
{
    if (lu_failed(status)) return;  // same value in every block: set by an earlier launch
    extern __shared__ __align__(16) float2 lsm[];
    float2 *tile = lsm;                        // rpb x kLuNb
    float2 *lcol = lsm + (size_t)rpb * kLuNb;  // rpb
    __shared__ float2 pv[kLuNb], rj[kLuNb];
    __shared__ unsigned sk[kLuThreads / 32];
    __shared__ int si[kLuThreads / 32], sq[kLuThreads / 32];
    __shared__ int s_row, s_wb, s_sing;
    const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int r0 = k0 + b * rpb, r1 = min(M, r0 + rpb), nr = max(0, r1 - r0);
    for (int e = tid; e < nr * w; e += blockDim.x) {
        const int i = e / w, c = e % w;
        tile[i * kLuNb + c] = A[(int64_t)(r0 + i) * M + k0 + c];
    }
    const unsigned tiny = __float_as_uint(__uint_as_float(*amax) * (float)M * 0x1p-50f);
    __syncthreads();
    for (int c = 0; c < w; c++) {
        const int j = k0 + c, par = c & 1;
        // this block's candidate: the largest |entry| of column c on its rows >= j
        unsigned key = 0;
        int row = INT_MAX;
        for (int i = tid; i < nr; i += blockDim.x) {
            const int gi = r0 + i;
            if (gi < j) continue;
            const unsigned kk = mag_key(tile[i * kLuNb + c]);
            if (row == INT_MAX || kk > key || (kk == key && gi < row)) { key = kk; row = gi; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned k2 = __shfl_xor_sync(0xffffffffu, key, o);
            const int r2 = __shfl_xor_sync(0xffffffffu, row, o);
            if (r2 != INT_MAX && (row == INT_MAX || k2 > key || (k2 == key && r2 < row))) { key = k2; row = r2; }
        }
        if (lane == 0) { sk[wid] = key; si[wid] = row; }
        __syncthreads();
        if (tid == 0) {
            unsigned bk = 0;
            int br = INT_MAX;
            for (int q = 0; q < kLuThreads / 32; q++)
                if (si[q] != INT_MAX && (br == INT_MAX || sk[q] > bk || (sk[q] == bk && si[q] < br))) {
                    bk = sk[q];
                    br = si[q];
                }
            ckey[par * nb + b] = bk;
            crow[par * nb + b] = br;
            s_row = br;
        }
        __syncthreads();
        {
            const int cr = s_row;
            if (cr != INT_MAX && tid < w) cval[((size_t)par * nb + b) * kLuNb + tid] = tile[(cr - r0) * kLuNb + tid];
            if (j >= r0 && j < r1 && tid < w) rjval[par * kLuNb + tid] = tile[(j - r0) * kLuNb + tid];
        }
        if (!grid_barrier(bar, nb, status)) return;
        {
            // the winner over the blocks' candidates: a thread per candidate, then the
            // block's (max key, smallest row) reduction
            unsigned bk = 0;
            int br = INT_MAX, bq = -1;
            for (int q = tid; q < nb; q += blockDim.x) {
                const int rr = __ldcg(&crow[par * nb + q]);
                if (rr == INT_MAX) continue;
                const unsigned kk = __ldcg(&ckey[par * nb + q]);
                if (bq < 0 || kk > bk || (kk == bk && rr < br)) { bk = kk; br = rr; bq = q; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned k2 = __shfl_xor_sync(0xffffffffu, bk, o);
                const int r2 = __shfl_xor_sync(0xffffffffu, br, o);
                const int q2 = __shfl_xor_sync(0xffffffffu, bq, o);
                if (q2 >= 0 && (bq < 0 || k2 > bk || (k2 == bk && r2 < br))) { bk = k2; br = r2; bq = q2; }
            }
            __syncthreads();  // sk, si reused
            if (lane == 0) { sk[wid] = bk; si[wid] = br; sq[wid] = bq; }
            __syncthreads();
            if (tid == 0) {
                bk = 0;
                br = INT_MAX;
                bq = -1;
                for (int q = 0; q < kLuThreads / 32; q++)
                    if (sq[q] >= 0 && (bq < 0 || sk[q] > bk || (sk[q] == bk && si[q] < br))) {
                        bk = sk[q];
                        br = si[q];
                        bq = sq[q];
                    }
                s_row = bq < 0 ? j : br;
                s_wb = bq;
                s_sing = bq < 0 || bk <= tiny || bk > kFInf;
                if (b == 0) piv[j] = s_row;
            }
        }
        __syncthreads();
        if (s_sing) {
            if (b == 0 && tid == 0) atomicOr(status, 4);
            break;  // every block takes the same branch
        }
        const int p = s_row, wb = s_wb;
        if (tid < w) {
            pv[tid] = __ldcg(&cval[((size_t)par * nb + wb) * kLuNb + tid]);
            rj[tid] = __ldcg(&rjval[par * kLuNb + tid]);
        }
        __syncthreads();
        // the interchange of rows j and p, within the panel
        if (j >= r0 && j < r1 && tid < w) tile[(j - r0) * kLuNb + tid] = pv[tid];
        if (p != j && p >= r0 && p < r1 && tid < w) tile[(p - r0) * kLuNb + tid] = rj[tid];
        __syncthreads();
        const df64 invp = df_rcp(ld(pv[c]));
        for (int i = tid; i < nr; i += blockDim.x) {
            if (r0 + i <= j) continue;
            const float2 l = pk(ld(tile[i * kLuNb + c]) * invp);
            tile[i * kLuNb + c] = l;
            lcol[i] = l;
        }
        __syncthreads();
        const int nc = w - c - 1;
        for (int e = tid; e < nr * nc; e += blockDim.x) {
            const int i = e / nc, cc = c + 1 + e % nc;
            if (r0 + i <= j) continue;
            tile[i * kLuNb + cc] = pk(df_fma(-ld(lcol[i]), ld(pv[cc]), ld(tile[i * kLuNb + cc])));
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * w; e += blockDim.x) {
        const int i = e / w, c = e % w;
        A[(int64_t)(r0 + i) * M + k0 + c] = tile[i * kLuNb + c];
    }
}

// the panel's interchanges, in order, on every column outside the panel
__global__ void k_lu_swap(int M, int k0, int w, float2 *A, const int *piv, const int *status)
{
    if (lu_failed(status)) return;
    __shared__ int sp[kLuNb];
    if (threadIdx.x < w) sp[threadIdx.x] = piv[k0 + threadIdx.x];
    __syncthreads();
    const int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (col >= M || (col >= k0 && col < k0 + w)) return;
    for (int c = 0; c < w; c++) {
        const int p = sp[c], j = k0 + c;
        if (p == j) continue;
        const float2 a = A[(int64_t)j * M + col], q = A[(int64_t)p * M + col];
        A[(int64_t)j * M + col] = q;
        A[(int64_t)p * M + col] = a;
    }
}

// U12 = L11^-1 A12 on 64 columns per block (column-oriented forward substitution)
__global__ void __launch_bounds__(kLuThreads)
k_lu_trsm(int M, int k0, int w, float2 *A, const int *status)
{
    if (lu_failed(status)) return;
    extern __shared__ __align__(16) float2 tsm[];
    float2 *Ls = tsm;                    // w x kLuPad
    float2 *Xs = tsm + kLuNb * kLuPad;   // w x kLuPad
    const int c0 = k0 + w + blockIdx.x * kLuTs, nc = min(kLuTs, M - c0);
    const int tid = threadIdx.x;
    for (int e = tid; e < w * w; e += blockDim.x) {
        const int r = e / w, t = e % w;
        Ls[r * kLuPad + t] = A[(int64_t)(k0 + r) * M + k0 + t];
    }
    for (int e = tid; e < w * kLuTs; e += blockDim.x) {
        const int r = e / kLuTs, cc = e % kLuTs;
        if (cc < nc) Xs[r * kLuPad + cc] = A[(int64_t)(k0 + r) * M + c0 + cc];
    }
    __syncthreads();
    for (int t = 0; t < w - 1; t++) {
        const int cnt = (w - 1 - t) * nc;
        for (int e = tid; e < cnt; e += blockDim.x) {
            const int r = t + 1 + e / nc, cc = e % nc;
            Xs[r * kLuPad + cc] = pk(df_fma(-ld(Ls[r * kLuPad + t]), ld(Xs[t * kLuPad + cc]), ld(Xs[r * kLuPad + cc])));
        }
        __syncthreads();
    }
    for (int e = tid; e < w * kLuTs; e += blockDim.x) {
        const int r = e / kLuTs, cc = e % kLuTs;
        if (cc < nc) A[(int64_t)(k0 + r) * M + c0 + cc] = Xs[r * kLuPad + cc];
    }
}

// ---- the trailing update on the tensor cores --------------------------------------
// A22 -= L21 U12 with K = w <= 64, the operands in double-float (~48-bit significands).
// The bf16 tensor-core products reach that precision by an exact split (Ozaki's scheme):
// each row i of L21 is scaled by 2^-e_i (|l_ik| 2^-e_i < 1, e_i from the row's largest
// entry), each column j of U12 by 2^-f_j, and the scaled values are cut into kOzS slices
// of 8 bits, x = sum_s v_s 2^(-8(s+1)), v_s a rounded integer (|v_0| <= 256, later
// |v_s| <= 128), exact in bf16.  A product of two slices is an integer below 2^16 and a
// sum of 64 of them, over the (s, t) with s + t = d, stays below 2^24: exact in the
// float accumulators of the MMA.  The update is then
//   (L21 U12)_ij = 2^(e_i + f_j) sum_d 2^(-8(d+2)) P_d,ij,  P_d = sum_{s+t=d} L_s U_t^T,
// with the pairs s + t > kOzD dropped (below 2^-48 of the row-times-column scale), and
// each tile combines its kOzD + 1 accumulators in double-float.
constexpr int kOzS = 6;              // slices per operand
constexpr int kOzD = 5;              // slice pairs with s + t <= kOzD
constexpr int kTcM = 128, kTcN = 64; // tile of A22 per CTA: 128 rows x 64 columns
constexpr int kTcLBytes = kTcM * kLuNb * 2;  // one bf16 slice of a 128-row block
constexpr int kTcUBytes = kTcN * kLuNb * 2;  // one bf16 slice of a 64-column block
constexpr int kTcSmem = kOzS * (kTcLBytes + kTcUBytes);
// instruction descriptor of tcgen05.mma kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

// element (r, k) of a K-major operand tile without swizzle, in bf16 units: 8 x 8 core
// matrices of 8 rows x 16 bytes, the 8 K-adjacent cores of an 8-row group 128 bytes
// apart (the descriptor's leading-dimension offset), the 8-row groups 1024 bytes apart
// (its stride-dimension offset)
__device__ __forceinline__ int core_off(int r, int k)
{
    return ((r >> 3) * 8 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (no swizzle): start address, leading- and
// stride-dimension byte offsets (all in 16-byte units), descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred P1;\n mbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
                 " selp.b32 %0, 1, 0, P1;\n}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes, one lane per thread
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t u[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                   "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]),
                   "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(u[i]);
}

// 2^x as a float, 0 below the normal range (x above 127 does not occur: the entries
// of S and its factors are far below 2^100)
__device__ __forceinline__ float pow2f(int x)
{
    return x < -126 ? 0.f : __int_as_float((min(x, 127) + 127) << 23);
}

// the exponent e with max < 2^e <= 2 max (0 for max = 0)
__device__ __forceinline__ int exp_above(float mx)
{
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e;
}

// kOzS slices of the eight values x[0..7] (each scaled to |x| < 1), packed as bf16 into
// out[s] (16 bytes: one row of a core matrix)
__device__ __forceinline__ void oz_split8(df64 (&x)[8], uint4 (&out)[kOzS])
{
#pragma unroll
    for (int sl = 0; sl < kOzS; sl++) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float th = x[i].hi * 256.f, tl = x[i].lo * 256.f;
            const float v = rintf(th);
            df_two_sum(th - v, tl, x[i].hi, x[i].lo);  // th - v is exact
            const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
            if (i & 1) w[i >> 1] |= b << 16;
            else w[i >> 1] = b;
        }
        out[sl] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Slices of L21 = A[k1.., k0 .. k0 + w) (k1 = k0 + w), rows in 128-row blocks: 8 threads
// a row, 8 columns each; Limg[rb][s] is the shared-memory image of slice s of block rb,
// el[rr] the exponent of row k1 + rr.  Rows past M and columns past w give zeros.
__global__ void __launch_bounds__(256)
k_oz_slice_rows(int M, int k0, int w, const float2 *A, uint4 *Limg, int *el, const int *status)
{
    if (lu_failed(status)) return;
    const int t = threadIdx.x, kg = t & 7;
    const int rr = blockIdx.x * 32 + (t >> 3), row = k0 + w + rr;
    df64 x[8];
    unsigned key = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int k = kg * 8 + i;
        const float2 v = (row < M && k < w) ? A[(int64_t)row * M + k0 + k] : make_float2(0.f, 0.f);
        x[i] = df64(v.x, v.y, 0);
        key = max(key, __float_as_uint(v.x) & 0x7fffffffu);
    }
    key = max(key, __shfl_xor_sync(0xffffffffu, key, 1));
    key = max(key, __shfl_xor_sync(0xffffffffu, key, 2));
    key = max(key, __shfl_xor_sync(0xffffffffu, key, 4));
    const int e = exp_above(__uint_as_float(key));
    const float sc = pow2f(-e);
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = df_ldexp(x[i], sc);
    uint4 out[kOzS];
    oz_split8(x, out);
    const int rb = rr >> 7, r = rr & 127;
#pragma unroll
    for (int sl = 0; sl < kOzS; sl++)
        Limg[((size_t)(rb * kOzS + sl) * kTcLBytes + 2 * core_off(r, kg * 8)) / 16] = out[sl];
    if (kg == 0) el[rr] = e;
}

// Slices of U12 = A[k0 .. k0 + w, k1 ..), columns in 64-column blocks: a block of 512
// threads per column block, (column, 8 rows of K) per thread; Uimg[cb][s] as above,
// eu[cc] the exponent of column k1 + cc.
__global__ void __launch_bounds__(512)
k_oz_slice_cols(int M, int k0, int w, const float2 *A, uint4 *Uimg, int *eu, const int *status)
{
    if (lu_failed(status)) return;
    __shared__ unsigned red[8][kTcN];
    const int t = threadIdx.x, jl = t & (kTcN - 1), kg = t >> 6;
    const int cb = blockIdx.x, col = k0 + w + cb * kTcN + jl;
    df64 x[8];
    unsigned key = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int k = kg * 8 + i;
        const float2 v = (col < M && k < w) ? A[(int64_t)(k0 + k) * M + col] : make_float2(0.f, 0.f);
        x[i] = df64(v.x, v.y, 0);
        key = max(key, __float_as_uint(v.x) & 0x7fffffffu);
    }
    red[kg][jl] = key;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; q++) key = max(key, red[q][jl]);
    const int e = exp_above(__uint_as_float(key));
    const float sc = pow2f(-e);
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = df_ldexp(x[i], sc);
    uint4 out[kOzS];
    oz_split8(x, out);
#pragma unroll
    for (int sl = 0; sl < kOzS; sl++)
        Uimg[((size_t)(cb * kOzS + sl) * kTcUBytes + 2 * core_off(jl, kg * 8)) / 16] = out[sl];
    if (kg == 0) eu[cb * kTcN + jl] = e;
}

// The trailing update as a persistent kernel, one CTA per SM taking work items of up to
// kTcChunk column blocks of one 128-row block (items c, c + grid, c + 2 grid, ... for CTA
// c, so every thread knows the sequence).  Warp 8 produces: one thread loads an item's
// row-block slices once (96 KB) and, per 128 x 64 tile, the column block's slices (48 KB)
// with bulk asynchronous copies, then issues the tile's 84 MMAs (21 slice pairs x 4 K
// steps of 16) into six TMEM accumulators of 64 columns and commits them.  Warps 0-7
// consume: per tile they read the accumulators (warp q: TMEM lanes 32 (q mod 4) ...,
// columns 32 (q / 4) ...), combine them in double-float, tell the producer that TMEM is
// free, stage the tile in shared memory and subtract it from A22 with coalesced loads and
// stores — while the producer already loads and multiplies the next tile.  mbarriers:
// row-block slices landed, column-block slices landed, MMAs done (the column buffer and
// TMEM are then free to reuse), accumulators read (8 arrivals).  Every wait is bounded; a
// wait that gives up records a time-out, and each side stops at its next tile (the
// consumers decide together, after a barrier of theirs); the CTA then frees its TMEM.
constexpr int kTcChunk = 8;                 // column blocks per work item
constexpr int kTcConsumers = 256;           // warps 0-7
constexpr int kTcThreads = kTcConsumers + 32;
constexpr int kTcVs = kTcN + 1;             // row stride of the staged tile (float2)
constexpr int kTcSmemAll = kTcSmem + kTcM * kTcVs * 8;

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, unsigned lim)
{
    for (unsigned spins = 0; spins < lim; spins++)
        if (mbar_test(mb, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, int bytes, uint32_t mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mb) : "memory");
}

__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" :: "r"(kTcConsumers) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_lu_gemm_tc(int M, int k1, int nrb, int ncb, const uint4 *Limg, const uint4 *Uimg, const int *el,
             const int *eu, float2 *A, int *status)
{
    if (lu_failed(status)) return;
    extern __shared__ __align__(128) uint4 gsm_tc[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long bar_l, bar_u, bar_mma, bar_free;
    __shared__ int s_abort, s_stop;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint4 *sL = gsm_tc, *sU = gsm_tc + kOzS * kTcLBytes / 16;
    float2 *vt = (float2 *)(gsm_tc + kTcSmem / 16);  // [kTcM][kTcVs]: the tile's products
    const uint32_t ml = smem_u32(&bar_l), mu = smem_u32(&bar_u), mm = smem_u32(&bar_mma),
                   mf = smem_u32(&bar_free);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(ml), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mu), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mm), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mf), "r"(kTcConsumers / 32) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const unsigned lim = wait_limit(status, kLuSpins);
    const int q = (ncb + kTcChunk - 1) / kTcChunk, nitems = nrb * q;
    auto give_up = [&]() {
        atomicOr(status, LBF_DEV_TIMEOUT);
        *(volatile int *)&s_abort = 1;
    };
    if (warp == kTcConsumers / 32) {
        // ---- producer ----
        if (lane == 0) {
            const uint32_t aL = smem_u32(sL), aU = smem_u32(sU);
            const uint64_t dL = tc_desc(aL), dU = tc_desc(aU);
            unsigned t = 0, nl = 0;
            int prev_rb = -1;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int rb = item / q, c0 = (item % q) * kTcChunk, c1 = min(ncb, c0 + kTcChunk);
                if (rb != prev_rb) {
                    // the row-block buffer is read until the last tile's MMAs are done
                    if (t > 0 && !(ok = mbar_wait(mm, (t - 1) & 1, lim))) break;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(ml), "r"(kOzS * kTcLBytes) : "memory");
                    bulk_g2s(aL, (const char *)Limg + (size_t)rb * kOzS * kTcLBytes, kOzS * kTcLBytes, ml);
                    if (!(ok = mbar_wait(ml, nl & 1, lim))) break;
                    nl++;
                    prev_rb = rb;
                }
                for (int cb = c0; cb < c1 && ok; cb++, t++) {
                    if (t > 0 && !(ok = mbar_wait(mm, (t - 1) & 1, lim))) break;  // column buffer free
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(mu), "r"(kOzS * kTcUBytes) : "memory");
                    bulk_g2s(aU, (const char *)Uimg + (size_t)cb * kOzS * kTcUBytes, kOzS * kTcUBytes, mu);
                    if (!(ok = mbar_wait(mu, t & 1, lim))) break;
                    if (t > 0 && !(ok = mbar_wait(mf, (t - 1) & 1, lim))) break;  // TMEM read
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int d = 0; d <= kOzD; d++)
#pragma unroll
                        for (int sl = 0; sl <= d; sl++)
#pragma unroll
                            for (int jk = 0; jk < kLuNb / 16; jk++)
                                tc_mma(tmem + (uint32_t)(d * kTcN),
                                       dL + (uint64_t)((sl * kTcLBytes + jk * 256) >> 4),
                                       dU + (uint64_t)(((d - sl) * kTcUBytes + jk * 256) >> 4),
                                       (sl > 0 || jk > 0) ? 1u : 0u);
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(mm) : "memory");
                }
            }
            if (!ok) {
                give_up();
                // copies or MMAs still in flight finish before the CTA lets go of its memory
                mbar_wait(mm, (t - 1) & 1, lim);
            } else if (t > 0) {
                mbar_wait(mm, (t - 1) & 1, lim);
            }
        }
    } else {
        // ---- consumers ----
        const int quarter = warp & 3, half = warp >> 2, rl = quarter * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
        unsigned t = 0;
        bool stop = false;
        for (int item = blockIdx.x; item < nitems && !stop; item += gridDim.x) {
            const int rb = item / q, c0 = (item % q) * kTcChunk, c1 = min(ncb, c0 + kTcChunk);
            const int i = k1 + rb * kTcM + rl;
            const float ri = i < M ? pow2f(el[rb * kTcM + rl] - 16) : 0.f;
            for (int cb = c0; cb < c1; cb++, t++) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait(mm, t & 1, lim);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok && lane == 0) give_up();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // 1. TMEM -> V_ij = sum_d P_d 2^(-8d) (times the row's scale), double-float
                float2 v[32];
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    float acc[kOzD + 1][16];
#pragma unroll
                    for (int d = 0; d <= kOzD; d++) tc_ld16(trow + (uint32_t)(d * kTcN + c), acc[d]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int qq = 0; qq < 16; qq++) {
                        float h = acc[kOzD][qq], l = 0.f;  // from the smallest term up
#pragma unroll
                        for (int d = kOzD - 1; d >= 0; d--) {
                            float e2;
                            df_two_sum(acc[d][qq], h * 0x1p-8f, h, e2);
                            l = e2 + l * 0x1p-8f;
                        }
                        const df64 vv = df_fast(h, l);
                        v[c + qq] = make_float2(vv.hi * ri, vv.lo * ri);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mf) : "memory");
                // 2. the previous tile's update is done everywhere: stage this one.  Whether to
                //    stop is read by one thread before the barrier and by all after it, so every
                //    consumer takes the same branch (the flag itself may change at any time)
                if (tid == 0) s_stop = *(volatile int *)&s_abort;
                consumers_sync();
                stop = s_stop != 0;
                if (stop) break;
#pragma unroll
                for (int c = 0; c < 32; c++) vt[rl * kTcVs + half * 32 + c] = v[c];
                consumers_sync();
                // 3. A22 -= V 2^f_j, lanes on consecutive columns of a row; all of a thread's
                //    loads before its stores (a store could alias a later load)
                constexpr int kStep = kTcConsumers / kTcN, kRows = kTcM / kStep;
                const int jl = tid % kTcN, j = k1 + cb * kTcN + jl, r0 = tid / kTcN;
                const float cj = j < M ? pow2f(eu[cb * kTcN + jl]) : 0.f;
                const int nrow = min(kTcM, M - (k1 + rb * kTcM));
                float2 *ap = A + (int64_t)(k1 + rb * kTcM) * M + j;
                const int64_t rs = (int64_t)kStep * M;
                if (j < M) {
                    float2 av[kRows];
#pragma unroll
                    for (int qq = 0; qq < kRows; qq++)
                        av[qq] = r0 + kStep * qq < nrow ? ap[r0 * (int64_t)M + qq * rs] : make_float2(0.f, 0.f);
#pragma unroll
                    for (int qq = 0; qq < kRows; qq++) {
                        const int r = r0 + kStep * qq;
                        if (r >= nrow) break;
                        const float2 w2 = vt[r * kTcVs + jl];
                        const df64 res = df64(av[qq].x, av[qq].y, 0) - df64(w2.x * cj, w2.y * cj, 0);
                        ap[r0 * (int64_t)M + qq * rs] = make_float2(res.hi, res.lo);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}


// Inverses of the diagonal blocks of L (unit lower) and U (upper), one kLuTs x kLuTs
// block per CUDA block, by substitution against the identity (columns in parallel);
// a short last block is padded with the identity.  dinv: [2][nB][kLuTs][kLuTs],
// L's inverses first.  The triangular solves then take each diagonal block as one
// matrix-vector product instead of kLuTs dependent steps.
__global__ void __launch_bounds__(kLuThreads)
k_lu_diaginv(int M, const float2 *__restrict__ A, float2 *__restrict__ dinv, const int *status)
{
    if (lu_failed(status)) return;
    extern __shared__ __align__(16) float2 dsm[];
    float2 *Ts = dsm;                    // the factor's diagonal block
    float2 *X = dsm + kLuTs * kLuPad;    // its inverse
    const int b = blockIdx.x, rb = b * kLuTs, nr = min(kLuTs, M - rb), tid = threadIdx.x;
    const int nB = gridDim.x;
    for (int which = 0; which < 2; which++) {  // 0: L, 1: U
        for (int e = tid; e < kLuTs * kLuTs; e += blockDim.x) {
            const int r = e >> 6, c = e & 63;
            float2 v = make_float2(r == c ? 1.f : 0.f, 0.f);
            if (r < nr && c < nr && (which == 0 ? c < r : c >= r)) v = A[(int64_t)(rb + r) * M + rb + c];
            Ts[r * kLuPad + c] = v;
            X[r * kLuPad + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
        }
        __syncthreads();
        if (which == 0) {
            for (int t = 0; t < kLuTs - 1; t++) {  // rows below t lose L[r][t] times row t
                for (int e = tid; e < (kLuTs - 1 - t) * kLuTs; e += blockDim.x) {
                    const int r = t + 1 + (e >> 6), c = e & 63;
                    X[r * kLuPad + c] = pk(df_fma(-ld(Ts[r * kLuPad + t]), ld(X[t * kLuPad + c]), ld(X[r * kLuPad + c])));
                }
                __syncthreads();
            }
        } else {
            for (int t = kLuTs - 1; t >= 0; t--) {  // row t divided by U[t][t], then rows above
                const df64 ip = df_rcp(ld(Ts[t * kLuPad + t]));
                if (tid < kLuTs) X[t * kLuPad + tid] = pk(ld(X[t * kLuPad + tid]) * ip);
                __syncthreads();
                for (int e = tid; e < t * kLuTs; e += blockDim.x) {
                    const int r = e >> 6, c = e & 63;
                    X[r * kLuPad + c] = pk(df_fma(-ld(Ts[r * kLuPad + t]), ld(X[t * kLuPad + c]), ld(X[r * kLuPad + c])));
                }
                __syncthreads();
            }
        }
        float2 *out = dinv + ((size_t)which * nB + b) * kLuTs * kLuTs;
        for (int e = tid; e < kLuTs * kLuTs; e += blockDim.x) out[e] = X[(e >> 6) * kLuPad + (e & 63)];
        __syncthreads();
    }
}

// perm from the interchanges (one block; in shared memory when it fits)
__global__ void k_lu_perm(int M, const int *piv, int *perm, int in_shared)
{
    extern __shared__ int ps[];
    int *p = in_shared ? ps : perm;
    for (int i = threadIdx.x; i < M; i += blockDim.x) p[i] = i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < M; k++) {
            const int q = piv[k];
            if (q != k && q >= 0 && q < M) {
                const int t = p[k];
                p[k] = p[q];
                p[q] = t;
            }
        }
    __syncthreads();
    if (in_shared)
        for (int i = threadIdx.x; i < M; i += blockDim.x) perm[i] = p[i];
}

__device__ __forceinline__ bool gate_shut(const int *gate) { return gate && *gate == 0; }

// z = P f (forward) or z = f (transposed), as double-float
__global__ void k_lu_gather(int M, const int *__restrict__ perm, const double *__restrict__ f,
                            float2 *__restrict__ z, int trans, const int *gate)
{
    if (gate_shut(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) z[i] = pk(df64(trans ? f[i] : f[perm[i]]));
}

// y = alpha z (forward) or y = alpha P^T z (transposed)
__global__ void k_lu_scatter(int M, const int *__restrict__ perm, const float2 *__restrict__ z,
                             double alpha, double *__restrict__ y, int trans, const int *gate)
{
    if (gate_shut(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double v = alpha * ((double)z[i].x + (double)z[i].y);
    y[trans ? perm[i] : i] = v;
}

// Triangular solve T x = x (in place, double-float), T from the factors:
//   mode 0: L (unit lower)   mode 1: U (upper)   mode 2: U^T (lower)   mode 3: L^T (unit upper).
// Row blocks of kLuTs rows are taken from a ticket counter in solve order (increasing
// for lower, decreasing for upper).  A block first prefetches its diagonal block's
// inverse (shared memory) and the off-diagonal tile it will need last (registers),
// then waits (bounded) for each block it depends on, in solve order, subtracting that
// block's part as it arrives, and finally multiplies by the diagonal inverse and
// publishes its rows by a flag word.  Every block it waits for took its ticket
// earlier and is running, so every wait ends.
// sw: [0] ticket, [1] finished blocks, [2] epoch, then one flag per row block; the last
// block to finish resets the counters and advances the epoch.
__global__ void __launch_bounds__(kLuThreads)
k_lu_trsv(int M, int mode, const float2 *__restrict__ A, const float2 *__restrict__ dinv,
          float2 *x, unsigned *sw, int *status, const int *gate)
{
    if (gate_shut(gate)) return;
    extern __shared__ __align__(16) float2 vsm[];
    float2 *T = vsm;                      // kLuTs x kLuPad: the diagonal block's inverse (as T)
    float2 *part = vsm + kLuTs * kLuPad;  // 4 x kLuTs partial sums
    __shared__ float2 xs[kLuTs], rv[kLuTs];
    __shared__ unsigned s_t, s_epoch;
    const bool lower = mode == 0 || mode == 2, trans = mode >= 2;
    const int nB = (M + kLuTs - 1) / kLuTs, tid = threadIdx.x;
    unsigned *flag = sw + 3;
    if (tid == 0) s_epoch = *(volatile unsigned *)&sw[2];
    __syncthreads();
    const unsigned epoch = s_epoch;
    // this thread's (row, quarter) of a tile product
    const int r = trans ? (tid & 63) : (tid >> 2), q = trans ? (tid >> 6) : (tid & 3);
    for (;;) {
        if (tid == 0) s_t = atomicAdd(&sw[0], 1u);
        __syncthreads();
        const unsigned t = s_t;
        __syncthreads();
        if (t >= (unsigned)nB) break;
        const int b = lower ? (int)t : nB - 1 - (int)t;
        const int rb = b * kLuTs, nr = min(kLuTs, M - rb);
        // the diagonal block's inverse: L^-1 (mode 0), U^-1 (1), U^-T (2), L^-T (3)
        {
            const float2 *D = dinv + ((size_t)((mode == 1 || mode == 2) ? 1 : 0) * nB + b) * kLuTs * kLuTs;
            for (int e = tid; e < kLuTs * kLuTs; e += blockDim.x) {
                const int rr = e >> 6, cc = e & 63;
                T[(trans ? cc : rr) * kLuPad + (trans ? rr : cc)] = D[e];
            }
        }
        const int nj = lower ? b : nB - 1 - b;
        // prefetch of the last off-diagonal tile (the one on the critical path)
        float2 pre[16];
        if (nj > 0) {
            const int j = lower ? b - 1 : b + 1, cb = j * kLuTs, nc = min(kLuTs, M - cb);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int c = q * 16 + k;
                pre[k] = make_float2(0.f, 0.f);
                if (r < nr && c < nc)
                    pre[k] = trans ? A[(int64_t)(cb + c) * M + rb + r] : A[(int64_t)(rb + r) * M + cb + c];
            }
        }
        df64 accp(0.f);
        for (int jj = 0; jj < nj; jj++) {
            const int j = lower ? jj : nB - 1 - jj;
            block_wait_flag(&flag[j], epoch + 1u, status, kLuSpins);
            const int cb = j * kLuTs, nc = min(kLuTs, M - cb);
            if (tid < nc) xs[tid] = __ldcg(&x[cb + tid]);
            __syncthreads();
            if (r < nr) {
                if (jj == nj - 1) {
#pragma unroll
                    for (int k = 0; k < 16; k++)
                        if (q * 16 + k < nc) accp = df_fma(ld(pre[k]), ld(xs[q * 16 + k]), accp);
                } else {
                    const int c1 = min(nc, q * 16 + 16);
                    if (!trans) {
                        const float2 *row = A + (int64_t)(rb + r) * M + cb;
                        for (int c = q * 16; c < c1; c++) accp = df_fma(ld(row[c]), ld(xs[c]), accp);
                    } else {
                        for (int c = q * 16; c < c1; c++)
                            accp = df_fma(ld(A[(int64_t)(cb + c) * M + rb + r]), ld(xs[c]), accp);
                    }
                }
            }
            __syncthreads();  // xs is refilled next
        }
        part[q * kLuTs + r] = pk(accp);
        __syncthreads();
        if (tid < kLuTs) {
            df64 v(0.f);
            if (tid < nr)
                v = ld(__ldcg(&x[rb + tid])) - (((ld(part[tid]) + ld(part[kLuTs + tid])) +
                                                 ld(part[2 * kLuTs + tid])) + ld(part[3 * kLuTs + tid]));
            rv[tid] = pk(v);
        }
        __syncthreads();
        {
            df64 a(0.f);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int c = q * 16 + k;
                a = df_fma(ld(T[r * kLuPad + c]), ld(rv[c]), a);
            }
            part[q * kLuTs + r] = pk(a);
        }
        __syncthreads();
        if (tid < nr)
            x[rb + tid] = pk(((ld(part[tid]) + ld(part[kLuTs + tid])) + ld(part[2 * kLuTs + tid])) +
                             ld(part[3 * kLuTs + tid]));
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(&flag[b], epoch + 1u);
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&sw[1], 1u) == gridDim.x - 1) {
            sw[0] = 0u;
            sw[1] = 0u;
            __threadfence();
            atomicExch(&sw[2], epoch + 1u);
        }
    }
}

// r = f - S z_nat (forward) or r = f - S^T z_nat (transposed) in double, where z holds
// the double-float solve in the triangular solves' order (z_nat = z forward; z_nat[perm[k]]
// = z[k] transposed): the residual of one refinement step against the double S.
__global__ void k_lu_resid(int M, const double *__restrict__ S, const int *__restrict__ perm,
                           const float2 *__restrict__ z, const double *__restrict__ f,
                           double *__restrict__ r, int trans, const int *gate)
{
    if (gate_shut(gate)) return;
    if (!trans) {  // a warp per row
        const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
        if (i >= M) return;
        double acc = 0.0;
        for (int m = lane; m < M; m += 32) acc = fma(S[(int64_t)i * M + m], (double)z[m].x + (double)z[m].y, acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) r[i] = f[i] - acc;
    } else {  // a thread per column of S, coalesced over the rows
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= M) return;
        double acc = 0.0;
        for (int k = 0; k < M; k++) acc = fma(S[(int64_t)perm[k] * M + i], (double)z[k].x + (double)z[k].y, acc);
        r[i] = f[i] - acc;
    }
}

// y = alpha (z0 + z1), both in the solves' order (see k_lu_scatter)
__global__ void k_lu_scatter2(int M, const int *__restrict__ perm, const float2 *__restrict__ z0,
                              const float2 *__restrict__ z1, double alpha, double *__restrict__ y,
                              int trans, const int *gate)
{
    if (gate_shut(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const df64 v = ld(z0[i]) + ld(z1[i]);
    y[trans ? perm[i] : i] = alpha * ((double)v.hi + (double)v.lo);
}

}  // namespace

// Scratch of the factorisation (plan time): the panel candidates and the grid barrier.
// row and column blocks of the trailing update's slice images for an M x M matrix
static int64_t oz_row_blocks(int M) { return (M + kTcM - 1) / kTcM; }
static int64_t oz_col_blocks(int M) { return (M + kTcN - 1) / kTcN; }

size_t lbf_lu_scratch_bytes(int M)
{
    return 256 + sizeof(unsigned) * 2 * kLuMaxPanelBlocks + sizeof(int) * 2 * kLuMaxPanelBlocks +
           sizeof(float2) * 2 * (size_t)kLuMaxPanelBlocks * kLuNb + sizeof(float2) * 2 * kLuNb +
           sizeof(GridBarrier) + (size_t)oz_row_blocks(M) * kOzS * kTcLBytes +
           (size_t)oz_col_blocks(M) * kOzS * kTcUBytes + sizeof(int) * (size_t)(oz_row_blocks(M) * kTcM) +
           sizeof(int) * (size_t)(oz_col_blocks(M) * kTcN) + 8 * 256;
}

int lbf_lu_sync_words(int M) { return 3 + (M + kLuTs - 1) / kLuTs; }

int64_t lbf_lu_dinv_entries(int M) { return 2 * (int64_t)((M + kLuTs - 1) / kLuTs) * kLuTs * kLuTs; }

// S (double, M x M, in pl->Sinv) -> its LU factors in place (double-float), pl->lu_piv,
// pl->lu_perm; on stream s.  scratch: lbf_lu_scratch_bytes(M) bytes of device memory.
int lbf_schur_lu_factor(lbf_plan *pl, cudaStream_t s, void *scratch)
{
    const int M = pl->M;
    float2 *A = (float2 *)pl->Sinv;
    char *p = (char *)scratch;
    auto take = [&](size_t b) {
        void *r = p;
        p += (b + 255) & ~size_t(255);
        return r;
    };
    unsigned *amax = (unsigned *)take(sizeof(unsigned));
    unsigned *ckey = (unsigned *)take(sizeof(unsigned) * 2 * kLuMaxPanelBlocks);
    int *crow = (int *)take(sizeof(int) * 2 * kLuMaxPanelBlocks);
    float2 *cval = (float2 *)take(sizeof(float2) * 2 * (size_t)kLuMaxPanelBlocks * kLuNb);
    float2 *rjval = (float2 *)take(sizeof(float2) * 2 * kLuNb);
    GridBarrier *bar = (GridBarrier *)take(sizeof(GridBarrier));
    uint4 *Limg = (uint4 *)take((size_t)oz_row_blocks(M) * kOzS * kTcLBytes);
    uint4 *Uimg = (uint4 *)take((size_t)oz_col_blocks(M) * kOzS * kTcUBytes);
    int *el = (int *)take(sizeof(int) * (size_t)(oz_row_blocks(M) * kTcM));
    int *eu = (int *)take(sizeof(int) * (size_t)(oz_col_blocks(M) * kTcN));
    int *status = pl->dev_status;
    LBF_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned), s));
    LBF_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s));
    lbf_inject_barrier(&bar->count, s);
    LBF_CUDA(cudaMemsetAsync(pl->lu_sync, 0, sizeof(unsigned) * lbf_lu_sync_words(M), s));
    const int64_t n2 = (int64_t)M * M;
    LBF_CUDA(cudaMemcpyAsync(pl->lu_S, pl->Sinv, sizeof(double) * (size_t)n2, cudaMemcpyDeviceToDevice, s));
    LBF_LAUNCH(k_lu_convert, (int)std::min<int64_t>(lbf_cdiv(n2, 256), 152 * 16), 256, 0, s, n2,
               pl->Sinv, amax);
    LBF_CHECK_LAUNCH();
    int dev = 0, nsm = 0, coop = 0;
    LBF_CUDA(cudaGetDevice(&dev));
    LBF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    LBF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return LBF_ECUDA;
    const size_t tile_smem = sizeof(float2) * 2 * kLuNb * kLuPad;
    LBF_CUDA(cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLuSmemCap));
    LBF_CUDA(cudaFuncSetAttribute(k_lu_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
    LBF_CUDA(cudaFuncSetAttribute(k_lu_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAll));
    for (int k0 = 0; k0 < M; k0 += kLuNb) {
        const int w = std::min(kLuNb, M - k0);
        const int rows = M - k0;
        int nblk = std::max(1, std::min(nsm, (rows + 31) / 32));
        int rpb = (rows + nblk - 1) / nblk;
        size_t smem = sizeof(float2) * ((size_t)rpb * kLuNb + rpb);
        if (smem > kLuSmemCap) return LBF_EINVAL;  // M above ~60,000
        int per_sm = 0;
        LBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_panel, kLuThreads, smem));
        if (per_sm < 1) return LBF_ECUDA;
        nblk = std::min(nblk, std::min(kLuMaxPanelBlocks, per_sm * nsm));
        rpb = (rows + nblk - 1) / nblk;
        smem = sizeof(float2) * ((size_t)rpb * kLuNb + rpb);
        int kk0 = k0, ww = w, rr = rpb;
        void *args[] = {(void *)&M, &kk0, &ww, &rr, &A, &pl->lu_piv, &amax, &ckey, &crow, &cval,
                        &rjval, &bar, &status};
        lbf_prof_mark(LBF_KERNEL_LU_PANEL, 1, s);
        LBF_CUDA(cudaLaunchCooperativeKernel((const void *)k_lu_panel, dim3(nblk), dim3(kLuThreads), args,
                                             smem, s));
        g_lbf_launches.fetch_add(1, std::memory_order_relaxed);
        lbf_prof_mark(LBF_KERNEL_LU_PANEL, 0, s);
        LBF_LAUNCH_P(LBF_KERNEL_LU_UPDATE, k_lu_swap, lbf_cdiv(M, 256), 256, 0, s, M, k0, w, A, pl->lu_piv,
                     status);
        const int rest = M - k0 - w;
        if (rest > 0) {
            const int nt = (rest + kLuTs - 1) / kLuTs;
            LBF_LAUNCH_P(LBF_KERNEL_LU_UPDATE, k_lu_trsm, nt, kLuThreads, tile_smem, s, M, k0, w, A, status);
            const int nrb = (rest + kTcM - 1) / kTcM, ncb = (rest + kTcN - 1) / kTcN;
            LBF_LAUNCH_P(LBF_KERNEL_LU_GEMM, k_oz_slice_rows, nrb * (kTcM / 32), 256, 0, s, M, k0, w, A,
                         Limg, el, status);
            LBF_LAUNCH_P(LBF_KERNEL_LU_GEMM, k_oz_slice_cols, ncb, 512, 0, s, M, k0, w, A, Uimg, eu,
                         status);
            const int items = nrb * ((ncb + kTcChunk - 1) / kTcChunk);
            LBF_LAUNCH_P(LBF_KERNEL_LU_GEMM, k_lu_gemm_tc, std::min(items, nsm), kTcThreads, kTcSmemAll, s, M,
                         k0 + w, nrb, ncb, Limg, Uimg, el, eu, A, status);
        }
        LBF_CHECK_LAUNCH();
    }
    {
        const int nB = (M + kLuTs - 1) / kLuTs;
        LBF_CUDA(cudaFuncSetAttribute(k_lu_diaginv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
        LBF_LAUNCH_P(LBF_KERNEL_LU_UPDATE, k_lu_diaginv, nB, kLuThreads, tile_smem, s, M, A, pl->lu_dinv, status);
        LBF_CHECK_LAUNCH();
    }
    const bool sh = (size_t)M * sizeof(int) <= kLuSmemCap;
    if (sh) LBF_CUDA(cudaFuncSetAttribute(k_lu_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLuSmemCap));
    LBF_LAUNCH(k_lu_perm, 1, 256, sh ? sizeof(int) * (size_t)M : 0, s, M, pl->lu_piv, pl->lu_perm, sh ? 1 : 0);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

// y = alpha S^-1 f (trans = 0) or y = alpha S^-T f (trans = 1), M-vectors (double),
// through the factors of lbf_schur_lu_factor.  accurate: one step of iterative
// refinement against the double S kept by the plan (z = z0 + LU^-1 (f - S z0)), which
// brings the rounding of the double-float solves (about cond(S) 2^-46) down to that of a
// double solve; the refinement's FP64 residuals use it, so their preconditioned residual
// has the same floor as with the double inverse.
int lbf_schur_lu_apply(lbf_plan *pl, const double *f, double alpha, double *y, int trans,
                       const int *gate, cudaStream_t s, int accurate)
{
    const int M = pl->M;
    const size_t smem = sizeof(float2) * (kLuTs * kLuPad + 4 * kLuTs);  // < 48 KB
    const int nB = (M + kLuTs - 1) / kLuTs;
    const int grid = std::min(nB, 2 * std::max(1, pl->nsm));
    const float2 *A = (const float2 *)pl->Sinv;
    auto solve = [&](const double *rhs, float2 *z) -> int {
        LBF_LAUNCH(k_lu_gather, lbf_cdiv(M, 256), 256, 0, s, M, pl->lu_perm, rhs, z, trans, gate);
        LBF_LAUNCH_P(LBF_KERNEL_LU_SOLVE, k_lu_trsv, grid, kLuThreads, smem, s, M, trans ? 2 : 0, A,
                     pl->lu_dinv, z, pl->lu_sync, pl->dev_status, gate);
        LBF_LAUNCH_P(LBF_KERNEL_LU_SOLVE, k_lu_trsv, grid, kLuThreads, smem, s, M, trans ? 3 : 1, A,
                     pl->lu_dinv, z, pl->lu_sync, pl->dev_status, gate);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    };
    int rc = solve(f, pl->lu_z);
    if (rc) return rc;
    if (!accurate) {
        LBF_LAUNCH(k_lu_scatter, lbf_cdiv(M, 256), 256, 0, s, M, pl->lu_perm, pl->lu_z, alpha, y, trans,
                   gate);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if (trans) LBF_LAUNCH(k_lu_resid, lbf_cdiv(M, 128), 128, 0, s, M, pl->lu_S, pl->lu_perm, pl->lu_z, f,
                          pl->lu_r, 1, gate);
    else LBF_LAUNCH(k_lu_resid, lbf_cdiv((int64_t)M * 32, 256), 256, 0, s, M, pl->lu_S, pl->lu_perm,
                    pl->lu_z, f, pl->lu_r, 0, gate);
    LBF_CHECK_LAUNCH();
    if ((rc = solve(pl->lu_r, pl->lu_z2))) return rc;
    LBF_LAUNCH(k_lu_scatter2, lbf_cdiv(M, 256), 256, 0, s, M, pl->lu_perm, pl->lu_z, pl->lu_z2, alpha, y,
               trans, gate);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}
