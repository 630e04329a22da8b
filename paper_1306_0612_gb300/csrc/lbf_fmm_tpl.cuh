// FMM kernels templated on the real type R (double: the accurate operator;
// float: the inner operator of iterative refinement).  The expansions,
// translations and near-field pair sums run in R; the final combine in double.
// The float path reads each node's coordinate relative to its own leaf (formed
// in double once per geometry) and moves it between box frames by powers of two
// and exact integer centre offsets, so its inner loops issue no double
// arithmetic (this GPU runs double at 1/64 of the float rate).
//
// Scaled expansions about a box centre c with half-width r:
//   multipole  phi(z) = sum_k a_k r^k / (z - c)^(k+1),  a_k = sum_j q_j ((xi_j - c)/r)^k
//   local      phi(z) = sum_l b_l ((z - c)/r)^l
// of the Cauchy potential phi(z) = sum_j q_j / (z - xi_j); the operator needs
// c_i = Im sum_{j != i} q_j / (xi_j - xi_i) = -Im phi(xi_i).
#pragma once

#include <type_traits>

#include "lbf_df64.cuh"
#include "lbf_internal.cuh"
#include "lbf_sync.cuh"

namespace fmm {

template <typename R> struct __align__(2 * sizeof(R)) cx {
    R x, y;
};

__device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ df64 fm(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }

// float and double-float read each node's leaf-local coordinate (rounded once per
// geometry) and move it between box frames by powers of two and integer offsets;
// double forms node offsets from the double positions
template <typename R> constexpr bool kLocal = !std::is_same<R, double>::value;
// largest level gap over which a leaf-local coordinate is rescaled into a coarser
// box's frame (its rounding grows by 2 per level; wider gaps use the positions)
template <typename R> constexpr int kMaxGap = std::is_same<R, float>::value ? 3 : 12;
// float: level gaps beyond kMaxGap (up to kDfGap, where box offsets stay exact in float)
// form the coordinate in double-float from the node's double-float leaf-local
// coordinate, so the cancellation between a large rescaled coordinate and the box
// offset happens in ~48 bits, then round it to float
constexpr int kDfGap = 20;

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
__device__ __forceinline__ df64 rcp(df64 a) { return df_rcp(a); }

// 1/a in double for a positive normal a in [2^-126, 2^126] (the near field's squared
// distances in units of a leaf half-width, the far-field arguments of M2P and P2L), with
// no instruction on the double pipe but the refinement: the float seed is a with its
// exponent rebiased and its mantissa cut to 20 bits, built with integer operations
// (relative error < 2^-20), the float reciprocal approximation of that, widened back by
// integer operations, then one third-order step of the series 1/a = x/(1 - e) =
// x (1 + e + e^2 + ...), e = 1 - a x: x <- x + x (e + e^2), three fused multiply-adds
// (the dropped terms are ~e^3 < 2^-59, below the rounding of the last one; two
// Newton-Raphson steps would take four).  On this GPU the double pipe is the bound of
// every double FMM kernel; a conversion instruction would occupy it like an arithmetic
// one.
__device__ __forceinline__ double rcp_near(double a)
{
    const int hi = __double2hiint(a);
    const float af = __int_as_float((hi - (896 << 20)) << 3);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(af));
    const unsigned yb = __float_as_uint(yf);
    const double x = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
    const double e = fma(-a, x, 1.0);
    return fma(x, fma(e, e, e), x);
}

template <typename R> __device__ __forceinline__ cx<R> crcp(cx<R> a)
{
    R d;
    if constexpr (std::is_same<R, double>::value) d = rcp_near(fma(a.x, a.x, a.y * a.y));
    else d = rcp(a.x * a.x + a.y * a.y);
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
    float invLf;  // 1/L rounded to float: 1/r of a level-l box is invLf 2^(l+1)
    df64 invLd;   // 1/L as a double-float
    double invL;  // 1/L in double
};

__device__ __forceinline__ void box_centre(const BoxGeo &g, int l, int ix, int iy, double &cx_,
                                           double &cy_, double &r)
{
    double w = ldexp(g.L, -l);
    r = 0.5 * w;
    cx_ = g.xmin + (ix + 0.5) * w;
    cy_ = g.ymin + (iy + 0.5) * w;
}

// The centre of a level-l box and 1/r, its half-width's reciprocal, with few instructions
// on the double pipe: ix + 1/2 from the integer's bits (2^52 + ix less 2^52 - 1/2, exact),
// the width L 2^-l and 1/r = (1/L) 2^(l+1) by exact power-of-two products (the same values
// as box_centre and 1.0 / r).
__device__ __forceinline__ void box_centre_ir(const BoxGeo &g, int l, int ix, int iy,
                                              double &cx_, double &cy_, double &ir);
// 2^e from the exponent bits (|e| well inside the normal range)
template <typename R> __device__ __forceinline__ R pow2(int e);
template <> __device__ __forceinline__ float pow2<float>(int e) { return __int_as_float((127 + e) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int e)
{
    return __longlong_as_double((long long)(1023 + e) << 52);
}
template <> __device__ __forceinline__ df64 pow2<df64>(int e) { return df64(pow2<float>(e)); }

__device__ __forceinline__ void box_centre_ir(const BoxGeo &g, int l, int ix, int iy,
                                              double &cx_, double &cy_, double &ir)
{
    const double w = g.L * pow2<double>(-l);
    const double hx = __hiloint2double(0x43300000, ix) - 4503599627370495.5;
    const double hy = __hiloint2double(0x43300000, iy) - 4503599627370495.5;
    cx_ = fma(hx, w, g.xmin);
    cy_ = fma(hy, w, g.ymin);
    ir = g.invL * pow2<double>(l + 1);
}

// 1/r of a level-l box in R without double arithmetic (float, double-float)
template <typename R> __device__ __forceinline__ R inv_half_width(const BoxGeo &g, int l);
template <> __device__ __forceinline__ float inv_half_width<float>(const BoxGeo &g, int l)
{
    return g.invLf * pow2<float>(l + 1);
}
template <> __device__ __forceinline__ df64 inv_half_width<df64>(const BoxGeo &g, int l)
{
    return df_ldexp(g.invLd, pow2<float>(l + 1));
}

// an expansion coefficient written by another block of the same launch (through L2)
__device__ __forceinline__ cx<double> ldcg_cx(const cx<double> *p)
{
    double2 v = __ldcg((const double2 *)p);
    return cx<double>{v.x, v.y};
}
__device__ __forceinline__ cx<float> ldcg_cx(const cx<float> *p)
{
    float2 v = __ldcg((const float2 *)p);
    return cx<float>{v.x, v.y};
}
__device__ __forceinline__ cx<df64> ldcg_cx(const cx<df64> *p)
{
    float4 v = __ldcg((const float4 *)p);
    return cx<df64>{df64(v.x, v.y, 0), df64(v.z, v.w, 0)};
}
template <typename R> __device__ __forceinline__ cx<R> offset_cx(float2 o)
{
    return cx<R>{R(o.x), R(o.y)};
}

// (c_a - c_b) / r_b for box a (level la) and box b (level lb), per axis
// (2 a + 1) 2^(lb - la) - (2 b + 1), formed in integers at the finer level and
// scaled once, so the float path needs no double arithmetic for box offsets
__device__ __forceinline__ float2 centre_offset(int la, int ax, int ay, int lb, int bx, int by)
{
    if (la >= lb) {
        const int sh = la - lb;
        const long long dx = (2LL * ax + 1) - ((2LL * bx + 1) << sh);
        const long long dy = (2LL * ay + 1) - ((2LL * by + 1) << sh);
        const float f = pow2<float>(-sh);
        return make_float2((float)(int)dx * f, (float)(int)dy * f);
    }
    const int sh = lb - la;
    const long long dx = ((2LL * ax + 1) << sh) - (2LL * bx + 1);
    const long long dy = ((2LL * ay + 1) << sh) - (2LL * by + 1);
    return make_float2((float)(int)dx, (float)(int)dy);
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

// s0 = sum_k C[k P + lc0] A[k], and s1 the same for lc1 when a lane holds two coefficients
// (two = P > 32, the same in every lane).  The test sits outside the loop: inside it the
// compiler predicates the second sum's multiply-adds, and an instruction whose lanes are all
// predicated off still takes its issue slots on the double pipe.
template <typename R>
__device__ __forceinline__ void coef_sums(const cx<R> *A, const R *C, int P, int lc0, int lc1,
                                          bool two, cx<R> &s0, cx<R> &s1)
{
    s0 = mk<R>(0, 0);
    s1 = mk<R>(0, 0);
    if (two) {
        for (int k = 0; k < P; k++) {
            const cx<R> a = A[k];
            const R c0 = C[k * P + lc0], c1 = C[k * P + lc1];
            s0.x = fm(c0, a.x, s0.x);
            s0.y = fm(c0, a.y, s0.y);
            s1.x = fm(c1, a.x, s1.x);
            s1.y = fm(c1, a.y, s1.y);
        }
    } else {
        for (int k = 0; k < P; k++) {
            const cx<R> a = A[k];
            const R c0 = C[k * P + lc0];
            s0.x = fm(c0, a.x, s0.x);
            s0.y = fm(c0, a.y, s0.y);
        }
    }
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
                     const double2 *__restrict__ xi, const cx<R> *__restrict__ uloc,
                     const cx<R> *__restrict__ q, cx<R> *mp, int *cnt, const int *gate,
                     int64_t slab)
{
    lbf_rhs(slab, q, mp, cnt, gate);
    if (gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl_len = (P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cl = (R *)sm_raw;  // Cl[k*P + l] = C(l, k) (0 for k > l)
    cx<R> *T = (cx<R> *)(sm_raw + cl_len) + (size_t)wid * P * 32;
    cx<R> *A = (cx<R> *)(sm_raw + cl_len) + (size_t)nw * P * 32 + (size_t)wid * 2 * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cl[e] = k <= l ? binom[l * LBF_MAX_TERMS + k] : R(0);
    }
    __syncthreads();
    int64_t t = blockIdx.x * (int64_t)nw + wid;
    if (t >= nleaf) return;
    int b = leaves[t];
    {
        double cxd = 0, cyd = 0, ir = 0;
        if constexpr (!kLocal<R>) {  // float and double-float read leaf-local coordinates
            double r;
            box_centre(g, level[b], ix[b], iy[b], cxd, cyd, r);
            ir = 1.0 / r;
        }
        cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
        for (int base = bg[b]; base < en[b]; base += 32) {
            int j = base + lane;
            cx<R> z = mk<R>(0, 0), term = mk<R>(0, 0);
            if (j < en[b]) {
                if constexpr (kLocal<R>) {
                    z = uloc[j];
                } else {
                    double2 x = xi[j];
                    z = mk<R>((R)((x.x - cxd) * ir), (R)((x.y - cyd) * ir));
                }
                term = q[j];
            }
            for (int k = 0; k < P; k++) {
                T[k * 32 + lane] = term;
                term = cmul(term, z);
            }
            __syncwarp();
            const int nin = min(32, en[b] - base);  // the chunk's nodes (the rest add 0)
            for (int k = lane; k < P; k += 32) {
                cx<R> s = mk<R>(0, 0);
                for (int m = 0; m < nin; m++) {
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
        if (P <= 32) {
            // Two children at a time, one per half-warp.  The M2M matrix C(l, k) (k <= l) is
            // triangular: lane j of a half sums the rows l = j and l = P - 1 - j, P + 1 terms
            // in one loop (it moves to the second row inside the loop); the halves' sums over
            // their children are added at the end.
            const int hf = lane >> 4, j = lane & 15;
            const unsigned hmask = hf ? 0xffff0000u : 0x0000ffffu;
            const int nr = (P + 1) / 2;
            const int r1 = j < nr ? j : 0, r2 = P - 1 - r1, n1 = r1 + 1;
            cx<R> *Ah = A + hf * P;
            cx<R> a1 = mk<R>(0, 0), a2 = mk<R>(0, 0);
            const int cend = child0[p] + nchild[p];
            for (int c0 = child0[p]; c0 < cend; c0 += 2) {
                const int c = c0 + hf;
                if (c < cend) {
                    const int d = (ix[c] & 1) + 2 * (iy[c] & 1);
                    const cx<R> *inv = d2inv(dtab, d);
                    for (int k = j; k < P; k += 16) Ah[k] = cmul(ldcg_cx(&mp[(int64_t)c * P + k]), inv[k]);
                    __syncwarp(hmask);
                    cx<R> acc = mk<R>(0, 0), s1 = mk<R>(0, 0);
                    for (int it = 0; it <= P; it++) {
                        const bool first = it < n1;
                        if (it == n1) {
                            s1 = acc;
                            acc = mk<R>(0, 0);
                        }
                        const int k = first ? it : it - n1, l = first ? r1 : r2;
                        const cx<R> a = Ah[k];
                        const R cc = Cl[k * P + l];
                        acc.x = fm(cc, a.x, acc.x);
                        acc.y = fm(cc, a.y, acc.y);
                    }
                    const cx<R> *dp = dpow(dtab, d);
                    a1 = cfma(dp[r1], s1, a1);
                    a2 = cfma(dp[r2], acc, a2);
                    __syncwarp(hmask);
                }
            }
            a1.x += __shfl_xor_sync(0xffffffffu, a1.x, 16);
            a1.y += __shfl_xor_sync(0xffffffffu, a1.y, 16);
            a2.x += __shfl_xor_sync(0xffffffffu, a2.x, 16);
            a2.y += __shfl_xor_sync(0xffffffffu, a2.y, 16);
            if (hf == 0 && j < nr) {
                mp[(int64_t)p * P + r1] = a1;
                if (r2 != r1) mp[(int64_t)p * P + r2] = a2;
            }
            cur = p;
            continue;
        }
        const int l0 = lane, l1 = lane + 32;
        const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
        cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
        for (int c = child0[p]; c < child0[p] + nchild[p]; c++) {
            int d = (ix[c] & 1) + 2 * (iy[c] & 1);
            const cx<R> *inv = d2inv(dtab, d);
            for (int k = lane; k < P; k += 32) {
                // written by other warps in this launch: read through L2
                const cx<R> a = ldcg_cx(&mp[(int64_t)c * P + k]);
                A[k] = cmul(a, inv[k]);
            }
            __syncwarp();
            cx<R> s0, s1;
            coef_sums(A, Cl, P, lc0, lc1, P > 32, s0, s1);
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

constexpr unsigned kPullSpins = 1u << 24;
constexpr unsigned kGrab = 1;

// Downward pass for one level (see lbf_fmm.cu): L2L + M2L (V) + P2L (X).
// P2L lanes take source nodes and run the power recurrence; their terms go
// through shared memory and lanes then take coefficients and sum in node order.
// Registers are held for three resident blocks of up to 8 warps per SM in float (a
// latency-bound pass) and two in double and double-float (whose shared memory allows two).
template <typename R> constexpr int kDownMinBlocks = std::is_same<R, float>::value ? 3 : 2;
template <typename R>
__global__ void __launch_bounds__(256, kDownMinBlocks<R>)
k_down(int64_t ls, int64_t le, const int32_t *__restrict__ level,
                       const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                       const int32_t *__restrict__ parent, const int32_t *__restrict__ vlist,
                       const int32_t *__restrict__ nv, const int32_t *__restrict__ xlist,
                       const int32_t *__restrict__ nx, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, BoxGeo g, int P,
                       const R *__restrict__ binom, const cx<R> *__restrict__ tpow,
                       const cx<R> *__restrict__ dtab, const double2 *__restrict__ xi,
                       const cx<R> *__restrict__ uloc, const cx<R> *__restrict__ q,
                       const cx<R> *__restrict__ mp, cx<R> *__restrict__ loc, const int *gate,
                       int with_l2l, unsigned *pull, int *status, const cx<df64> *__restrict__ udf,
                       int64_t slab)
{
    lbf_rhs(slab, q, mp, loc, gate, pull);
    if (gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nw = blockDim.x >> 5;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = (2 * P * P * (int)sizeof(R) + 15) / 16 * 16;
    R *Cm = (R *)sm_raw;          // Cm[k*P + l] = C(k+l, l)
    R *Cd = Cm + P * P;           // Cd[k*P + l] = C(k, l) (0 for k < l)
    cx<R> *A = (cx<R> *)(sm_raw + tl) + (size_t)wid * 2 * P;
    cx<R> *T = (cx<R> *)(sm_raw + tl) + (size_t)nw * 2 * P + (size_t)wid * P * 32;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int k = e / P, l = e % P;
        Cm[e] = binom[(k + l) * LBF_MAX_TERMS + l];
        Cd[e] = k >= l ? binom[k * LBF_MAX_TERMS + l] : R(0);
    }
    __syncthreads();
    const int l0 = lane, l1 = lane + 32;
    const int lc0 = l0 < P ? l0 : 0, lc1 = l1 < P ? l1 : 0;
    // with_l2l == 2: every box in one launch, in two phases.  Phase 1 takes runs of
    // boxes from a counter and writes each one's M2L + P2L part; phase 2 takes them
    // again in increasing index order (level by level) and adds the parent's full expansion
    // shifted down (L2L), once the parent is done.  Every box a warp waits for was
    // taken earlier by a running warp, so each wait ends.  The last warp to finish
    // resets the counters and advances the epoch that marks a box done.
    // pull: [0] phase-1 counter, [1] finished warps, [2] epoch, [3] phase-2 counter,
    // then per box the epoch of its phase-1 part and of its full expansion.
    unsigned *part = pull + 4, *done = pull + 4 + (le - ls);
    unsigned epoch = 0;
    if (with_l2l == 2) {
        if (lane == 0) epoch = *(volatile unsigned *)&pull[2];
        epoch = __shfl_sync(0xffffffffu, epoch, 0);
    }
    unsigned cb = 0, ce = 0;  // the warp's current run of boxes (kGrab at a time)
    for (int64_t it = 0;; it++) {
    int64_t b;
    if (with_l2l == 2) {
        if (cb == ce) {
            unsigned bi = 0;
            if (lane == 0) bi = atomicAdd(&pull[0], kGrab);
            cb = __shfl_sync(0xffffffffu, bi, 0);
            ce = cb + kGrab;
        }
        b = ls + (int64_t)cb++;
    } else {
        b = it == 0 ? ls + blockIdx.x * (int64_t)nw + wid : le;
    }
    if (b >= le) break;
    int bx = ix[b], by = iy[b];
    cx<R> accL0 = mk<R>(0, 0), accL1 = mk<R>(0, 0);
    // L2L: b'_l = (2d)^-l sum_{k>=l} C(k,l) d^k b_k, from the parent's full local expansion
    // (with_l2l == 1: written by the previous launch; 2: by another warp of this launch)
    auto l2l = [&]() {
        int p = parent[b];
        int d = (bx & 1) + 2 * (by & 1);
        const cx<R> *dp = dpow(dtab, d);
        for (int k = lane; k < P; k += 32) A[k] = cmul(ldcg_cx(&loc[(int64_t)p * P + k]), dp[k]);
        __syncwarp();
        cx<R> s0, s1;
        coef_sums(A, Cd, P, lc0, lc1, P > 32, s0, s1);
        const cx<R> *inv = d2inv(dtab, d);
        accL0 = cmul(inv[l0], s0);
        if (l1 < P) accL1 = cmul(inv[l1], s1);
        __syncwarp();
    };
    if (with_l2l == 1 && level[b] >= 3) l2l();
    // M2L: (-1)^l t^(l+1) sum_k C(k+l, l) t^k a_k,  t = 1/(2 (dx + i dy))  (times 1/r below)
    cx<R> accF0 = mk<R>(0, 0), accF1 = mk<R>(0, 0);
    if (P <= 16) {
        // two half-warps take two V-list boxes at a time; lane gl of a half-warp owns
        // coefficient gl, and the halves are summed at the end
        // the V list's boxes and offset indices are loaded once, a lane per entry (at most
        // 27), and the next pair's multipole coefficients are fetched one step ahead
        const int grp = lane >> 4, gl = lane & 15;
        const int glc = gl < P ? gl : 0;
        cx<R> *Ag = A + grp * P;
        const int nvb = nv[b];
        int vs = 0, vo = 0;
        if (lane < nvb) {
            vs = vlist[b * 27 + lane];
            vo = (bx - ix[vs] + 3) * 7 + (by - iy[vs] + 3);
        }
        cx<R> mnext = mk<R>(0, 0);
        {
            const int s0 = __shfl_sync(0xffffffffu, vs, grp);
            if (grp < nvb && gl < P) mnext = mp[(int64_t)s0 * P + gl];
        }
        for (int v0 = 0; v0 < nvb; v0 += 2) {
            const int vq = v0 + grp;
            const bool on = vq < nvb;
            const int o = __shfl_sync(0xffffffffu, vo, vq & 31);
            const int sn = __shfl_sync(0xffffffffu, vs, (vq + 2) & 31);
            const cx<R> mcur = mnext;
            if (vq + 2 < nvb && gl < P) mnext = mp[(int64_t)sn * P + gl];
            const cx<R> *tp = tpow + (size_t)(on ? o : 0) * (LBF_MAX_TERMS + 1);
            if (on && gl < P) Ag[gl] = cmul(mcur, tp[gl]);
            __syncwarp();
            if (on && gl < P) {
                cx<R> s0 = mk<R>(0, 0);
                for (int k = 0; k < P; k++) {
                    cx<R> a = Ag[k];
                    R c0 = Cm[k * P + glc];
                    s0.x = fm(c0, a.x, s0.x);
                    s0.y = fm(c0, a.y, s0.y);
                }
                cx<R> f0 = tp[gl + 1];
                if (gl & 1) { f0.x = -f0.x; f0.y = -f0.y; }
                accF0 = cfma(f0, s0, accF0);
            }
            __syncwarp();
        }
        accF0.x += __shfl_down_sync(0xffffffffu, accF0.x, 16);
        accF0.y += __shfl_down_sync(0xffffffffu, accF0.y, 16);
        if (lane >= 16) accF0 = mk<R>(0, 0);
    } else {
        bool done = false;
        if constexpr (std::is_same<R, double>::value) {
            if (nv[b] >= 4) {
                done = true;
                // Native double, four or more V-list boxes: a masked lane occupies the double pipe
                // like an active one, so the nv x P (box, coefficient) slots run flattened, 32 at a
                // time, instead of a box at a time on P of the 32 lanes.  The scaled multipoles
                // t^k a_k of all the boxes go to shared memory first; slot (v, l) forms
                // sum_k C(k+l, l) t_v^k a_{v,k} and adds (-1)^l t_v^(l+1) times it into the
                // coefficient l of a per-warp accumulator.  Lanes i and i + P of a round hold the
                // same l (P >= 17 here, so no third): they add in two steps, so every coefficient
                // takes its boxes in list order, the same operations in the same order as the
                // box-at-a-time loop.
                const int nvb = nv[b];
                int vs = 0, vo = 0;
                if (lane < nvb) {
                    vs = vlist[b * 27 + lane];
                    vo = (bx - ix[vs] + 3) * 7 + (by - iy[vs] + 3);
                }
                const int ns = nvb * P;
                cx<R> *Af = T;  // nv x P scaled multipoles (T holds 32 P)
                for (int s0 = 0; s0 < ns; s0 += 32) {
                    const int sl = s0 + lane, v = sl / P, k = sl - v * P;
                    const int src = __shfl_sync(0xffffffffu, vs, v & 31);
                    const int o = __shfl_sync(0xffffffffu, vo, v & 31);
                    if (sl < ns)
                        Af[sl] = cmul(mp[(int64_t)src * P + k], tpow[(size_t)o * (LBF_MAX_TERMS + 1) + k]);
                }
                for (int l = lane; l < P; l += 32) A[l] = mk<R>(0, 0);
                __syncwarp();
                for (int s0 = 0; s0 < ns; s0 += 32) {
                    const int sl = s0 + lane, v = sl / P, l = sl - v * P;
                    const int o = __shfl_sync(0xffffffffu, vo, v & 31);
                    const bool on = sl < ns;
                    cx<R> sa = mk<R>(0, 0);
                    if (on) {
                        const cx<R> *av = Af + v * P;
                        for (int k = 0; k < P; k++) {
                            const cx<R> a = av[k];
                            const R c = Cm[k * P + l];
                            sa.x = fm(c, a.x, sa.x);
                            sa.y = fm(c, a.y, sa.y);
                        }
                    }
                    cx<R> f = on ? tpow[(size_t)o * (LBF_MAX_TERMS + 1) + l + 1] : mk<R>(0, 0);
                    if (l & 1) { f.x = -f.x; f.y = -f.y; }
                    if (on && lane < P) A[l] = cfma(f, sa, A[l]);
                    __syncwarp();
                    if (on && lane >= P) A[l] = cfma(f, sa, A[l]);
                    __syncwarp();
                }
                if (l0 < P) accF0 = A[l0];
                if (l1 < P) accF1 = A[l1];
                __syncwarp();
            }
        }
        if (!done) {
            // V-list records loaded once (a lane per entry); with P <= 32 the next box's
            // coefficients are fetched one step ahead
            const int nvb = nv[b];
            int vs = 0, vo = 0;
            if (lane < nvb) {
                vs = vlist[b * 27 + lane];
                vo = (bx - ix[vs] + 3) * 7 + (by - iy[vs] + 3);
            }
            cx<R> mnext = mk<R>(0, 0);
            const int sfirst = __shfl_sync(0xffffffffu, vs, 0);
            if (P <= 32 && nvb > 0 && lane < P) mnext = mp[(int64_t)sfirst * P + lane];
            for (int vq = 0; vq < nvb; vq++) {
                const int s = __shfl_sync(0xffffffffu, vs, vq);
                const int o = __shfl_sync(0xffffffffu, vo, vq);
                const int sn = __shfl_sync(0xffffffffu, vs, (vq + 1) & 31);
                const cx<R> *tp = tpow + (size_t)o * (LBF_MAX_TERMS + 1);
                if (P <= 32) {
                    const cx<R> mcur = mnext;
                    if (vq + 1 < nvb && lane < P) mnext = mp[(int64_t)sn * P + lane];
                    if (lane < P) A[lane] = cmul(mcur, tp[lane]);
                } else {
                    for (int k = lane; k < P; k += 32) A[k] = cmul(mp[(int64_t)s * P + k], tp[k]);
                }
                __syncwarp();
                cx<R> s0, s1;
                coef_sums(A, Cm, P, lc0, lc1, P > 32, s0, s1);
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
        }
    }
    // P2L: (-1)^l sum_j q_j tau_j^(l+1), tau_j = r / (c - xi_j)  (times 1/r below)
    const int lb = level[b];
    double cxd = 0, cyd = 0, ir = 0;
    bool have_c = false;
    auto need_centre = [&]() {  // double centre: the double path and float fallbacks only
        if (have_c) return;
        double r;
        box_centre(g, lb, bx, by, cxd, cyd, r);
        ir = 1.0 / r;
        have_c = true;
    };
    if constexpr (!kLocal<R>) need_centre();
    // the X list's box records (at most 16), a lane per box, then broadcast
    const int nxb = nx[b];
    int xr_s = 0, xr_l = 0, xr_x = 0, xr_y = 0, xr_b = 0, xr_e = 0;
    if (lane < nxb) {
        xr_s = xlist[b * 16 + lane];
        xr_l = level[xr_s];
        xr_x = ix[xr_s];
        xr_y = iy[xr_s];
        xr_b = bg[xr_s];
        xr_e = en[xr_s];
    }
    if constexpr (std::is_same<R, double>::value) {
        // native double: the X-list boxes' nodes (all taken relative to this box's centre
        // in double) run as one list, 32 at a time, so short source boxes share a round
        const int xn = lane < nxb ? xr_e - xr_b : 0;
        int inc = xn;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const int nxt = __shfl_sync(0xffffffffu, inc, 31), xoff = inc - xn;
        if (nxt > 0) need_centre();
        for (int base = 0; base < nxt; base += 32) {
            const int gi = base + lane;
            int j = -1;
            for (int xq = 0; xq < nxb; xq++) {
                const int o = __shfl_sync(0xffffffffu, xoff, xq);
                const int n = __shfl_sync(0xffffffffu, xn, xq);
                const int b0 = __shfl_sync(0xffffffffu, xr_b, xq);
                if (gi >= o && gi < o + n) j = b0 + gi - o;
            }
            cx<R> tau = mk<R>(0, 0), term = mk<R>(0, 0);
            if (j >= 0) {
                const double2 z = xi[j];
                tau = crcp(mk<R>((R)((cxd - z.x) * ir), (R)((cyd - z.y) * ir)));
                term = cmul(q[j], tau);  // l = 0
            }
            for (int l = 0; l < P; l++) {
                T[l * 32 + lane] = (l & 1) ? mk<R>(-term.x, -term.y) : term;
                term = cmul(term, tau);
            }
            __syncwarp();
            const int nin = min(32, nxt - base);
            for (int l = lane; l < P; l += 32) {
                cx<R> sm = mk<R>(0, 0);
                for (int m = 0; m < nin; m++) {
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
    for (int xq = 0; xq < (std::is_same<R, double>::value ? 0 : nxb); xq++) {
        const int ls = __shfl_sync(0xffffffffu, xr_l, xq);
        const int sx_ = __shfl_sync(0xffffffffu, xr_x, xq), sy_ = __shfl_sync(0xffffffffu, xr_y, xq);
        const int sbg = __shfl_sync(0xffffffffu, xr_b, xq), sen = __shfl_sync(0xffffffffu, xr_e, xq);
        // float, double-float: the source's leaf-local coordinate rescaled into this box's frame
        bool local = false, dfp = false;
        R fs = R(0.0f);
        cx<R> os = mk<R>(R(0.0f), R(0.0f));
        if constexpr (kLocal<R>) {
            local = lb >= ls && lb - ls <= kMaxGap<R>;
            if constexpr (std::is_same<R, float>::value)
                dfp = !local && udf && lb >= ls && lb - ls <= kDfGap;
            if (local || dfp) {
                fs = R(pow2<float>(lb - ls));
                os = offset_cx<R>(centre_offset(ls, sx_, sy_, lb, bx, by));
            }
        }
        for (int base = sbg; base < sen; base += 32) {
            int j = base + lane;
            cx<R> tau = mk<R>(0, 0), term = mk<R>(0, 0);
            if (j < sen) {
                if (local) {
                    const cx<R> uu = uloc[j];
                    tau = crcp(mk<R>(-(uu.x * fs + os.x), -(uu.y * fs + os.y)));
                } else if (dfp) {
                    if constexpr (std::is_same<R, float>::value) {
                        const cx<df64> ud = udf[j];
                        tau = crcp(mk<R>(-df_round(df_ldexp(ud.x, fs) + df64(os.x)),
                                         -df_round(df_ldexp(ud.y, fs) + df64(os.y))));
                    }
                } else {
                    need_centre();
                    double2 z = xi[j];
                    tau = crcp(mk<R>((R)((cxd - z.x) * ir), (R)((cyd - z.y) * ir)));
                }
                term = cmul(q[j], tau);  // l = 0
            }
            for (int l = 0; l < P; l++) {
                T[l * 32 + lane] = (l & 1) ? mk<R>(-term.x, -term.y) : term;
                term = cmul(term, tau);
            }
            __syncwarp();
            const int nin = min(32, sen - base);
            for (int l = lane; l < P; l += 32) {
                cx<R> sm = mk<R>(0, 0);
                for (int m = 0; m < nin; m++) {
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
    R irr;
    if constexpr (kLocal<R>) irr = inv_half_width<R>(g, lb);
    else irr = (R)ir;
    if (l0 < P) loc[b * P + l0] = mk<R>(accL0.x + accF0.x * irr, accL0.y + accF0.y * irr);
    if (l1 < P) loc[b * P + l1] = mk<R>(accL1.x + accF1.x * irr, accL1.y + accF1.y * irr);
    if (with_l2l == 2) {
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicExch(&part[b - ls], epoch + 1u);
    }
    }  // boxes
    if (with_l2l != 2) return;
    // phase 2: full expansions, top down
    auto wait_for = [&](const unsigned *flag) {
        if (lane == 0) {
            unsigned spins = 0;
            const unsigned lim = wait_limit(status, kPullSpins);
            while (*(volatile const unsigned *)flag != epoch + 1u)
                if (++spins > lim) {
                    atomicOr(status, LBF_DEV_TIMEOUT);
                    break;
                }
        }
        __syncwarp();
        __threadfence();
    };
    if (P <= 32) {
        // Two boxes a warp, one per half-warp.  The L2L matrix C(k, l) (k >= l) is
        // triangular: lane j of a half sums the rows l = j and l = P - 1 - j, P + 1 terms in
        // one loop (it moves to the second row inside the loop), each row's terms in the
        // order of the full-row loop without its zero terms.  Each half waits for its own
        // box's part and parent; when the parent is the other half's box, the other half
        // marks it done first.
        const int hf = lane >> 4, j = lane & 15;
        const unsigned hmask = hf ? 0xffff0000u : 0x0000ffffu;
        const int nr = (P + 1) / 2;  // lanes of a half with rows
        const int r1 = j < nr ? j : 0, r2 = P - 1 - r1, n1 = P - r1;
        cx<R> *Ah = A + hf * P;
        auto wait_half = [&](const unsigned *flag) {
            if (j == 0) {
                unsigned spins = 0;
                const unsigned lim = wait_limit(status, kPullSpins);
                while (*(volatile const unsigned *)flag != epoch + 1u)
                    if (++spins > lim) {
                        atomicOr(status, LBF_DEV_TIMEOUT);
                        break;
                    }
            }
            __syncwarp(hmask);
            __threadfence();
        };
        for (;;) {
            unsigned bi = 0;
            if (lane == 0) bi = atomicAdd(&pull[3], 2u);
            const int64_t bpair = ls + (int64_t)__shfl_sync(0xffffffffu, bi, 0);
            if (bpair >= le) break;
            const int64_t b = bpair + hf;
            if (b >= le) continue;
            wait_half(&part[b - ls]);
            if (level[b] >= 3) {
                const int p = parent[b];
                wait_half(&done[p - ls]);
                const int bx = ix[b], by = iy[b], d = (bx & 1) + 2 * (by & 1);
                const cx<R> *dp = dpow(dtab, d);
                for (int k = j; k < P; k += 16) Ah[k] = cmul(ldcg_cx(&loc[(int64_t)p * P + k]), dp[k]);
                __syncwarp(hmask);
                cx<R> acc = mk<R>(0, 0), s1 = mk<R>(0, 0);
                for (int it = 0; it <= P; it++) {
                    const bool first = it < n1;
                    if (it == n1) {
                        s1 = acc;
                        acc = mk<R>(0, 0);
                    }
                    const int k = first ? r1 + it : r2 + (it - n1), l = first ? r1 : r2;
                    const cx<R> a = Ah[k];
                    const R c = Cd[k * P + l];
                    acc.x = fm(c, a.x, acc.x);
                    acc.y = fm(c, a.y, acc.y);
                }
                const cx<R> *inv = d2inv(dtab, d);
                if (j < nr) {
                    const cx<R> own = ldcg_cx(&loc[b * P + r1]);
                    loc[b * P + r1] = cfma(inv[r1], s1, own);
                    if (r2 != r1) {
                        const cx<R> own2 = ldcg_cx(&loc[b * P + r2]);
                        loc[b * P + r2] = cfma(inv[r2], acc, own2);
                    }
                }
                __threadfence();
                __syncwarp(hmask);
            }
            if (j == 0) atomicExch(&done[b - ls], epoch + 1u);
        }
    } else {
        cb = ce = 0;
        for (;;) {
            if (cb == ce) {
                unsigned bi = 0;
                if (lane == 0) bi = atomicAdd(&pull[3], kGrab);
                cb = __shfl_sync(0xffffffffu, bi, 0);
                ce = cb + kGrab;
            }
            const int64_t b = ls + (int64_t)cb++;
            if (b >= le) break;
            wait_for(&part[b - ls]);
            if (level[b] >= 3) {
                const int p = parent[b];
                wait_for(&done[p - ls]);
                const int bx = ix[b], by = iy[b], d = (bx & 1) + 2 * (by & 1);
                const cx<R> *dp = dpow(dtab, d);
                for (int k = lane; k < P; k += 32) A[k] = cmul(ldcg_cx(&loc[(int64_t)p * P + k]), dp[k]);
                __syncwarp();
                cx<R> s0, s1;
                coef_sums(A, Cd, P, lc0, lc1, P > 32, s0, s1);
                const cx<R> *inv = d2inv(dtab, d);
                if (l0 < P) {
                    const cx<R> own = ldcg_cx(&loc[b * P + l0]);
                    loc[b * P + l0] = cfma(inv[l0], s0, own);
                }
                if (l1 < P) {
                    const cx<R> own = ldcg_cx(&loc[b * P + l1]);
                    loc[b * P + l1] = cfma(inv[l1], s1, own);
                }
                __threadfence();
                __syncwarp();
            }
            if (lane == 0) atomicExch(&done[b - ls], epoch + 1u);
        }
    }
    if (lane == 0) {
        const unsigned total = gridDim.x * (unsigned)nw;
        if (atomicAdd(&pull[1], 1u) == total - 1u) {
            pull[0] = 0u;
            pull[1] = 0u;
            pull[3] = 0u;
            __threadfence();
            atomicExch(&pull[2], epoch + 1u);
        }
    }
}

constexpr int kLeafWarps = 4;  // default warps per block of the leaf kernel
constexpr int kSrcChunk = 256;
constexpr int kLeafExtra = 64 * 16;  // per warp: 32 target positions, 32 pairs of partial sums

template <typename R> struct LeafSrc {
    cx<R> z, q;
};
// dynamic shared memory of the leaf kernel for lw warps per block
template <typename R, int MODE> constexpr size_t leaf_smem(int lw)
{
    return (size_t)lw * (kSrcChunk * sizeof(LeafSrc<R>) +
                         (std::is_same<R, double>::value && MODE == 0 ? kLeafExtra : 0));
}
__device__ __forceinline__ bool positive(float x) { return x > 0.0f; }
__device__ __forceinline__ bool positive(double x) { return x > 0.0; }
__device__ __forceinline__ bool positive(df64 x) { return x.hi > 0.0f; }
// far below any squared distance between distinct nodes in units of a leaf half-width,
// and its reciprocal stays finite in R
template <typename R> __device__ __forceinline__ R tiny_sq();
template <> __device__ __forceinline__ float tiny_sq<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_sq<double>() { return 1e-30; }
template <> __device__ __forceinline__ df64 tiny_sq<df64>() { return df64(1e-30f); }

// What the leaf kernel writes for node i (all with the self pair excluded):
//   kLeafForward   v_i = 2 [ (1/2pi) Im sum_j q_j/(xi_j - xi_i) + dself_i sigma_i + s ],
//                  the double-layer rows of Eq. disc_sphere (s = beta.sigma);
//   kLeafTranspose v_i = 2 [ (1/2pi) Im(w_i Phi(xi_i)) + dself_i sigma_i + beta_i s ],
//                  Phi(z) = sum_j q_j/(z - xi_j) with real charges q_j = tau_j and
//                  s = sum_j tau_j: the transposed rows (K^T tau)_i;
//   kLeafDeriv     Phi'(xi_i) = -sum_j q_j/(xi_i - xi_j)^2 as a double2.
constexpr int kLeafForward = 0, kLeafTranspose = 1, kLeafDeriv = 2;

// Per leaf: far field (L2P of the leaf's full local expansion and M2P from W(b)),
// near field (P2P over U(b)), then the output above.  A lane
// owns one target; the sources of U(b) pass through shared memory in chunks and
// every lane reads each one (broadcast).  Near-field positions are taken relative
// to the leaf centre in units of its half-width r, so close nodes cancel before
// any rounding to R: in double from the node positions, in float from each node's
// own leaf-local coordinate rescaled by a power of two and shifted by the exact
// offset between box centres (double positions only where a source box is much
// coarser).
template <typename R, int MODE>
__global__ void k_leaf(int64_t nleaf, const int32_t *__restrict__ leaves,
                       const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                       const int32_t *__restrict__ iy, const int32_t *__restrict__ bg,
                       const int32_t *__restrict__ en, const int32_t *__restrict__ uptr,
                       const int32_t *__restrict__ uidx, const int32_t *__restrict__ wptr,
                       const int32_t *__restrict__ widx, BoxGeo g, int P,
                       const double2 *__restrict__ xi, const cx<R> *__restrict__ uloc,
                       const cx<R> *__restrict__ q, const cx<R> *__restrict__ mp,
                       const cx<R> *__restrict__ loc, const double *__restrict__ sigma,
                       const double *__restrict__ dself, const double2 *__restrict__ w,
                       const double *__restrict__ beta, const double *__restrict__ bsig,
                       double *__restrict__ v, const int *gate, const cx<df64> *__restrict__ udf,
                       int l2p, const int32_t *__restrict__ isl, const double *__restrict__ imean,
                       const double *__restrict__ iacoef, int M, int64_t slab,
                       const double *__restrict__ nearv)
{
    lbf_rhs(slab, q, mp, loc, sigma, bsig, v, gate, imean, nearv);
    if (gate_closed(gate)) return;
    constexpr bool kF32 = kLocal<R>;  // leaf-local coordinates (float, double-float)
    // per warp, kSrcChunk staged sources (position in units of r, charge); the warps per
    // block (the near-field tile) is a launch parameter
    extern __shared__ __align__(16) unsigned char leaf_sm[];
    LeafSrc<R>(*ss)[kSrcChunk] = (LeafSrc<R>(*)[kSrcChunk])leaf_sm;
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the double forward rows split the near field's (target, source) pairs evenly over
    // the lanes (below); the others give each target 32/TP lanes
    constexpr bool kFlat = std::is_same<R, double>::value && MODE == kLeafForward;
    double2 *tz = (double2 *)(leaf_sm + (blockDim.x >> 5) * kSrcChunk * sizeof(LeafSrc<R>)) +
                  (size_t)wid * 64;
    double2 *part = tz + 32;
    int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + wid;
    if (t >= nleaf) return;
    const int b = leaves[t];
    const int lt = level[b], tx = ix[b], ty = iy[b];
    double cxd = 0, cyd = 0, ir = 0;
    bool have_c = false;
    auto need_centre = [&]() {  // double centre: the double path and float fallbacks only
        if (have_c) return;
        double r;
        box_centre(g, lt, tx, ty, cxd, cyd, r);
        ir = 1.0 / r;
        have_c = true;
    };
    R irr;
    if constexpr (kF32) {
        irr = inv_half_width<R>(g, lt);
    } else {
        need_centre();
        irr = (R)ir;
    }
    const cx<R> *lb = loc + (int64_t)b * P;
    for (int tb = bg[b]; tb < en[b]; tb += 32) {
        const int nt = min(32, en[b] - tb);
        const int i = tb + lane;
        const bool act = lane < nt;  // this lane's far field and output
        // near field: TP >= nt target slots, 32/TP lanes per target splitting the sources
        const int TP = nt <= 1 ? 1 : 1 << (32 - __clz(nt - 1));
        const int slot = lane & (TP - 1), grp = lane / TP, G = 32 / TP;
        const bool pact = slot < nt;
        cx<R> u = mk<R>(0, 0);  // (z - c)/r
        cx<R> phi = mk<R>(0, 0);  // far field: Phi (or Phi' in kLeafDeriv)
        if (act) {
            if constexpr (kF32) {
                u = uloc[i];
            } else {
                double2 zi = xi[i];
                u = mk<R>((zi.x - cxd) * ir, (zi.y - cyd) * ir);
            }
            // (the double forward rows take their far field below, flattened)
            if constexpr (!kFlat) {
            if constexpr (MODE == kLeafDeriv) {
                // d/dz sum_l b_l ((z - c)/r)^l = (1/r) sum_{l>=1} l b_l u^(l-1)
                cx<R> d = mk<R>((R)(P - 1) * lb[P - 1].x, (R)(P - 1) * lb[P - 1].y);
                for (int l = P - 2; l >= 1; l--)
                    d = cfma(d, u, mk<R>((R)l * lb[l].x, (R)l * lb[l].y));
                phi = mk<R>(d.x * irr, d.y * irr);
            } else if (l2p) {
                phi = lb[P - 1];
                for (int l = P - 2; l >= 0; l--) phi = cfma(phi, u, lb[l]);
            }
            for (int wq = wptr[b]; wq < wptr[b + 1]; wq++) {
                const int s = widx[wq];
                const int ls = level[s];
                cx<R> zs;  // (z - c_s)/r_s
                R isr;
                bool local = false;
                if constexpr (kF32) {
                    local = ls >= lt && ls - lt <= kMaxGap<R>;
                    if (local) {
                        const R f = R(pow2<float>(ls - lt));
                        const cx<R> o = offset_cx<R>(centre_offset(lt, tx, ty, ls, ix[s], iy[s]));
                        zs = mk<R>(u.x * f + o.x, u.y * f + o.y);
                        isr = irr * f;
                    }
                    if constexpr (std::is_same<R, float>::value) {
                        if (!local && udf && ls >= lt && ls - lt <= kDfGap) {
                            const float f = pow2<float>(ls - lt);
                            const float2 o = centre_offset(lt, tx, ty, ls, ix[s], iy[s]);
                            const cx<df64> ud = udf[i];
                            zs = mk<R>(df_round(df_ldexp(ud.x, f) + df64(o.x)),
                                       df_round(df_ldexp(ud.y, f) + df64(o.y)));
                            isr = irr * f;
                            local = true;
                        }
                    }
                }
                if (!local) {
                    double2 zi = xi[i];
                    double sxd, syd, sr;
                    box_centre(g, ls, ix[s], iy[s], sxd, syd, sr);
                    const double isd = 1.0 / sr;
                    zs = mk<R>((R)((zi.x - sxd) * isd), (R)((zi.y - syd) * isd));
                    isr = (R)isd;
                }
                const cx<R> rho = crcp(zs);  // r_s / (z - c_s)
                const cx<R> *a = mp + (int64_t)s * P;
                if constexpr (MODE == kLeafDeriv) {
                    // -(1/r^2) sum_k (k+1) a_k rho^(k+2)
                    cx<R> ps = mk<R>((R)P * a[P - 1].x, (R)P * a[P - 1].y);
                    for (int k = P - 2; k >= 0; k--)
                        ps = cfma(ps, rho, mk<R>((R)(k + 1) * a[k].x, (R)(k + 1) * a[k].y));
                    ps = cmul(ps, cmul(rho, rho));
                    phi.x -= ps.x * isr * isr;
                    phi.y -= ps.y * isr * isr;
                } else {
                    cx<R> ps = a[P - 1];
                    for (int k = P - 2; k >= 0; k--) ps = cfma(ps, rho, a[k]);
                    ps = cmul(ps, rho);
                    phi.x += ps.x * isr;
                    phi.y += ps.y * isr;
                }
            }
            }
        }
        // near field, in units of r: sum over sources of q conj(dz)/|dz|^2 (Im part only
        // in the forward mode) or q conj(dz)^2/|dz|^4, dz = xi_s - z
        const cx<R> ut = mk<R>(__shfl_sync(0xffffffffu, u.x, slot),
                               __shfl_sync(0xffffffffu, u.y, slot));
        R accI = 0;
        cx<R> acc = mk<R>(0, 0);
        int fill = 0;
        double phiI = 0.0;  // the double forward rows: Im of the far field at target lane
        if constexpr (kFlat) {
            if (act) tz[lane] = make_double2((double)u.x, (double)u.y);
            __syncwarp();
            // Far field as nt x (1 + |W(b)|) items, 32 at a time, source-major (the lanes of a
            // round mostly share one expansion): item (0, t) is the L2P of the leaf's own
            // local expansion at target t, item (s, t) the M2P of the s-th W-list box.  Both
            // are a Horner sum of P terms at a point x, times a factor w: x = w = 1 for the
            // L2P; x = rho = r_s/(z - c_s) and w = rho/r_s for the M2P.  Each target then
            // adds its items of the round in item order.
            const int wb = wptr[b], nit = nt * (wptr[b + 1] - wb + (l2p ? 1 : 0));
            const int s_off = l2p ? 0 : 1;
            for (int i0 = 0; i0 < nit; i0 += 32) {
                const int it = min(i0 + lane, nit - 1);
                const int sq = it / nt + s_off, t = it - (sq - s_off) * nt;
                const cx<double> *cf;
                cx<double> x, w;
                if (sq == 0) {
                    cf = (const cx<double> *)lb;
                    x = mk<double>(tz[t].x, tz[t].y);
                    w = mk<double>(1.0, 0.0);
                } else {
                    const int sb = widx[wb + sq - 1];
                    double sxd, syd, sir;
                    box_centre_ir(g, level[sb], ix[sb], iy[sb], sxd, syd, sir);
                    const double2 zi = xi[tb + t];
                    x = crcp(mk<double>((zi.x - sxd) * sir, (zi.y - syd) * sir));
                    w = mk<double>(x.x * sir, x.y * sir);
                    cf = (const cx<double> *)mp + (int64_t)sb * P;
                }
                cx<double> h = cf[P - 1];
                for (int l = P - 2; l >= 0; l--) h = cfma(h, x, cf[l]);
                part[lane].x = fma(w.x, h.y, w.y * h.x);  // Im(w h)
                __syncwarp();
                if (lane < nt) {
                    for (int L = (lane - i0 % nt + nt) % nt; L < 32 && i0 + L < nit; L += nt)
                        phiI += part[L].x;
                }
                __syncwarp();
            }
        }
        // Double forward rows: a masked lane occupies the double pipe like an active one,
        // so the nt x fill (target, source) pairs of a staged chunk, target-major, are
        // cut into 32 runs of W = ceil(nt fill / 32); a run spans at most two targets
        // (W <= fill), and each target then sums the partial sums of the runs that
        // cover it, in lane order (a fixed order: the result does not depend on timing).
        auto process_flat = [&]() {
            __syncwarp();
            const int tot = nt * fill, W = (tot + 31) >> 5;
            const int a0 = min(lane * W, tot), a1 = min(a0 + W, tot);
            // one loop of a1 - a0 steps (the same for all but the last runs); a run that
            // reaches the end of its first target moves on to the next one inside it, so
            // the warp does not execute the two targets' parts one after the other
            double p = 0.0, pfirst = 0.0;
            bool second = false;
            {
                const int t = a0 < tot ? a0 / fill : 0;
                int m = a0 - t * fill;
                double2 z = tz[t];
#pragma unroll 4
                for (int k = a0; k < a1; k++, m++) {
                    if (m == fill) {
                        pfirst = p;
                        p = 0.0;
                        m = 0;
                        z = tz[t + 1];
                        second = true;
                    }
                    const LeafSrc<R> sm = ss[wid][m];
                    const double dr = (double)sm.z.x - z.x, di = (double)sm.z.y - z.y;
                    const double ir2 = rcp_near(fma(dr, dr, fma(di, di, 1e-30)));
                    p = fma(fma((double)sm.q.y, dr, -(double)sm.q.x * di), ir2, p);
                }
            }
            part[lane] = second ? make_double2(pfirst, p) : make_double2(p, 0.0);
            __syncwarp();
            if (lane < nt) {
                const int lo = (lane * fill) / W, hi = ((lane + 1) * fill - 1) / W;
                double sum = 0.0;
                for (int L = lo; L <= hi; L++) {
                    const double2 pv = part[L];
                    sum += (L * W) / fill == lane ? pv.x : pv.y;  // the run's first target?
                }
                accI += (R)sum;
            }
            __syncwarp();
            fill = 0;
        };
        auto process = [&]() {
            if constexpr (kFlat) {
                process_flat();
                return;
            }
            __syncwarp();
            if (pact) {
#pragma unroll 4
                for (int m = grp; m < fill; m += G) {
                    const LeafSrc<R> sm = ss[wid][m];
                    const cx<R> zs = sm.z, qq = sm.q;
                    const R dr = zs.x - ut.x, di = zs.y - ut.y;
                    // the target itself (the only source at distance 0) adds nothing: with a
                    // tiny shift of |dz|^2 its term is 0 x (finite), so the forward and
                    // transposed rows need no test; the derivative rows (|dz|^-4) test
                    R ir2;
                    if constexpr (MODE == kLeafDeriv) {
                        const R d2 = fm(dr, dr, di * di);
                        ir2 = positive(d2) ? rcp(d2) : R(0.0f);
                    } else if constexpr (std::is_same<R, double>::value) {
                        ir2 = rcp_near(fma(dr, dr, fma(di, di, tiny_sq<R>())));
                    } else {
                        ir2 = rcp(fm(dr, dr, di * di) + tiny_sq<R>());
                    }
                    if constexpr (MODE == kLeafForward) {
                        accI = fm(fm(qq.y, dr, -qq.x * di), ir2, accI);
                    } else if constexpr (MODE == kLeafTranspose) {
                        acc.x = fm(fm(qq.x, dr, qq.y * di), ir2, acc.x);
                        acc.y = fm(fm(qq.y, dr, -qq.x * di), ir2, acc.y);
                    } else {
                        // q conj(dz)^2 / |dz|^4
                        const R er = (dr * dr - di * di) * ir2 * ir2, ei = -2 * dr * di * ir2 * ir2;
                        acc.x = fm(qq.x, er, fm(-qq.y, ei, acc.x));
                        acc.y = fm(qq.x, ei, fm(qq.y, er, acc.y));
                    }
                }
            }
            __syncwarp();
            fill = 0;
        };
        // (nearv given: the near field of these rows was summed by k_near_multi)
        for (int uq = uptr[b]; !nearv && uq < uptr[b + 1]; uq++) {
            const int s = uidx[uq];
            int sb = bg[s], se = en[s];
            bool local = false, dfp = false;
            R fs = R(0.0f);
            cx<R> os = mk<R>(R(0.0f), R(0.0f));
            if constexpr (kF32) {
                const int ls = level[s];
                local = ls >= lt && ls - lt <= 16;
                if constexpr (std::is_same<R, float>::value)
                    dfp = !local && udf && ls < lt && lt - ls <= kDfGap;  // a coarser source leaf
                if (local || dfp) {
                    fs = R(pow2<float>(lt - ls));
                    os = offset_cx<R>(centre_offset(ls, ix[s], iy[s], lt, tx, ty));
                }
            }
            while (sb < se) {
                int take = min(se - sb, kSrcChunk - fill);
                for (int m = lane; m < take; m += 32) {
                    cx<R> zr;  // (z_j - c)/r
                    if (local) {
                        const cx<R> uu = uloc[sb + m];
                        zr = mk<R>(uu.x * fs + os.x, uu.y * fs + os.y);
                    } else if (dfp) {
                        if constexpr (std::is_same<R, float>::value) {
                            const cx<df64> ud = udf[sb + m];
                            zr = mk<R>(df_round(df_ldexp(ud.x, fs) + df64(os.x)),
                                       df_round(df_ldexp(ud.y, fs) + df64(os.y)));
                        }
                    } else {
                        need_centre();
                        double2 zs = xi[sb + m];
                        zr = mk<R>((R)((zs.x - cxd) * ir), (R)((zs.y - cyd) * ir));
                    }
                    ss[wid][fill + m] = LeafSrc<R>{zr, q[sb + m]};
                }
                fill += take;
                sb += take;
                if (fill == kSrcChunk) process();
            }
        }
        if (fill > 0) process();
        if constexpr (!kFlat) {
            for (int o = TP; o < 32; o <<= 1) {  // sum the source groups of each target
                accI += __shfl_xor_sync(0xffffffffu, accI, o);
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
        }
        if (act) {
            if constexpr (MODE == kLeafForward) {
                double c = (double)(-(kFlat ? (R)phiI : phi.y)) + (double)(accI * irr);
                if (nearv) c += nearv[i];
                // with island means m split off (isl given): the sums saw sigma - m; the
                // means' rows are a_k m_k + 2 n m_(enclosing island) (the beta . m part is
                // in bsig, formed from sigma)
                double mk = 0.0, mrow = 0.0;
                if (isl) {
                    const int k = isl[i];
                    mk = imean[k];
                    const int ke = (int)imean[M + 1];
                    mrow = iacoef[k] * mk + (ke >= 0 ? imean[M + 2] * imean[ke] : 0.0);
                }
                v[i] = 2.0 * (c * (1.0 / (2.0 * LBF_PI)) + dself[i] * (sigma[i] - mk) + *bsig) + mrow;
            } else if constexpr (MODE == kLeafTranspose) {
                // Phi = far - near sum (the near sum above is sum q/(xi_s - z))
                const double pr = (double)phi.x - (double)(acc.x * irr);
                const double pi = (double)phi.y - (double)(acc.y * irr);
                const double2 ww = w[i];
                const double im = ww.x * pi + ww.y * pr;
                v[i] = 2.0 * (im * (1.0 / (2.0 * LBF_PI)) + dself[i] * sigma[i] + beta[i] * *bsig);
            } else {
                const double i2 = (double)irr * (double)irr;
                ((double2 *)v)[i] = make_double2((double)phi.x - (double)acc.x * i2,
                                                 (double)phi.y - (double)acc.y * i2);
            }
        }
        __syncwarp();
    }
}

// The far field of the float operator's forward rows, a thread per node: every
// ancestor's own local expansion (levels >= 2, the leaf included) at the node, from its
// leaf-local coordinate u: (z - c_a)/r_a = 2((ix_b - 2^s ix_a + 1/2) 2^-s - 1/2) + u 2^-s
// for a depth gap s (ix_b - 2^s ix_a = the low s bits of ix_b).  Adds the far-field
// term of the forward rows, 2 (1/2pi) (-Im Phi), to v (the leaf kernel wrote the rest).
// A parallel alternative to shifting the expansions down the tree (L2L): no serial
// chain, and the nodes of a leaf share their ancestors' coefficients in L1.
__global__ void k_l2p_walk(int64_t N, int P, const int32_t *__restrict__ leaf_of,
                           const int32_t *__restrict__ level, const int32_t *__restrict__ ix,
                           const int32_t *__restrict__ iy, const int32_t *__restrict__ anc,
                           const float2 *__restrict__ u32, const cx<float> *__restrict__ loc,
                           double *__restrict__ v, const int *gate, int64_t slab)
{
    lbf_rhs(slab, loc, v, gate);
    if (gate_closed(gate)) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = leaf_of[i];
    const float2 uu = u32[i];
    const int lv = level[b], bx = ix[b], by = iy[b];
    const int32_t *ab = anc + (int64_t)b * LBF_ANC_STRIDE;
    auto at = [&](int sh) {  // the node in ancestor sh's frame, and its coefficients
        const float sc = pow2<float>(-sh);
        const int dxi = bx & ((1 << sh) - 1), dyi = by & ((1 << sh) - 1);
        return mk<float>(2.0f * (((float)dxi + 0.5f) * sc - 0.5f) + uu.x * sc,
                         2.0f * (((float)dyi + 0.5f) * sc - 0.5f) + uu.y * sc);
    };
    // two ancestors at a time: two independent Horner chains
    float acc = 0.0f;
    const int na = lv - 1;
    int sh = 0;
    for (; sh + 1 < na; sh += 2) {
        const cx<float> *la = loc + (int64_t)ab[sh] * P, *lb = loc + (int64_t)ab[sh + 1] * P;
        const cx<float> ua = at(sh), ub = at(sh + 1);
        cx<float> ta = la[P - 1], tb = lb[P - 1];
        for (int l = P - 2; l >= 0; l--) {
            ta = cfma(ta, ua, la[l]);
            tb = cfma(tb, ub, lb[l]);
        }
        acc += ta.y + tb.y;
    }
    if (sh < na) {
        const cx<float> *la = loc + (int64_t)ab[sh] * P;
        const cx<float> ua = at(sh);
        cx<float> t = la[P - 1];
        for (int l = P - 2; l >= 0; l--) t = cfma(t, ua, la[l]);
        acc += t.y;
    }
    v[i] += 2.0 * (-(double)acc * (1.0 / (2.0 * LBF_PI)));
}

// Near field of several right-hand sides at once (solves in lockstep): the forward rows'
// P2P sum over U(b) for nr densities.  With the charges q_j = c_j w_j (c_j the density, less
// its island mean where the float operator splits it, w_j the node's complex weight), a
// pair's term Im(q_j conj(dz)) / |dz|^2 is c_j G with G = Im(w_j conj(dz)) / |dz|^2: the
// pair's geometry (dz, the reciprocal, G) is formed once and each right-hand side adds
// c_j G, one multiply-add, where the single-density kernel spends the whole pair on it.
// Lanes hold targets as in k_leaf (32 / TP lanes a target splitting the sources), each
// with NR sums; positions are leaf-local as there.  Two warps share a leaf, taking its
// chunks of 32 targets in turn (warp 2 t + c: chunks c, c + 2, ...), so a small system
// still has a warp per chunk of most leaves.  Writes near_r[i] = (1/r) sum, the
// near part of the forward row k_leaf adds when given nearv (r: the target leaf's
// half-width).  Right-hand side k's buffers (sigma, imean, near, its gate) sit k slab
// bytes after the first's; those beyond nr add zeros.
template <typename R> constexpr int kMultiChunk = std::is_same<R, double>::value ? 64 : 128;
template <typename R, int NR> constexpr size_t near_multi_smem(int lw)
{
    return (size_t)lw * kMultiChunk<R> * (2 * sizeof(cx<R>) + NR * sizeof(R));
}
template <typename R, int NR>
__global__ void __launch_bounds__(128)
k_near_multi(int64_t nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ level,
             const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
             const int32_t *__restrict__ bg, const int32_t *__restrict__ en,
             const int32_t *__restrict__ uptr, const int32_t *__restrict__ uidx, BoxGeo g,
             const double2 *__restrict__ xi, const cx<R> *__restrict__ uloc,
             const cx<df64> *__restrict__ udf, const double2 *__restrict__ w,
             const double *__restrict__ sigma, const int32_t *__restrict__ isl,
             const double *__restrict__ imean, int nr, int64_t slab, double *__restrict__ near,
             const int *gate)
{
    constexpr bool kF32 = kLocal<R>;
    constexpr int CH = kMultiChunk<R>;
    int open = gate ? 0 : nr;  // right-hand sides whose gate is open (no gate: all)
    for (int k = 0; gate && k < nr; k++)
        open += gate_closed((const int *)((const char *)gate + k * slab)) ? 0 : 1;
    if (open == 0) return;
    extern __shared__ __align__(16) unsigned char nm_sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t per = (size_t)CH * (2 * sizeof(cx<R>) + NR * sizeof(R));
    cx<R> *sz = (cx<R> *)(nm_sm + wid * per), *sw = sz + CH;
    R(*sc)[NR] = (R(*)[NR])(sw + CH);
    const int64_t wt = blockIdx.x * (int64_t)(blockDim.x >> 5) + wid;
    if (wt >= 2 * nleaf) return;
    const int b = leaves[wt >> 1];
    const int lt = level[b], tx = ix[b], ty = iy[b];
    double cxd = 0, cyd = 0, ir = 0;
    bool have_c = false;
    auto need_centre = [&]() {
        if (have_c) return;
        double r;
        box_centre(g, lt, tx, ty, cxd, cyd, r);
        ir = 1.0 / r;
        have_c = true;
    };
    R irr;
    if constexpr (kF32) {
        irr = inv_half_width<R>(g, lt);
    } else {
        need_centre();
        irr = (R)ir;
    }
    for (int tb = bg[b] + 32 * (int)(wt & 1); tb < en[b]; tb += 64) {
        const int nt = min(32, en[b] - tb);
        const int TP = nt <= 1 ? 1 : 1 << (32 - __clz(nt - 1));
        const int slot = lane & (TP - 1), grp = lane / TP, G = 32 / TP;
        cx<R> u = mk<R>(0, 0);
        if (slot < nt) {
            if constexpr (kF32) {
                u = uloc[tb + slot];
            } else {
                const double2 zi = xi[tb + slot];
                u = mk<R>((zi.x - cxd) * ir, (zi.y - cyd) * ir);
            }
        }
        R acc[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) acc[k] = R(0.0f);
        int fill = 0;
        auto process = [&]() {
            __syncwarp();
            if (slot < nt) {
#pragma unroll 2
                for (int m = grp; m < fill; m += G) {
                    const cx<R> zs = sz[m], ww = sw[m];
                    const R dr = zs.x - u.x, di = zs.y - u.y;
                    R ir2;
                    if constexpr (std::is_same<R, double>::value)
                        ir2 = rcp_near(fma(dr, dr, fma(di, di, tiny_sq<R>())));
                    else
                        ir2 = rcp(fm(dr, dr, di * di) + tiny_sq<R>());
                    const R gm = fm(ww.y, dr, -ww.x * di) * ir2;
#pragma unroll
                    for (int k = 0; k < NR; k++) acc[k] = fm(sc[m][k], gm, acc[k]);
                }
            }
            __syncwarp();
            fill = 0;
        };
        for (int uq = uptr[b]; uq < uptr[b + 1]; uq++) {
            const int s = uidx[uq];
            int sb = bg[s], se = en[s];
            bool local = false, dfp = false;
            R fs = R(0.0f);
            cx<R> os = mk<R>(R(0.0f), R(0.0f));
            if constexpr (kF32) {
                const int ls = level[s];
                local = ls >= lt && ls - lt <= 16;
                if constexpr (std::is_same<R, float>::value)
                    dfp = !local && udf && ls < lt && lt - ls <= kDfGap;
                if (local || dfp) {
                    fs = R(pow2<float>(lt - ls));
                    os = offset_cx<R>(centre_offset(ls, ix[s], iy[s], lt, tx, ty));
                }
            }
            while (sb < se) {
                const int take = min(se - sb, CH - fill);
                for (int m = lane; m < take; m += 32) {
                    const int j = sb + m;
                    cx<R> zr;
                    if (local) {
                        const cx<R> uu = uloc[j];
                        zr = mk<R>(uu.x * fs + os.x, uu.y * fs + os.y);
                    } else if (dfp) {
                        if constexpr (std::is_same<R, float>::value) {
                            const cx<df64> ud = udf[j];
                            zr = mk<R>(df_round(df_ldexp(ud.x, fs) + df64(os.x)),
                                       df_round(df_ldexp(ud.y, fs) + df64(os.y)));
                        }
                    } else {
                        need_centre();
                        const double2 zs = xi[j];
                        zr = mk<R>((R)((zs.x - cxd) * ir), (R)((zs.y - cyd) * ir));
                    }
                    sz[fill + m] = zr;
                    const double2 wj = w[j];
                    sw[fill + m] = mk<R>((R)wj.x, (R)wj.y);
                    const int kj = isl ? isl[j] : 0;
#pragma unroll
                    for (int k = 0; k < NR; k++) {
                        double c = 0.0;
                        if (k < nr) {
                            const int64_t o = (int64_t)k * slab;
                            c = *(const double *)((const char *)(sigma + j) + o);
                            if (isl) c -= *(const double *)((const char *)(imean + kj) + o);
                        }
                        sc[fill + m][k] = (R)c;
                    }
                }
                fill += take;
                sb += take;
                if (fill == CH) process();
            }
        }
        if (fill > 0) process();
        for (int o = TP; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < NR; k++) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        }
        if (grp == 0 && slot < nt) {
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (k < nr)
                    *(double *)((char *)(near + tb + slot) + (int64_t)k * slab) = (double)(acc[k] * irr);
        }
        __syncwarp();
    }
}

}  // namespace fmm
