// Adaptive quadtree on the projected nodes (Sec. 6 Example 3: boxes are split
// until no more than a preset number of nodes remain; the stereographic
// distortion makes the tree deep, 16-22 levels in the paper) and the adaptive
// FMM interaction lists U, V, W, X (Carrier, Greengard & Rokhlin).
//
// Integer specification (bit-exact, checked against the oracle's independent
// reference tree):
//   L    = max(xmax - xmin, ymax - ymin) * (1 + 2^-20), or 1 if that is 0
//   cell = min(2^D - 1, floor((v - vmin) / L * 2^D)) in IEEE double
//   key  = bit interleave of the cells, y bit above x bit at every level
//   nodes sorted stably by key (ties keep the caller's order)
//   a box at level l splits while it holds more than leaf_size nodes and l < D;
//   empty children are dropped; boxes are numbered level by level, in Morton
//   order within a level.
#include <vector>

#include "lbf_internal.cuh"

namespace {

constexpr int kUnit = 1024;  // radix-sort items per warp

__device__ __forceinline__ uint64_t spread_bits(uint64_t v)
{
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// ---- bounding square ---------------------------------------------------------
__global__ void k_bbox_partial(int64_t N, const double2 *__restrict__ xi, double *__restrict__ part)
{
    __shared__ double s[4][256];
    double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        double2 z = xi[j];
        mnx = fmin(mnx, z.x); mxx = fmax(mxx, z.x);
        mny = fmin(mny, z.y); mxy = fmax(mxy, z.y);
    }
    int t = threadIdx.x;
    s[0][t] = mnx; s[1][t] = mxx; s[2][t] = mny; s[3][t] = mxy;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) {
            s[0][t] = fmin(s[0][t], s[0][t + o]);
            s[1][t] = fmax(s[1][t], s[1][t + o]);
            s[2][t] = fmin(s[2][t], s[2][t + o]);
            s[3][t] = fmax(s[3][t], s[3][t + o]);
        }
        __syncthreads();
    }
    if (t < 4) part[4 * blockIdx.x + t] = s[t][0];
}

// one warp: lanes strided over the block partials, then shuffles (min and max are
// exact, so the result does not depend on the order)
__global__ void k_bbox_final(int nb, const double *__restrict__ part, double *__restrict__ bbox)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int b = lane; b < nb; b += 32) {
        mnx = fmin(mnx, part[4 * b]); mxx = fmax(mxx, part[4 * b + 1]);
        mny = fmin(mny, part[4 * b + 2]); mxy = fmax(mxy, part[4 * b + 3]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fmin(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mxx = fmax(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mny = fmin(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxy = fmax(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if (lane != 0) return;
    double ex = __dsub_rn(mxx, mnx), ey = __dsub_rn(mxy, mny);
    double L = __dmul_rn(ex > ey ? ex : ey, 1.0 + 0x1p-20);
    if (!(L > 0.0)) L = 1.0;
    bbox[0] = mnx;
    bbox[1] = mny;
    bbox[2] = L;
}

__global__ void k_keys(int64_t N, const double2 *__restrict__ xi, const double *__restrict__ bbox,
                       int D, uint64_t *__restrict__ keys, int32_t *__restrict__ perm)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    double xmin = bbox[0], ymin = bbox[1], L = bbox[2];
    double scale = ldexp(1.0, D);
    double2 z = xi[j];
    double fx = floor(__dmul_rn(__ddiv_rn(__dsub_rn(z.x, xmin), L), scale));
    double fy = floor(__dmul_rn(__ddiv_rn(__dsub_rn(z.y, ymin), L), scale));
    uint64_t cmax = (1ull << D) - 1ull;
    uint64_t cx = (uint64_t)fx, cy = (uint64_t)fy;
    if (cx > cmax) cx = cmax;
    if (cy > cmax) cy = cmax;
    keys[j] = spread_bits(cx) | (spread_bits(cy) << 1);
    perm[j] = (int32_t)j;
}

// ---- exclusive scan (int32) ------------------------------------------------------
__global__ void k_scan_block(const int32_t *__restrict__ in, int32_t *out, int64_t n,
                             int32_t *__restrict__ sums)
{
    __shared__ int32_t wsum[32];
    int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int64_t i0 = blockIdx.x * 2048ll + 2 * t, i1 = i0 + 1;
    int32_t a = i0 < n ? in[i0] : 0, b = i1 < n ? in[i1] : 0;
    int32_t sv = a + b, x = sv;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int32_t excl = x - sv + (wid > 0 ? wsum[wid - 1] : 0);
    if (i0 < n) out[i0] = excl;
    if (i1 < n) out[i1] = excl + a;
    if (t == 1023 && sums) sums[blockIdx.x] = excl + sv;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *__restrict__ sums)
{
    int64_t i = blockIdx.x * 2048ll + threadIdx.x;
    int32_t add = sums[blockIdx.x];
    if (i < n) out[i] += add;
    if (i + 1024 < n) out[i + 1024] += add;
}

// ---- stable LSD radix sort, 8-bit digits -------------------------------------------
// Each warp owns a unit of kUnit consecutive items; per-unit digit counts are
// scanned digit-major so that scattering unit by unit, in item order, is stable.
__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                          int32_t *__restrict__ hist, int64_t nunits)
{
    __shared__ int32_t cnt[8][256];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) cnt[wid][d] = 0;
    __syncwarp();
    int64_t u = blockIdx.x * 8ll + wid;
    if (u >= nunits) return;
    int64_t b = u * kUnit, e = b + kUnit < n ? b + kUnit : n;
    for (int64_t i = b + lane; i < e; i += 32) atomicAdd(&cnt[wid][(keys[i] >> shift) & 255u], 1);
    __syncwarp();
    for (int d = lane; d < 256; d += 32) hist[(int64_t)d * nunits + u] = cnt[wid][d];
}

__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n,
                             int shift, const int32_t *__restrict__ off, int64_t nunits)
{
    __shared__ int32_t cnt[8][256];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) cnt[wid][d] = 0;
    __syncwarp();
    int64_t u = blockIdx.x * 8ll + wid;
    if (u >= nunits) return;
    int64_t b = u * kUnit, e = b + kUnit < n ? b + kUnit : n;
    unsigned lt = (1u << lane) - 1u;
    for (int64_t base = b; base < e; base += 32) {
        int64_t i = base + lane;
        bool act = i < e;
        unsigned mask = __ballot_sync(0xffffffffu, act);
        if (act) {
            uint64_t k = kin[i];
            int d = (int)((k >> shift) & 255u);
            unsigned peers = __match_any_sync(mask, d);
            int r = __popc(peers & lt);
            int pos = off[(int64_t)d * nunits + u] + cnt[wid][d] + r;
            kout[pos] = k;
            vout[pos] = vin[i];
            __syncwarp(mask);
            if (lane == __ffs(peers) - 1) cnt[wid][d] += __popc(peers);
        }
        __syncwarp();
    }
}

// ---- level-by-level split ------------------------------------------------------------
__device__ __forceinline__ int digit_at(uint64_t k, int shift) { return (int)((k >> shift) & 3ull); }

// first index in [b, e) whose digit is >= d (digits are non-decreasing there)
__device__ __forceinline__ int32_t first_digit_ge(const uint64_t *keys, int32_t b, int32_t e,
                                                  int shift, int d)
{
    while (b < e) {
        int32_t m = b + ((e - b) >> 1);
        if (digit_at(keys[m], shift) < d) b = m + 1; else e = m;
    }
    return b;
}

__global__ void k_split_count(int64_t ls, int64_t le, int l, int D, int leaf,
                              const uint64_t *__restrict__ keys, const int32_t *__restrict__ bg,
                              const int32_t *__restrict__ en, int32_t *__restrict__ nchild)
{
    int64_t b = ls + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= le) return;
    int32_t s = bg[b], e = en[b];
    int nc = 0;
    if (e - s > leaf && l < D) {
        int shift = 2 * (D - l - 1);
        int32_t cut[5];
        cut[0] = s; cut[4] = e;
        for (int d = 1; d < 4; d++) cut[d] = first_digit_ge(keys, s, e, shift, d);
        for (int d = 0; d < 4; d++) nc += cut[d + 1] > cut[d];
    }
    nchild[b] = nc;
}

__global__ void k_split_write(int64_t ls, int64_t le, int l, int D, const uint64_t *__restrict__ keys,
                              int32_t *__restrict__ level, int32_t *__restrict__ ix,
                              int32_t *__restrict__ iy, int32_t *__restrict__ parent,
                              int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                              int32_t *__restrict__ bg, int32_t *__restrict__ en,
                              const int32_t *__restrict__ off)
{
    int64_t b = ls + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= le) return;
    if (nchild[b] == 0) {
        child0[b] = -1;
        return;
    }
    int32_t s = bg[b], e = en[b];
    int shift = 2 * (D - l - 1);
    int32_t cut[5];
    cut[0] = s; cut[4] = e;
    for (int d = 1; d < 4; d++) cut[d] = first_digit_ge(keys, s, e, shift, d);
    int32_t c = (int32_t)(le + off[b - ls]);
    child0[b] = c;
    for (int d = 0; d < 4; d++) {
        if (cut[d + 1] > cut[d]) {
            level[c] = l + 1;
            ix[c] = 2 * ix[b] + (d & 1);
            iy[c] = 2 * iy[b] + (d >> 1);
            parent[c] = (int32_t)b;
            bg[c] = cut[d];
            en[c] = cut[d + 1];
            c++;
        }
    }
}

__global__ void k_leaf_flags(int64_t nb, const int32_t *__restrict__ nchild, int32_t *__restrict__ f)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nb) f[b] = nchild[b] == 0;
}

__global__ void k_leaf_compact(int64_t nb, const int32_t *__restrict__ nchild,
                               const int32_t *__restrict__ pos, int32_t *__restrict__ leaves)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nb && nchild[b] == 0) leaves[pos[b]] = (int32_t)b;
}

// ---- interaction lists --------------------------------------------------------------
struct TreeView {
    const int32_t *level, *ix, *iy, *parent, *child0, *nchild;
};

// closed boxes a and b touch (or overlap): integer test at the finer level
__device__ __forceinline__ bool touches(const TreeView &T, int32_t a, int32_t b)
{
    int la = T.level[a], lb = T.level[b];
    int64_t xa = T.ix[a], ya = T.iy[a], xb = T.ix[b], yb = T.iy[b];
    if (la > lb) {
        int t = la; la = lb; lb = t;
        int64_t u = xa; xa = xb; xb = u;
        u = ya; ya = yb; yb = u;
    }
    int s = lb - la;
    return xb <= ((xa + 1) << s) && xb + 1 >= (xa << s) && yb <= ((ya + 1) << s) &&
           yb + 1 >= (ya << s);
}

__global__ void k_root_lists(int32_t *coll, int32_t *nv, int32_t *ncoarse, int32_t *nx)
{
    if (threadIdx.x < 9) coll[threadIdx.x] = threadIdx.x == 0 ? 0 : -1;
    if (threadIdx.x == 0) { nv[0] = 0; ncoarse[0] = 0; nx[0] = 0; }
}

// colleagues (same level, touching, self included), V, coarse neighbours and X
// of every box at one level, from its parent's lists.
__global__ void k_lists_level(int64_t ls, int64_t le, TreeView T, int32_t *__restrict__ coll,
                              int32_t *__restrict__ vlist, int32_t *__restrict__ nv,
                              int32_t *__restrict__ coarse, int32_t *__restrict__ ncoarse,
                              int32_t *__restrict__ xlist, int32_t *__restrict__ nx,
                              int *__restrict__ status)
{
    int64_t bb = ls + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (bb >= le) return;
    int32_t b = (int32_t)bb;
    int32_t P = T.parent[b];
    int nc = 0, nvv = 0;
    int bx = T.ix[b], by = T.iy[b];
    for (int q = 0; q < 9; q++) {
        int32_t C = coll[P * 9 + q];
        if (C < 0) continue;
        int k = T.nchild[C];
        for (int c = T.child0[C]; k > 0 && c < T.child0[C] + k; c++) {
            if (abs(T.ix[c] - bx) <= 1 && abs(T.iy[c] - by) <= 1) {
                if (nc < 9) coll[b * 9 + nc] = c;
                nc++;
            } else {
                if (nvv < 27) vlist[b * 27 + nvv] = c;
                nvv++;
            }
        }
    }
    for (int q = nc; q < 9; q++) coll[b * 9 + q] = -1;
    int nco = 0, nxx = 0;
    // shallower leaves touching the parent: its leaf colleagues and its own coarse neighbours
    for (int q = 0; q < 9 + 8; q++) {
        int32_t c;
        if (q < 9) {
            c = coll[P * 9 + q];
            if (c < 0 || c == P || T.nchild[c] != 0) continue;
        } else {
            if (q - 9 >= ncoarse[P]) break;
            c = coarse[P * 8 + (q - 9)];
        }
        if (touches(T, c, b)) {
            if (nco < 8) coarse[b * 8 + nco] = c;
            nco++;
        } else {
            if (nxx < 16) xlist[b * 16 + nxx] = c;
            nxx++;
        }
    }
    if (nc > 9 || nvv > 27 || nco > 8 || nxx > 16) atomicOr(status, 8);
    nv[b] = nvv < 27 ? nvv : 27;
    ncoarse[b] = nco < 8 ? nco : 8;
    nx[b] = nxx < 16 ? nxx : 16;
}

// U and W of every leaf (count pass: fill == 0; fill pass writes at the CSR offsets).
// U: the leaf, its leaf colleagues, shallower touching leaves, and deeper touching
// leaves found by descending into non-leaf colleagues; W: boxes met in that descent
// that do not touch the leaf (their parent does).
__global__ void k_lists_uw(int64_t nleaf, const int32_t *__restrict__ leaves, TreeView T,
                           const int32_t *__restrict__ coll, const int32_t *__restrict__ coarse,
                           const int32_t *__restrict__ ncoarse, int fill,
                           int32_t *__restrict__ ucnt, int32_t *__restrict__ wcnt,
                           const int32_t *__restrict__ uptr, const int32_t *__restrict__ wptr,
                           int32_t *__restrict__ uidx, int32_t *__restrict__ widx,
                           int *__restrict__ status)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int32_t b = leaves[t];
    int nu = 0, nw = 0;
    int32_t u0 = fill ? uptr[b] : 0, w0 = fill ? wptr[b] : 0;
#define EMIT_U(v) do { if (fill) uidx[u0 + nu] = (v); nu++; } while (0)
#define EMIT_W(v) do { if (fill) widx[w0 + nw] = (v); nw++; } while (0)
    EMIT_U(b);
    int32_t stack[128];
    for (int q = 0; q < 9; q++) {
        int32_t C = coll[b * 9 + q];
        if (C < 0 || C == b) continue;
        if (T.nchild[C] == 0) {
            EMIT_U(C);
            continue;
        }
        int sp = 0;
        for (int c = T.child0[C] + T.nchild[C] - 1; c >= T.child0[C]; c--) stack[sp++] = c;
        while (sp > 0) {
            int32_t d = stack[--sp];
            if (touches(T, d, b)) {
                if (T.nchild[d] == 0) {
                    EMIT_U(d);
                } else {
                    if (sp + 4 > 128) { atomicOr(status, 8); break; }
                    for (int c = T.child0[d] + T.nchild[d] - 1; c >= T.child0[d]; c--) stack[sp++] = c;
                }
            } else {
                EMIT_W(d);
            }
        }
    }
    for (int q = 0; q < ncoarse[b]; q++) EMIT_U(coarse[b * 8 + q]);
#undef EMIT_U
#undef EMIT_W
    if (!fill) {
        ucnt[b] = nu;
        wcnt[b] = nw;
    }
}

__global__ void k_export_boxes(int64_t nb, TreeView T, const int32_t *__restrict__ bg,
                               const int32_t *__restrict__ en, int32_t *__restrict__ out)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t *o = out + 8 * b;
    o[0] = T.level[b]; o[1] = T.ix[b]; o[2] = T.iy[b]; o[3] = T.parent[b];
    o[4] = T.nchild[b] > 0 ? T.child0[b] : -1; o[5] = T.nchild[b]; o[6] = bg[b]; o[7] = en[b];
}

// fixed-capacity list (stride cap per box, count array) -> CSR counts
__global__ void k_fixed_counts(int64_t nb, const int32_t *__restrict__ cnt, int32_t *__restrict__ out)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nb) out[b] = cnt[b];
}

__global__ void k_fixed_fill(int64_t nb, int stride, const int32_t *__restrict__ lst,
                             const int32_t *__restrict__ cnt, const int32_t *__restrict__ ptr,
                             int32_t *__restrict__ idx)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int k = 0; k < cnt[b]; k++) idx[ptr[b] + k] = lst[b * stride + k];
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

int lbf_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *scratch, int64_t scratch_len,
                 cudaStream_t s)
{
    if (n <= 0) return LBF_OK;
    int64_t nb = lbf_cdiv(n, 2048);
    if (nb == 1) {
        LBF_LAUNCH(k_scan_block, 1, 1024, 0, s, in, out, n, (int32_t *)nullptr);
        LBF_CHECK_LAUNCH();
        return LBF_OK;
    }
    if (scratch_len < nb) return LBF_EWORKSPACE;
    int32_t *sums = scratch;
    LBF_LAUNCH(k_scan_block, nb, 1024, 0, s, in, out, n, sums);
    LBF_CHECK_LAUNCH();
    int rc = lbf_scan_i32(sums, sums, nb, scratch + nb, scratch_len - nb, s);
    if (rc) return rc;
    LBF_LAUNCH(k_scan_add, nb, 1024, 0, s, out, n, sums);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

static int read_i32(const int32_t *d, int32_t *h, cudaStream_t s)
{
    LBF_CUDA(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

int lbf_radix_sort(uint64_t *keys, uint64_t *keys_alt, int32_t *vals, int32_t *vals_alt, int64_t n,
                   int bits, int32_t *scratch, int64_t scratch_len, cudaStream_t s)
{
    if (n <= 0) return LBF_OK;
    int64_t nunits = lbf_cdiv(n, kUnit);
    int32_t *hist = scratch;
    int32_t *sc = scratch + 256 * nunits;
    int64_t sc_len = scratch_len - 256 * nunits;
    if (sc_len < 0) return LBF_EWORKSPACE;
    int passes = (int)lbf_cdiv(bits, 8);
    uint64_t *ka = keys, *kb = keys_alt;
    int32_t *va = vals, *vb = vals_alt;
    for (int ps = 0; ps < passes; ps++) {
        int shift = 8 * ps;
        LBF_LAUNCH(k_rs_hist, lbf_cdiv(nunits, 8), 256, 0, s, ka, n, shift, hist, nunits);
        LBF_CHECK_LAUNCH();
        int rc = lbf_scan_i32(hist, hist, 256 * nunits, sc, sc_len, s);
        if (rc) return rc;
        LBF_LAUNCH(k_rs_scatter, lbf_cdiv(nunits, 8), 256, 0, s, ka, va, kb, vb, n, shift, hist,
                   nunits);
        LBF_CHECK_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        LBF_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        LBF_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return LBF_OK;
}

int lbf_tree_build(lbf_plan *pl, cudaStream_t s, const double2 *xi_o, uint64_t *keys,
                   uint64_t *keys_alt, int32_t *perm_alt, int32_t *scratch, int64_t scratch_len,
                   int64_t *box_needed)
{
    Tree &T = pl->tree;
    int64_t N = pl->N;
    int D = pl->opt.max_depth;
    int leaf = pl->opt.leaf_size;
    // bounding square
    int nbb = (int)std::min<int64_t>(lbf_cdiv(N, 256), 1024);
    double *part = (double *)scratch;  // 4 * nbb doubles
    double *bbox = part + 4 * nbb;
    LBF_LAUNCH(k_bbox_partial, nbb, 256, 0, s, N, xi_o, part);
    LBF_LAUNCH(k_bbox_final, 1, 32, 0, s, nbb, part, bbox);
    LBF_CHECK_LAUNCH();
    double hb[3];
    LBF_CUDA(cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, s));
    LBF_LAUNCH(k_keys, lbf_cdiv(N, 256), 256, 0, s, N, xi_o, bbox, D, keys, pl->perm);
    LBF_CHECK_LAUNCH();
    LBF_CUDA(cudaStreamSynchronize(s));
    T.xmin = hb[0];
    T.ymin = hb[1];
    T.L = hb[2];

    // radix sort (keys, perm)
    int rc = lbf_radix_sort(keys, keys_alt, pl->perm, perm_alt, N, 2 * D, scratch, scratch_len, s);
    if (rc) return rc;

    // root box
    int32_t root[8] = {0, 0, 0, -1, -1, 0, 0, (int32_t)N};
    LBF_CUDA(cudaMemcpyAsync(T.level, &root[0], 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.ix, &root[1], 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.iy, &root[2], 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.parent, &root[3], 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.begin, &root[6], 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.end, &root[7], 4, cudaMemcpyHostToDevice, s));
    int64_t ls = 0, le = 1;
    T.lev_start[0] = 0;
    int l = 0;
    int32_t *off = scratch;
    int32_t *sc2 = scratch + T.cap;
    int64_t sc2_len = scratch_len - T.cap;
    for (;; l++) {
        int64_t nlev = le - ls;
        LBF_LAUNCH(k_split_count, lbf_cdiv(nlev, 256), 256, 0, s, ls, le, l, D, leaf, keys,
                   T.begin, T.end, T.nchild);
        LBF_CHECK_LAUNCH();
        int rc = lbf_scan_i32(T.nchild + ls, off, nlev, sc2, sc2_len, s);
        if (rc) return rc;
        int32_t last_off = 0, last_n = 0;
        if ((rc = read_i32(off + nlev - 1, &last_off, s))) return rc;
        if ((rc = read_i32(T.nchild + le - 1, &last_n, s))) return rc;
        int64_t nnew = (int64_t)last_off + last_n;
        if (le + nnew > T.cap) {
            if (box_needed) *box_needed = 2 * (le + nnew) + 1024;
            return LBF_EWORKSPACE;
        }
        LBF_LAUNCH(k_split_write, lbf_cdiv(nlev, 256), 256, 0, s, ls, le, l, D, keys, T.level,
                   T.ix, T.iy, T.parent, T.child0, T.nchild, T.begin, T.end, off);
        LBF_CHECK_LAUNCH();
        T.lev_start[l + 1] = le;
        if (nnew == 0) break;
        if (l + 1 > LBF_MAX_LEVELS - 1) return LBF_EDEPTH;
        ls = le;
        le = le + nnew;
    }
    T.nlev = l + 1;
    T.nbox = le;
    // last level: its boxes are leaves; child0/nchild were written by the final count/write
    // leaves
    int32_t *flags = scratch;
    int32_t *pos = scratch + T.nbox;
    LBF_LAUNCH(k_leaf_flags, lbf_cdiv(T.nbox, 256), 256, 0, s, T.nbox, T.nchild, flags);
    LBF_CHECK_LAUNCH();
    rc = lbf_scan_i32(flags, pos, T.nbox, scratch + 2 * T.nbox, scratch_len - 2 * T.nbox, s);
    if (rc) return rc;
    int32_t lp = 0, lf = 0;
    if ((rc = read_i32(pos + T.nbox - 1, &lp, s))) return rc;
    if ((rc = read_i32(flags + T.nbox - 1, &lf, s))) return rc;
    T.nleaf = (int64_t)lp + lf;
    LBF_LAUNCH(k_leaf_compact, lbf_cdiv(T.nbox, 256), 256, 0, s, T.nbox, T.nchild, pos, T.leaves);
    LBF_CHECK_LAUNCH();
    return LBF_OK;
}

int lbf_lists_build(lbf_plan *pl, cudaStream_t s, int32_t *scratch, int64_t scratch_len,
                    int64_t *box_needed)
{
    Tree &T = pl->tree;
    TreeView V{T.level, T.ix, T.iy, T.parent, T.child0, T.nchild};
    LBF_LAUNCH(k_root_lists, 1, 32, 0, s, T.coll, T.nv, T.ncoarse, T.nx);
    LBF_CHECK_LAUNCH();
    for (int l = 1; l < T.nlev; l++) {
        int64_t ls = T.lev_start[l], le = T.lev_start[l + 1];
        if (le <= ls) continue;
        LBF_LAUNCH(k_lists_level, lbf_cdiv(le - ls, 128), 128, 0, s, ls, le, V, T.coll, T.vlist,
                   T.nv, T.coarse, T.ncoarse, T.xlist, T.nx, pl->dev_status);
        LBF_CHECK_LAUNCH();
    }
    int64_t nb = T.nbox;
    int32_t *ucnt = scratch, *wcnt = scratch + nb;
    LBF_LAUNCH(k_fill_i32, lbf_cdiv(2 * nb, 256), 256, 0, s, scratch, 2 * nb, 0);
    LBF_LAUNCH(k_lists_uw, lbf_cdiv(T.nleaf, 128), 128, 0, s, T.nleaf, T.leaves, V, T.coll,
               T.coarse, T.ncoarse, 0, ucnt, wcnt, (const int32_t *)nullptr,
               (const int32_t *)nullptr, (int32_t *)nullptr, (int32_t *)nullptr, pl->dev_status);
    LBF_CHECK_LAUNCH();
    int rc = lbf_scan_i32(ucnt, T.u_ptr, nb, scratch + 2 * nb, scratch_len - 2 * nb, s);
    if (rc) return rc;
    rc = lbf_scan_i32(wcnt, T.w_ptr, nb, scratch + 2 * nb, scratch_len - 2 * nb, s);
    if (rc) return rc;
    int32_t a = 0, b = 0, c = 0, d = 0;
    if ((rc = read_i32(T.u_ptr + nb - 1, &a, s))) return rc;
    if ((rc = read_i32(ucnt + nb - 1, &b, s))) return rc;
    if ((rc = read_i32(T.w_ptr + nb - 1, &c, s))) return rc;
    if ((rc = read_i32(wcnt + nb - 1, &d, s))) return rc;
    T.u_len = (int64_t)a + b;
    T.w_len = (int64_t)c + d;
    // CSR terminators
    int32_t ul = (int32_t)T.u_len, wl = (int32_t)T.w_len;
    LBF_CUDA(cudaMemcpyAsync(T.u_ptr + nb, &ul, 4, cudaMemcpyHostToDevice, s));
    LBF_CUDA(cudaMemcpyAsync(T.w_ptr + nb, &wl, 4, cudaMemcpyHostToDevice, s));
    if (T.u_len > T.u_cap || T.w_len > T.w_cap) {
        if (box_needed) {
            double f = std::max((double)T.u_len / (double)T.u_cap, (double)T.w_len / (double)T.w_cap);
            *box_needed = (int64_t)(T.cap * f * 1.25) + 1024;
        }
        return LBF_EWORKSPACE;
    }
    LBF_LAUNCH(k_lists_uw, lbf_cdiv(T.nleaf, 128), 128, 0, s, T.nleaf, T.leaves, V, T.coll,
               T.coarse, T.ncoarse, 1, ucnt, wcnt, T.u_ptr, T.w_ptr, T.u_idx, T.w_idx,
               pl->dev_status);
    LBF_CHECK_LAUNCH();
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

extern "C" int lbf_tree_export(const lbf_plan *pl, int32_t *perm, int32_t *boxes, lbf_stream_t stream)
{
    if (!pl) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Tree &T = pl->tree;
    if (perm) LBF_CUDA(cudaMemcpyAsync(perm, pl->perm, sizeof(int32_t) * pl->N, cudaMemcpyDeviceToDevice, s));
    if (boxes && T.nbox > 0) {
        TreeView V{T.level, T.ix, T.iy, T.parent, T.child0, T.nchild};
        LBF_LAUNCH(k_export_boxes, lbf_cdiv(T.nbox, 256), 256, 0, s, T.nbox, V, T.begin, T.end, boxes);
        LBF_CHECK_LAUNCH();
    }
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}

extern "C" int lbf_list_export(const lbf_plan *pl, int kind, int32_t *ptr, int32_t *idx, int64_t *len,
                               lbf_stream_t stream)
{
    if (!pl || kind < 0 || kind > 3 || !len) return LBF_EINVAL;
    if (pl->opt.matvec != LBF_MATVEC_FMM) return LBF_ENOTBUILT;
    cudaStream_t s = (cudaStream_t)stream;
    const Tree &T = pl->tree;
    int64_t nb = T.nbox;
    if (kind == 0 || kind == 2) {
        const int32_t *p = kind == 0 ? T.u_ptr : T.w_ptr;
        const int32_t *ix = kind == 0 ? T.u_idx : T.w_idx;
        *len = kind == 0 ? T.u_len : T.w_len;
        if (ptr) LBF_CUDA(cudaMemcpyAsync(ptr, p, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToDevice, s));
        if (idx && *len > 0)
            LBF_CUDA(cudaMemcpyAsync(idx, ix, sizeof(int32_t) * (*len), cudaMemcpyDeviceToDevice, s));
        LBF_CUDA(cudaStreamSynchronize(s));
        return LBF_OK;
    }
    // V and X are stored with a fixed capacity per box: build CSR offsets on the fly
    const int32_t *cnt = kind == 1 ? T.nv : T.nx;
    const int32_t *lst = kind == 1 ? T.vlist : T.xlist;
    int stride = kind == 1 ? 27 : 16;
    if (!ptr) return LBF_EINVAL;
    LBF_LAUNCH(k_fixed_counts, lbf_cdiv(nb, 256), 256, 0, s, nb, cnt, ptr);
    LBF_CHECK_LAUNCH();
    // exclusive scan of the counts on the host (inspection path, not the hot path)
    std::vector<int32_t> h(nb + 1);
    LBF_CUDA(cudaMemcpyAsync(h.data(), ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; b++) { int32_t c = h[b]; h[b] = (int32_t)acc; acc += c; }
    h[nb] = (int32_t)acc;
    *len = acc;
    LBF_CUDA(cudaMemcpyAsync(ptr, h.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    if (idx && acc > 0) {
        LBF_LAUNCH(k_fixed_fill, lbf_cdiv(nb, 256), 256, 0, s, nb, stride, lst, cnt, ptr, idx);
        LBF_CHECK_LAUNCH();
    }
    LBF_CUDA(cudaStreamSynchronize(s));
    return LBF_OK;
}
