// Autotuner of the FMM's free parameters for one geometry: the expansion order p, the
// leaf size (the quadtree splits a box holding more nodes) and the near-field tile (warps
// of the leaf pass per block).  The paper fixes none of them (Sec. 6 states only the
// FMM tolerance); here they are chosen by timed trials on the caller's geometry against
// an accuracy target for the density operator (I + 2K) sigma:
//   1. a reference application at high order (p = 44, leaf 48) on a seeded density;
//   2. for each leaf size, increasing p until the relative l2 error against the
//      reference is at most target / 4 (the first such p is the cheapest at that leaf
//      size: a higher order only adds work), then time it (median of 3 after a warm-up);
//   3. for the fastest (p, leaf), the near-field tile of 2, 4 and 8 warps, timed.
// A trial's time is what a solve spends on the operator: the double (or double-float)
// application, plus, for FP32_REFINE options, kFloatPerDouble times the float one (the
// refinement's inner solves apply the float operator about ten times per FP64 residual:
// 41 to 4 on the 16,384-island benchmark, 239,211 to 24,578 on the 512 batched
// geometries), so the leaf size and tile suit the operator the solve mostly runs.
// Every trial plan is built without the border (the border does not depend on these
// parameters) in the caller's workspace, one at a time.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbf_internal.cuh"

namespace {

// seeded density in [-1, 1): splitmix64 of (seed, index), top 53 bits
__global__ void k_tune_density(int64_t n, unsigned long long seed, double *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    out[i] = 2.0 * ((double)(z >> 11) * 0x1p-53) - 1.0;
}

// rel-l2 of a - b against b: partial sums per block, the last block adds them in order
__global__ void k_tune_err(int64_t n, const double *a, const double *b, double *part,
                           unsigned *count, double *out)
{
    __shared__ double s1[32], s2[32];
    __shared__ bool last;
    double d2 = 0.0, r2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = a[i] - b[i];
        d2 = fma(d, d, d2);
        r2 = fma(b[i], b[i], r2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = d2; s2[threadIdx.x >> 5] = r2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { t1 += s1[w]; t2 += s2[w]; }
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t1 = 0.0, t2 = 0.0;
        for (unsigned q = 0; q < gridDim.x; q++) {
            t1 += ((volatile double *)part)[2 * q];
            t2 += ((volatile double *)part)[2 * q + 1];
        }
        out[0] = t2 > 0.0 ? sqrt(t1 / t2) : 0.0;
        *count = 0u;
    }
}

constexpr int kErrBlocks = 304;
constexpr double kFloatPerDouble = 10.0;

struct Trial {
    int p, leaf, warps;
    double err, ms, ms64, ms32;
    int status;
};

}  // namespace

extern "C" int lbf_autotune(int M, const int64_t *island_ptr, const double *x, const double *dx,
                            const double *d2x, const double *centres, const double *pole_rotation,
                            const lbf_options *base, double target, void *workspace, size_t bytes,
                            size_t *bytes_needed, lbf_options *best, char *table, size_t table_len,
                            lbf_stream_t stream)
{
    if (!island_ptr || !base || !best || !(target > 0.0) || M < 1) return LBF_EINVAL;
    const int64_t N = island_ptr[M];
    const int leaves[] = {32, 48, 64};
    const int orders[] = {16, 18, 20, 22, 24, 26, 28, 30, 34, 38};
    const int p_ref = 44, leaf_ref = 48;
    // workspace: the largest trial plan, then 4 N doubles and the reduction scratch
    lbf_options o = *base;
    o.border = 0;
    o.matvec = LBF_MATVEC_FMM;
    o.box_capacity = 0;
    size_t plan_bytes = 0;
    for (int lf : {16, 32, 48, 64}) {
        o.leaf_size = lf;
        o.p = p_ref;
        size_t b = 0;
        int rc = lbf_workspace_size(M, island_ptr, &o, &b);
        if (rc) return rc;
        plan_bytes = std::max(plan_bytes, b);
    }
    plan_bytes = (plan_bytes + 255) & ~size_t(255);
    const size_t vec_bytes = sizeof(double) * (size_t)(4 * N + 2 * kErrBlocks + 8);
    const size_t need = plan_bytes + vec_bytes + 256;
    if (bytes_needed) *bytes_needed = need;
    if (!workspace || bytes < need) return workspace ? LBF_EWORKSPACE : LBF_OK;
    if (!x || !dx || !d2x || !centres) return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    char *wsp = (char *)workspace;
    double *sig = (double *)(wsp + plan_bytes), *ref = sig + N, *out = ref + N;
    double *part = out + 2 * N, *errv = part + 2 * kErrBlocks;
    unsigned *count = (unsigned *)(errv + 2);
    LBF_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
    LBF_LAUNCH(k_tune_density, lbf_cdiv(N, 256), 256, 0, s, N, 0x5eedull, sig);
    LBF_CHECK_LAUNCH();
    cudaEvent_t e0, e1;
    LBF_CUDA(cudaEventCreate(&e0));
    LBF_CUDA(cudaEventCreate(&e1));
    std::vector<Trial> trials;
    // one trial: plan, apply, error against the reference (when it exists), time
    auto run = [&](int p, int leaf, int warps, bool as_ref, bool time_it, Trial &t) -> int {
        t = Trial{p, leaf, warps, -1.0, -1.0, -1.0, -1.0, 0};
        lbf_options q = o;
        q.p = p;
        q.leaf_size = leaf;
        q.p2p_warps = warps;
        lbf_plan *pl = nullptr;
        int64_t need_box = 0;
        int rc = lbf_plan_create(&pl, M, island_ptr, x, dx, d2x, centres, pole_rotation, &q, wsp,
                                 plan_bytes, &need_box, stream);
        if (rc) {
            t.status = rc;
            return rc;
        }
        double *dst = as_ref ? ref : out;
        rc = lbf_apply(pl, LBF_OP_K_ONLY, sig, dst, stream);
        if (!rc && !as_ref) {
            LBF_LAUNCH(k_tune_err, kErrBlocks, 256, 0, s, N, out, ref, part, count, errv);
            double h = 0.0;
            if (cudaMemcpyAsync(&h, errv, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = LBF_ECUDA;
            t.err = h;
        }
        // median of 3 timed applications of op after a warm-up
        auto time_op = [&](int op, double &ms_out) {
            std::vector<float> ts;
            for (int r = 0; r < 4 && !rc; r++) {
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = LBF_ECUDA;
                if (!rc) rc = lbf_apply(pl, op, sig, out, stream);
                if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    rc = LBF_ECUDA;
                float ms = 0.f;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LBF_ECUDA;
                if (r > 0) ts.push_back(ms);  // the first is a warm-up
            }
            if (!rc) {
                std::sort(ts.begin(), ts.end());
                ms_out = ts[ts.size() / 2];
            }
        };
        if (!rc && time_it) {
            time_op(LBF_OP_K_ONLY, t.ms64);
            t.ms = t.ms64;
            if (!rc && o.precision == LBF_PRECISION_FP32_REFINE) {
                time_op(LBF_OP_K_ONLY | LBF_OP_FP32, t.ms32);
                if (!rc) t.ms = t.ms64 + kFloatPerDouble * t.ms32;
            }
        }
        int rs = lbf_sync_status(pl, stream);
        lbf_plan_destroy(pl);
        t.status = rc ? rc : rs;
        return t.status;
    };
    Trial tr;
    int rc = run(p_ref, leaf_ref, 0, true, false, tr);
    const double goal = 0.25 * target;
    int bp = -1, bl = -1, bw = 0;
    double bms = 1e300;
    if (!rc) {
        for (int leaf : leaves) {
            for (int p : orders) {
                if (p + 1 > LBF_MAX_TERMS) break;
                Trial t;
                run(p, leaf, 0, false, true, t);
                trials.push_back(t);
                if (t.status) break;
                if (t.err >= 0.0 && t.err <= goal) {
                    if (t.ms < bms) { bms = t.ms; bp = p; bl = leaf; }
                    break;
                }
            }
        }
        if (bp >= 0) {
            for (int w : {2, 8}) {
                Trial t;
                run(bp, bl, w, false, true, t);
                trials.push_back(t);
                if (!t.status && t.err <= goal && t.ms < bms) { bms = t.ms; bw = w; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = *base;
    if (bp >= 0) {
        best->p = bp;
        best->leaf_size = bl;
        best->p2p_warps = bw;
    }
    if (table && table_len) {
        std::string js = "{\"target\": " + std::to_string(target) + ", \"reference\": {\"p\": " +
                         std::to_string(p_ref) + ", \"leaf\": " + std::to_string(leaf_ref) +
                         "}, \"trials\": [";
        char buf[256];
        for (size_t i = 0; i < trials.size(); i++) {
            const Trial &t = trials[i];
            snprintf(buf, sizeof(buf),
                     "%s{\"p\": %d, \"leaf\": %d, \"warps\": %d, \"err\": %.3e, \"ms\": %.4f, "
                     "\"ms64\": %.4f, \"ms32\": %.4f, \"status\": %d}",
                     i ? ", " : "", t.p, t.leaf, t.warps ? t.warps : 4, t.err, t.ms, t.ms64, t.ms32,
                     t.status);
            js += buf;
        }
        snprintf(buf, sizeof(buf), "], \"best\": {\"p\": %d, \"leaf\": %d, \"warps\": %d, \"ms\": %.4f}}",
                 bp, bl, bw ? bw : 4, bp >= 0 ? bms : -1.0);
        js += buf;
        const size_t n = std::min(js.size(), table_len - 1);
        memcpy(table, js.data(), n);
        table[n] = 0;
    }
    if (rc) return rc;
    return bp >= 0 ? LBF_OK : LBF_NOCONV;
}
