// Tracing (CUDA events around selected kernels) and FMM work counts.
#include <mutex>
#include <vector>

#include "lbf_internal.cuh"

namespace {

struct Rec {
    int id;
    int begin;
    cudaEvent_t ev;
};

struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<Rec> recs;
} g_prof;

constexpr size_t kPool = 1 << 16;

__global__ void k_counts(int64_t nbox, const int32_t *__restrict__ level,
                         const int32_t *__restrict__ nchild, const int32_t *__restrict__ bg,
                         const int32_t *__restrict__ en, const int32_t *__restrict__ uptr,
                         const int32_t *__restrict__ uidx, const int32_t *__restrict__ wptr,
                         const int32_t *__restrict__ nv, const int32_t *__restrict__ xlist,
                         const int32_t *__restrict__ nx, unsigned long long *__restrict__ c)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    unsigned long long nb = (unsigned long long)(en[b] - bg[b]);
    if (nchild[b] == 0) {
        unsigned long long su = 0;
        for (int q = uptr[b]; q < uptr[b + 1]; q++) su += (unsigned long long)(en[uidx[q]] - bg[uidx[q]]);
        atomicAdd(&c[1], nb * su);
        atomicAdd(&c[5], nb * (unsigned long long)(wptr[b + 1] - wptr[b]));
        atomicAdd(&c[7], 1ull);
    }
    if (level[b] >= 1) atomicAdd(&c[2], 1ull);  // every non-root box shifts into its parent
    if (level[b] >= 3) atomicAdd(&c[4], 1ull);  // locals are non-zero from level 2 down
    atomicAdd(&c[3], (unsigned long long)nv[b]);
    unsigned long long sx = 0;
    for (int q = 0; q < nx[b]; q++) {
        int s = xlist[b * 16 + q];
        sx += (unsigned long long)(en[s] - bg[s]);
    }
    atomicAdd(&c[6], sx);
}

}  // namespace

namespace {
thread_local bool t_capturing = false;
}

void lbf_prof_capture(bool on) { t_capturing = on; }

void lbf_prof_mark(int id, int begin, cudaStream_t s)
{
    if (!g_prof.on || t_capturing) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on || g_prof.next >= g_prof.pool.size()) return;
    cudaEvent_t ev = g_prof.pool[g_prof.next++];
    if (cudaEventRecord(ev, s) != cudaSuccess) return;
    g_prof.recs.push_back({id, begin, ev});
}

extern "C" {

int lbf_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (on && g_prof.pool.empty()) {
        g_prof.pool.resize(kPool);
        for (auto &e : g_prof.pool)
            if (cudaEventCreate(&e) != cudaSuccess) return LBF_ECUDA;
    }
    g_prof.on = on != 0;
    return LBF_OK;
}

int lbf_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto &r : g_prof.recs) cudaEventSynchronize(r.ev);
    g_prof.recs.clear();
    g_prof.next = 0;
    return LBF_OK;
}

int lbf_profile_read(int kernel, int64_t *launches, double *total_ms)
{
    if (kernel < 0 || kernel >= LBF_KERNEL_COUNT || !launches || !total_ms) return LBF_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    int64_t n = 0;
    double t = 0.0;
    const Rec *open = nullptr;
    for (const auto &r : g_prof.recs) {
        if (r.id != kernel) continue;
        if (r.begin) {
            open = &r;
        } else if (open) {
            if (cudaEventSynchronize(r.ev) != cudaSuccess) return LBF_ECUDA;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, open->ev, r.ev) != cudaSuccess) return LBF_ECUDA;
            t += ms;
            n++;
            open = nullptr;
        }
    }
    *launches = n;
    *total_ms = t;
    return LBF_OK;
}

int lbf_plan_counts(const lbf_plan *pl, int64_t counts[8], lbf_stream_t stream)
{
    if (!pl || !counts) return LBF_EINVAL;
    for (int k = 0; k < 8; k++) counts[k] = 0;
    counts[0] = pl->N;
    if (pl->opt.matvec != LBF_MATVEC_FMM) {
        counts[1] = pl->N * (pl->N - 1);
        return LBF_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Tree &T = pl->tree;
    unsigned long long *c = (unsigned long long *)pl->red;  // 8 counters in the reduction scratch
    LBF_CUDA(cudaMemsetAsync(c, 0, 8 * sizeof(unsigned long long), s));
    LBF_LAUNCH(k_counts, lbf_cdiv(T.nbox, 256), 256, 0, s, T.nbox, T.level, T.nchild, T.begin,
               T.end, T.u_ptr, T.u_idx, T.w_ptr, T.nv, T.xlist, T.nx, c);
    LBF_CHECK_LAUNCH();
    unsigned long long h[8];
    LBF_CUDA(cudaMemcpyAsync(h, c, sizeof(h), cudaMemcpyDeviceToHost, s));
    LBF_CUDA(cudaStreamSynchronize(s));
    for (int k = 1; k < 8; k++) counts[k] = (int64_t)h[k];
    counts[1] -= pl->N;  // each leaf lists itself in U: drop the self pairs
    return LBF_OK;
}

}  // extern "C"
