// Batched solves of independent geometries (many instances of the system of Sec. 5,
// each with several right-hand sides).  A host-side scheduler: worker threads, each
// with its own CUDA stream, take whole instances largest-first (plan, every
// right-hand side's solve and evaluation, plan destroyed) so that the small,
// latency-bound solves of different instances overlap on the GPU.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "lbf_internal.cuh"

namespace {

int run_item(lbf_batch_item &it, const lbf_options &opt_all, cudaStream_t s)
{
    lbf_plan *pl = nullptr;
    int64_t need = 0;
    lbf_options opt = opt_all;
    opt.box_capacity = it.box_capacity;
    int rc = lbf_plan_create(&pl, it.M, it.island_ptr, it.x, it.dx, it.d2x, it.centres, nullptr,
                             &opt, it.workspace, it.bytes, &need, (lbf_stream_t)s);
    if (rc) {
        it.box_capacity_needed = need;
        return rc;
    }
    const int64_t N = pl->N;
    int worst = LBF_OK;
    // the right-hand sides in lockstep when the item's workspace holds their buffers
    // after the plan's (lbf_batch_workspace_size)
    size_t pbytes = 0, mbytes = 0;
    const bool sized = lbf_workspace_size(it.M, it.island_ptr, &opt, &pbytes) == LBF_OK;
    pbytes = (pbytes + 255) & ~size_t(255);
    const bool lock = sized && it.nrhs > 1 && lbf_gmres_workspace_many(pl, it.nrhs, &mbytes) == LBF_OK &&
                      mbytes > 0 && it.bytes >= pbytes + mbytes;
    if (lock) {
        std::vector<int> its(it.nrhs, 0);
        std::vector<double> rr(it.nrhs, 0.0);
        rc = lbf_gmres_solve_many(pl, it.nrhs, it.g, it.sigma, it.a, its.data(), rr.data(),
                                  (char *)it.workspace + pbytes, it.bytes - pbytes, (lbf_stream_t)s);
        if (rc < 0) {
            worst = rc;
        } else {
            if (rc == LBF_NOCONV) worst = LBF_NOCONV;
            for (int r = 0; r < it.nrhs; r++) {
                it.iters += its[r];
                it.max_rel_res = std::max(it.max_rel_res, rr[r]);
            }
            int64_t st[4];
            lbf_solve_stats(pl, st);
            it.fp64_applies += st[1];
            it.fp32_applies += st[2];
            for (int r = 0; r < it.nrhs && it.T > 0 && it.u && worst >= 0; r++) {
                rc = lbf_evaluate(pl, it.sigma + r * N, it.a ? it.a + (int64_t)r * it.M : nullptr,
                                  it.T, it.targets, it.u + r * it.T, (lbf_stream_t)s);
                if (rc) worst = rc;
            }
        }
    }
    for (int r = 0; r < it.nrhs && worst >= 0 && !lock; r++) {
        int its = 0;
        double rr = 0.0;
        rc = lbf_gmres_solve(pl, it.g + r * N, it.sigma + r * N, it.a ? it.a + (int64_t)r * it.M : nullptr,
                             nullptr, &its, &rr, (lbf_stream_t)s);
        if (rc < 0) {
            worst = rc;
            break;
        }
        if (rc == LBF_NOCONV) worst = LBF_NOCONV;
        it.iters += its;
        it.max_rel_res = std::max(it.max_rel_res, rr);
        int64_t st[4];
        lbf_solve_stats(pl, st);
        it.fp64_applies += st[1];
        it.fp32_applies += st[2];
        if (it.T > 0 && it.u) {
            rc = lbf_evaluate(pl, it.sigma + r * N, it.a ? it.a + (int64_t)r * it.M : nullptr, it.T,
                              it.targets, it.u + r * it.T, (lbf_stream_t)s);
            if (rc) worst = rc;
        }
    }
    // every path: the item's kernels finish before its plan (and the caller's view of
    // its workspace) is released
    if (cudaStreamSynchronize(s) != cudaSuccess && worst >= 0) worst = LBF_ECUDA;
    lbf_plan_destroy(pl);
    return worst;
}

}  // namespace

extern "C" int lbf_batch_run(int nitems, lbf_batch_item *items, const lbf_options *opt,
                             int nworkers)
{
    if (nitems < 0 || (nitems > 0 && !items) || !opt || nworkers < 1) return LBF_EINVAL;
    for (int q = 0; q < nitems; q++) {
        lbf_batch_item &it = items[q];
        if (it.nrhs < 0 || it.M < 1 || !it.island_ptr || !it.workspace || (it.nrhs > 0 && (!it.g || !it.sigma)) ||
            it.T < 0 || (it.T > 0 && it.u && !it.targets))
            return LBF_EINVAL;
        it.status = LBF_OK;
        it.iters = 0;
        it.fp64_applies = it.fp32_applies = 0;
        it.max_rel_res = 0.0;
        it.box_capacity_needed = 0;
    }
    // largest first: sum of nodes times right-hand sides
    std::vector<int> order(nitems);
    for (int q = 0; q < nitems; q++) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int64_t wx = items[x].island_ptr[items[x].M] * std::max(items[x].nrhs, 1);
        const int64_t wy = items[y].island_ptr[items[y].M] * std::max(items[y].nrhs, 1);
        return wx > wy;
    });
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBF_ECUDA;
    std::atomic<int> next{0};
    std::atomic<int> fail{0};
    auto worker = [&]() {
        if (cudaSetDevice(dev) != cudaSuccess) {
            fail.store(1);
            return;
        }
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            fail.store(1);
            return;
        }
        for (;;) {
            int k = next.fetch_add(1);
            if (k >= nitems) break;
            lbf_batch_item &it = items[order[k]];
            it.status = run_item(it, *opt, s);
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    const int nw = std::max(1, std::min(nworkers, std::max(nitems, 1)));
    std::vector<std::thread> pool;
    pool.reserve(nw);
    for (int w = 0; w < nw; w++) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    return fail.load() ? LBF_ECUDA : LBF_OK;
}
