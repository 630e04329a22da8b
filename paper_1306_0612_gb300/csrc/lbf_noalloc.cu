// lbf_evaluate_noalloc: the off-curve evaluation of the double-layer
// representation with every byte of scratch in a file-scope static device
// array, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where no allocator is reachable or allowed --
// a host thread with a fixed memory budget handed out at start-up (real-time
// or embedded loops), a foreign-language binding with no access to the
// framework's allocator, or a plugin inside another library's callback that
// must not grow that library's pool.  Such callers can still pass their own
// inputs and outputs; this entry point needs nothing else.
//
// Limits and sharing:
//   - at most LBF_NOALLOC_MAX_NODES nodes (the array holds q = sigma w for each
//     node plus the reduction partials: about 4 MB, held by every GPU that loads
//     the library until the process exits);
//   - every call, on every stream, uses the same array and leaves its contents
//     behind: two calls whose work overlaps on the GPU race and give wrong
//     results.  Serialise them (same stream, or events);
//   - the first call on a device looks up the array's device address (set-up)
//     with that device current; make that first call before any stream capture.
#include <algorithm>
#include <mutex>

#include "lbf_internal.cuh"

namespace {

constexpr int kNaBlocks = 1024;
constexpr int64_t kNaScratchDoubles = 2 * (int64_t)LBF_NOALLOC_MAX_NODES + kNaBlocks + 64;

// q (2 doubles per node) | block partials (kNaBlocks) | beta.sigma | counter
static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

std::mutex g_na_mu;
double *g_na_addr[64] = {};

__device__ __forceinline__ double na_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// q_j = sigma_j w_j and sum_j beta_j sigma_j with
// beta_j = -(1/2pi) Im(conj(xi_j) w_j / (1 + |xi_j|^2)) (the sphere correction of
// the planar double layer, Eq. dlpC), the last block summing the partials in order.
__global__ void k_na_prep(int64_t N, const double2 *__restrict__ xi, const double2 *__restrict__ w,
                          const double *__restrict__ sigma, double *scr)
{
    double2 *q = (double2 *)scr;
    double *part = scr + 2 * (int64_t)LBF_NOALLOC_MAX_NODES;
    double *bsig = part + kNaBlocks;
    unsigned *count = (unsigned *)(bsig + 1);
    __shared__ double sh[32];
    __shared__ bool last;
    double acc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        double s = sigma[j];
        double2 z = xi[j], ww = w[j];
        q[j] = make_double2(s * ww.x, s * ww.y);
        double beta = -(1.0 / (2.0 * LBF_PI)) * (z.x * ww.y - z.y * ww.x) / (1.0 + z.x * z.x + z.y * z.y);
        acc = fma(beta, s, acc);
    }
    acc = na_warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
        part[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) t += ((volatile double *)part)[b];
        *bsig = t;
        *count = 0u;
    }
}

// u(t) = (1/2pi) Im sum_j q_j / (xi_j - xi_t) + beta.sigma + sum_m a_m G(t, c_m), one warp per target.
__global__ void k_na_eval(int64_t N, int M, const double2 *__restrict__ xi, const double *scr,
                          const double *__restrict__ a, const double *__restrict__ c, int64_t T,
                          const double *__restrict__ t, double *__restrict__ u)
{
    const double2 *q = (const double2 *)scr;
    const double *bsig = scr + 2 * (int64_t)LBF_NOALLOC_MAX_NODES + kNaBlocks;
    int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (wid >= T) return;
    double p0 = t[3 * wid], p1 = t[3 * wid + 1], p2 = t[3 * wid + 2];
    double wz = 1.0 - p2;
    double acc = 0.0;
    if (wz > 0.0) {
        double zx = p0 / wz, zy = p1 / wz;
        for (int64_t j = lane; j < N; j += 32) {
            double dr = xi[j].x - zx, di = xi[j].y - zy;
            double2 qq = q[j];
            acc += (qq.y * dr - qq.x * di) / (dr * dr + di * di);
        }
    }
    acc = na_warp_sum(acc) * (1.0 / (2.0 * LBF_PI));
    if (lane == 0) {
        double s = acc + *bsig;
        for (int m = 0; m < M; m++) {
            double d0 = p0 - c[3 * m], d1 = p1 - c[3 * m + 1], d2 = p2 - c[3 * m + 2];
            s += a[m] * (1.0 / (4.0 * LBF_PI)) * log(2.0 / (d0 * d0 + d1 * d1 + d2 * d2));
        }
        u[wid] = s;
    }
}

// device address of the static scratch for the current device (set-up on first use)
int na_scratch(double **out)
{
    int dev = 0;
    LBF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LBF_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        LBF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_addr[dev] = (double *)p;
    }
    *out = g_na_addr[dev];
    return LBF_OK;
}

}  // namespace

extern "C" int lbf_evaluate_noalloc(int64_t N, const double *xi, const double *weight,
                                    const double *sigma, int M, const double *a,
                                    const double *centres, int64_t T, const double *targets,
                                    double *u, lbf_stream_t stream)
{
    if (N < 1 || N > LBF_NOALLOC_MAX_NODES) return LBF_EINVAL;
    if (!xi || !weight || !sigma || T < 0 || (T > 0 && (!targets || !u)) || M < 0 ||
        (M > 0 && (!a || !centres)))
        return LBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *scr = nullptr;
    int rc = na_scratch(&scr);
    if (rc) return rc;
    // the last block of every call that ran to completion leaves the reduction counter at
    // zero; this reset only recovers a counter left behind by a launch that never
    // completed (an aborted context).  It does not make overlapping calls safe:
    // serialise them.
    unsigned *count = (unsigned *)(scr + 2 * (int64_t)LBF_NOALLOC_MAX_NODES + kNaBlocks + 1);
    LBF_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
    int nb = (int)std::min<int64_t>(lbf_cdiv(N, 256), kNaBlocks);
    LBF_LAUNCH(k_na_prep, nb, 256, 0, s, N, (const double2 *)xi, (const double2 *)weight, sigma, scr);
    LBF_CHECK_LAUNCH();
    if (T > 0) {
        LBF_LAUNCH(k_na_eval, lbf_cdiv(T * 32, 256), 256, 0, s, N, M, (const double2 *)xi, scr, a,
                   centres, T, targets, u);
        LBF_CHECK_LAUNCH();
    }
    return LBF_OK;
}
