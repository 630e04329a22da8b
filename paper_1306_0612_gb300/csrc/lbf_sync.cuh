// Bounded device-wide waits shared by the cooperative kernels (the inverse and the
// LU factorisation of the Schur complement) and the in-launch dependency chains.
//
// Every wait polls at most a fixed number of times, then sets LBF_DEV_TIMEOUT in the
// plan's status word and gives up, so a kernel always ends.  The poll limit is the
// plan's status word's neighbour status[1] when that is non-zero (a caller may lower
// it to make a wait run out on purpose: lbf_debug_wait_limit), else the default.
#pragma once

#include "lbf_internal.cuh"

constexpr unsigned kBarrierSpins = 1u << 22;

static __device__ __forceinline__ unsigned wait_limit(const int *status, unsigned dflt)
{
    const unsigned v = (unsigned)((const volatile int *)status)[1];
    return v ? v : dflt;
}

struct GridBarrier {
    unsigned count, gen;
};

// all nb blocks of a cooperative launch meet here; false (status set) on time-out
static __device__ __noinline__ bool grid_barrier(GridBarrier *bar, unsigned nb, int *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned lim = wait_limit(status, kBarrierSpins);
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
                if (++it > lim) {
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

// thread 0 waits until *flag == want (another block of the same launch sets it);
// false (status set) on time-out; the whole block returns the same value
static __device__ __noinline__ bool block_wait_flag(const unsigned *flag, unsigned want, int *status,
                                            unsigned dflt_spins)
{
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned lim = wait_limit(status, dflt_spins);
        unsigned it = 0;
        while (*(const volatile unsigned *)flag != want) {
            if (++it > lim) {
                atomicOr(status, LBF_DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}
