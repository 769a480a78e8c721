// Grid barrier and CTA reductions for the persistent cooperative kernels.
#pragma once

#include "common.cuh"

#define HQS_BARRIER_LIMIT_CYCLES 2000000000ll

namespace hqs {

HQS_DEV unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (cooperative launch: all CTAs are resident).  Returns
// false when the wait exceeded `limit` SM clock cycles (about a second by
// default) or another CTA reported an error.
HQS_DEV bool grid_barrier(unsigned* bar, unsigned* err, long long limit = HQS_BARRIER_LIMIT_CYCLES) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (*(volatile unsigned*)err) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > limit) {
                    atomicOr(err, HQS_DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

HQS_DEV double cta_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        red[32] = t;
    }
    __syncthreads();
    t = red[32];
    __syncthreads();
    return t;
}

}  // namespace hqs
