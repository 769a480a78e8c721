// Measured FP32 FMA throughput of the GPU (no counterpart in the paper): the
// denominator of the ALU roofline that the L2-resident persistent solve is
// reported against.  Every thread runs 8 independent FMA chains, so the FMA
// pipes stay busy at full occupancy; the rate is timed with CUDA events.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_probe(float* __restrict__ sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
#pragma unroll 16
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.f) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

extern "C" int hqs_probe_fp32_peak(double* tflops, void* stream) {
    if (!tflops) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    HQS_CUDA_TRY(cudaGetDevice(&dev));
    HQS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8, threads = 256, iters = 16384;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HQS_CUDA_TRY(cudaEventCreate(&e0));
    HQS_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<float> ms;
    int rc = HQS_OK;
    for (int rep = 0; rep < 4 && rc == HQS_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = HQS_ERR_CUDA;
        k_fma_probe<<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999f, 1e-4f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            rc = HQS_ERR_CUDA;
        float t = 0.f;
        if (rc == HQS_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = HQS_ERR_CUDA;
        if (rep > 0) ms.push_back(t);   // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != HQS_OK) return rc;
    std::sort(ms.begin(), ms.end());
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *tflops = flops / (ms[ms.size() / 2] * 1e-3) / 1e12;
    return HQS_OK;
}
