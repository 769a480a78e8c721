// Shared device/host helpers for the sm_103a kernels of the HQS hot path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hqs.h"

#define HQS_DEV __device__ __forceinline__

// ---------------------------------------------------------------- complex
HQS_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
HQS_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
HQS_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
HQS_DEV float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
HQS_DEV float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
HQS_DEV float2 cfma(float2 a, float2 b, float2 acc) {   // acc + a*b
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}
// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg; both
// addresses 16-byte aligned), and the wait for every copy this thread issued.
HQS_DEV void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
HQS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Programmatic dependent launch (kernels launched with launch_pdl): the
// kernel lets the next kernel of the stream launch its CTAs early and waits
// until the previous kernel of the stream has completed and its memory is
// visible; both are no-ops without a programmatic dependency.  A kernel entered
// this way touches no global memory before the wait.
HQS_DEV void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
HQS_DEV void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#define HQS_PDL_ENTRY()              \
    do {                             \
        griddep_launch_dependents(); \
        griddep_wait();              \
    } while (0)

// multiply by -i (forward) or +i (inverse)
template <bool INV> HQS_DEV float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------- errors
#define HQS_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            hqs_note_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return (e_ == cudaErrorMemoryAllocation) ? HQS_ERR_OOM : HQS_ERR_CUDA; \
        }                                                    \
    } while (0)

void hqs_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Device error word bits (per plan), read back at sync points.
#define HQS_DEVERR_TIMEOUT   1u
#define HQS_DEVERR_BREAKDOWN 2u
#define HQS_DEVERR_BOUNDS    4u

// Launch with programmatic stream serialisation: the kernel's CTAs may start
// while the previous kernel of the stream finishes (the kernel begins with
// HQS_PDL_ENTRY), which hides the launch gap between the passes of an operator.
template <class... KArgs, class... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- math
static inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
