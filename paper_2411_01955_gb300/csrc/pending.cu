// Entry points of the solver variants that are declared in the C ABI but
// not built yet: they fail loudly with HQS_ERR_UNSUPPORTED instead of
// falling back to another path.
#include "solve.cuh"

int launch_toeplitz_mixed(hqs_plan_s*, const float2*, float2*, int, cudaStream_t) {
    return HQS_ERR_UNSUPPORTED;
}
