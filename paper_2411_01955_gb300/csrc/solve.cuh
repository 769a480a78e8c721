// Declarations shared by the operator, solver and outer-loop translation units.
#pragma once

#include "plan.cuh"

#define HQS_TRY_RC(expr)               \
    do {                               \
        int rc__ = (expr);             \
        if (rc__ != HQS_OK) return rc__; \
    } while (0)

enum CgScalarMode { CG_INIT = 0, CG_ALPHA = 1, CG_RES = 2, CG_BETA = 3, CG_BETA0 = 4 };

struct ToepArgs {
    int n, L, LC, nchunk;
    const float2* smaps;   // [n][n][L]
    const float* khat;     // [2n][2n]
    const float2* tw;      // 2n-point twiddles
    float2* T;             // [n][2n][L] intermediate
    float2* chunk;         // [nchunk][n][n] per-chunk coil sums (nchunk > 1)
};

int toep_partial_count(const hqs_plan_s* p);

ToepArgs toep_args(hqs_plan_s* p);

int launch_toeplitz_ex(hqs_plan_s* p, const float2* src, float2* pvec, int fuse, float2* out,
                       const float2* pmul, float a, float b, int mode, double* part,
                       const CgScalars* cg, cudaStream_t st);
int launch_toeplitz_mixed(hqs_plan_s* p, const float2* x, float2* out, int precision, cudaStream_t st);
int launch_toeplitz_mixed_ex(hqs_plan_s* p, const float2* x, float2* out, const float2* pmul, float a, float b,
                             int mode, double* part, int precision, cudaStream_t st);
int mixed_partial_count(const hqs_plan_s* p);
int launch_precond_ex(hqs_plan_s* p, float a, float b, const float2* r, float2* z, bool rows_done,
                      const CgScalars* cg, double* part, cudaStream_t st);

int pcg_plain(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter,
              double rel_tol, int precond, bool x0_zero, cudaStream_t st, int precision = HQS_PREC_FP32);
int pcg_fused(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter,
              double rel_tol, int precond, int precision, bool x0_zero, cudaStream_t st);
int fcg_learned(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter,
                double rel_tol, bool x0_zero, cudaStream_t st);
int read_solve_info(hqs_plan_s* p, hqs_solve_info* info, cudaStream_t st);
