// Toeplitz-embedded normal operator A^H A (a4) and the preconditioned CG
// data-consistency solve (a5) of Sec. 3.4.
//
// A^H A x = sum_l conj(S_l) crop(IFFT_2N(Khat * FFT_2N(pad(S_l x)))) in three
// passes over a coil-innermost [n][2n][L] intermediate:
//   P1 (rows, n of them):   S_l * x, zero-pad to 2n, FFT along x
//   P2 (columns, 2n):       zero-pad to 2n, FFT along y, * Khat, IFFT, keep n rows
//   P3 (rows, n):           IFFT along x, keep n, sum_l conj(S_l) * . over coils
// The CG recursion is fused into P1 (p = z + beta p) and P3 (q = a A^H A p +
// b p with the fp64 partial of <p, q>).  Inner products accumulate in fp64
// with a fixed-order reduction, so the solve is deterministic.
#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "plan.cuh"
#include "solve.cuh"

using namespace hqs;

#include "toep_items.cuh"

// --------------------------------------------------------- plain kernels
template <int N2>
__global__ void k_toep_rows_fwd(ToepArgs A, const float2* __restrict__ src, float2* __restrict__ pvec,
                                int fuse, const CgScalars* __restrict__ cg) {
    HQS_PDL_ENTRY();
    if (cg && cg->done) return;
    extern __shared__ __align__(16) float2 s[];
    const float beta = (fuse && cg) ? (float)cg->beta : 0.f;
    toep_rows_fwd_item<N2>(A, blockIdx.x, blockIdx.y, src, pvec, beta, fuse != 0, s);
}

template <int N2>
__global__ void k_toep_cols(ToepArgs A, const CgScalars* __restrict__ cg) {
    HQS_PDL_ENTRY();
    if (cg && cg->done) return;
    extern __shared__ __align__(16) float2 s[];
    toep_cols_item<N2>(A, blockIdx.x, blockIdx.y, s);
}

template <int N2>
__global__ void k_toep_rows_adj(ToepArgs A, float2* __restrict__ out, const float2* __restrict__ pvec,
                                float a, float b, int mode, double* __restrict__ part,
                                const CgScalars* __restrict__ cg) {
    HQS_PDL_ENTRY();
    if (cg && cg->done) return;
    extern __shared__ __align__(16) float2 s[];
    __shared__ double red[32];
    const double v = toep_rows_adj_item<N2>(A, blockIdx.x, blockIdx.y, out, pvec, a, b, mode, s);
    if (part && A.nchunk == 1) {
        const double t = block_sum(v, red);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// Several coil chunks: sum the chunk partials in a fixed order, then the
// CG epilogue; partials of Re<p, q> per block.
__global__ void k_toep_chunk_epilogue(ToepArgs A, float2* __restrict__ out, const float2* __restrict__ pvec,
                                      float a, float b, int mode, double* __restrict__ part,
                                      const CgScalars* __restrict__ cg) {
    HQS_PDL_ENTRY();
    if (cg && cg->done) return;
    __shared__ double red[32];
    const int count = A.n * A.n;
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        for (int c = 0; c < A.nchunk; ++c) v = cadd(v, A.chunk[(int64_t)c * count + e]);
        out[e] = toep_epilogue(v, e, pvec, a, b, mode, acc);
    }
    if (part) {
        const double t = block_sum(acc, red);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// p = z + beta p (used instead of the fused update when there are several chunks)
__global__ void k_cg_pupdate(const float2* __restrict__ z, float2* __restrict__ p, int count,
                             const CgScalars* __restrict__ cg) {
    if (cg->done) return;
    const float beta = (float)cg->beta;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        float2 v = z[e];
        if (beta != 0.f) {
            const float2 pv = p[e];
            v.x = fmaf(beta, pv.x, v.x);
            v.y = fmaf(beta, pv.y, v.y);
        }
        p[e] = v;
    }
}

// r = rhs - q (q == nullptr: the start is x = 0, written here, and r = rhs);
// partials ||r||^2 and ||rhs||^2
__global__ void k_cg_init_r(const float2* __restrict__ rhs, const float2* __restrict__ q,
                            float2* __restrict__ r, float2* __restrict__ x, int count,
                            double* __restrict__ part_rr, double* __restrict__ part_bb) {
    __shared__ double red[32];
    double rr = 0.0, bb = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 b = rhs[e];
        float2 v = b;
        if (q) v = csub(b, q[e]);
        else x[e] = make_float2(0.f, 0.f);
        r[e] = v;
        rr += (double)v.x * v.x + (double)v.y * v.y;
        bb += (double)b.x * b.x + (double)b.y * b.y;
    }
    const double t1 = block_sum(rr, red);
    const double t2 = block_sum(bb, red);
    if (threadIdx.x == 0) {
        part_rr[blockIdx.x] = t1;
        part_bb[blockIdx.x] = t2;
    }
}

// x += alpha p; r -= alpha q; partial ||r||^2
__global__ void k_cg_update(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                            const float2* __restrict__ q, int count, double* __restrict__ part_rr,
                            const CgScalars* __restrict__ cg) {
    if (cg->done) return;
    __shared__ double red[32];
    const float alpha = (float)cg->alpha;
    double rr = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 pv = p[e], qv = q[e];
        float2 xv = x[e], rv = r[e];
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        x[e] = xv;
        r[e] = rv;
        rr += (double)rv.x * rv.x + (double)rv.y * rv.y;
    }
    const double t = block_sum(rr, red);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = t;
}

__global__ void k_zero_if_flag(float2* __restrict__ x, int count, const CgScalars* __restrict__ cg) {
    if (!cg->zero_rhs) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        x[e] = make_float2(0.f, 0.f);
}

HQS_DEV double fixed_sum(const double* part, int nb, double* red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[i];
    return block_sum(v, red);
}

// Scalar steps of the CG recursion, one block, fixed reduction order.
__global__ void k_cg_scalar(CgScalars* __restrict__ cg, const double* __restrict__ partials, int mode,
                            int nb, double rz_scale, int use_rz, double* __restrict__ hist) {
    __shared__ double red[32];
    if (mode != CG_INIT && cg->done) return;
    if (mode == CG_INIT) {
        const double rr = fixed_sum(partials + SLOT_RR * HQS_MAX_BLOCKS, nb, red);
        const double bb = fixed_sum(partials + SLOT_BB * HQS_MAX_BLOCKS, nb, red);
        if (threadIdx.x == 0) {
            cg->it = 0;
            cg->bnorm = sqrt(bb);
            cg->rr = rr;
            cg->tol2 = cg->tol2 * bb;       // tol2 holds rel_tol^2 on entry
            cg->beta = 0.0;
            cg->alpha = 0.0;
            cg->status = HQS_OK;
            cg->zero_rhs = 0;
            cg->done = 0;
            hist[0] = rr;
            if (!(bb == bb) || !(rr == rr) || isinf(bb) || isinf(rr)) {
                cg->status = HQS_ERR_BREAKDOWN;
                cg->done = 1;
            } else if (bb == 0.0) {
                cg->zero_rhs = 1;
                cg->rr = 0.0;
                hist[0] = 0.0;
                cg->done = 1;
            } else if (rr <= cg->tol2 || cg->max_iter == 0) {
                cg->done = 1;
                if (rr > cg->tol2 && cg->tol2 > 0.0) cg->status = HQS_ERR_NOT_CONVERGED;
            }
        }
    } else if (mode == CG_ALPHA) {
        const double pq = fixed_sum(partials + SLOT_PQ * HQS_MAX_BLOCKS, nb, red);
        if (threadIdx.x == 0) {
            cg->pq = pq;
            if (!(pq > 0.0) || isinf(pq)) {
                cg->status = HQS_ERR_BREAKDOWN;
                cg->done = 1;
            } else {
                cg->alpha = cg->rz / pq;
            }
        }
    } else if (mode == CG_RES) {
        const double rr = fixed_sum(partials + SLOT_RR * HQS_MAX_BLOCKS, nb, red);
        if (threadIdx.x == 0) {
            cg->rr = rr;
            cg->it += 1;
            hist[cg->it] = rr;
            if (!(rr == rr) || isinf(rr)) {
                cg->status = HQS_ERR_BREAKDOWN;
                cg->done = 1;
            } else if (rr <= cg->tol2) {
                cg->done = 1;
            } else if (cg->it >= cg->max_iter) {
                cg->done = 1;
                if (cg->tol2 > 0.0) cg->status = HQS_ERR_NOT_CONVERGED;
            }
        }
    } else {  // CG_BETA / CG_BETA0
        double rz;
        if (use_rz)
            rz = fixed_sum(partials + SLOT_RZ * HQS_MAX_BLOCKS, nb, red) * rz_scale;
        else
            rz = cg->rr;
        if (threadIdx.x == 0) {
            if (mode == CG_BETA0) {
                cg->beta = 0.0;
            } else {
                cg->beta = rz / cg->rz;
            }
            cg->rz = rz;
            if (!(rz > 0.0) || isinf(rz)) {
                cg->status = HQS_ERR_BREAKDOWN;
                cg->done = 1;
            }
        }
    }
}

__global__ void k_cg_setup(CgScalars* cg, int max_iter, double rel_tol) {
    cg->max_iter = max_iter;
    cg->tol2 = rel_tol * rel_tol;
    cg->done = 0;
    cg->status = HQS_OK;
    cg->it = 0;
    cg->fallback = 0;
}

// ------------------------------------------------------------ launchers
ToepArgs toep_args(hqs_plan_s* p) {
    ToepArgs A;
    A.n = p->n;
    A.L = p->L;
    A.LC = p->LC;
    A.nchunk = p->nchunk;
    A.smaps = p->smaps;
    A.khat = p->khat;
    A.tw = plan_twiddles(p, p->n2);
    A.T = p->work;
    A.chunk = p->chunk_buf;
    return A;
}

// Number of partial-sum slots written by the A^H A epilogue (rows or blocks).
int toep_partial_count(const hqs_plan_s* p) {
    return p->nchunk == 1 ? p->n : std::min(ceil_div(p->n * p->n, 256), 1024);
}

template <int N2>
static int toep_impl(hqs_plan_s* p, const float2* src, float2* pvec, int fuse, float2* out,
                     const float2* pmul, float a, float b, int mode, double* part,
                     const CgScalars* cg, cudaStream_t st) {
    ToepArgs A = toep_args(p);
    const int th = fft_threads<N2>(p->LC);
    const size_t sm = toep_smem_floats2<N2>(p->n) * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_toep_rows_fwd<N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_toep_cols<N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_toep_rows_adj<N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const dim3 grows(p->n, p->nchunk), gcols(N2, p->nchunk);
    if (fuse && p->nchunk > 1) {
        k_cg_pupdate<<<std::min(ceil_div(p->n * p->n, 256), 1024), 256, 0, st>>>(src, pvec, p->n * p->n, cg);
        src = pvec;
        fuse = 0;
    }
    HQS_CUDA_TRY(launch_pdl(k_toep_rows_fwd<N2>, grows, th, sm, st, A, src, pvec, fuse, cg));
    HQS_CUDA_TRY(launch_pdl(k_toep_cols<N2>, gcols, th, sm, st, A, cg));
    HQS_CUDA_TRY(launch_pdl(k_toep_rows_adj<N2>, grows, th, sm, st, A, out, pmul, a, b, mode, part, cg));
    if (p->nchunk > 1)
        HQS_CUDA_TRY(launch_pdl(k_toep_chunk_epilogue, dim3(toep_partial_count(p)), dim3(256), 0, st, A, out, pmul, a,
                                b, mode, part, cg));
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

int launch_toeplitz_ex(hqs_plan_s* p, const float2* src, float2* pvec, int fuse, float2* out,
                       const float2* pmul, float a, float b, int mode, double* part,
                       const CgScalars* cg, cudaStream_t st) {
    return dispatch_fft_size(p->n2, [&]<int NN>() {
        return toep_impl<NN>(p, src, pvec, fuse, out, pmul, a, b, mode, part, cg, st);
    });
}

int launch_toeplitz(hqs_plan_s* p, const float2* x, float2* out, cudaStream_t st) {
    return launch_toeplitz_ex(p, x, nullptr, 0, out, nullptr, 1.f, 0.f, 0, nullptr, nullptr, st);
}

extern "C" int hqs_toeplitz_normal(hqs_plan p, const hqs_c64* x, hqs_c64* out, int precision,
                                   void* stream) {
    if (!p || !x || !out) return HQS_ERR_INVALID_ARG;
    if (precision == HQS_PREC_FP32)
        return launch_toeplitz(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(out),
                               (cudaStream_t)stream);
    if (precision == HQS_PREC_BF16X3 || precision == HQS_PREC_FP16X3)
        return launch_toeplitz_mixed(p, reinterpret_cast<const float2*>(x),
                                     reinterpret_cast<float2*>(out), precision, (cudaStream_t)stream);
    return HQS_ERR_INVALID_ARG;
}

// ------------------------------------------------------- plain PCG driver
// One launch per stage; the host reads the stop flag after every iteration.
// H p with the CG epilogue (q = a A^H A p + b p, partials of <p, q>); FP32
// in-house FFTs, or the tensor-core DFT-GEMM passes for the mixed precisions
// (p = z + beta p then runs as its own kernel).  Returns the partial count.
static int toep_apply(hqs_plan_s* p, int precision, const float2* src, float2* pvec, int fuse, float2* out,
                      const float2* pmul, float a, float b, double* part, const CgScalars* cg,
                      cudaStream_t st, int* nparts) {
    if (precision == HQS_PREC_FP32) {
        *nparts = toep_partial_count(p);
        return launch_toeplitz_ex(p, src, pvec, fuse, out, pmul, a, b, 1, part, cg, st);
    }
    if (fuse) {
        k_cg_pupdate<<<std::min(ceil_div(p->n * p->n, 256), 1024), 256, 0, st>>>(src, pvec, p->n * p->n, cg);
        src = pvec;
    }
    *nparts = mixed_partial_count(p);
    return launch_toeplitz_mixed_ex(p, src, out, pmul, a, b, 1, part, precision, st);
}

int pcg_plain(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter,
              double rel_tol, int precond, bool x0_zero, cudaStream_t st, int precision) {
    const int n = p->n, count = n * n;
    const int nb_vec = std::min(ceil_div(count, 256), HQS_MAX_BLOCKS);
    double* part = p->partials;
    double* P_PQ = part + SLOT_PQ * HQS_MAX_BLOCKS;
    double* P_RR = part + SLOT_RR * HQS_MAX_BLOCKS;
    double* P_BB = part + SLOT_BB * HQS_MAX_BLOCKS;
    double* P_RZ = part + SLOT_RZ * HQS_MAX_BLOCKS;
    const bool dc = precond == HQS_PRECOND_DC;
    const double rz_scale = 1.0 / ((double)n * n);
    const int nb_pc = ceil_div(n, p->q_rows);
    const float2* zsrc = dc ? p->cg_z : p->cg_r;

    k_cg_setup<<<1, 1, 0, st>>>(p->cg, max_iter, rel_tol);
    int nparts = 0;
    // q = H x (skipped for a zero start)
    if (!x0_zero)
        HQS_TRY_RC(toep_apply(p, precision, x, nullptr, 0, p->cg_q, x, a, b, nullptr, nullptr, st, &nparts));
    k_cg_init_r<<<nb_vec, 256, 0, st>>>(rhs, x0_zero ? nullptr : p->cg_q, p->cg_r, x, count, P_RR, P_BB);
    k_cg_scalar<<<1, 256, 0, st>>>(p->cg, part, CG_INIT, nb_vec, rz_scale, 0, p->hist);
    if (dc) HQS_TRY_RC(launch_precond_ex(p, a, b, p->cg_r, p->cg_z, false, p->cg, P_RZ, st));
    k_cg_scalar<<<1, 256, 0, st>>>(p->cg, part, CG_BETA0, dc ? nb_pc : nb_vec, rz_scale, dc ? 1 : 0, p->hist);
    k_zero_if_flag<<<nb_vec, 256, 0, st>>>(x, count, p->cg);
    HQS_CUDA_TRY(cudaGetLastError());
    for (int it = 0; it < max_iter; ++it) {
        HQS_CUDA_TRY(cudaMemcpyAsync(p->h_cg, p->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        if (p->h_cg->done) break;
        // p = z + beta p; q = H p; <p, q>
        HQS_TRY_RC(toep_apply(p, precision, zsrc, p->cg_p, 1, p->cg_q, p->cg_p, a, b, P_PQ, p->cg, st, &nparts));
        k_cg_scalar<<<1, 256, 0, st>>>(p->cg, part, CG_ALPHA, nparts, rz_scale, 0, p->hist);
        k_cg_update<<<nb_vec, 256, 0, st>>>(x, p->cg_r, p->cg_p, p->cg_q, count, P_RR, p->cg);
        k_cg_scalar<<<1, 256, 0, st>>>(p->cg, part, CG_RES, nb_vec, rz_scale, 0, p->hist);
        if (dc) HQS_TRY_RC(launch_precond_ex(p, a, b, p->cg_r, p->cg_z, false, p->cg, P_RZ, st));
        k_cg_scalar<<<1, 256, 0, st>>>(p->cg, part, CG_BETA, dc ? nb_pc : nb_vec, rz_scale, dc ? 1 : 0, p->hist);
        HQS_CUDA_TRY(cudaGetLastError());
    }
    return HQS_OK;
}

int read_solve_info(hqs_plan_s* p, hqs_solve_info* info, cudaStream_t st) {
    HQS_CUDA_TRY(cudaMemcpyAsync(p->h_cg, p->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(p->h_hist, p->hist, sizeof(double) * (HQS_MAX_ITERS + 1),
                                 cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(p->h_err, p->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    const CgScalars& c = *p->h_cg;
    const int status = (*p->h_err & HQS_DEVERR_TIMEOUT) ? HQS_ERR_TIMEOUT : c.status;
    if (!info) return status;
    info->iterations = c.it;
    info->status = status;
    info->fallback = c.fallback;
    info->reserved = 0;
    info->rhs_norm = c.bnorm;
    const double bn = c.bnorm > 0 ? c.bnorm : 1.0;
    info->rel_residual = c.bnorm > 0 ? sqrt(std::max(c.rr, 0.0)) / bn : 0.0;
    for (int i = 0; i <= HQS_MAX_ITERS; ++i)
        info->res_history[i] = (i <= c.it) ? sqrt(std::max(p->h_hist[i], 0.0)) / bn : 0.0;
    if (c.bnorm == 0) info->res_history[0] = 0.0;
    return status;
}

extern "C" int hqs_last_solve_info(hqs_plan p, hqs_solve_info* info, void* stream) {
    if (!p || !info) return HQS_ERR_INVALID_ARG;
    int rc = read_solve_info(p, info, (cudaStream_t)stream);
    return rc < 0 && rc != HQS_ERR_NOT_CONVERGED && rc != HQS_ERR_BREAKDOWN && rc != HQS_ERR_TIMEOUT ? rc
                                                                                                    : HQS_OK;
}

extern "C" int hqs_dc_solve(hqs_plan p, float a, float b, const hqs_c64* rhs, hqs_c64* x,
                            int max_iter, double rel_tol, int precond, int mode, int precision,
                            hqs_solve_info* info, void* stream) {
    if (!p || !rhs || !x || !(b > 0.f) || !(a == a) || max_iter < 0 || max_iter > HQS_MAX_ITERS ||
        !(rel_tol >= 0.0))
        return HQS_ERR_INVALID_ARG;
    if (precond != HQS_PRECOND_NONE && precond != HQS_PRECOND_DC && precond != HQS_PRECOND_LEARNED)
        return HQS_ERR_INVALID_ARG;
    const bool x0_zero = (mode & HQS_SOLVE_X0_ZERO) != 0;
    mode &= ~HQS_SOLVE_X0_ZERO;
    if (mode != HQS_SOLVE_PLAIN && mode != HQS_SOLVE_FUSED) return HQS_ERR_INVALID_ARG;
    if (precision != HQS_PREC_FP32 && precision != HQS_PREC_BF16X3 && precision != HQS_PREC_FP16X3)
        return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const float2* r = reinterpret_cast<const float2*>(rhs);
    float2* xx = reinterpret_cast<float2*>(x);
    int rc;
    if (precond == HQS_PRECOND_LEARNED) {
        if (precision != HQS_PREC_FP32) return HQS_ERR_UNSUPPORTED;
        rc = fcg_learned(p, a, b, r, xx, max_iter, rel_tol, x0_zero, st);
    } else if (mode == HQS_SOLVE_FUSED) {
        rc = pcg_fused(p, a, b, r, xx, max_iter, rel_tol, precond, precision, x0_zero, st);
    } else {
        rc = pcg_plain(p, a, b, r, xx, max_iter, rel_tol, precond, x0_zero, st, precision);
    }
    if (rc != HQS_OK) return rc;
    if (info) return read_solve_info(p, info, st);
    return HQS_OK;
}
