// Persistent cooperative PCG for the data-consistency step of Sec. 3.4
// (the fused solve, HQS_SOLVE_FUSED): one launch runs the whole solve.
//
// Every CTA loops over the work items of each stage (rows, columns or row
// blocks), then meets the others at a grid barrier.  Per iteration:
//   A  rows:        z row = IFFT_N(pc spectrum row)/N^2 (or r row), p = z + beta p,
//                   S_l p zero-padded, FFT along x          -> T
//   B  columns:     FFT along y, * Khat, IFFT, keep n rows   -> T
//   C  rows:        IFFT along x, crop, sum_l conj(S_l) .    -> q = a A^H A p + b p, <p,q>
//   D  row blocks:  x += alpha p, r -= alpha q, ||r||^2, FFT rows of r
//   E  col blocks:  FFT columns, * s^-1/2, <r,z> by Parseval, IFFT columns
// z is never stored.  Scalars are reduced by every CTA from the per-CTA
// partials in the same fixed order, so all CTAs take identical decisions and
// the result is deterministic.  Barrier waits are bounded (about a second):
// on expiry the kernel records HQS_DEVERR_TIMEOUT and returns.
#include <algorithm>
#include <cmath>

#include "plan.cuh"
#include "solve.cuh"
#include "persist.cuh"
#include "toep_items.cuh"

using namespace hqs;


struct FusedArgs {
    ToepArgs A;
    float a, b;
    const float2* rhs;
    float2* x;
    float2* r;
    float2* p;
    float2* q;
    float2* pcb;        // [n][n] preconditioner spectrum / row FFTs
    const float* lam;
    const float2* twN;  // n-point twiddles
    int Q;              // preconditioner lines per item
    int precond;
    int x0_zero;        // start from x = 0 (no initial A^H A apply)
    int max_iter;
    double rel_tol2;
    double* part;       // [NSLOTS][HQS_MAX_BLOCKS]
    CgScalars* cg;
    double* hist;
    unsigned* bar;      // [0] arrivals, [1] generation
    unsigned* err;
    unsigned long long* trace;  // optional: globaltimer stamp after each barrier
    int trace_max;
    int skip_cta;               // test hook: this CTA leaves before the first barrier (-1: none)
    long long barrier_limit;    // grid barrier wait limit, SM clock cycles
};



// Sum of the per-CTA partials of one slot, identical in every CTA.
HQS_DEV double grid_total(const double* part, double* red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(part + i);
    return cta_sum(v, red);
}

HQS_DEV void put_partial(double* part, double v, double* red) {
    const double t = cta_sum(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// z row iy into zs[0..n): IFFT_N of the preconditioner spectrum row / N^2,
// or the residual row when there is no preconditioner.
template <int N>
HQS_DEV void z_row(const FusedArgs& F, int iy, float2* s, const float2* twN, float2* zs) {
    const int n = F.A.n;
    if (!F.precond) {
        for (int ix = threadIdx.x; ix < n; ix += blockDim.x) zs[ix] = __ldcg(F.r + (int64_t)iy * n + ix);
        __syncthreads();
        return;
    }
    const float sc = 1.0f / ((float)N * (float)N);
    const float2* row = F.pcb + (int64_t)iy * N;
    __syncthreads();
    block_fft_io<N, true, false, false>(
        s, 1, twN, [&](int, int pos, bool) { return __ldcg(row + pos); }, NoIO{},
        [&](int, int pos, float2 v) { zs[pos] = cscale(v, sc); });
    __syncthreads();
    (void)n;
}

// Row block [r0, r0+Q): optional CG update, ||r||^2, FFT of the r rows -> pcb.
template <int N, int BD>
HQS_DEV double update_rows(const FusedArgs& F, int r0, float alpha, bool update, float2* s,
                           const float2* twN) {
    constexpr int n = N;
    const int lines = min(F.Q, n - r0);
    double rr = 0.0;
    auto body = [&](int e) {
        const int q_ = e / n, ix = e - q_ * n;
        const int64_t idx = (int64_t)(r0 + q_) * n + ix;
        float2 rv = __ldcg(F.r + idx);
        if (update) {
            const float2 pv = __ldcg(F.p + idx), qv = __ldcg(F.q + idx);
            float2 xv = __ldcg(F.x + idx);
            xv.x = fmaf(alpha, pv.x, xv.x);
            xv.y = fmaf(alpha, pv.y, xv.y);
            rv.x = fmaf(-alpha, qv.x, rv.x);
            rv.y = fmaf(-alpha, qv.y, rv.y);
            F.x[idx] = xv;
            F.r[idx] = rv;
        }
        rr += (double)rv.x * rv.x + (double)rv.y * rv.y;
        if (F.precond) s[ix * kLines + q_] = rv;
    };
    if (lines == kLines) {
        unrolled<kLines * N / BD, BD>(threadIdx.x, body);
    } else {
        for (int e = threadIdx.x; e < lines * n; e += blockDim.x) body(e);
    }
    if (F.precond) {
        // row FFTs, the last stage stores the spectra straight to pcb
        __syncthreads();
        block_fft_io<N, false, false, false>(
            s, lines, twN, NoIO{}, NoIO{},
            [&](int line, int pos, float2 v) { F.pcb[(int64_t)(r0 + line) * N + pos] = v; });
    }
    __syncthreads();
    return rr;
}

// Column block [c0, c0+Q) of the row spectra: FFT, * s^-1/2, partial of
// sum m |R|^2 (= N^2 <r, z>), IFFT; in place in pcb.
template <int N, int BD>
HQS_DEV double precond_cols(const FusedArgs& F, int c0, float2* s, const float2* twN) {
    const int lines = min(F.Q, N - c0);
    if (lines == kLines) {
        unrolled<kLines * N / BD, BD>(threadIdx.x, [&](int e) {
            s[e] = __ldcg(F.pcb + (int64_t)(e / kLines) * N + c0 + (e % kLines));
        });
    } else {
        for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
            const int pos = e / lines, q_ = e - pos * lines;
            s[pos * kLines + q_] = __ldcg(F.pcb + (int64_t)pos * N + c0 + q_);
        }
    }
    __syncthreads();
    block_fft<N, false>(s, lines, twN);
    double acc = 0.0;
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int pos = e / lines, q_ = e - pos * lines;
        const float l = F.lam[(int64_t)pos * N + c0 + q_];
        const float m = rsqrtf(fmaxf(fmaf(F.a, fmaxf(l, 0.f), F.b), 0.25f * F.b));
        const float2 v = s[pos * kLines + q_];
        acc += (double)(m * (v.x * v.x + v.y * v.y));
        s[pos * kLines + q_] = cscale(v, m);
    }
    __syncthreads();
    block_fft<N, true>(s, lines, twN);
    if (lines == kLines) {
        unrolled<kLines * N / BD, BD>(threadIdx.x, [&](int e) {
            F.pcb[(int64_t)(e / kLines) * N + c0 + (e % kLines)] = s[e];
        });
    } else {
        for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
            const int pos = e / lines, q_ = e - pos * lines;
            F.pcb[(int64_t)pos * N + c0 + q_] = s[pos * kLines + q_];
        }
    }
    __syncthreads();
    return acc;
}

template <int N2, int N> constexpr size_t fused_smem_floats2() {
    return (size_t)N2 * kLines + N + N2 + N + N;   // lines | row | tw N2 | tw N | z row
}

template <int N2, int N>
__global__ void __launch_bounds__(FftSize<N2>::TPL * kLines,
                                  (512 / (FftSize<N2>::TPL * kLines)) > 1 ? 512 / (FftSize<N2>::TPL * kLines) : 1)
    k_pcg_persistent(FusedArgs F) {
    extern __shared__ __align__(16) float2 s[];
    __shared__ double red[33];
    constexpr int BD = FftSize<N2>::TPL * kLines;   // == blockDim.x
    const ToepArgs& A = F.A;
    const int n = A.n, nch = A.nchunk;
    const int G = gridDim.x, bid = blockIdx.x;
    if (bid == F.skip_cta) return;   // test hook: the others' first barrier wait runs out
    const int count = n * n;
    const int npc = (n + F.Q - 1) / F.Q;
    float2* twN = s + (size_t)N2 * kLines + N + N2;
    float2* zs = twN + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) twN[i] = F.twN[i];
    double* P_PQ = F.part + SLOT_PQ * HQS_MAX_BLOCKS;
    double* P_RR = F.part + SLOT_RR * HQS_MAX_BLOCKS;
    double* P_BB = F.part + SLOT_BB * HQS_MAX_BLOCKS;
    double* P_RZ = F.part + SLOT_RZ * HQS_MAX_BLOCKS;
    const bool lead = bid == 0 && threadIdx.x == 0;
    int ntrace = 0;
    if (lead && F.trace && F.trace_max > 0) F.trace[ntrace++] = global_ns();
#define BARRIER()                                                            \
    do {                                                                     \
        if (!grid_barrier(F.bar, F.err, F.barrier_limit)) return;            \
        if (lead && F.trace && ntrace < F.trace_max) F.trace[ntrace++] = global_ns(); \
    } while (0)

    // ---- r = rhs - H x  (x = 0: r = rhs without an A^H A apply)
    if (!F.x0_zero) {
        for (int it = bid; it < n * nch; it += G) toep_rows_fwd_item<N2>(A, it % n, it / n, F.x, nullptr, 0.f, false, s);
        BARRIER();
        for (int it = bid; it < N2 * nch; it += G) toep_cols_item<N2>(A, it % N2, it / N2, s);
        BARRIER();
        for (int it = bid; it < n * nch; it += G) toep_rows_adj_item<N2>(A, it % n, it / n, F.q, F.x, F.a, F.b, 1, s);
        if (nch > 1) {
            BARRIER();
            double dummy = 0.0;
            for (int e = bid * blockDim.x + threadIdx.x; e < count; e += G * blockDim.x) {
                float2 v = make_float2(0.f, 0.f);
                for (int c = 0; c < nch; ++c) v = cadd(v, __ldcg(A.chunk + (int64_t)c * count + e));
                F.q[e] = toep_epilogue(v, e, F.x, F.a, F.b, 1, dummy);
            }
        }
        BARRIER();
    }
    {
        double rr = 0.0, bb = 0.0;
        for (int e = bid * blockDim.x + threadIdx.x; e < count; e += G * blockDim.x) {
            const float2 bv = F.rhs[e];
            float2 v = bv;
            if (F.x0_zero) F.x[e] = make_float2(0.f, 0.f);
            else v = csub(bv, __ldcg(F.q + e));
            F.r[e] = v;
            rr += (double)v.x * v.x + (double)v.y * v.y;
            bb += (double)bv.x * bv.x + (double)bv.y * bv.y;
        }
        put_partial(P_RR, rr, red);
        put_partial(P_BB, bb, red);
    }
    BARRIER();
    double rr = grid_total(P_RR, red);
    const double bb = grid_total(P_BB, red);
    const double tol2 = F.rel_tol2 * bb;
    int status = HQS_OK, zero_rhs = 0, done = 0, it = 0;
    if (lead) F.hist[0] = rr;
    if (!(bb == bb) || !(rr == rr) || isinf(bb) || isinf(rr)) {
        status = HQS_ERR_BREAKDOWN;
        done = 1;
    } else if (bb == 0.0) {
        zero_rhs = 1;
        done = 1;
        rr = 0.0;
        if (lead) F.hist[0] = 0.0;
        for (int e = bid * blockDim.x + threadIdx.x; e < count; e += G * blockDim.x) F.x[e] = make_float2(0.f, 0.f);
    } else if (rr <= tol2 || F.max_iter == 0) {
        done = 1;
        if (rr > tol2 && tol2 > 0.0) status = HQS_ERR_NOT_CONVERGED;
    }
    double rz = rr, alpha = 0.0, beta = 0.0;
    if (!done && F.precond) {
        for (int ib = bid; ib < npc; ib += G) update_rows<N, BD>(F, ib * F.Q, 0.f, false, s, twN);
        BARRIER();
        double acc = 0.0;
        for (int ib = bid; ib < npc; ib += G) acc += precond_cols<N, BD>(F, ib * F.Q, s, twN);
        put_partial(P_RZ, acc, red);
        BARRIER();
        rz = grid_total(P_RZ, red) / ((double)N * N);
        if (!(rz > 0.0) || isinf(rz)) {
            status = HQS_ERR_BREAKDOWN;
            done = 1;
        }
    }
    while (!done) {
        // A: p = z + beta p, S_l p, FFT rows
        const float fb = (float)beta;
        if (nch == 1) {
            for (int iy = bid; iy < n; iy += G) {
                z_row<N>(F, iy, s, twN, zs);
                toep_rows_fwd_item<N2>(A, iy, 0, nullptr, F.p, fb, true, s, zs);
            }
        } else {
            for (int iy = bid; iy < n; iy += G) {
                z_row<N>(F, iy, s, twN, zs);
                for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                    const int64_t e = (int64_t)iy * n + ix;
                    float2 v = zs[ix];
                    if (fb != 0.f) {
                        const float2 pv = __ldcg(F.p + e);
                        v.x = fmaf(fb, pv.x, v.x);
                        v.y = fmaf(fb, pv.y, v.y);
                    }
                    F.p[e] = v;
                }
                __syncthreads();
            }
            BARRIER();
            for (int w = bid; w < n * nch; w += G) toep_rows_fwd_item<N2>(A, w % n, w / n, F.p, nullptr, 0.f, false, s);
        }
        BARRIER();
        // B: columns
        for (int w = bid; w < N2 * nch; w += G) toep_cols_item<N2>(A, w % N2, w / N2, s);
        BARRIER();
        // C: q = a A^H A p + b p, <p, q>
        double pq = 0.0;
        for (int w = bid; w < n * nch; w += G) pq += toep_rows_adj_item<N2>(A, w % n, w / n, F.q, F.p, F.a, F.b, 1, s);
        if (nch > 1) {
            BARRIER();
            pq = 0.0;
            for (int e = bid * blockDim.x + threadIdx.x; e < count; e += G * blockDim.x) {
                float2 v = make_float2(0.f, 0.f);
                for (int c = 0; c < nch; ++c) v = cadd(v, __ldcg(A.chunk + (int64_t)c * count + e));
                F.q[e] = toep_epilogue(v, e, F.p, F.a, F.b, 1, pq);
            }
        }
        put_partial(P_PQ, pq, red);
        BARRIER();
        const double pqt = grid_total(P_PQ, red);
        if (!(pqt > 0.0) || isinf(pqt)) {
            status = HQS_ERR_BREAKDOWN;
            break;
        }
        alpha = rz / pqt;
        // D: x, r update, ||r||^2, row FFTs of r
        double racc = 0.0;
        for (int ib = bid; ib < npc; ib += G) racc += update_rows<N, BD>(F, ib * F.Q, (float)alpha, true, s, twN);
        put_partial(P_RR, racc, red);
        BARRIER();
        rr = grid_total(P_RR, red);
        ++it;
        if (lead) F.hist[it] = rr;
        if (!(rr == rr) || isinf(rr)) {
            status = HQS_ERR_BREAKDOWN;
            break;
        }
        if (rr <= tol2) break;
        if (it >= F.max_iter) {
            if (tol2 > 0.0) status = HQS_ERR_NOT_CONVERGED;
            break;
        }
        // E: preconditioner columns, <r, z>
        double rz_new = rr;
        if (F.precond) {
            double acc = 0.0;
            for (int ib = bid; ib < npc; ib += G) acc += precond_cols<N, BD>(F, ib * F.Q, s, twN);
            put_partial(P_RZ, acc, red);
            BARRIER();
            rz_new = grid_total(P_RZ, red) / ((double)N * N);
        }
        if (!(rz_new > 0.0) || isinf(rz_new)) {
            status = HQS_ERR_BREAKDOWN;
            break;
        }
        beta = rz_new / rz;
        rz = rz_new;
    }
#undef BARRIER
    if (lead) {
        CgScalars* c = F.cg;
        c->rz = rz;
        c->alpha = alpha;
        c->beta = beta;
        c->bnorm = sqrt(bb);
        c->rr = rr;
        c->tol2 = tol2;
        c->it = it;
        c->done = 1;
        c->status = status;
        c->zero_rhs = zero_rhs;
        c->max_iter = F.max_iter;
        c->fallback = 0;
        if (F.trace && ntrace < F.trace_max) F.trace[ntrace++] = global_ns();
        if (F.trace) F.trace[F.trace_max] = ntrace;
    }
}

template <int N2, int N>
static int pcg_fused_impl(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter,
                          double rel_tol, int precond, bool x0_zero, cudaStream_t st) {
    FusedArgs F;
    F.A = toep_args(p);
    F.a = a;
    F.b = b;
    F.rhs = rhs;
    F.x = x;
    F.r = p->cg_r;
    F.p = p->cg_p;
    F.q = p->cg_q;
    F.pcb = p->pc_buf;
    F.lam = p->lam;
    F.twN = plan_twiddles(p, N);
    F.Q = std::max(1, std::min(p->pc_lines, kLines));
    F.precond = precond == HQS_PRECOND_DC ? 1 : 0;
    F.x0_zero = x0_zero ? 1 : 0;
    F.max_iter = max_iter;
    F.rel_tol2 = rel_tol * rel_tol;
    F.part = p->partials;
    F.cg = p->cg;
    F.hist = p->hist;
    F.bar = p->barrier;
    F.err = p->dev_err;
    F.trace = p->trace;
    F.trace_max = p->trace ? HQS_TRACE_MAX : 0;
    auto kern = k_pcg_persistent<N2, N>;
    const int threads = FftSize<N2>::TPL * kLines;
    const size_t sm = fused_smem_floats2<N2, N>() * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, nsm = 0, dev = 0;
    HQS_CUDA_TRY(cudaGetDevice(&dev));
    HQS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm));
    if (per_sm < 1) return HQS_ERR_UNSUPPORTED;
    int grid = std::min(per_sm * nsm, N2 * p->nchunk);
    grid = std::min(grid, HQS_MAX_BLOCKS);
    if (p->fused_grid > 0) grid = std::min(grid, p->fused_grid);
    // test hook (one-shot): the last CTA leaves at once and the waits are cut to
    // about 10 ms, so the solve ends with HQS_ERR_TIMEOUT instead of a result
    F.skip_cta = p->debug_barrier_skip ? grid - 1 : -1;
    F.barrier_limit = p->debug_barrier_skip ? 20000000ll : HQS_BARRIER_LIMIT_CYCLES;
    p->debug_barrier_skip = 0;
    HQS_CUDA_TRY(cudaMemsetAsync(p->barrier, 0, 2 * sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaMemsetAsync(p->dev_err, 0, sizeof(unsigned), st));
    void* args[] = {&F};
    HQS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, sm, st));
    return HQS_OK;
}

int pcg_fused(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter, double rel_tol,
              int precond, int precision, bool x0_zero, cudaStream_t st) {
    if (precision != HQS_PREC_FP32) return HQS_ERR_UNSUPPORTED;
    switch (p->n) {
        case 16: return pcg_fused_impl<32, 16>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 32: return pcg_fused_impl<64, 32>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 64: return pcg_fused_impl<128, 64>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 128: return pcg_fused_impl<256, 128>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 256: return pcg_fused_impl<512, 256>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 320: return pcg_fused_impl<640, 320>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        case 384: return pcg_fused_impl<768, 384>(p, a, b, rhs, x, max_iter, rel_tol, precond, x0_zero, st);
        default: return HQS_ERR_INVALID_ARG;
    }
}

extern "C" int hqs_debug_phase_trace(hqs_plan p, int enable, unsigned long long* out, int max_out,
                                     void* stream) {
    if (!p) return HQS_ERR_INVALID_ARG;
    if (enable && !p->trace) {
        HQS_CUDA_TRY(cudaMalloc(&p->trace, (HQS_TRACE_MAX + 1) * sizeof(unsigned long long)));
        HQS_CUDA_TRY(cudaMemset(p->trace, 0, (HQS_TRACE_MAX + 1) * sizeof(unsigned long long)));
        return 0;
    }
    if (!p->trace) return 0;
    unsigned long long h[HQS_TRACE_MAX + 1];
    HQS_CUDA_TRY(cudaMemcpyAsync(h, p->trace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    HQS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const int cnt = (int)std::min<unsigned long long>(h[HQS_TRACE_MAX], HQS_TRACE_MAX);
    if (out)
        for (int i = 0; i < cnt && i < max_out; ++i) out[i] = h[i];
    return cnt;
}

extern "C" int hqs_plan_set_tuning(hqs_plan p, int key, int value) {
    if (!p) return HQS_ERR_INVALID_ARG;
    switch (key) {
        case HQS_TUNE_FUSED_GRID:
            if (value < 0) return HQS_ERR_INVALID_ARG;
            p->fused_grid = value;
            return HQS_OK;
        case HQS_TUNE_PC_LINES:
            if (value < 1 || value > kLines) return HQS_ERR_INVALID_ARG;
            p->pc_lines = value;
            return HQS_OK;
        case HQS_TUNE_SPREAD_TILE:
            return hqs_plan_retile(p, value, nullptr);
        case HQS_TUNE_DEBUG_BARRIER_SKIP:
            if (value != 0 && value != 1) return HQS_ERR_INVALID_ARG;
            p->debug_barrier_skip = value;
            return HQS_OK;
        default:
            return HQS_ERR_INVALID_ARG;
    }
}
