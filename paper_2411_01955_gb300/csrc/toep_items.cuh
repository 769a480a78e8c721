// Device bodies of the three A^H A passes, shared by the per-stage kernels
// and the persistent solver.
#pragma once

#include "fft.cuh"
#include "solve.cuh"

namespace hqs {

// ------------------------------------------------------------ A^H A passes
// Each CTA handles one row/column for the coils of chunk `ch` (<= 16 coils);
// the FFT body must not sit inside a runtime loop (register allocation
// collapses), so coil chunks are a grid dimension.

// Shared memory of the A^H A passes: [N2][kLines] lines | [n] image row |
// [N2] twiddles.
template <int N2> constexpr size_t toep_smem_floats2(int n) { return (size_t)N2 * kLines + n + N2; }

// P1: v = src (or p = src + beta p when fused, single chunk only), S_l v,
// zero-pad to N2, FFT along x.
// src_row, when given, is the row already in shared memory (the persistent
// solver rebuilds z there); otherwise the row is read from src.  tws, when given,
// holds the 2n-point twiddles already staged in shared memory (else this item
// stages them after the image row).  Vectors
// written by other CTAs earlier in the same launch are read with ld.global.cg
// (L2), never from a possibly stale L1 line.
template <int N2, int BD = FftSize<N2>::TPL * kLines>
HQS_DEV void toep_rows_fwd_item(const ToepArgs& A, int iy, int ch, const float2* __restrict__ src,
                                float2* __restrict__ pvec, float beta, bool fuse, float2* s,
                                const float2* src_row = nullptr, const float2* tws = nullptr) {
    const int n = A.n, L = A.L;
    float2* rowv = s + N2 * kLines;
    const float2* tw = tws ? tws : stage_twiddles<N2>(rowv + n, A.tw);
    for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
        const int64_t e = (int64_t)iy * n + ix;
        float2 v = src_row ? src_row[ix] : __ldcg(src + e);
        if (fuse) {
            if (beta != 0.f) {
                const float2 pv = __ldcg(pvec + e);
                v.x = fmaf(beta, pv.x, v.x);
                v.y = fmaf(beta, pv.y, v.y);
            }
            pvec[e] = v;
        }
        rowv[ix] = v;
    }
    const int l0 = ch * A.LC;
    const int lines = min(A.LC, L - l0);
    const float2* sm = A.smaps + (int64_t)iy * n * L + l0;
    float2* dst = A.T + (int64_t)iy * N2 * L + l0;
    __syncthreads();
    // S_l v straight into the first radix stage (upper half is the zero
    // padding), last stage straight to T
    block_fft_io<N2, false, true, false>(
        s, lines, tw, [&](int line, int p, bool) { return cmul(sm[(int64_t)p * L + line], rowv[p]); }, NoIO{},
        [&](int line, int p, float2 v) { dst[(int64_t)p * L + line] = v; });
    __syncthreads();
}

// P2: column kx: zero-pad, FFT along y, * Khat, IFFT, keep the first n rows.
template <int N2, int BD = FftSize<N2>::TPL * kLines>
HQS_DEV void toep_cols_item(const ToepArgs& A, int kx, int ch, float2* s, const float2* tws = nullptr) {
    const int n = A.n, L = A.L;
    const float2* tw = tws ? tws : stage_twiddles<N2>(s + N2 * kLines + n, A.tw);
    const int l0 = ch * A.LC;
    const int lines = min(A.LC, L - l0);
    float2* col = A.T + (int64_t)kx * L + l0;
    const int64_t rs = (int64_t)N2 * L;
    const float* kh = A.khat + (int64_t)kx * N2;   // Khat stored transposed: column kx contiguous
    // the column of Khat (N2 floats) goes to the image-row region asynchronously while
    // the forward stages run; the pair's middle stage waits for it before its barrier
    float* khs = reinterpret_cast<float*>(s + N2 * kLines);
    for (int c = threadIdx.x; c < N2 / 4; c += blockDim.x) cp_async16(khs + 4 * c, kh + 4 * c);
    __syncthreads();
    // column straight into the first stage (zero-padded upper half), * Khat between
    // the last forward and the first inverse stage (on registers), IFFT, first n rows
    // straight back to T
    block_fft_pair<N2, true, true>(
        s, lines, tw, [&](int line, int p, bool) { return __ldcg(col + line + p * rs); },
        [&](int, int p, float2 v) { return cscale(v, khs[p]); },
        [&](int line, int p, float2 v) { col[line + p * rs] = v; });
    __syncthreads();
}

// P2 over nl consecutive (column, coil) lines of the flattened index f = kx L + l
// (f0 .. f0 + nl - 1, nl <= kLines): the data of line f at position p is
// T[f + p N2 L], so an item's lines are contiguous whichever columns they belong
// to, and chunks of fewer than kLines coils need not leave threads idle.  Khat of
// the item's first column is staged with cp.async; a line of a later column reads
// its Khat through L1.
template <int N2, int BD = FftSize<N2>::TPL * kLines>
HQS_DEV void toep_cols_flat_item(const ToepArgs& A, int f0, int nl, float2* s, const float2* tws = nullptr) {
    const int n = A.n, L = A.L;
    const float2* tw = tws ? tws : stage_twiddles<N2>(s + N2 * kLines + n, A.tw);
    float2* col = A.T + f0;
    const int64_t rs = (int64_t)N2 * L;
    const int kx0 = f0 / L;
    const float* kh0 = A.khat + (int64_t)kx0 * N2;
    const float* khat = A.khat;
    float* khs = reinterpret_cast<float*>(s + N2 * kLines);
    for (int c = threadIdx.x; c < N2 / 4; c += blockDim.x) cp_async16(khs + 4 * c, kh0 + 4 * c);
    __syncthreads();
    block_fft_pair<N2, true, true>(
        s, nl, tw, [&](int line, int p, bool) { return __ldcg(col + line + p * rs); },
        [&](int line, int p, float2 v) {
            const int kx = (f0 + line) / L;
            return cscale(v, kx == kx0 ? khs[p] : __ldg(khat + (int64_t)kx * N2 + p));
        },
        [&](int line, int p, float2 v) { col[line + p * rs] = v; });
    __syncthreads();
}

// CG epilogue on one pixel: mode 0 returns v = A^H A p; mode 1 returns
// q = a v + b p and adds Re<p, q> to part.
HQS_DEV float2 toep_epilogue_pv(float2 v, float2 pv, float a, float b, double& part) {
    v = make_float2(fmaf(a, v.x, b * pv.x), fmaf(a, v.y, b * pv.y));
    part += (double)pv.x * v.x + (double)pv.y * v.y;
    return v;
}
HQS_DEV float2 toep_epilogue(float2 v, int64_t e, const float2* __restrict__ pvec, float a, float b,
                             int mode, double& part) {
    if (mode == 1) v = toep_epilogue_pv(v, __ldcg(pvec + e), a, b, part);
    return v;
}

// P3: row iy: IFFT along x, keep n, sum_l conj(S_l) . over the chunk's coils.
// One chunk: epilogue and store here (returns the thread's partial); several
// chunks: the raw chunk sum goes to A.chunk[ch] for k_toep_chunk_epilogue.
template <int N2, int BD = FftSize<N2>::TPL * kLines>
HQS_DEV double toep_rows_adj_item(const ToepArgs& A, int iy, int ch, float2* __restrict__ out,
                                  const float2* __restrict__ pvec, float a, float b, int mode,
                                  float2* s, const float2* tws = nullptr) {
    const int n = A.n, L = A.L;
    const float2* tw = tws ? tws : stage_twiddles<N2>(s + N2 * kLines + n, A.tw);
    const int l0 = ch * A.LC;
    const int lines = min(A.LC, L - l0);
    const float2* src = A.T + (int64_t)iy * N2 * L + l0;
    const float2* sm = A.smaps + (int64_t)iy * n * L + l0;
    // Maps in 16-byte pieces (an even number of coils at an even offset): the row's
    // maps of the chunk go with cp.async to the upper half of the lines buffer
    // ([n][kLines], `lines` used per pixel) once the last stage has read it (that
    // stage writes the lower half only), issued by the stage's active threads, so
    // their latency overlaps the stage; with one chunk and mode 1 the row of pvec
    // (when 16-byte aligned) goes to the image-row region at the start.  Callers
    // declare the dynamic shared memory 16-byte aligned.
    constexpr int TPL = FftSize<N2>::TPL;
    const bool pre_m = (lines % 2) == 0 && (L % 2) == 0 && (l0 % 2) == 0;
    const bool pre_p = mode == 1 && A.nchunk == 1 && ((uintptr_t)pvec & 15u) == 0;
    float2* msm = s + (int64_t)n * kLines;   // upper half: [n][kLines]
    float2* prow = s + N2 * kLines;          // image-row region: [n]
    if (pre_p)
        for (int c = threadIdx.x; c < n / 2; c += blockDim.x) cp_async16(prow + 2 * c, pvec + (int64_t)iy * n + 2 * c);
    bool issued = false;
    __syncthreads();
    // row straight from T into the first stage; only the first n columns are kept
    block_fft_io<N2, true, false, true>(
        s, lines, tw, [&](int line, int p, bool) { return __ldcg(src + (int64_t)p * L + line); },
        [&](int line, int, float2 v) {
            if (pre_m && !issued) {
                issued = true;
                // active threads: (line < lines, t < TPL), numbered t * lines + line
                const int me = (int)(threadIdx.x / (blockDim.x / TPL)) * lines + line;
                const int per = lines / 2;
                for (int e = me; e < n * per; e += lines * TPL) {
                    const int ix = e / per, h = e - ix * per;
                    cp_async16(msm + ix * kLines + 2 * h, sm + (int64_t)ix * L + 2 * h);
                }
            }
            return v;
        },
        NoIO{});
    if (pre_m || pre_p) {
        cp_async_wait_all();
        __syncthreads();
    }
    double part = 0.0;
    for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        const float2* smx = pre_m ? msm + ix * kLines : sm + (int64_t)ix * L;
        if (pre_m && lines == kLines) {
            // a full chunk of 16 coils is 128 contiguous, 16-byte aligned bytes
            const float4* s4 = reinterpret_cast<const float4*>(msm + ix * kLines);
            float4 sv4[kLines / 2];
#pragma unroll
            for (int h = 0; h < kLines / 2; ++h) sv4[h] = s4[h];
#pragma unroll
            for (int h = 0; h < kLines / 2; ++h) {
                const float2 g0 = s[ix * kLines + 2 * h], g1 = s[ix * kLines + 2 * h + 1];
                acc.x += sv4[h].x * g0.x + sv4[h].y * g0.y + sv4[h].z * g1.x + sv4[h].w * g1.y;
                acc.y += sv4[h].x * g0.y - sv4[h].y * g0.x + sv4[h].z * g1.y - sv4[h].w * g1.x;
            }
        } else {
            for (int ll = 0; ll < lines; ++ll) {
                const float2 sv = smx[ll];
                const float2 g = s[ix * kLines + ll];
                acc.x += sv.x * g.x + sv.y * g.y;
                acc.y += sv.x * g.y - sv.y * g.x;
            }
        }
        const int64_t e = (int64_t)iy * n + ix;
        if (A.nchunk == 1)
            out[e] = pre_p ? toep_epilogue_pv(acc, prow[ix], a, b, part) : toep_epilogue(acc, e, pvec, a, b, mode, part);
        else
            A.chunk[(int64_t)ch * n * n + e] = acc;
    }
    __syncthreads();
    return part;
}

HQS_DEV double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}


}  // namespace hqs
