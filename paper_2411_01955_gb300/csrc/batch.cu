// Batched annealed PnP-HQS over slices of uneven size (a9): one persistent
// cooperative launch runs, for every slice s and outer iteration k
// (Sec. 3.3, the prox in the metric P = c0 I + c1 A^H A of Sec. 3.4),
//   u = x_k;  rhs = A^H y + mu_k (c0 x_k + c1 A^H A x_k);  cg_iters DC-
//   preconditioned CG iterations on ((1 + c1 mu_k) A^H A + c0 mu_k I) u = rhs
//   from u;  x_{k+1} = G_{s_k} u
// with the Gaussian-smoothing denoiser of std s_k = kappa sigma_k / sigma_0.
// The CG start u = x_k needs A^H A x_k anyway (for H u), so the c1 term of the
// right-hand side costs no extra operator apply.
// The work items of all slices (rows, columns, preconditioner row blocks,
// denoiser tiles) are dealt to the CTAs together in every phase, so slices of
// 256^2, 320^2 and 384^2 with 8-20 coils share the GPU without per-slice
// launches.  Every CTA reduces the per-slice partials in the same fixed order,
// so the per-slice scalars agree everywhere.  hqs_batch_run records the
// per-slice adjoints (A^H y) and the persistent kernel into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "persist.cuh"
#include "plan.cuh"
#include "solve.cuh"
#include "toep_items.cuh"

using namespace hqs;

#define HQS_BATCH_MAX 64
#define HQS_BATCH_BD 256
#define HQS_BATCH_MAXR 24

namespace {

enum BatchSlot { BS_PQ = 0, BS_RR = 1, BS_BB = 2, BS_RZ = 3, BS_N = 4 };
enum BatchList { BL_ROWS = 0, BL_COLS = 1, BL_PC = 2, BL_IMG = 3, BL_BLUR = 4, BL_EPI = 5, BL_ZP = 6, BL_N = 7 };

struct BatchSlice {
    ToepArgs A;
    int colcap;   // > 0: column items of colcap flattened (column, coil) lines; 0: one column per chunk
    const float2* twN;
    const float* lam;
    const float2* b0;
    float2* x;
    float2* u;
    float2* rhs;
    float2* r;
    float2* p;
    float2* q;
    float2* pcb;
};

struct BatchArgs {
    const BatchSlice* sl;
    int ns;
    const int* off;      // [BL_N][ns + 1] prefix item counts
    int K, k0, cg_iters;
    float c0, c1;
    const float* mu;     // [K]
    const float* taps;   // [K][2 MAXR + 1], normalised
    const int* radius;   // [K], -1: identity
    double* part;        // [BS_N][ns][gridDim]
    double* res;         // [ns] final ||r||^2 / ||rhs||^2 of the last DC step
    unsigned* bar;
    unsigned* err;
};

HQS_DEV int find_slice(const int* off, int ns, int g) {
    int s = 0;
    while (s + 1 < ns && off[s + 1] <= g) ++s;
    return s;
}

// per-slice totals of a slot, identical in every CTA (fixed order)
HQS_DEV void slice_totals(const double* part, int ns, double* out) {
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        double v = 0.0;
        for (int c = lane; c < G; c += 32) v += __ldcg(part + (size_t)s * G + c);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) out[s] = v;
    }
    __syncthreads();
}

HQS_DEV void put_slice_partials(double* part, int ns, const double* acc) {
    for (int s = threadIdx.x; s < ns; s += blockDim.x) part[(size_t)s * gridDim.x + blockIdx.x] = acc[s];
}

// ---- per-size item bodies (BD = HQS_BATCH_BD)
// z rows per item in the p-update phase: as many n-point lines as the CTA holds
// (up to 2 kLines: 32 lines of 320 points fill the 256 threads, so the 16 slices'
// items of this phase fit in one round of the grid)
template <int N> constexpr int batch_zq() {
    return (HQS_BATCH_BD / FftSize<N>::TPL) < 2 * kLines ? HQS_BATCH_BD / FftSize<N>::TPL : 2 * kLines;
}

// rows [r0, r0 + lines): z = IFFT_N(pc spectrum rows) / N^2, p = z + beta p
template <int N2, int N>
HQS_DEV void z_and_p_rows(const BatchSlice& S, int r0, float beta, bool first, float2* s, const float2* twN) {
    constexpr int n = N;
    const int lines = min(batch_zq<N>(), n - r0);
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
        const int q = e / N, pos = e - q * N;
        s[line_elem<N>(pos, q)] = __ldcg(S.pcb + (size_t)(r0 + q) * N + pos);
    }
    __syncthreads();
    block_fft<N, true, false, false, true>(s, lines, twN);
    const float sc = 1.0f / ((float)N * (float)N);
    for (int e2 = threadIdx.x; e2 < lines * n; e2 += blockDim.x) {
        const int q = e2 / n, ix = e2 - q * n;
        const size_t e = (size_t)(r0 + q) * n + ix;
        float2 v = cscale(s[line_elem<N>(ix, q)], sc);
        if (!first && beta != 0.f) {
            const float2 pv = __ldcg(S.p + e);
            v.x = fmaf(beta, pv.x, v.x);
            v.y = fmaf(beta, pv.y, v.y);
        }
        S.p[e] = v;
    }
    __syncthreads();
}

// preconditioner lines per item: as many n-point lines as the CTA holds (<= 2 kLines)
template <int N> constexpr int batch_pq() {
    return (HQS_BATCH_BD / FftSize<N>::TPL) < 2 * kLines ? HQS_BATCH_BD / FftSize<N>::TPL : 2 * kLines;
}

template <int N>
HQS_DEV double pc_rows(const BatchSlice& S, int r0, float alpha, bool update, float2* s, const float2* twN) {
    const int lines = min(batch_pq<N>(), N - r0);
    double rr = 0.0;
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
        const int q_ = e / N, ix = e - q_ * N;
        const size_t idx = (size_t)(r0 + q_) * N + ix;
        float2 rv = __ldcg(S.r + idx);
        if (update) {
            const float2 pv = __ldcg(S.p + idx), qv = __ldcg(S.q + idx);
            float2 uv = __ldcg(S.u + idx);
            uv.x = fmaf(alpha, pv.x, uv.x);
            uv.y = fmaf(alpha, pv.y, uv.y);
            rv.x = fmaf(-alpha, qv.x, rv.x);
            rv.y = fmaf(-alpha, qv.y, rv.y);
            S.u[idx] = uv;
            S.r[idx] = rv;
        }
        rr += (double)rv.x * rv.x + (double)rv.y * rv.y;
        s[line_elem<N>(ix, q_)] = rv;
    }
    __syncthreads();
    block_fft<N, false, false, false, true>(s, lines, twN);
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
        const int q_ = e / N, pos = e - q_ * N;
        S.pcb[(size_t)(r0 + q_) * N + pos] = s[line_elem<N>(pos, q_)];
    }
    __syncthreads();
    return rr;
}

template <int N>
HQS_DEV double pc_cols(const BatchSlice& S, int c0, float a, float b, float2* s, const float2* twN) {
    const int lines = min(batch_pq<N>(), N - c0);
    // column FFT, * s^-1/2 (accumulating <r, z> = sum s^-1/2 |r_hat|^2), column IFFT as
    // one forward x factor x inverse pair, loads and stores straight from / to pcb
    double acc = 0.0;
    float2* col = S.pcb + c0;
    const float* lcol = S.lam + c0;
    block_fft_pair<N, false, false, true>(
        s, lines, twN, [&](int line, int pos, bool) { return __ldcg(col + (size_t)pos * N + line); },
        [&](int line, int pos, float2 v) {
            const float l = __ldg(lcol + (size_t)pos * N + line);
            const float m = rsqrtf(fmaxf(fmaf(a, fmaxf(l, 0.f), b), 0.25f * b));
            acc += (double)(m * (v.x * v.x + v.y * v.y));
            return cscale(v, m);
        },
        [&](int line, int pos, float2 v) { col[(size_t)pos * N + line] = v; });
    __syncthreads();
    return acc;
}

#define HQS_BATCH_DISPATCH(n, ...)                                         \
    switch (n) {                                                           \
        case 64: { constexpr int N2 = 128, N = 64; __VA_ARGS__; break; }   \
        case 128: { constexpr int N2 = 256, N = 128; __VA_ARGS__; break; } \
        case 256: { constexpr int N2 = 512, N = 256; __VA_ARGS__; break; } \
        case 320: { constexpr int N2 = 640, N = 320; __VA_ARGS__; break; } \
        default: { constexpr int N2 = 768, N = 384; __VA_ARGS__; break; }  \
    }

// Gaussian blur of one 32x32 tile of u into x (periodic), radius r >= 0
HQS_DEV void blur_tile(const BatchSlice& S, int tile, const float* g, int r, float2* sb) {
    const int n = S.A.n;
    const int tpr = (n + 31) / 32;
    const int y0 = (tile / tpr) * 32, x0 = (tile % tpr) * 32;
    const int E = 32 + 2 * r;
    float2* t = sb;
    float2* mid = sb + E * E;
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        const int ty = e / E, tx = e - ty * E;
        int gy = (y0 + ty - r) % n, gx = (x0 + tx - r) % n;
        if (gy < 0) gy += n;
        if (gx < 0) gx += n;
        t[e] = __ldcg(S.u + (size_t)gy * n + gx);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E * 32; e += blockDim.x) {
        const int ty = e / 32, tx = e - ty * 32;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i <= 2 * r; ++i) {
            const float2 v = t[ty * E + tx + i];
            acc.x = fmaf(g[i], v.x, acc.x);
            acc.y = fmaf(g[i], v.y, acc.y);
        }
        mid[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int ty = e / 32, tx = e - ty * 32;
        const int gy = y0 + ty, gx = x0 + tx;
        if (gy >= n || gx >= n) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i <= 2 * r; ++i) {
            const float2 v = mid[(ty + i) * 32 + tx];
            acc.x = fmaf(g[i], v.x, acc.x);
            acc.y = fmaf(g[i], v.y, acc.y);
        }
        S.x[(size_t)gy * n + gx] = acc;
    }
    __syncthreads();
}

// smem: lines buffer [768][16] | row [384] | tw 2n [768]; the n-point twiddles
// of the preconditioner FFTs are read from global memory (L1), which keeps two
// CTAs resident per SM.
constexpr size_t kBatchSmemF2 = (size_t)768 * kLines + 384 + 768;
// the preconditioner items' lines (up to 2 kLines per item) fit the lines buffer
static_assert(2 * 64 * kLines <= 768 * kLines && 2 * 320 * kLines <= 768 * kLines &&
                  batch_pq<384>() <= kLines && batch_pq<128>() <= kLines && batch_pq<256>() <= kLines,
              "preconditioner items exceed the lines buffer");

__global__ void __launch_bounds__(HQS_BATCH_BD, 2) k_hqs_batch(BatchArgs B) {
    extern __shared__ __align__(16) float2 s[];
    __shared__ double red[33];
    __shared__ double acc[2][HQS_BATCH_MAX];
    __shared__ double tot[2][HQS_BATCH_MAX];
    __shared__ double rzs[HQS_BATCH_MAX], alphas[HQS_BATCH_MAX], betas[HQS_BATCH_MAX];
    __shared__ int sl_cache, tw_cur;
    const int ns = B.ns, G = gridDim.x, bid = blockIdx.x;
    const float2* twN = nullptr;   // n-point twiddles of the current slice (global)
    // the 2n-point twiddles of the Toeplitz items stay in the shared region after the
    // largest lines buffer and its image row (the blur and preconditioner items use
    // less than the lines buffer), restaged only when the slice size changes
    float2* twT = s + (size_t)768 * kLines + 384;
    if (threadIdx.x == 0) tw_cur = 0;
#define STAGE_TW2(AA)                                                                    \
    if (tw_cur != 2 * (AA).n) {                                                          \
        __syncthreads();                                                                 \
        for (int i_ = threadIdx.x; i_ < 2 * (AA).n; i_ += blockDim.x) twT[i_] = (AA).tw[i_]; \
        __syncthreads();                                                                 \
        if (threadIdx.x == 0) tw_cur = 2 * (AA).n;                                       \
        __syncthreads();                                                                 \
    }
#define BB_BARRIER()                                \
    do {                                            \
        if (!grid_barrier(B.bar, B.err)) return;    \
    } while (0)
    // the chunk epilogue reads what the row-adjoint pass wrote: its barrier is needed
    // only when some slice has several coil chunks
    const bool has_epi = B.off[BL_EPI * (ns + 1) + ns] > 0;
#define EPI_BARRIER()                   \
    do {                                \
        if (has_epi) BB_BARRIER();      \
    } while (0)
#define FOR_ITEMS(list, ...)                                                               \
    {                                                                                      \
        const int* off_ = B.off + (list) * (ns + 1);                                       \
        for (int g_ = bid; g_ < off_[ns]; g_ += G) {                                       \
            const int si = find_slice(off_, ns, g_);                                       \
            const int it_ = g_ - off_[si];                                                 \
            const BatchSlice& S = B.sl[si];                                                \
            __VA_ARGS__;                                                                   \
        }                                                                                  \
    }
#define STAGE_TWN(S, si) twN = (S).twN;
#define CLEAR_ACC()                                                      \
    for (int i_ = threadIdx.x; i_ < 2 * HQS_BATCH_MAX; i_ += blockDim.x) \
        (&acc[0][0])[i_] = 0.0;                                          \
    __syncthreads();

    (void)sl_cache;
    for (int k = B.k0; k < B.K; ++k) {
        const float muk = B.mu[k];
        const float acoef = 1.0f + B.c1 * muk, bcoef = B.c0 * muk;
        // with c1 != 0 the first operator pass keeps v = A^H A u (epilogue mode 0);
        // the residual phase forms H u = a v + b u and the rhs term mu c1 v
        const int mode0 = B.c1 != 0.f ? 0 : 1;
        // PREP: u = x, rhs = A^H y + mu c0 x
        FOR_ITEMS(BL_IMG, {
            const int n = S.A.n;
            for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                const size_t e = (size_t)it_ * n + ix;
                const float2 xv = __ldcg(S.x + e), bv = S.b0[e];
                S.u[e] = xv;
                S.rhs[e] = make_float2(fmaf(bcoef, xv.x, bv.x), fmaf(bcoef, xv.y, bv.y));
            }
        });
        BB_BARRIER();
        // q = H u
        FOR_ITEMS(BL_ROWS, {
            const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
            STAGE_TW2(S.A);
            HQS_BATCH_DISPATCH(n, (toep_rows_fwd_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.u, nullptr, 0.f, false, s,
                                                                        nullptr, twT)));
        });
        BB_BARRIER();
        FOR_ITEMS(BL_COLS, {
            const int n = S.A.n, N2v = 2 * n, ch = it_ / N2v, kx = it_ - ch * N2v;
            STAGE_TW2(S.A);
            if (S.colcap > 0) {
                const int f0 = it_ * S.colcap, nl = min(S.colcap, N2v * S.A.L - f0);
                HQS_BATCH_DISPATCH(n, (toep_cols_flat_item<N2, HQS_BATCH_BD>(S.A, f0, nl, s, twT)));
            } else {
                HQS_BATCH_DISPATCH(n, (toep_cols_item<N2, HQS_BATCH_BD>(S.A, kx, ch, s, twT)));
            }
        });
        BB_BARRIER();
        FOR_ITEMS(BL_ROWS, {
            const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
            STAGE_TW2(S.A);
            HQS_BATCH_DISPATCH(n, (toep_rows_adj_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.q, S.u, acoef, bcoef, mode0, s,
                                                                        twT)));
        });
        EPI_BARRIER();
        FOR_ITEMS(BL_EPI, {   // several coil chunks: fixed-order chunk sum + epilogue
            const int n = S.A.n, cnt = n * n;
            for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                const size_t e = (size_t)it_ * n + ix;
                float2 v = make_float2(0.f, 0.f);
                for (int c = 0; c < S.A.nchunk; ++c) v = cadd(v, __ldcg(S.A.chunk + (size_t)c * cnt + e));
                double dummy = 0.0;
                S.q[e] = toep_epilogue(v, e, S.u, acoef, bcoef, mode0, dummy);
            }
        });
        BB_BARRIER();
        // r = rhs - q; ||r||^2, ||rhs||^2 per slice (c1 != 0: q holds v = A^H A u;
        // rhs += mu c1 v and q = a v + b u, in the epilogue's arithmetic)
        CLEAR_ACC();
        FOR_ITEMS(BL_IMG, {
            const int n = S.A.n;
            double a1 = 0.0, a2 = 0.0;
            for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                const size_t e = (size_t)it_ * n + ix;
                float2 bv = __ldcg(S.rhs + e);
                float2 qv = __ldcg(S.q + e);
                if (mode0 == 0) {
                    const float mc1 = muk * B.c1;
                    bv.x = fmaf(mc1, qv.x, bv.x);
                    bv.y = fmaf(mc1, qv.y, bv.y);
                    S.rhs[e] = bv;
                    double dummy = 0.0;
                    qv = toep_epilogue(qv, e, S.u, acoef, bcoef, 1, dummy);
                    S.q[e] = qv;
                }
                const float2 v = csub(bv, qv);
                S.r[e] = v;
                a1 += (double)v.x * v.x + (double)v.y * v.y;
                a2 += (double)bv.x * bv.x + (double)bv.y * bv.y;
            }
            a1 = cta_sum(a1, red);
            a2 = cta_sum(a2, red);
            if (threadIdx.x == 0) {
                acc[0][si] += a1;
                acc[1][si] += a2;
            }
        });
        __syncthreads();
        put_slice_partials(B.part + (size_t)BS_RR * ns * G, ns, acc[0]);
        put_slice_partials(B.part + (size_t)BS_BB * ns * G, ns, acc[1]);
        BB_BARRIER();
        slice_totals(B.part + (size_t)BS_BB * ns * G, ns, tot[1]);
        // preconditioner of the initial residual
        FOR_ITEMS(BL_PC, {
            STAGE_TWN(S, si);
            HQS_BATCH_DISPATCH(S.A.n, (pc_rows<N>(S, it_ * batch_pq<N>(), 0.f, false, s, twN)));
        });
        BB_BARRIER();
        CLEAR_ACC();
        FOR_ITEMS(BL_PC, {
            STAGE_TWN(S, si);
            double v = 0.0;
            HQS_BATCH_DISPATCH(S.A.n, (v = pc_cols<N>(S, it_ * batch_pq<N>(), acoef, bcoef, s, twN)));
            v = cta_sum(v, red);
            if (threadIdx.x == 0) acc[0][si] += v;
        });
        __syncthreads();
        put_slice_partials(B.part + (size_t)BS_RZ * ns * G, ns, acc[0]);
        BB_BARRIER();
        slice_totals(B.part + (size_t)BS_RZ * ns * G, ns, tot[0]);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const int n = B.sl[i].A.n;
            rzs[i] = tot[0][i] / ((double)n * n);
            betas[i] = 0.0;
        }
        __syncthreads();
        for (int cg = 0; cg < B.cg_iters; ++cg) {
            // A0: z rows and p = z + beta p
            FOR_ITEMS(BL_ZP, {
                STAGE_TWN(S, si);
                HQS_BATCH_DISPATCH(S.A.n, (z_and_p_rows<N2, N>(S, it_ * batch_zq<N>(), (float)betas[si], cg == 0, s, twN)));
            });
            BB_BARRIER();
            FOR_ITEMS(BL_ROWS, {
                const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
                STAGE_TW2(S.A);
                HQS_BATCH_DISPATCH(n, (toep_rows_fwd_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.p, nullptr, 0.f, false, s,
                                                                            nullptr, twT)));
            });
            BB_BARRIER();
            FOR_ITEMS(BL_COLS, {
                const int n = S.A.n, N2v = 2 * n, ch = it_ / N2v, kx = it_ - ch * N2v;
                STAGE_TW2(S.A);
                if (S.colcap > 0) {
                    const int f0 = it_ * S.colcap, nl = min(S.colcap, N2v * S.A.L - f0);
                    HQS_BATCH_DISPATCH(n, (toep_cols_flat_item<N2, HQS_BATCH_BD>(S.A, f0, nl, s, twT)));
                } else {
                    HQS_BATCH_DISPATCH(n, (toep_cols_item<N2, HQS_BATCH_BD>(S.A, kx, ch, s, twT)));
                }
            });
            BB_BARRIER();
            CLEAR_ACC();
            FOR_ITEMS(BL_ROWS, {
                const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
                double v = 0.0;
                STAGE_TW2(S.A);
                HQS_BATCH_DISPATCH(n, (v = toep_rows_adj_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.q, S.p, acoef, bcoef, 1, s,
                                                                                 twT)));
                v = cta_sum(v, red);
                if (threadIdx.x == 0) acc[0][si] += v;
            });
            EPI_BARRIER();
            FOR_ITEMS(BL_EPI, {
                const int n = S.A.n, cnt = n * n;
                double v = 0.0;
                for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                    const size_t e = (size_t)it_ * n + ix;
                    float2 w = make_float2(0.f, 0.f);
                    for (int c = 0; c < S.A.nchunk; ++c) w = cadd(w, __ldcg(S.A.chunk + (size_t)c * cnt + e));
                    S.q[e] = toep_epilogue(w, e, S.p, acoef, bcoef, 1, v);
                }
                v = cta_sum(v, red);
                if (threadIdx.x == 0) acc[0][si] += v;
            });
            __syncthreads();
            put_slice_partials(B.part + (size_t)BS_PQ * ns * G, ns, acc[0]);
            BB_BARRIER();
            slice_totals(B.part + (size_t)BS_PQ * ns * G, ns, tot[0]);
            for (int i = threadIdx.x; i < ns; i += blockDim.x) {
                const double pq = tot[0][i];
                alphas[i] = (pq > 0.0 && !isinf(pq)) ? rzs[i] / pq : 0.0;
            }
            __syncthreads();
            // D: u, r update, ||r||^2, row FFTs of r
            CLEAR_ACC();
            FOR_ITEMS(BL_PC, {
                STAGE_TWN(S, si);
                double v = 0.0;
                HQS_BATCH_DISPATCH(S.A.n, (v = pc_rows<N>(S, it_ * batch_pq<N>(), (float)alphas[si], true, s, twN)));
                v = cta_sum(v, red);
                if (threadIdx.x == 0) acc[1][si] += v;
            });
            __syncthreads();
            put_slice_partials(B.part + (size_t)BS_RR * ns * G, ns, acc[1]);
            BB_BARRIER();
            if (cg == B.cg_iters - 1) break;
            // E: preconditioner columns, <r, z>
            CLEAR_ACC();
            FOR_ITEMS(BL_PC, {
                STAGE_TWN(S, si);
                double v = 0.0;
                HQS_BATCH_DISPATCH(S.A.n, (v = pc_cols<N>(S, it_ * batch_pq<N>(), acoef, bcoef, s, twN)));
                v = cta_sum(v, red);
                if (threadIdx.x == 0) acc[0][si] += v;
            });
            __syncthreads();
            put_slice_partials(B.part + (size_t)BS_RZ * ns * G, ns, acc[0]);
            BB_BARRIER();
            slice_totals(B.part + (size_t)BS_RZ * ns * G, ns, tot[0]);
            for (int i = threadIdx.x; i < ns; i += blockDim.x) {
                const int n = B.sl[i].A.n;
                const double rz_new = tot[0][i] / ((double)n * n);
                betas[i] = rzs[i] > 0.0 ? rz_new / rzs[i] : 0.0;
                rzs[i] = rz_new;
            }
            __syncthreads();
        }
        if (k == B.K - 1) {
            slice_totals(B.part + (size_t)BS_RR * ns * G, ns, tot[0]);
            if (bid == 0)
                for (int i = threadIdx.x; i < ns; i += blockDim.x)
                    B.res[i] = tot[1][i] > 0.0 ? tot[0][i] / tot[1][i] : 0.0;
        }
        // denoiser: x = G(u)
        const int rk = B.radius[k];
        const float* gk = B.taps + (size_t)k * (2 * HQS_BATCH_MAXR + 1);
        FOR_ITEMS(BL_BLUR, {
            if (rk < 0) {
                const int n = S.A.n, tpr = (n + 31) / 32;
                const int y0 = (it_ / tpr) * 32, x0 = (it_ % tpr) * 32;
                for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
                    const int gy = y0 + e / 32, gx = x0 + e % 32;
                    if (gy < n && gx < n) S.x[(size_t)gy * n + gx] = __ldcg(S.u + (size_t)gy * n + gx);
                }
            } else {
                blur_tile(S, it_, gk, rk, s);
            }
        });
        BB_BARRIER();
    }
#undef BB_BARRIER
#undef EPI_BARRIER
#undef FOR_ITEMS
#undef STAGE_TWN
#undef STAGE_TW2
#undef CLEAR_ACC
}


// ---------------------------------------------------------------------------
// Batched data-consistency solve: DC-preconditioned CG on (a A^H A + b I) x =
// rhs for every slice from x = 0 to its own relative tolerance, in one
// cooperative launch (the same per-slice work items as the HQS kernel, so the
// phases of all slices share the GPU and one slice's phase tail is filled by
// the others' items).  A slice that converges (or breaks down) drops out of
// the item lists; every CTA takes the same decisions from the same totals.
struct DcBatchArgs {
    const BatchSlice* sl;   // u = caller's x, rhs = caller's right-hand side
    int ns;
    const int* off;
    float a, b;
    int max_iter;
    double tol2;            // rel_tol^2
    double* part;           // [BS_N][ns][gridDim]
    double* res;            // [ns] final ||r||^2 / ||rhs||^2
    int* iters;             // [ns]
    int* status;            // [ns] HQS_OK / HQS_ERR_NOT_CONVERGED / HQS_ERR_BREAKDOWN
    unsigned* bar;
    unsigned* err;
    unsigned long long* trace;   // optional: globaltimer stamp at the start, after each grid barrier, at the end
    int trace_max;
};

__global__ void __launch_bounds__(HQS_BATCH_BD, 2) k_pcg_batch(DcBatchArgs B) {
    extern __shared__ __align__(16) float2 s[];
    __shared__ double red[33];
    __shared__ double acc[2][HQS_BATCH_MAX];
    __shared__ double tot[2][HQS_BATCH_MAX];
    __shared__ double rzs[HQS_BATCH_MAX], alphas[HQS_BATCH_MAX], betas[HQS_BATCH_MAX];
    __shared__ double bbs[HQS_BATCH_MAX], rrs[HQS_BATCH_MAX];
    __shared__ int active[HQS_BATCH_MAX], its[HQS_BATCH_MAX], stat[HQS_BATCH_MAX];
    __shared__ int nact, tw_cur;
    const int ns = B.ns, G = gridDim.x, bid = blockIdx.x;
    const float a = B.a, bcoef = B.b;
    // the 2n-point twiddles of the Toeplitz items stay in a fixed shared region after
    // the largest transform buffer and its image row, restaged only when the size changes
    float2* twT = s + (size_t)768 * kLines + 384;
    if (threadIdx.x == 0) tw_cur = 0;
#define STAGE_TW2(AA)                                                                    \
    if (tw_cur != 2 * (AA).n) {                                                          \
        __syncthreads();                                                                 \
        for (int i_ = threadIdx.x; i_ < 2 * (AA).n; i_ += blockDim.x) twT[i_] = (AA).tw[i_]; \
        __syncthreads();                                                                 \
        if (threadIdx.x == 0) tw_cur = 2 * (AA).n;                                       \
        __syncthreads();                                                                 \
    }
    const float2* twN = nullptr;
    // optional phase trace, kept by thread 0 of CTA 0 (count in shared memory: no registers)
    __shared__ int ntr;
    if (B.trace && bid == 0 && threadIdx.x == 0) {
        ntr = 0;
        if (B.trace_max > 0) B.trace[ntr++] = global_ns();
    }
#define BB_BARRIER()                                                                         \
    do {                                                                                     \
        if (!grid_barrier(B.bar, B.err)) return;                                             \
        if (B.trace && bid == 0 && threadIdx.x == 0 && ntr < B.trace_max) B.trace[ntr++] = global_ns(); \
    } while (0)
    // the chunk epilogue reads what the row-adjoint pass wrote: its barrier is needed
    // only when some slice has several coil chunks (the trace keeps the stamp)
    const bool has_epi = B.off[BL_EPI * (ns + 1) + ns] > 0;
#define EPI_BARRIER()                                                                        \
    do {                                                                                     \
        if (has_epi) {                                                                       \
            BB_BARRIER();                                                                    \
        } else if (B.trace && bid == 0 && threadIdx.x == 0 && ntr < B.trace_max) {           \
            B.trace[ntr++] = global_ns();                                                    \
        }                                                                                    \
    } while (0)
    // Each phase deals its items in the opposite slice order to the phase before, so
    // that it starts on the slices whose data the previous phase touched last (still
    // in L2 when the batch's intermediates do not all fit).
    int pdir = 0;
#define FOR_ITEMS(list, ...)                                                               \
    {                                                                                      \
        const int* off_ = B.off + (list) * (ns + 1);                                       \
        const int tot_ = off_[ns];                                                         \
        pdir ^= 1;                                                                         \
        for (int k_ = bid; k_ < tot_; k_ += G) {                                           \
            const int g_ = pdir ? tot_ - 1 - k_ : k_;                                      \
            const int si = find_slice(off_, ns, g_);                                       \
            if (!active[si]) continue;                                                     \
            const int it_ = g_ - off_[si];                                                 \
            const BatchSlice& S = B.sl[si];                                                \
            __VA_ARGS__;                                                                   \
        }                                                                                  \
    }
#define STAGE_TWN(S, si) twN = (S).twN;
#define CLEAR_ACC()                                                      \
    for (int i_ = threadIdx.x; i_ < 2 * HQS_BATCH_MAX; i_ += blockDim.x) \
        (&acc[0][0])[i_] = 0.0;                                          \
    __syncthreads();
#define COUNT_ACTIVE()                                               \
    if (threadIdx.x == 0) {                                          \
        int c_ = 0;                                                  \
        for (int i_ = 0; i_ < ns; ++i_) c_ += active[i_];            \
        nact = c_;                                                   \
    }                                                                \
    __syncthreads();

    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        active[i] = 1;
        its[i] = 0;
        stat[i] = HQS_OK;
        betas[i] = 0.0;
    }
    __syncthreads();
    // x = 0, r = rhs, ||rhs||^2
    CLEAR_ACC();
    FOR_ITEMS(BL_IMG, {
        const int n = S.A.n;
        double a1 = 0.0;
        for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
            const size_t e = (size_t)it_ * n + ix;
            const float2 bv = S.rhs[e];
            S.u[e] = make_float2(0.f, 0.f);
            S.r[e] = bv;
            a1 += (double)bv.x * bv.x + (double)bv.y * bv.y;
        }
        a1 = cta_sum(a1, red);
        if (threadIdx.x == 0) acc[0][si] += a1;
    });
    __syncthreads();
    put_slice_partials(B.part + (size_t)BS_BB * ns * G, ns, acc[0]);
    BB_BARRIER();
    slice_totals(B.part + (size_t)BS_BB * ns * G, ns, tot[0]);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const double bb = tot[0][i];
        bbs[i] = bb;
        rrs[i] = bb;
        if (!(bb == bb) || isinf(bb)) {
            stat[i] = HQS_ERR_BREAKDOWN;
            active[i] = 0;
        } else if (bb == 0.0 || B.tol2 >= 1.0) {
            active[i] = 0;
        } else if (B.max_iter == 0) {
            stat[i] = HQS_ERR_NOT_CONVERGED;
            active[i] = 0;
        }
    }
    __syncthreads();
    // preconditioner of the initial residual, <r, z>
    FOR_ITEMS(BL_PC, {
        STAGE_TWN(S, si);
        HQS_BATCH_DISPATCH(S.A.n, (pc_rows<N>(S, it_ * batch_pq<N>(), 0.f, false, s, twN)));
    });
    BB_BARRIER();
    CLEAR_ACC();
    FOR_ITEMS(BL_PC, {
        STAGE_TWN(S, si);
        double v = 0.0;
        HQS_BATCH_DISPATCH(S.A.n, (v = pc_cols<N>(S, it_ * batch_pq<N>(), a, bcoef, s, twN)));
        v = cta_sum(v, red);
        if (threadIdx.x == 0) acc[0][si] += v;
    });
    __syncthreads();
    put_slice_partials(B.part + (size_t)BS_RZ * ns * G, ns, acc[0]);
    BB_BARRIER();
    slice_totals(B.part + (size_t)BS_RZ * ns * G, ns, tot[0]);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const int n = B.sl[i].A.n;
        rzs[i] = tot[0][i] / ((double)n * n);
        if (active[i] && !(rzs[i] > 0.0 && !isinf(rzs[i]))) {
            stat[i] = HQS_ERR_BREAKDOWN;
            active[i] = 0;
        }
    }
    __syncthreads();
    COUNT_ACTIVE();
    for (int cg = 0; cg < B.max_iter && nact > 0; ++cg) {
        // p = z + beta p
        FOR_ITEMS(BL_ZP, {
            STAGE_TWN(S, si);
            HQS_BATCH_DISPATCH(S.A.n, (z_and_p_rows<N2, N>(S, it_ * batch_zq<N>(), (float)betas[si], cg == 0, s, twN)));
        });
        BB_BARRIER();
        // q = a A^H A p + b p, <p, q>
        FOR_ITEMS(BL_ROWS, {
            const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
            STAGE_TW2(S.A);
            HQS_BATCH_DISPATCH(n, (toep_rows_fwd_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.p, nullptr, 0.f, false, s,
                                                                        nullptr, twT)));
        });
        BB_BARRIER();
        FOR_ITEMS(BL_COLS, {
            const int n = S.A.n, N2v = 2 * n, ch = it_ / N2v, kx = it_ - ch * N2v;
            STAGE_TW2(S.A);
            if (S.colcap > 0) {
                const int f0 = it_ * S.colcap, nl = min(S.colcap, N2v * S.A.L - f0);
                HQS_BATCH_DISPATCH(n, (toep_cols_flat_item<N2, HQS_BATCH_BD>(S.A, f0, nl, s, twT)));
            } else {
                HQS_BATCH_DISPATCH(n, (toep_cols_item<N2, HQS_BATCH_BD>(S.A, kx, ch, s, twT)));
            }
        });
        BB_BARRIER();
        CLEAR_ACC();
        FOR_ITEMS(BL_ROWS, {
            const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
            double v = 0.0;
            STAGE_TW2(S.A);
            HQS_BATCH_DISPATCH(n, (v = toep_rows_adj_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.q, S.p, a, bcoef, 1, s, twT)));
            v = cta_sum(v, red);
            if (threadIdx.x == 0) acc[0][si] += v;
        });
        EPI_BARRIER();
        FOR_ITEMS(BL_EPI, {   // several coil chunks: fixed-order chunk sum + epilogue
            const int n = S.A.n, cnt = n * n;
            double v = 0.0;
            for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                const size_t e = (size_t)it_ * n + ix;
                float2 w = make_float2(0.f, 0.f);
                for (int c = 0; c < S.A.nchunk; ++c) w = cadd(w, __ldcg(S.A.chunk + (size_t)c * cnt + e));
                S.q[e] = toep_epilogue(w, e, S.p, a, bcoef, 1, v);
            }
            v = cta_sum(v, red);
            if (threadIdx.x == 0) acc[0][si] += v;
        });
        __syncthreads();
        put_slice_partials(B.part + (size_t)BS_PQ * ns * G, ns, acc[0]);
        BB_BARRIER();
        slice_totals(B.part + (size_t)BS_PQ * ns * G, ns, tot[0]);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const double pq = tot[0][i];
            alphas[i] = (pq > 0.0 && !isinf(pq)) ? rzs[i] / pq : 0.0;
            if (active[i] && !(pq > 0.0 && !isinf(pq))) {
                stat[i] = HQS_ERR_BREAKDOWN;
                active[i] = 0;
            }
        }
        __syncthreads();
        // x += alpha p, r -= alpha q, ||r||^2, row FFTs of r
        CLEAR_ACC();
        FOR_ITEMS(BL_PC, {
            STAGE_TWN(S, si);
            double v = 0.0;
            HQS_BATCH_DISPATCH(S.A.n, (v = pc_rows<N>(S, it_ * batch_pq<N>(), (float)alphas[si], true, s, twN)));
            v = cta_sum(v, red);
            if (threadIdx.x == 0) acc[1][si] += v;
        });
        __syncthreads();
        put_slice_partials(B.part + (size_t)BS_RR * ns * G, ns, acc[1]);
        BB_BARRIER();
        slice_totals(B.part + (size_t)BS_RR * ns * G, ns, tot[1]);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            if (!active[i]) continue;
            const double rr = tot[1][i];
            its[i] += 1;
            rrs[i] = rr;
            if (!(rr == rr) || isinf(rr)) {
                stat[i] = HQS_ERR_BREAKDOWN;
                active[i] = 0;
            } else if (rr <= B.tol2 * bbs[i]) {
                active[i] = 0;
            } else if (its[i] >= B.max_iter) {
                if (B.tol2 > 0.0) stat[i] = HQS_ERR_NOT_CONVERGED;
                active[i] = 0;
            }
        }
        __syncthreads();
        COUNT_ACTIVE();
        if (nact == 0) break;
        // preconditioner columns, <r, z>, beta
        CLEAR_ACC();
        FOR_ITEMS(BL_PC, {
            STAGE_TWN(S, si);
            double v = 0.0;
            HQS_BATCH_DISPATCH(S.A.n, (v = pc_cols<N>(S, it_ * batch_pq<N>(), a, bcoef, s, twN)));
            v = cta_sum(v, red);
            if (threadIdx.x == 0) acc[0][si] += v;
        });
        __syncthreads();
        put_slice_partials(B.part + (size_t)BS_RZ * ns * G, ns, acc[0]);
        BB_BARRIER();
        slice_totals(B.part + (size_t)BS_RZ * ns * G, ns, tot[0]);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const int n = B.sl[i].A.n;
            const double rz_new = tot[0][i] / ((double)n * n);
            if (active[i] && !(rz_new > 0.0 && !isinf(rz_new))) {
                stat[i] = HQS_ERR_BREAKDOWN;
                active[i] = 0;
            }
            betas[i] = rzs[i] > 0.0 ? rz_new / rzs[i] : 0.0;
            rzs[i] = rz_new;
        }
        __syncthreads();
        COUNT_ACTIVE();
    }
    if (bid == 0)
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            B.res[i] = bbs[i] > 0.0 ? rrs[i] / bbs[i] : 0.0;
            B.iters[i] = its[i];
            B.status[i] = stat[i];
        }
    if (B.trace && bid == 0 && threadIdx.x == 0) {
        if (ntr < B.trace_max) B.trace[ntr++] = global_ns();
        B.trace[B.trace_max] = ntr;
    }
#undef BB_BARRIER
#undef EPI_BARRIER
#undef FOR_ITEMS
#undef STAGE_TWN
#undef CLEAR_ACC
#undef STAGE_TW2
#undef COUNT_ACTIVE
}

}  // namespace

// Batched normal operator: out_i = A_i^H A_i x_i for every slice of a batch in
// one cooperative launch (Sec. 3.4's A^H A, the Toeplitz form of the per-stage
// operator): the three Toeplitz passes, each dealing the items of all slices to
// all CTAs, with a grid barrier between passes (and the fixed-order coil-chunk
// sum when a slice has several chunks).  The per-slice arithmetic is that of
// the per-stage passes.
struct AhaBatchArgs {
    const BatchSlice* sl;   // u = caller's x, q = caller's out
    int ns;
    const int* off;
    unsigned* bar;
    unsigned* err;
};

__global__ void __launch_bounds__(HQS_BATCH_BD, 2) k_aha_batch(AhaBatchArgs B) {
    extern __shared__ __align__(16) float2 s[];
    __shared__ int tw_cur;
    const int ns = B.ns, G = gridDim.x, bid = blockIdx.x;
    float2* twT = s + (size_t)768 * kLines + 384;
    if (threadIdx.x == 0) tw_cur = 0;
    __syncthreads();
#define STAGE_TW2(AA)                                                                    \
    if (tw_cur != 2 * (AA).n) {                                                          \
        __syncthreads();                                                                 \
        for (int i_ = threadIdx.x; i_ < 2 * (AA).n; i_ += blockDim.x) twT[i_] = (AA).tw[i_]; \
        __syncthreads();                                                                 \
        if (threadIdx.x == 0) tw_cur = 2 * (AA).n;                                       \
        __syncthreads();                                                                 \
    }
#define AB_BARRIER()                                \
    do {                                            \
        if (!grid_barrier(B.bar, B.err)) return;    \
    } while (0)
#define FOR_ITEMS(list, ...)                                                               \
    {                                                                                      \
        const int* off_ = B.off + (list) * (ns + 1);                                       \
        for (int g_ = bid; g_ < off_[ns]; g_ += G) {                                       \
            const int si = find_slice(off_, ns, g_);                                       \
            const int it_ = g_ - off_[si];                                                 \
            const BatchSlice& S = B.sl[si];                                                \
            __VA_ARGS__;                                                                   \
        }                                                                                  \
    }
    FOR_ITEMS(BL_ROWS, {
        const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
        STAGE_TW2(S.A);
        HQS_BATCH_DISPATCH(n, (toep_rows_fwd_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.u, nullptr, 0.f, false, s, nullptr,
                                                                    twT)));
    });
    AB_BARRIER();
    FOR_ITEMS(BL_COLS, {
        const int n = S.A.n, N2v = 2 * n, ch = it_ / N2v, kx = it_ - ch * N2v;
        STAGE_TW2(S.A);
        if (S.colcap > 0) {
            const int f0 = it_ * S.colcap, nl = min(S.colcap, N2v * S.A.L - f0);
            HQS_BATCH_DISPATCH(n, (toep_cols_flat_item<N2, HQS_BATCH_BD>(S.A, f0, nl, s, twT)));
        } else {
            HQS_BATCH_DISPATCH(n, (toep_cols_item<N2, HQS_BATCH_BD>(S.A, kx, ch, s, twT)));
        }
    });
    AB_BARRIER();
    FOR_ITEMS(BL_ROWS, {
        const int n = S.A.n, ch = it_ / n, iy = it_ - ch * n;
        STAGE_TW2(S.A);
        HQS_BATCH_DISPATCH(n, (toep_rows_adj_item<N2, HQS_BATCH_BD>(S.A, iy, ch, S.q, nullptr, 1.f, 0.f, 0, s, twT)));
    });
    if (B.off[BL_EPI * (ns + 1) + ns] > 0) {   // several coil chunks: fixed-order chunk sum
        AB_BARRIER();
        FOR_ITEMS(BL_EPI, {
            const int n = S.A.n, cnt = n * n;
            for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
                const size_t e = (size_t)it_ * n + ix;
                float2 v = make_float2(0.f, 0.f);
                for (int c = 0; c < S.A.nchunk; ++c) v = cadd(v, __ldcg(S.A.chunk + (size_t)c * cnt + e));
                S.q[e] = v;
            }
        });
    }
#undef AB_BARRIER
#undef FOR_ITEMS
#undef STAGE_TW2
}

struct hqs_batch_s {
    int device = 0;
    int ns = 0;
    int K = 0;
    std::vector<hqs_plan_s*> plans;
    BatchSlice* d_slices = nullptr;
    int* d_off = nullptr;
    float* d_mu = nullptr;
    float* d_taps = nullptr;
    int* d_radius = nullptr;
    double* d_part = nullptr;
    double* d_res = nullptr;
    unsigned* d_bar = nullptr;
    unsigned* d_err = nullptr;
    float* h_mu = nullptr;        // pinned staging (read when the graph replays)
    float* h_taps = nullptr;
    int* h_radius = nullptr;
    int grid = 0;        // CTAs of a launch: every resident CTA of the kernel
    int grid_cap = 0;    // hqs_batch_set_grid: at most this many (0: no cap)
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;  // y / x pointers the graph was recorded with
    int key_K = -1, key_k0 = -1, key_cg = -1, key_grid = -1;
    float key_c0 = 0.f, key_c1 = 0.f;
    std::vector<float2*> chunks;   // per-slice coil-chunk partial sums
    // batched data-consistency solve: its own slice table (u = x, rhs = the
    // caller's), rebuilt when the caller's pointers change
    std::vector<BatchSlice> dc_host;
    BatchSlice* d_slices_dc = nullptr;
    int* d_iters = nullptr;
    int* d_status = nullptr;
    std::vector<const void*> dc_key;
    unsigned long long* d_trace = nullptr;   // optional phase trace of the batched solve
    // batched A^H A: its own slice table (u = x, q = out), rebuilt when the pointers change
    std::vector<BatchSlice> ap_host;
    BatchSlice* d_slices_ap = nullptr;
    std::vector<const void*> ap_key;
    // batched forward / adjoint: the lower-half passes' argument tables of the slices
    // that take them, grouped by grid size (rebuilt when the pointers change)
    struct HalfGroup {
        int G, n, maxchunk, first, count;
    };
    void* d_half[2] = {nullptr, nullptr};   // [0] forward, [1] adjoint
    std::vector<HalfGroup> half_groups[2];
    std::vector<const void*> half_key[2];
};

static void batch_free(hqs_batch_s* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_slices);
    cudaFree(b->d_off);
    cudaFree(b->d_mu);
    cudaFree(b->d_taps);
    cudaFree(b->d_radius);
    cudaFree(b->d_part);
    cudaFree(b->d_res);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    cudaFreeHost(b->h_mu);
    cudaFreeHost(b->h_taps);
    cudaFreeHost(b->h_radius);
    for (float2* c : b->chunks) cudaFree(c);
    cudaFree(b->d_slices_dc);
    cudaFree(b->d_iters);
    cudaFree(b->d_status);
    cudaFree(b->d_trace);
    cudaFree(b->d_slices_ap);
    cudaFree(b->d_half[0]);
    cudaFree(b->d_half[1]);
    delete b;
}

extern "C" void hqs_batch_destroy(hqs_batch b) { batch_free(b); }

// CTAs of one cooperative launch of a batch kernel: every CTA the kernel keeps
// resident (at most b->grid, the partial-sum slots), or the caller's cap
static int batch_grid(const hqs_batch_s* b, int resident) {
    const int g = std::min(b->grid, resident);
    return b->grid_cap > 0 ? std::min(g, b->grid_cap) : g;
}

extern "C" int hqs_batch_set_grid(hqs_batch b, int ctas) {
    if (!b || ctas < 0) return HQS_ERR_INVALID_ARG;
    b->grid_cap = ctas;
    return HQS_OK;
}


// preconditioner lines per item for a slice of size n (host side of batch_pq)
static int batch_pq_host(int n) {
    switch (n) {
        case 64: return batch_pq<64>();
        case 128: return batch_pq<128>();
        case 256: return batch_pq<256>();
        case 320: return batch_pq<320>();
        default: return batch_pq<384>();
    }
}

extern "C" int hqs_batch_create(hqs_batch* out, hqs_plan* plans, int n, int max_outer) {
    if (!out || !plans || n <= 0 || n > HQS_BATCH_MAX || max_outer <= 0 || max_outer > 4096)
        return HQS_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const hqs_plan_s* p = plans[i];
        if (!p) return HQS_ERR_INVALID_ARG;
        if (p->n != 64 && p->n != 128 && p->n != 256 && p->n != 320 && p->n != 384) return HQS_ERR_UNSUPPORTED;
    }
    hqs_batch_s* b = new (std::nothrow) hqs_batch_s();
    if (!b) return HQS_ERR_OOM;
    cudaGetDevice(&b->device);
    b->ns = n;
    b->K = max_outer;
    b->plans.assign(plans, plans + n);
    auto fail = [&](int rc) {
        batch_free(b);
        return rc;
    };
    // slice table and item lists
    std::vector<BatchSlice> hs(n);
    std::vector<int> off((size_t)BL_N * (n + 1), 0);
    for (int i = 0; i < n; ++i) {
        hqs_plan_s* p = plans[i];
        BatchSlice& S = hs[i];
        S.A = toep_args(p);
        // coil chunk: as many lines as fill the CTA at this FFT size (16 lines of
        // 640 points, 8 of 512 or 768), chunks of equal size
        const int tpl = dispatch_fft_size(p->n2, [&]<int NN>() { return FftSize<NN>::TPL; });
        const int lcmax = std::max(1, std::min(kLines, HQS_BATCH_BD / tpl));
        const int nch = ceil_div(p->L, lcmax);
        S.A.nchunk = nch;
        S.A.LC = ceil_div(p->L, nch);
        S.A.chunk = nullptr;
        if (nch > 1) {
            float2* cb = nullptr;
            if (cudaMalloc(&cb, (size_t)nch * p->n * p->n * sizeof(float2))) return fail(HQS_ERR_OOM);
            b->chunks.push_back(cb);
            S.A.chunk = cb;
        }
        S.twN = plan_twiddles(p, p->n);
        S.lam = p->lam;
        S.b0 = p->img_b0;
        S.x = nullptr;   // set per run
        S.u = p->img_u;
        S.rhs = p->img_rhs;
        S.r = p->cg_r;
        S.p = p->cg_p;
        S.q = p->cg_q;
        S.pcb = p->pc_buf;
        // column items: with chunks of fewer than lcmax coils, items of lcmax flattened
        // (column, coil) lines instead of one column per chunk
        const bool pack = S.A.LC < lcmax;
        S.colcap = pack ? lcmax : 0;
        const int ncols = pack ? ceil_div(2 * p->n * p->L, lcmax) : 2 * p->n * nch;
        const int zq = dispatch_fft_size(p->n, [&]<int NN>() { return batch_zq<NN>(); });
        const int cnt[BL_N] = {p->n * nch, ncols, ceil_div(p->n, batch_pq_host(p->n)), p->n,
                               ceil_div(p->n, 32) * ceil_div(p->n, 32), nch > 1 ? p->n : 0, ceil_div(p->n, zq)};
        for (int l = 0; l < BL_N; ++l) off[(size_t)l * (n + 1) + i + 1] = off[(size_t)l * (n + 1) + i] + cnt[l];
    }
    const size_t sm = kBatchSmemF2 * sizeof(float2);
    int per_sm = 0, nsm = 0;
    if (cudaFuncSetAttribute(k_hqs_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hqs_batch, HQS_BATCH_BD, sm) ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device) || per_sm < 1)
        return fail(HQS_ERR_CUDA);
    b->grid = per_sm * nsm;
    if (cudaMalloc(&b->d_slices, n * sizeof(BatchSlice)) || cudaMalloc(&b->d_off, off.size() * sizeof(int)) ||
        cudaMalloc(&b->d_mu, max_outer * sizeof(float)) ||
        cudaMalloc(&b->d_taps, (size_t)max_outer * (2 * HQS_BATCH_MAXR + 1) * sizeof(float)) ||
        cudaMalloc(&b->d_radius, max_outer * sizeof(int)) ||
        cudaMalloc(&b->d_part, (size_t)BS_N * n * b->grid * sizeof(double)) ||
        cudaMalloc(&b->d_res, n * sizeof(double)) || cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) ||
        cudaMalloc(&b->d_err, sizeof(unsigned)) || cudaMallocHost(&b->h_mu, max_outer * sizeof(float)) ||
        cudaMallocHost(&b->h_taps, (size_t)max_outer * (2 * HQS_BATCH_MAXR + 1) * sizeof(float)) ||
        cudaMallocHost(&b->h_radius, max_outer * sizeof(int)) ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking))
        return fail(HQS_ERR_OOM);
    b->dc_host = hs;
    b->ap_host = hs;
    if (cudaMalloc(&b->d_slices_dc, n * sizeof(BatchSlice)) || cudaMalloc(&b->d_iters, n * sizeof(int)) ||
        cudaMalloc(&b->d_status, n * sizeof(int)) || cudaMalloc(&b->d_slices_ap, n * sizeof(BatchSlice)))
        return fail(HQS_ERR_OOM);
    if (cudaMemcpy(b->d_slices, hs.data(), n * sizeof(BatchSlice), cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice))
        return fail(HQS_ERR_CUDA);
    *out = b;
    return HQS_OK;
}

// Everything one batch step enqueues (recorded into the graph).
static int batch_enqueue(hqs_batch_s* b, const hqs_c64* const* y, hqs_c64* const* x, int K, int k0, int cg_iters,
                         float c0, float c1, cudaStream_t st) {
    const int n = b->ns;
    for (int i = 0; i < n; ++i)
        HQS_TRY_RC(launch_adj(b->plans[i], reinterpret_cast<const float2*>(y[i]), b->plans[i]->img_b0, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(b->d_mu, b->h_mu, K * sizeof(float), cudaMemcpyHostToDevice, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(b->d_taps, b->h_taps, (size_t)K * (2 * HQS_BATCH_MAXR + 1) * sizeof(float),
                                 cudaMemcpyHostToDevice, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(b->d_radius, b->h_radius, K * sizeof(int), cudaMemcpyHostToDevice, st));
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), st));
    BatchArgs A;
    A.sl = b->d_slices;
    A.ns = n;
    A.off = b->d_off;
    A.K = K;
    A.k0 = k0;
    A.cg_iters = cg_iters;
    A.c0 = c0;
    A.c1 = c1;
    A.mu = b->d_mu;
    A.taps = b->d_taps;
    A.radius = b->d_radius;
    A.part = b->d_part;
    A.res = b->d_res;
    A.bar = b->d_bar;
    A.err = b->d_err;
    void* args[] = {&A};
    HQS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_hqs_batch, dim3(batch_grid(b, b->grid)), dim3(HQS_BATCH_BD), args,
                                             kBatchSmemF2 * sizeof(float2), st));
    return HQS_OK;
}

extern "C" int hqs_batch_run(hqs_batch b, const hqs_c64* const* y, hqs_c64* const* x, const float* mu,
                             const float* sigma, int K, int k0, int cg_iters, float c0, float c1,
                             const hqs_gauss_params* gauss, int use_graph, void* stream) {
    if (!b || !y || !x || !mu || !sigma || K <= 0 || K > b->K || k0 < 0 || k0 >= K || cg_iters < 1 ||
        cg_iters > HQS_MAX_ITERS || !(c0 > 0.f) || !(c1 == c1))
        return HQS_ERR_INVALID_ARG;
    for (int i = 0; i < b->ns; ++i)
        if (!x[i] || (!y[i] && b->plans[i]->M > 0)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // a previous step may still read the slice table and the staging buffers
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    // the x pointers live in the device slice table
    std::vector<BatchSlice> hs(b->ns);
    HQS_CUDA_TRY(cudaMemcpy(hs.data(), b->d_slices, b->ns * sizeof(BatchSlice), cudaMemcpyDeviceToHost));
    bool xchg = false;
    for (int i = 0; i < b->ns; ++i) {
        float2* xi = reinterpret_cast<float2*>(x[i]);
        if (hs[i].x != xi) xchg = true;
        hs[i].x = xi;
    }
    if (xchg) HQS_CUDA_TRY(cudaMemcpy(b->d_slices, hs.data(), b->ns * sizeof(BatchSlice), cudaMemcpyHostToDevice));
    // schedules and denoiser taps (host, into pinned staging)
    const float kappa = gauss ? gauss->kappa : 1.5f;
    const float s0 = gauss ? gauss->sigma0 : sigma[0];
    for (int k = 0; k < K; ++k) {
        if (!(mu[k] > 0.f) || !(sigma[k] >= 0.f)) return HQS_ERR_INVALID_ARG;
        b->h_mu[k] = mu[k];
        const double sd = s0 > 0.f ? (double)kappa * sigma[k] / s0 : (double)sigma[k];
        float* g = b->h_taps + (size_t)k * (2 * HQS_BATCH_MAXR + 1);
        if (sd < 0.1) {
            b->h_radius[k] = -1;
            continue;
        }
        const int r = (int)std::ceil(3.0 * sd);
        if (r > HQS_BATCH_MAXR) return HQS_ERR_INVALID_ARG;
        b->h_radius[k] = r;
        double sum = 0.0;
        std::vector<double> gg(2 * r + 1);
        for (int i = -r; i <= r; ++i) sum += gg[i + r] = std::exp(-(double)i * i / (2.0 * sd * sd));
        for (int i = 0; i <= 2 * r; ++i) g[i] = (float)(gg[i] / sum);
    }
    if (!use_graph) return batch_enqueue(b, y, x, K, k0, cg_iters, c0, c1, st);
    std::vector<const void*> key;
    for (int i = 0; i < b->ns; ++i) {
        key.push_back(y[i]);
        key.push_back(x[i]);
    }
    if (!b->exec || key != b->key || K != b->key_K || k0 != b->key_k0 || cg_iters != b->key_cg || c0 != b->key_c0 ||
        c1 != b->key_c1 || b->grid_cap != b->key_grid) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        HQS_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = batch_enqueue(b, y, x, K, k0, cg_iters, c0, c1, b->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc != HQS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        HQS_CUDA_TRY(e);
        b->graph = g;
        HQS_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
        b->key = key;
        b->key_K = K;
        b->key_k0 = k0;
        b->key_cg = cg_iters;
        b->key_c0 = c0;
        b->key_c1 = c1;
        b->key_grid = b->grid_cap;
    }
    HQS_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return HQS_OK;
}

extern "C" int hqs_batch_status(hqs_batch b, double* rel_res, void* stream) {
    if (!b) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned err = 0;
    HQS_CUDA_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    std::vector<double> r(b->ns);
    HQS_CUDA_TRY(cudaMemcpyAsync(r.data(), b->d_res, b->ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    if (rel_res)
        for (int i = 0; i < b->ns; ++i) rel_res[i] = std::sqrt(std::max(r[i], 0.0));
    return (err & HQS_DEVERR_TIMEOUT) ? HQS_ERR_TIMEOUT : HQS_OK;
}

extern "C" int hqs_batch_dc_solve(hqs_batch b, const hqs_c64* const* rhs, hqs_c64* const* x, float a, float bcoef,
                                  int max_iter, double rel_tol, void* stream) {
    if (!b || !rhs || !x || !(a == a) || !(bcoef > 0.f) || max_iter < 0 || max_iter > HQS_MAX_ITERS ||
        !(rel_tol >= 0.0))
        return HQS_ERR_INVALID_ARG;
    for (int i = 0; i < b->ns; ++i)
        if (!rhs[i] || !x[i]) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<const void*> key;
    for (int i = 0; i < b->ns; ++i) {
        key.push_back(rhs[i]);
        key.push_back(x[i]);
    }
    if (key != b->dc_key) {
        // a previous solve may still read the table
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < b->ns; ++i) {
            b->dc_host[i].u = reinterpret_cast<float2*>(x[i]);
            b->dc_host[i].rhs = const_cast<float2*>(reinterpret_cast<const float2*>(rhs[i]));
            b->dc_host[i].x = nullptr;
        }
        HQS_CUDA_TRY(cudaMemcpy(b->d_slices_dc, b->dc_host.data(), b->ns * sizeof(BatchSlice),
                                cudaMemcpyHostToDevice));
        b->dc_key = key;
    }
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), st));
    DcBatchArgs A;
    A.sl = b->d_slices_dc;
    A.ns = b->ns;
    A.off = b->d_off;
    A.a = a;
    A.b = bcoef;
    A.max_iter = max_iter;
    A.tol2 = rel_tol * rel_tol;
    A.part = b->d_part;
    A.res = b->d_res;
    A.iters = b->d_iters;
    A.status = b->d_status;
    A.bar = b->d_bar;
    A.err = b->d_err;
    A.trace = b->d_trace;
    A.trace_max = b->d_trace ? HQS_TRACE_MAX : 0;
    const size_t sm = kBatchSmemF2 * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pcg_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, nsm = 0;
    HQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batch, HQS_BATCH_BD, sm));
    HQS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    if (per_sm < 1) return HQS_ERR_UNSUPPORTED;
    const int grid = batch_grid(b, per_sm * nsm);   // d_part holds b->grid partials per slot
    void* args[] = {&A};
    HQS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_pcg_batch, dim3(grid), dim3(HQS_BATCH_BD), args, sm, st));
    return HQS_OK;
}

extern "C" int hqs_batch_toeplitz_normal(hqs_batch b, const hqs_c64* const* x, hqs_c64* const* out, void* stream) {
    if (!b || !x || !out) return HQS_ERR_INVALID_ARG;
    for (int i = 0; i < b->ns; ++i)
        if (!x[i] || !out[i]) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<const void*> key;
    for (int i = 0; i < b->ns; ++i) {
        key.push_back(x[i]);
        key.push_back(out[i]);
    }
    if (key != b->ap_key) {
        // a previous apply may still read the table
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < b->ns; ++i) {
            b->ap_host[i].u = const_cast<float2*>(reinterpret_cast<const float2*>(x[i]));
            b->ap_host[i].q = reinterpret_cast<float2*>(out[i]);
            b->ap_host[i].x = nullptr;
        }
        HQS_CUDA_TRY(cudaMemcpy(b->d_slices_ap, b->ap_host.data(), b->ns * sizeof(BatchSlice),
                                cudaMemcpyHostToDevice));
        b->ap_key = key;
    }
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), st));
    AhaBatchArgs A;
    A.sl = b->d_slices_ap;
    A.ns = b->ns;
    A.off = b->d_off;
    A.bar = b->d_bar;
    A.err = b->d_err;
    const size_t sm = kBatchSmemF2 * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_aha_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, nsm = 0;
    HQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_aha_batch, HQS_BATCH_BD, sm));
    HQS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    if (per_sm < 1) return HQS_ERR_UNSUPPORTED;
    const int grid = batch_grid(b, per_sm * nsm);
    void* args[] = {&A};
    HQS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_aha_batch, dim3(grid), dim3(HQS_BATCH_BD), args, sm, st));
    return HQS_OK;
}

// Argument tables of the batched lower-half passes (dir 0: forward x -> grid,
// dir 1: adjoint grid -> x with the axpy term z), grouped by grid size in slice
// order; uploaded when the image pointers differ from the last call.
static int half_tables(hqs_batch_s* b, int dir, const float2* const* xin, float2* const* xout,
                       const float2* const* z, cudaStream_t st) {
    std::vector<const void*> key;
    for (int i = 0; i < b->ns; ++i) {
        key.push_back(xin ? (const void*)xin[i] : nullptr);
        key.push_back(xout ? (const void*)xout[i] : nullptr);
        key.push_back(z ? (const void*)z[i] : nullptr);
    }
    if (b->d_half[dir] && key == b->half_key[dir]) return HQS_OK;
    // a previous call may still read the table
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    const size_t sz = half_args_bytes();
    if (!b->d_half[dir]) HQS_CUDA_TRY(cudaMalloc(&b->d_half[dir], sz * b->ns));
    std::vector<unsigned char> host(sz * b->ns);
    std::vector<hqs_batch_s::HalfGroup> groups;
    std::vector<int> done(b->ns, 0);
    int slot = 0;
    for (int i = 0; i < b->ns; ++i) {
        const hqs_plan_s* p = b->plans[i];
        if (done[i] || !plan_half_passes(p)) continue;
        hqs_batch_s::HalfGroup g{p->G, p->n, 0, slot, 0};
        for (int j = i; j < b->ns; ++j) {
            const hqs_plan_s* q = b->plans[j];
            if (done[j] || !plan_half_passes(q) || q->G != p->G) continue;
            fill_half_args(q, xin ? xin[j] : nullptr, xout ? xout[j] : nullptr, z ? z[j] : nullptr,
                           host.data() + sz * slot);
            g.maxchunk = std::max(g.maxchunk, q->nchunk);
            ++g.count;
            ++slot;
            done[j] = 1;
        }
        groups.push_back(g);
    }
    if (slot > 0) HQS_CUDA_TRY(cudaMemcpy(b->d_half[dir], host.data(), sz * slot, cudaMemcpyHostToDevice));
    b->half_groups[dir] = groups;
    b->half_key[dir] = key;
    return HQS_OK;
}

extern "C" int hqs_batch_adjoint_axpy(hqs_batch b, const hqs_c64* const* y, float zc, const hqs_c64* const* z,
                                      hqs_c64* const* x, void* stream) {
    if (!b || !y || !x || !(zc == zc)) return HQS_ERR_INVALID_ARG;
    for (int i = 0; i < b->ns; ++i)
        if (!x[i] || (!y[i] && b->plans[i]->M > 0)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    auto X = reinterpret_cast<float2* const*>(x);
    auto Z = reinterpret_cast<const float2* const*>(z);
    HQS_TRY_RC(half_tables(b, 1, nullptr, X, Z, st));
    // spreading per slice (the others take their whole per-slice adjoint)
    for (int i = 0; i < b->ns; ++i) {
        hqs_plan_s* p = b->plans[i];
        const float2* yi = reinterpret_cast<const float2*>(y[i]);
        if (plan_half_passes(p))
            HQS_TRY_RC(launch_spread(p, yi, st));
        else
            HQS_TRY_RC(launch_adj_axpy(p, yi, zc, Z ? Z[i] : nullptr, X[i], st));
    }
    const size_t sz = half_args_bytes();
    for (const auto& g : b->half_groups[1])
        HQS_TRY_RC(launch_half_group(g.G, g.n, g.maxchunk, g.count,
                                     static_cast<unsigned char*>(b->d_half[1]) + sz * g.first, 1, zc, st));
    for (int i = 0; i < b->ns; ++i)
        if (plan_half_passes(b->plans[i])) HQS_TRY_RC(launch_adj_chunks(b->plans[i], X[i], zc, Z ? Z[i] : nullptr, st));
    return HQS_OK;
}

extern "C" int hqs_batch_forward(hqs_batch b, const hqs_c64* const* x, hqs_c64* const* y, void* stream) {
    if (!b || !x || !y) return HQS_ERR_INVALID_ARG;
    for (int i = 0; i < b->ns; ++i)
        if (!x[i] || (!y[i] && b->plans[i]->M > 0)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    auto Xin = reinterpret_cast<const float2* const*>(x);
    auto Y = reinterpret_cast<float2* const*>(y);
    HQS_TRY_RC(half_tables(b, 0, Xin, nullptr, nullptr, st));
    const size_t sz = half_args_bytes();
    for (const auto& g : b->half_groups[0])
        HQS_TRY_RC(launch_half_group(g.G, g.n, g.maxchunk, g.count,
                                     static_cast<unsigned char*>(b->d_half[0]) + sz * g.first, 0, 0.f, st));
    for (int i = 0; i < b->ns; ++i) {
        hqs_plan_s* p = b->plans[i];
        if (plan_half_passes(p))
            HQS_TRY_RC(launch_interp(p, Y[i], st));
        else
            HQS_TRY_RC(launch_fwd(p, Xin[i], Y[i], st));
    }
    return HQS_OK;
}

extern "C" int hqs_batch_dc_info(hqs_batch b, int* iterations, double* rel_residual, int* status, void* stream) {
    if (!b) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned err = 0;
    std::vector<int> it(b->ns), stt(b->ns);
    std::vector<double> r(b->ns);
    HQS_CUDA_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(it.data(), b->d_iters, b->ns * sizeof(int), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(stt.data(), b->d_status, b->ns * sizeof(int), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(r.data(), b->d_res, b->ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < b->ns; ++i) {
        if (iterations) iterations[i] = it[i];
        if (rel_residual) rel_residual[i] = std::sqrt(std::max(r[i], 0.0));
        if (status) status[i] = stt[i];
    }
    return (err & HQS_DEVERR_TIMEOUT) ? HQS_ERR_TIMEOUT : HQS_OK;
}

extern "C" int hqs_batch_debug_trace(hqs_batch b, int enable, unsigned long long* out, int max_out, void* stream) {
    if (!b) return HQS_ERR_INVALID_ARG;
    if (enable && !b->d_trace) {
        HQS_CUDA_TRY(cudaMalloc(&b->d_trace, (HQS_TRACE_MAX + 1) * sizeof(unsigned long long)));
        HQS_CUDA_TRY(cudaMemset(b->d_trace, 0, (HQS_TRACE_MAX + 1) * sizeof(unsigned long long)));
        return 0;
    }
    if (!b->d_trace) return 0;
    std::vector<unsigned long long> h(HQS_TRACE_MAX + 1);
    HQS_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d_trace, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
    HQS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const int cnt = (int)std::min<unsigned long long>(h[HQS_TRACE_MAX], HQS_TRACE_MAX);
    if (out)
        for (int i = 0; i < cnt && i < max_out; ++i) out[i] = h[i];
    return cnt;
}
