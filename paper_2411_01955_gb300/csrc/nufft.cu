// Gridding NUFFT of the multicoil operator of Eq. (1) (Sec. 2.1):
//   forward (a2): apodise + coil-multiply + zero-pad fused into the row FFT,
//                 column FFT, Kaiser-Bessel interpolation (gather);
//   adjoint (a3): shared-memory tiled KB spreading, column IFFT, row IFFT
//                 fused with crop + deapodisation + conj(S_l) coil sum.
// All grids are coil-innermost ([gy][gx][l]) so a grid tap is L contiguous
// complex values.
#include <algorithm>

#include "fft.cuh"
#include "plan.cuh"

using namespace hqs;

// phi(t) = I0(beta sqrt(1 - (2t/W)^2)) on |t| <= W/2.
HQS_DEV float kb_phi(float t, float W, float beta) {
    const float z = 2.0f * t / W;
    const float s = 1.0f - z * z;
    return s >= 0.f ? cyl_bessel_i0f(beta * sqrtf(s)) : 0.f;
}

// image pixel held at oversampled-grid position p (centred layout), or -1
HQS_DEV int grid_to_pix(int p, int n, int G) {
    const int h = n >> 1;
    if (p < h) return p + h;
    if (p >= G - h) return p - G + h;
    return -1;
}
HQS_DEV int pix_to_grid(int i, int n, int G) {
    const int c = i - (n >> 1);
    return c >= 0 ? c : c + G;
}

// ---------------------------------------------------------------- forward
// Shared memory of the FFT passes: [G][kLines] lines | [G] twiddles.
template <int G> constexpr size_t nufft_smem_floats2() { return (size_t)G * kLines + G; }

// Row iy for the coils of chunk blockIdx.y: S_l x / (phihat phihat) placed at
// n mod G, FFT along x -> U[iy][gx][l].
template <int G>
__global__ void k_fwd_rows(const float2* __restrict__ x, const float2* __restrict__ smaps,
                           const float* __restrict__ apod, int n, int L, int LC, int nchunk,
                           float scale, const float2* __restrict__ twg, float2* __restrict__ U) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<G>(s + G * kLines, twg);
    const int iy = blockIdx.x;
    const float ay = apod[iy] * scale;
    const int l0 = blockIdx.y * LC;
    const int lines = min(LC, L - l0);
    const int pst = blockDim.x / lines;
    const int l = threadIdx.x % lines, p0 = threadIdx.x / lines;
    if (p0 < pst) {
#pragma unroll 4
        for (int p = p0; p < G; p += pst) {
            const int ix = grid_to_pix(p, n, G);
            float2 v = make_float2(0.f, 0.f);
            if (ix >= 0) {
                const int64_t pix = (int64_t)iy * n + ix;
                v = cscale(cmul(smaps[pix * L + l0 + l], x[pix]), ay * apod[ix]);
            }
            s[p * kLines + l] = v;
        }
    }
    __syncthreads();
    block_fft<G, false>(s, lines, tw);
    float2* dst = U + (int64_t)iy * G * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 4
        for (int p = p0; p < G; p += pst) dst[(int64_t)p * L] = s[p * kLines + l];
    }
}

// Column gx: image rows at n mod G, zeros elsewhere, FFT along y -> Ghat.
template <int G>
__global__ void k_fwd_cols(const float2* __restrict__ U, int n, int L, int LC, int nchunk,
                           const float2* __restrict__ twg, float2* __restrict__ Gh) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<G>(s + G * kLines, twg);
    const int gx = blockIdx.x;
    const int l0 = blockIdx.y * LC;
    const int lines = min(LC, L - l0);
    const int pst = blockDim.x / lines;
    const int l = threadIdx.x % lines, p0 = threadIdx.x / lines;
    const int64_t rs = (int64_t)G * L;
    const float2* col = U + (int64_t)gx * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 8
        for (int p = p0; p < G; p += pst) {
            const int iy = grid_to_pix(p, n, G);
            s[p * kLines + l] = iy >= 0 ? col[iy * rs] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    block_fft<G, false>(s, lines, tw);
    float2* dst = Gh + (int64_t)gx * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 4
        for (int p = p0; p < G; p += pst) dst[p * rs] = s[p * kLines + l];
    }
}

// Type-2 interpolation: 16 lanes per point (lane = coil, looping over coils
// beyond 16), the 2W separable weights computed once per point by lanes
// 0..2W-1 and broadcast with shuffles.
template <int W>
__global__ void __launch_bounds__(256) k_interp(const float2* __restrict__ Gh, const int4* __restrict__ pts,
                                                const int* __restrict__ perm, int M, int G, int L,
                                                float beta, float2* __restrict__ y) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4);
    const int h = threadIdx.x & 15;
    const int base = threadIdx.x & 16;
    const bool valid = j < M;
    const int4 pt = valid ? pts[j] : make_int4(0, 0, 0, 0);
    const float dx = __int_as_float(pt.z), dy = __int_as_float(pt.w);
    float wm = 0.f;
    if (valid && h < 2 * W) wm = kb_phi(h < W ? dx - (float)h : dy - (float)(h - W), (float)W, beta);
    float wx[W], wy[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        wx[w] = __shfl_sync(0xffffffffu, wm, base + w);
        wy[w] = __shfl_sync(0xffffffffu, wm, base + W + w);
    }
    if (!valid) return;
    int gxs[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        int gx = pt.x + b;
        gxs[b] = gx >= G ? gx - G : gx;
    }
    const int dst = perm[j];
    for (int l = h; l < L; l += 16) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            int gy = pt.y + a;
            if (gy >= G) gy -= G;
            const float2* row = Gh + (int64_t)gy * G * L + l;
            float2 ra = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float2 g = __ldg(row + (int64_t)gxs[b] * L);
                ra.x = fmaf(wx[b], g.x, ra.x);
                ra.y = fmaf(wx[b], g.y, ra.y);
            }
            acc.x = fmaf(wy[a], ra.x, acc.x);
            acc.y = fmaf(wy[a], ra.y, acc.y);
        }
        y[(int64_t)l * M + dst] = acc;
    }
}

// ---------------------------------------------------------------- adjoint
// Type-1 spreading of one sub-problem (<= HQS_SPREAD_MAXPTS points of one
// TB x TB bin) into a (TB+W-1)^2 x LC patch in shared memory with shared
// atomics, then one pass of vector float2 atomics into the global grid.
template <int W>
__global__ void k_spread(const float2* __restrict__ y, const int4* __restrict__ pts,
                         const int* __restrict__ perm, const int4* __restrict__ subs, int M, int G,
                         int L, int LC, int nchunk, int TB, int nbx, float beta,
                         float2* __restrict__ grid) {
    extern __shared__ float4 smem4[];
    const int P = TB + W - 1;
    float2* patch = reinterpret_cast<float2*>(smem4);
    float* wts = reinterpret_cast<float*>(patch + P * P * LC);
    int2* loc = reinterpret_cast<int2*>(wts + HQS_SPREAD_MAXPTS * 2 * W);
    const int4 sb = subs[blockIdx.x];
    const int bin = sb.x, start = sb.y, cnt = sb.z;
    const int bx = bin % nbx, by = bin / nbx;
    const int ox = bx * TB - W / 2, oy = by * TB - W / 2;
    for (int i = threadIdx.x; i < cnt * 2 * W; i += blockDim.x) {
        const int pi = i / (2 * W), hh = i - pi * 2 * W;
        const int4 pt = pts[start + pi];
        const float t = hh < W ? __int_as_float(pt.z) - (float)hh : __int_as_float(pt.w) - (float)(hh - W);
        wts[i] = kb_phi(t, (float)W, beta);
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int4 pt = pts[start + i];
        int cx = pt.x + W / 2, cy = pt.y + W / 2;
        if (cx >= G) cx -= G;
        if (cy >= G) cy -= G;
        loc[i] = make_int2(cx - bx * TB, cy - by * TB);
    }
    for (int ch = blockIdx.y; ch < nchunk; ch += gridDim.y) {
        const int l0 = ch * LC;
        const int lines = min(LC, L - l0);
        for (int e = threadIdx.x; e < P * P * lines; e += blockDim.x) patch[e] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int wi = threadIdx.x; wi < cnt * lines; wi += blockDim.x) {
            const int i = wi / lines, l = wi - i * lines;
            const float2 v = y[(int64_t)(l0 + l) * M + perm[start + i]];
            const int2 c0 = loc[i];
            const float* wv = wts + i * 2 * W;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const float wyv = wv[W + a];
                const float2 va = make_float2(v.x * wyv, v.y * wyv);
                float2* prow = patch + ((c0.y + a) * P + c0.x) * lines + l;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float wxv = wv[b];
                    atomicAdd(&prow[b * lines].x, va.x * wxv);
                    atomicAdd(&prow[b * lines].y, va.y * wxv);
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P * P * lines; e += blockDim.x) {
            const float2 v = patch[e];
            if (v.x == 0.f && v.y == 0.f) continue;
            const int l = e % lines, cell = e / lines;
            const int cy = cell / P, cx = cell - cy * P;
            int gx = ox + cx, gy = oy + cy;
            gx = gx < 0 ? gx + G : (gx >= G ? gx - G : gx);
            gy = gy < 0 ? gy + G : (gy >= G ? gy - G : gy);
            atomicAdd(&grid[((int64_t)gy * G + gx) * L + l0 + l], v);
        }
        __syncthreads();
    }
}

// Column gx: IFFT along y of the spread grid, keep the image rows -> V[iy][gx][l].
template <int G>
__global__ void k_adj_cols(const float2* __restrict__ Hg, int n, int L, int LC, int nchunk,
                           const float2* __restrict__ twg, float2* __restrict__ V) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<G>(s + G * kLines, twg);
    const int gx = blockIdx.x;
    const int l0 = blockIdx.y * LC;
    const int lines = min(LC, L - l0);
    const int pst = blockDim.x / lines;
    const int l = threadIdx.x % lines, p0 = threadIdx.x / lines;
    const int64_t rs = (int64_t)G * L;
    const float2* col = Hg + (int64_t)gx * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 8
        for (int p = p0; p < G; p += pst) s[p * kLines + l] = col[p * rs];
    }
    __syncthreads();
    block_fft<G, true>(s, lines, tw);
    float2* dst = V + (int64_t)gx * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 4
        for (int iy = p0; iy < n; iy += pst) dst[iy * rs] = s[pix_to_grid(iy, n, G) * kLines + l];
    }
}

// Row IFFT + crop + conj(S_l) sum over the coils of chunk blockIdx.y.  With
// one chunk the deapodised image is written directly; otherwise the chunk's
// partial sum goes to part[chunk] and k_adj_chunk_sum finishes.
template <int G>
__global__ void k_adj_rows(const float2* __restrict__ V, const float2* __restrict__ smaps,
                           const float* __restrict__ apod, int n, int L, int LC, int nchunk,
                           float scale, const float2* __restrict__ twg, float2* x,
                           float2* __restrict__ part, float zc, const float2* z) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<G>(s + G * kLines, twg);
    const int iy = blockIdx.x;
    const int l0 = blockIdx.y * LC;
    const int lines = min(LC, L - l0);
    const int pst = blockDim.x / lines;
    const int l = threadIdx.x % lines, p0 = threadIdx.x / lines;
    const float2* src = V + (int64_t)iy * G * L + l0 + l;
    if (p0 < pst) {
#pragma unroll 8
        for (int p = p0; p < G; p += pst) s[p * kLines + l] = src[(int64_t)p * L];
    }
    __syncthreads();
    block_fft<G, true>(s, lines, tw);
    const float ay = apod[iy] * scale;
    for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
        const int p = pix_to_grid(ix, n, G);
        const float2* sm = smaps + ((int64_t)iy * n + ix) * L + l0;
        float2 a = make_float2(0.f, 0.f);
        for (int ll = 0; ll < lines; ++ll) {
            const float2 sv = sm[ll];
            const float2 g = s[p * kLines + ll];
            a.x += sv.x * g.x + sv.y * g.y;
            a.y += sv.x * g.y - sv.y * g.x;
        }
        if (nchunk == 1) {
            const int64_t e = (int64_t)iy * n + ix;
            float2 v = cscale(a, ay * apod[ix]);
            if (z) {
                const float2 zv = z[e];
                v.x = fmaf(zc, zv.x, v.x);
                v.y = fmaf(zc, zv.y, v.y);
            }
            x[e] = v;
        } else {
            part[((int64_t)blockIdx.y * n + iy) * n + ix] = a;
        }
    }
}

__global__ void k_adj_chunk_sum(const float2* __restrict__ part, const float* __restrict__ apod, int n,
                                int nchunk, float scale, float2* x, float zc, const float2* z) {
    const int count = n * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        float2 a = make_float2(0.f, 0.f);
        for (int c = 0; c < nchunk; ++c) a = cadd(a, part[(int64_t)c * count + e]);
        const int iy = e / n, ix = e - iy * n;
        float2 v = cscale(a, apod[iy] * apod[ix] * scale);
        if (z) {
            const float2 zv = z[e];
            v.x = fmaf(zc, zv.x, v.x);
            v.y = fmaf(zc, zv.y, v.y);
        }
        x[e] = v;
    }
}

// ---------------------------------------------------------------- launchers
template <int G>
static int fwd_fft_impl(hqs_plan_s* p, const float2* x, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, G);
    const int th = fft_threads<G>(p->LC);
    const size_t sm = nufft_smem_floats2<G>() * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fwd_rows<G><<<dim3(p->n, p->nchunk), th, sm, st>>>(x, p->smaps, p->apod, p->n, p->L, p->LC,
                                                         p->nchunk, p->scale, tw, p->work);
    k_fwd_cols<G><<<dim3(G, p->nchunk), th, sm, st>>>(p->work, p->n, p->L, p->LC, p->nchunk, tw, p->grid);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int G>
static int adj_fft_impl(hqs_plan_s* p, float2* x, float zc, const float2* z, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, G);
    const int th = fft_threads<G>(p->LC);
    const size_t sm = nufft_smem_floats2<G>() * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_adj_cols<G><<<dim3(G, p->nchunk), th, sm, st>>>(p->grid, p->n, p->L, p->LC, p->nchunk, tw, p->work);
    k_adj_rows<G><<<dim3(p->n, p->nchunk), th, sm, st>>>(p->work, p->smaps, p->apod, p->n, p->L, p->LC,
                                                         p->nchunk, p->scale, tw, x, p->chunk_buf, zc, z);
    if (p->nchunk > 1)
        k_adj_chunk_sum<<<std::min(ceil_div(p->n * p->n, 256), 1024), 256, 0, st>>>(
            p->chunk_buf, p->apod, p->n, p->nchunk, p->scale, x, zc, z);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int W>
static int interp_impl(hqs_plan_s* p, float2* y, cudaStream_t st) {
    if (p->M == 0) return HQS_OK;
    const int64_t threads = p->M * 16;
    k_interp<W><<<(unsigned)ceil_div64(threads, 256), 256, 0, st>>>(p->grid, p->pts, p->perm, (int)p->M,
                                                                    p->G, p->L, (float)p->beta, y);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int W>
static int spread_impl(hqs_plan_s* p, const float2* y, cudaStream_t st) {
    if (p->nsub == 0) return HQS_OK;
    const int P = p->tile + W - 1;
    // coil chunks of <= 8 on the grid's y dimension: a smaller shared patch per
    // CTA keeps more CTAs resident to hide the shared-atomic latency
    const int nch = ceil_div(p->L, 8);
    const int lc = ceil_div(p->L, nch);
    const size_t sm = (size_t)P * P * lc * sizeof(float2) + HQS_SPREAD_MAXPTS * 2 * W * sizeof(float) +
                      HQS_SPREAD_MAXPTS * sizeof(int2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_spread<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_spread<W><<<dim3(p->nsub, nch), 256, sm, st>>>(y, p->pts, p->perm, p->subs, (int)p->M, p->G, p->L, lc,
                                                     nch, p->tile, p->nbx, (float)p->beta, p->grid);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <class F> static int dispatch_w(int W, F&& f) {
    switch (W) {
        case 2: return f.template operator()<2>();
        case 3: return f.template operator()<3>();
        case 4: return f.template operator()<4>();
        case 5: return f.template operator()<5>();
        case 6: return f.template operator()<6>();
        case 7: return f.template operator()<7>();
        case 8: return f.template operator()<8>();
        default: return HQS_ERR_INVALID_ARG;
    }
}

int launch_fwd(hqs_plan_s* p, const float2* x, float2* y, cudaStream_t st) {
    int rc = dispatch_fft_size(p->G, [&]<int GG>() { return fwd_fft_impl<GG>(p, x, st); });
    if (rc != HQS_OK) return rc;
    return dispatch_w(p->W, [&]<int WW>() { return interp_impl<WW>(p, y, st); });
}

int launch_adj_axpy(hqs_plan_s* p, const float2* y, float zc, const float2* z, float2* x, cudaStream_t st) {
    HQS_CUDA_TRY(cudaMemsetAsync(p->grid, 0, (size_t)p->G * p->G * p->L * sizeof(float2), st));
    int rc = dispatch_w(p->W, [&]<int WW>() { return spread_impl<WW>(p, y, st); });
    if (rc != HQS_OK) return rc;
    return dispatch_fft_size(p->G, [&]<int GG>() { return adj_fft_impl<GG>(p, x, zc, z, st); });
}

int launch_adj(hqs_plan_s* p, const float2* y, float2* x, cudaStream_t st) {
    return launch_adj_axpy(p, y, 0.f, nullptr, x, st);
}

extern "C" int hqs_forward(hqs_plan p, const hqs_c64* x, hqs_c64* y, void* stream) {
    if (!p || !x || (!y && p->M > 0)) return HQS_ERR_INVALID_ARG;
    return launch_fwd(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                      (cudaStream_t)stream);
}

extern "C" int hqs_adjoint(hqs_plan p, const hqs_c64* y, hqs_c64* x, void* stream) {
    if (!p || !x || (!y && p->M > 0)) return HQS_ERR_INVALID_ARG;
    return launch_adj(p, reinterpret_cast<const float2*>(y), reinterpret_cast<float2*>(x),
                      (cudaStream_t)stream);
}

extern "C" int hqs_adjoint_axpy(hqs_plan p, const hqs_c64* y, float c, const hqs_c64* z, hqs_c64* x,
                                void* stream) {
    if (!p || !x || !z || (!y && p->M > 0)) return HQS_ERR_INVALID_ARG;
    return launch_adj_axpy(p, reinterpret_cast<const float2*>(y), c, reinterpret_cast<const float2*>(z),
                           reinterpret_cast<float2*>(x), (cudaStream_t)stream);
}
