// Annealed PnP-HQS outer loop (a6, a7; Sec. 3.3 and 3.4), the built-in
// Gaussian-smoothing denoiser and the power iteration for ||A^H A||.
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.cuh"
#include "solve.cuh"

#define HQS_BLUR_TILE 32
#define HQS_BLUR_MAXR 24

struct BlurTaps {
    int r;
    float g[2 * HQS_BLUR_MAXR + 1];
};

// One pass over a 32x32 output tile: the tile plus an r-pixel periodic halo
// is staged in shared memory, blurred along x into a second buffer (rows of
// the halo included), then along y into the output.
__global__ void k_gauss_blur(const float2* __restrict__ in, float2* __restrict__ out, int ny, int nx,
                             BlurTaps taps) {
    extern __shared__ float2 sb[];
    const int r = taps.r;
    const int E = HQS_BLUR_TILE + 2 * r;
    float2* tile = sb;             // [E][E]
    float2* mid = sb + E * E;      // [E][TILE]
    const int y0 = blockIdx.y * HQS_BLUR_TILE, x0 = blockIdx.x * HQS_BLUR_TILE;
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        const int ty = e / E, tx = e - ty * E;
        int gy = (y0 + ty - r) % ny;
        int gx = (x0 + tx - r) % nx;
        if (gy < 0) gy += ny;
        if (gx < 0) gx += nx;
        tile[e] = in[(int64_t)gy * nx + gx];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E * HQS_BLUR_TILE; e += blockDim.x) {
        const int ty = e / HQS_BLUR_TILE, tx = e - ty * HQS_BLUR_TILE;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i <= 2 * r; ++i) {
            const float2 v = tile[ty * E + tx + i];
            acc.x = fmaf(taps.g[i], v.x, acc.x);
            acc.y = fmaf(taps.g[i], v.y, acc.y);
        }
        mid[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < HQS_BLUR_TILE * HQS_BLUR_TILE; e += blockDim.x) {
        const int ty = e / HQS_BLUR_TILE, tx = e - ty * HQS_BLUR_TILE;
        const int gy = y0 + ty, gx = x0 + tx;
        if (gy >= ny || gx >= nx) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i <= 2 * r; ++i) {
            const float2 v = mid[(ty + i) * HQS_BLUR_TILE + tx];
            acc.x = fmaf(taps.g[i], v.x, acc.x);
            acc.y = fmaf(taps.g[i], v.y, acc.y);
        }
        out[(int64_t)gy * nx + gx] = acc;
    }
}

extern "C" int hqs_gaussian_denoise(void* user, const hqs_c64* in, hqs_c64* out, int ny, int nx,
                                    float sigma, void* stream) {
    if (!in || !out || ny <= 0 || nx <= 0 || !(sigma >= 0.f)) return HQS_ERR_INVALID_ARG;
    float s = sigma;
    if (user) {
        const hqs_gauss_params* gp = static_cast<const hqs_gauss_params*>(user);
        if (gp->sigma0 > 0.f) s = gp->kappa * sigma / gp->sigma0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (s < 0.1f) {
        if (in != out)
            HQS_CUDA_TRY(cudaMemcpyAsync(out, in, (size_t)ny * nx * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        return HQS_OK;
    }
    BlurTaps taps;
    taps.r = (int)std::ceil(3.0 * (double)s);
    if (taps.r > HQS_BLUR_MAXR || taps.r >= std::min(ny, nx)) return HQS_ERR_INVALID_ARG;
    double sum = 0.0;
    std::vector<double> g(2 * taps.r + 1);
    for (int i = -taps.r; i <= taps.r; ++i) {
        g[i + taps.r] = std::exp(-(double)i * i / (2.0 * (double)s * (double)s));
        sum += g[i + taps.r];
    }
    for (int i = 0; i <= 2 * taps.r; ++i) taps.g[i] = (float)(g[i] / sum);
    const int E = HQS_BLUR_TILE + 2 * taps.r;
    const size_t sm = (size_t)(E * E + E * HQS_BLUR_TILE) * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_gauss_blur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid(ceil_div(nx, HQS_BLUR_TILE), ceil_div(ny, HQS_BLUR_TILE));
    k_gauss_blur<<<grid, 256, sm, st>>>(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                                        ny, nx, taps);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// out = a * u + b * v (+ c * w if w)
__global__ void k_axpbypcz(float2* __restrict__ out, const float2* __restrict__ u, float a,
                           const float2* __restrict__ v, float b, const float2* __restrict__ w, float c,
                           int count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        float2 o = cscale(u[e], a);
        const float2 vv = v[e];
        o.x = fmaf(b, vv.x, o.x);
        o.y = fmaf(b, vv.y, o.y);
        if (w) {
            const float2 ww = w[e];
            o.x = fmaf(c, ww.x, o.x);
            o.y = fmaf(c, ww.y, o.y);
        }
        out[e] = o;
    }
}

extern "C" int hqs_run(hqs_plan p, const hqs_c64* y, hqs_c64* x, const float* mu, const float* sigma,
                       int K, int k0, int cg_iters, float c0, float c1, hqs_denoiser_fn denoiser,
                       void* user, void* stream) {
    if (!p || !x || (!y && p->M > 0) || !mu || !sigma || K < 0 || k0 < 0 || k0 > K || cg_iters < 0 ||
        cg_iters > HQS_MAX_ITERS || !(c0 > 0.f))
        return HQS_ERR_INVALID_ARG;
    for (int k = k0; k < K; ++k)
        if (!(mu[k] > 0.f) || !(sigma[k] >= 0.f)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->n, count = n * n;
    const int nb = std::min(ceil_div(count, 256), 1024);
    float2* xx = reinterpret_cast<float2*>(x);
    hqs_gauss_params gp_default = {1.5f, sigma[0]};
    if (!denoiser && !user) user = &gp_default;
    if (!denoiser) denoiser = hqs_gaussian_denoise;
    HQS_TRY_RC(launch_adj(p, reinterpret_cast<const float2*>(y), p->img_b0, st));
    for (int k = k0; k < K; ++k) {
        const float m = mu[k];
        const float a = 1.0f + c1 * m, b = c0 * m;
        const float2* w = nullptr;
        if (c1 != 0.f) {
            HQS_TRY_RC(launch_toeplitz(p, xx, p->img_tmp, st));
            w = p->img_tmp;
        }
        k_axpbypcz<<<nb, 256, 0, st>>>(p->img_rhs, p->img_b0, 1.0f, xx, m * c0, w, m * c1, count);
        HQS_CUDA_TRY(cudaMemcpyAsync(p->img_u, xx, (size_t)count * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        // the persistent solve (one launch per outer step); per-stage launches for
        // sizes it does not cover
        int rc = pcg_fused(p, a, b, p->img_rhs, p->img_u, cg_iters, 0.0, HQS_PRECOND_DC, HQS_PREC_FP32, false, st);
        if (rc == HQS_ERR_INVALID_ARG || rc == HQS_ERR_UNSUPPORTED)
            rc = pcg_plain(p, a, b, p->img_rhs, p->img_u, cg_iters, 0.0, HQS_PRECOND_DC, false, st);
        HQS_TRY_RC(rc);
        const int drc = denoiser(user, reinterpret_cast<const hqs_c64*>(p->img_u), x, n, n, sigma[k], stream);
        if (drc != 0) return HQS_ERR_CALLBACK;
    }
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// PnP-PGD (Sec. 3.3) in the metric P = c0 I + c1 A^H A of Sec. 3.4:
//   g = A^H A x - A^H y;  u = x - gamma_k (c0 g + c1 A^H A g);  x = D_{sigma_k}(u)
extern "C" int hqs_pgd_run(hqs_plan p, const hqs_c64* y, hqs_c64* x, const float* gamma, const float* sigma,
                           int K, float c0, float c1, hqs_denoiser_fn denoiser, void* user, void* stream) {
    if (!p || !x || (!y && p->M > 0) || !gamma || !sigma || K < 0) return HQS_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (!(gamma[k] > 0.f) || !(sigma[k] >= 0.f)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->n, count = n * n;
    const int nb = std::min(ceil_div(count, 256), 1024);
    float2* xx = reinterpret_cast<float2*>(x);
    hqs_gauss_params gp_default = {1.5f, K > 0 ? sigma[0] : 1.f};
    if (!denoiser && !user) user = &gp_default;
    if (!denoiser) denoiser = hqs_gaussian_denoise;
    HQS_TRY_RC(launch_adj(p, reinterpret_cast<const float2*>(y), p->img_b0, st));
    for (int k = 0; k < K; ++k) {
        HQS_TRY_RC(launch_toeplitz(p, xx, p->img_tmp, st));
        k_axpbypcz<<<nb, 256, 0, st>>>(p->img_rhs, p->img_tmp, 1.0f, p->img_b0, -1.0f, nullptr, 0.f, count);
        const float2* h = nullptr;
        if (c1 != 0.f) {
            HQS_TRY_RC(launch_toeplitz(p, p->img_rhs, p->img_tmp2, st));
            h = p->img_tmp2;
        }
        k_axpbypcz<<<nb, 256, 0, st>>>(p->img_u, xx, 1.0f, p->img_rhs, -gamma[k] * c0, h, -gamma[k] * c1, count);
        const int drc = denoiser(user, reinterpret_cast<const hqs_c64*>(p->img_u), x, n, n, sigma[k], stream);
        if (drc != 0) return HQS_ERR_CALLBACK;
    }
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// ------------------------------------------------------ power iteration
__global__ void k_dot_norm(const float2* __restrict__ v, const float2* __restrict__ w, int count,
                           double* __restrict__ part) {
    __shared__ double red[2][32];
    double vw = 0.0, ww = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 a = v[e], b = w[e];
        vw += (double)a.x * b.x + (double)a.y * b.y;
        ww += (double)b.x * b.x + (double)b.y * b.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        vw += __shfl_xor_sync(0xffffffffu, vw, o);
        ww += __shfl_xor_sync(0xffffffffu, ww, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = vw;
        red[1][threadIdx.x >> 5] = ww;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_scale_into(float2* __restrict__ v, const float2* __restrict__ w, int count, float s) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        v[e] = cscale(w[e], s);
}

extern "C" int hqs_power_iteration(hqs_plan p, int iters, double* lam_max, void* stream) {
    if (!p || !lam_max || iters <= 0) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->n, count = n * n;
    const int nb = std::min(ceil_div(count, 256), 256);
    std::vector<float2> h(count);
    uint64_t s = 0x9E3779B97F4A7C15ull;
    double nrm = 0.0;
    for (int i = 0; i < count; ++i) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const float a = (float)((s >> 40) & 0xFFFFFF) / 16777216.0f - 0.5f;
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const float b = (float)((s >> 40) & 0xFFFFFF) / 16777216.0f - 0.5f;
        h[i] = make_float2(a, b);
        nrm += (double)a * a + (double)b * b;
    }
    const float inv = (float)(1.0 / std::sqrt(nrm));
    for (auto& v : h) v = make_float2(v.x * inv, v.y * inv);
    float2* v = p->img_tmp;
    float2* w = p->img_tmp2;
    HQS_CUDA_TRY(cudaMemcpyAsync(v, h.data(), count * sizeof(float2), cudaMemcpyHostToDevice, st));
    std::vector<double> part(2 * nb);
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        HQS_TRY_RC(launch_toeplitz(p, v, w, st));
        k_dot_norm<<<nb, 256, 0, st>>>(v, w, count, p->partials);
        HQS_CUDA_TRY(cudaMemcpyAsync(part.data(), p->partials, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        double vw = 0.0, ww = 0.0;
        for (int b = 0; b < nb; ++b) {
            vw += part[2 * b];
            ww += part[2 * b + 1];
        }
        lam = vw;
        if (!(ww > 0.0)) break;
        k_scale_into<<<nb, 256, 0, st>>>(v, w, count, (float)(1.0 / std::sqrt(ww)));
    }
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    *lam_max = lam;
    return HQS_OK;
}
