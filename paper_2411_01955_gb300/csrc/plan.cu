// Plan creation for the multicoil non-Cartesian operator (step a1):
// point coordinates and bin sort on the GPU, Kaiser-Bessel deapodisation
// table, twiddle tables, coil maps in coil-innermost layout, the Toeplitz
// kernel t(d) of A^H A (Sec. 3.4) with its 2N FFT, and the density symbol of
// the circulant CG preconditioner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fft.cuh"
#include "plan.cuh"

using namespace hqs;

static thread_local char g_last_cuda_error[256] = {0};

void hqs_note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s:%d %s -> %s", file, line, what,
             cudaGetErrorString(e));
    if (getenv("HQS_VERBOSE")) fprintf(stderr, "[hqs] %s\n", g_last_cuda_error);
}

extern "C" const char* hqs_status_string(int s) {
    switch (s) {
        case HQS_OK: return "ok";
        case HQS_ERR_INVALID_ARG: return "invalid argument";
        case HQS_ERR_OOM: return "device out of memory";
        case HQS_ERR_NOT_CONVERGED: return "not converged";
        case HQS_ERR_BREAKDOWN: return "CG breakdown (non-positive curvature or non-finite value)";
        case HQS_ERR_TIMEOUT: return "device wait timed out";
        case HQS_ERR_CALLBACK: return "denoiser callback failed";
        case HQS_ERR_CUDA: return g_last_cuda_error[0] ? g_last_cuda_error : "CUDA error";
        case HQS_ERR_UNSUPPORTED: return "unsupported by this build";
        default: return "unknown status";
    }
}

const float2* plan_twiddles(const hqs_plan_s* p, int N) {
    for (int i = 0; i < 4; ++i)
        if (p->tw_sizes[i] == N) return p->tw + p->tw_offs[i];
    return nullptr;
}

// ------------------------------------------------------------- kernels

// (L, n, n) -> (n, n, L)
__global__ void k_smaps_to_coil_inner(const float2* __restrict__ in, float2* __restrict__ out,
                                      int n, int L) {
    const int64_t total = (int64_t)n * n * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % L);
        const int64_t pix = e / L;
        out[e] = in[(int64_t)l * n * n + pix];
    }
}

// Per point: tap origin i0 in [0, G), fractional offset d = u - i0 (u =
// k G / 2 pi wrapped to [0, G), i0 = ceil(u - W/2)), spreading bin, and the
// split phase a = k / 2 pi (mod 1) = a_hi + a_lo used by the Toeplitz kernel.
__global__ void k_point_coords(const float* __restrict__ traj, int M, int G, int W, int TB,
                               int nbx, int4* __restrict__ raw, int* __restrict__ bin,
                               int* __restrict__ counts, float4* __restrict__ phase) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int i0v[2];
    float dv[2];
    float ah[2], al[2];
    int cb[2];
    for (int ax = 0; ax < 2; ++ax) {
        const double k = (double)traj[2 * j + ax];
        double u = (k * (double)G) / (2.0 * 3.141592653589793);
        if (u < 0.0) u += (double)G;
        const double i0 = ceil(u - 0.5 * (double)W);
        const double d = u - i0;
        int ii = (int)i0;
        if (ii < 0) ii += G;
        if (ii >= G) ii -= G;
        i0v[ax] = ii;
        dv[ax] = (float)d;
        int c = ii + W / 2;
        if (c >= G) c -= G;
        cb[ax] = c / TB;
        double a = k / (2.0 * 3.141592653589793);
        a -= rint(a);
        const double hi = rint(a * 8192.0) / 8192.0;
        ah[ax] = (float)hi;
        al[ax] = (float)(a - hi);
    }
    raw[j] = make_int4(i0v[0], i0v[1], __float_as_int(dv[0]), __float_as_int(dv[1]));
    const int b = cb[1] * nbx + cb[0];
    bin[j] = b;
    atomicAdd(&counts[b], 1);
    phase[j] = make_float4(ah[0], al[0], ah[1], al[1]);
}

__global__ void k_point_scatter(const int4* __restrict__ raw, const int* __restrict__ bin, int M,
                                int* __restrict__ cursor, int4* __restrict__ pts,
                                int* __restrict__ perm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int pos = atomicAdd(&cursor[bin[j]], 1);
    pts[pos] = raw[j];
    perm[pos] = j;
}

__global__ void k_invert_perm(const int* __restrict__ perm, int M, int* __restrict__ inv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) inv[perm[j]] = j;
}

// Toeplitz kernel c[py][px] = Npix^-1 sum_j exp(+i (kx_j dx + ky_j dy)), d the
// circulant offset of position p, as a complex GEMM Ey^T Ex whose operands are
// generated in shared memory.  Phases are formed in turns from the split
// a = a_hi + a_lo (a_hi d exact in fp32), products accumulate in fp32 over
// 256 points and then in fp64.
__global__ void __launch_bounds__(256) k_toeplitz_kernel(const float4* __restrict__ phase, int M,
                                                          int n, int n2, double inv_npix,
                                                          float2* __restrict__ c) {
    __shared__ float2 sEy[32][64];
    __shared__ float2 sEx[32][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int py0 = blockIdx.y * 64, px0 = blockIdx.x * 64;
    float2 acc[4][4];
    double accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[i][k] = make_float2(0.f, 0.f);
            accr[i][k] = 0.0;
            acci[i][k] = 0.0;
        }
    int chunk = 0;
    for (int j0 = 0; j0 < M; j0 += 32, ++chunk) {
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            const int jj = e >> 6, dd = e & 63;
            const int j = j0 + jj;
            float2 vy = make_float2(0.f, 0.f), vx = make_float2(0.f, 0.f);
            if (j < M) {
                const float4 a = phase[j];
                const int py = py0 + dd, px = px0 + dd;
                if (py < n2) {
                    const float d = (float)(py < n ? py : py - n2);
                    float tr = a.z * d;
                    tr -= rintf(tr);
                    tr = fmaf(a.w, d, tr);
                    float sn, cs;
                    sincospif(2.0f * tr, &sn, &cs);
                    vy = make_float2(cs, sn);
                }
                if (px < n2) {
                    const float d = (float)(px < n ? px : px - n2);
                    float tr = a.x * d;
                    tr -= rintf(tr);
                    tr = fmaf(a.y, d, tr);
                    float sn, cs;
                    sincospif(2.0f * tr, &sn, &cs);
                    vx = make_float2(cs, sn);
                }
            }
            sEy[jj][dd] = vy;
            sEx[jj][dd] = vx;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            float2 ey[4], ex[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ey[i] = sEy[jj][ty + 16 * i];
#pragma unroll
            for (int k = 0; k < 4; ++k) ex[k] = sEx[jj][tx + 16 * k];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = cfma(ey[i], ex[k], acc[i][k]);
        }
        __syncthreads();
        if ((chunk & 7) == 7) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    accr[i][k] += (double)acc[i][k].x;
                    acci[i][k] += (double)acc[i][k].y;
                    acc[i][k] = make_float2(0.f, 0.f);
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int py = py0 + ty + 16 * i, px = px0 + tx + 16 * k;
            if (py < n2 && px < n2) {
                double re = (accr[i][k] + (double)acc[i][k].x) * inv_npix;
                double im = (acci[i][k] + (double)acc[i][k].y) * inv_npix;
                if (py == n || px == n) re = im = 0.0;
                c[(int64_t)py * n2 + px] = make_float2((float)re, (float)im);
            }
        }
}

// First column of T. Chan's optimal circulant on the N-grid: per axis the
// offsets q (weight (N-q)/N) and q-N (weight q/N).
__global__ void k_chan_column(const float2* __restrict__ c, int n, int n2, float2* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int qy = e / n, qx = e % n;
    const int dys[2] = {qy, qy - n};
    const int dxs[2] = {qx, qx - n};
    const float wys[2] = {(float)(n - qy) / n, (float)qy / n};
    const float wxs[2] = {(float)(n - qx) / n, (float)qx / n};
    float2 acc = make_float2(0.f, 0.f);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int py = (dys[a] + n2) % n2, px = (dxs[b] + n2) % n2;
            const float w = wys[a] * wxs[b];
            const float2 v = c[(int64_t)py * n2 + px];
            acc.x += w * v.x;
            acc.y += w * v.y;
        }
    out[e] = acc;
}

__global__ void k_real_scaled(const float2* __restrict__ in, float* __restrict__ out, int count,
                              float scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) out[e] = in[e].x * scale;
}

// out[c][r] = Re in[r][c] * scale (Khat kept transposed so that a column of
// the Toeplitz spectrum is contiguous for the column pass)
__global__ void k_real_scaled_T(const float2* __restrict__ in, float* __restrict__ out, int nn,
                                float scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nn * nn) return;
    const int r = e / nn, c = e - r * nn;
    out[(int64_t)c * nn + r] = in[e].x * scale;
}

// ------------------------------------------------------------- host side

// Continuous transform of the KB kernel: W sinh(r)/r, r = sqrt(beta^2 - (pi W nu)^2).
static double kb_phihat(double nu, int W, double beta) {
    const double r2 = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
    if (r2 > 1e-300) {
        const double r = sqrt(r2);
        return W * sinh(r) / r;
    }
    if (r2 < -1e-300) {
        const double r = sqrt(-r2);
        return W * sin(r) / r;
    }
    return (double)W;
}

template <class T> static int dev_alloc(hqs_plan_s* p, T** ptr, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) {
        hqs_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        *ptr = nullptr;
        return HQS_ERR_OOM;
    }
    p->allocs.push_back(v);
    p->bytes += count * sizeof(T);
    *ptr = static_cast<T*>(v);
    return HQS_OK;
}

#define HQS_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != HQS_OK) return rc_; \
    } while (0)

static void plan_free(hqs_plan_s* p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    mixed_free(p);
    spread_free(p);
    for (void* v : p->allocs) cudaFree(v);
    if (p->trace) cudaFree(p->trace);
    if (p->h_cg) cudaFreeHost(p->h_cg);
    if (p->h_hist) cudaFreeHost(p->h_hist);
    if (p->h_err) cudaFreeHost(p->h_err);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

static int plan_build(hqs_plan_s* p, const float* traj, const float2* smaps_user, cudaStream_t s) {
    const int n = p->n, L = p->L, G = p->G, n2 = p->n2;
    const int M = (int)p->M;
    // coil chunking for the FFT passes
    p->nchunk = ceil_div(L, HQS_MAX_LC);
    p->LC = ceil_div(L, p->nchunk);
    p->tile = 8;   // every supported G is a multiple of 8
    p->nbx = G / p->tile;
    p->q_rows = 16;
    const int maxg = std::max(G, n2);

    HQS_TRY(dev_alloc(p, &p->smaps, (size_t)n * n * L));
    HQS_TRY(dev_alloc(p, &p->apod, (size_t)n));
    HQS_TRY(dev_alloc(p, &p->pts, (size_t)std::max(M, 1)));
    HQS_TRY(dev_alloc(p, &p->perm, (size_t)std::max(M, 1)));
    HQS_TRY(dev_alloc(p, &p->invperm, (size_t)std::max(M, 1)));
    HQS_TRY(dev_alloc(p, &p->spread.ysort, (size_t)std::max(M, 1) * L));
    HQS_TRY(dev_alloc(p, &p->spread.kbw, (size_t)std::max(M, 1) * 2 * p->W));
    HQS_TRY(dev_alloc(p, &p->khat, (size_t)n2 * n2));
    HQS_TRY(dev_alloc(p, &p->lam, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->grid, (size_t)G * G * L));
    HQS_TRY(dev_alloc(p, &p->work, (size_t)n * maxg * L));
    HQS_TRY(dev_alloc(p, &p->cg_r, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->cg_z, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->cg_p, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->cg_q, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->img_tmp, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->img_tmp2, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->pc_buf, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->img_b0, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->img_rhs, (size_t)n * n));
    HQS_TRY(dev_alloc(p, &p->img_u, (size_t)n * n));
    if (p->nchunk > 1) HQS_TRY(dev_alloc(p, &p->chunk_buf, (size_t)p->nchunk * n * n));
    HQS_TRY(dev_alloc(p, &p->partials, (size_t)NSLOTS * HQS_MAX_BLOCKS));
    HQS_TRY(dev_alloc(p, &p->cg, (size_t)1));
    HQS_TRY(dev_alloc(p, &p->hist, (size_t)HQS_MAX_ITERS + 1));
    HQS_TRY(dev_alloc(p, &p->dev_err, (size_t)4));
    HQS_TRY(dev_alloc(p, &p->barrier, (size_t)64));
    HQS_CUDA_TRY(cudaMallocHost(&p->h_cg, sizeof(CgScalars)));
    HQS_CUDA_TRY(cudaMallocHost(&p->h_hist, sizeof(double) * (HQS_MAX_ITERS + 1)));
    HQS_CUDA_TRY(cudaMallocHost(&p->h_err, sizeof(unsigned)));
    HQS_CUDA_TRY(cudaMemsetAsync(p->cg, 0, sizeof(CgScalars), s));
    HQS_CUDA_TRY(cudaMemsetAsync(p->dev_err, 0, 4 * sizeof(unsigned), s));
    HQS_CUDA_TRY(cudaMemsetAsync(p->barrier, 0, 64 * sizeof(unsigned), s));

    // twiddle bank for the distinct FFT sizes (forward roots, fp64 -> fp32)
    {
        int sizes[3] = {G, n2, n};
        int ns = 0, total = 0;
        for (int i = 0; i < 3; ++i) {
            bool seen = false;
            for (int k = 0; k < ns; ++k) seen |= (p->tw_sizes[k] == sizes[i]);
            if (!seen) {
                p->tw_sizes[ns] = sizes[i];
                p->tw_offs[ns] = total;
                total += sizes[i];
                ++ns;
            }
        }
        std::vector<float2> h(total);
        for (int k = 0; k < ns; ++k)
            for (int m = 0; m < p->tw_sizes[k]; ++m) {
                const double a = -2.0 * M_PI * (double)m / (double)p->tw_sizes[k];
                h[p->tw_offs[k] + m] = make_float2((float)cos(a), (float)sin(a));
            }
        HQS_TRY(dev_alloc(p, &p->tw, (size_t)total));
        HQS_CUDA_TRY(cudaMemcpyAsync(p->tw, h.data(), total * sizeof(float2), cudaMemcpyHostToDevice, s));
        HQS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // deapodisation 1/phihat((i - n/2)/G)
    {
        std::vector<float> h(n);
        for (int i = 0; i < n; ++i) h[i] = (float)(1.0 / kb_phihat((double)(i - n / 2) / G, p->W, p->beta));
        HQS_CUDA_TRY(cudaMemcpyAsync(p->apod, h.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
        HQS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // coil maps
    k_smaps_to_coil_inner<<<std::min(ceil_div(n * n * L, 256), 4096), 256, 0, s>>>(smaps_user, p->smaps, n, L);
    HQS_CUDA_TRY(cudaGetLastError());

    // points: coordinates, histogram, host scan + sub-problems, scatter
    const int nbins = p->nbx * p->nbx;
    int4* raw = nullptr;
    int* bin = nullptr;
    int* counts = nullptr;
    float4* phase = nullptr;
    float2* cbuf = nullptr;
    float2* chan = nullptr;
    auto cleanup = [&]() {
        cudaFree(raw);
        cudaFree(bin);
        cudaFree(counts);
        cudaFree(phase);
        cudaFree(cbuf);
        cudaFree(chan);
    };
    int rc = HQS_OK;
    do {
        const int Mp = std::max(M, 1);
        if (cudaMalloc(&raw, Mp * sizeof(int4)) || cudaMalloc(&bin, Mp * sizeof(int)) ||
            cudaMalloc(&counts, nbins * sizeof(int)) || cudaMalloc(&phase, Mp * sizeof(float4)) ||
            cudaMalloc(&cbuf, (size_t)n2 * n2 * sizeof(float2)) ||
            cudaMalloc(&chan, (size_t)n * n * sizeof(float2))) {
            rc = HQS_ERR_OOM;
            break;
        }
        if (cudaMemsetAsync(counts, 0, nbins * sizeof(int), s)) { rc = HQS_ERR_CUDA; break; }
        if (M > 0) {
            k_point_coords<<<ceil_div(M, 256), 256, 0, s>>>(traj, M, G, p->W, p->tile, p->nbx, raw,
                                                            bin, counts, phase);
        }
        std::vector<int> hc(nbins);
        if (cudaMemcpyAsync(hc.data(), counts, nbins * sizeof(int), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { rc = HQS_ERR_CUDA; break; }
        std::vector<int> offs(nbins);
        int acc = 0;
        for (int b = 0; b < nbins; ++b) {
            offs[b] = acc;
            acc += hc[b];
        }
        if (cudaMemcpyAsync(counts, offs.data(), nbins * sizeof(int), cudaMemcpyHostToDevice, s)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        if (M > 0) {
            k_point_scatter<<<ceil_div(M, 256), 256, 0, s>>>(raw, bin, M, counts, p->pts, p->perm);
            k_invert_perm<<<ceil_div(M, 256), 256, 0, s>>>(p->perm, M, p->invperm);
        }
        if ((rc = launch_point_weights(p, s)) != HQS_OK) break;
        if ((rc = spread_build(p, hc, s)) != HQS_OK) break;

        // Toeplitz kernel, its FFT (Khat, real, scaled by 1/n2^2) and the density symbol
        dim3 gg(ceil_div(n2, 64), ceil_div(n2, 64));
        if (M > 0 && !p->nufft_only) {
            k_toeplitz_kernel<<<gg, 256, 0, s>>>(phase, M, n, n2, 1.0 / ((double)n * n), cbuf);
        } else if (cudaMemsetAsync(cbuf, 0, (size_t)n2 * n2 * sizeof(float2), s)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        k_chan_column<<<ceil_div(n * n, 256), 256, 0, s>>>(cbuf, n, n2, chan);
        if ((rc = launch_fft2d(p, cbuf, n2, false, s)) != HQS_OK) break;
        k_real_scaled_T<<<ceil_div(n2 * n2, 256), 256, 0, s>>>(cbuf, p->khat, n2,
                                                               1.0f / ((float)n2 * (float)n2));
        if ((rc = launch_fft2d(p, chan, n, false, s)) != HQS_OK) break;
        k_real_scaled<<<ceil_div(n * n, 256), 256, 0, s>>>(chan, p->lam, n * n, 1.0f);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            rc = HQS_ERR_CUDA;
            break;
        }
    } while (0);
    cleanup();
    return rc;
}

extern "C" int hqs_plan_create(hqs_plan* out, const float* traj, int64_t M, int ny, int nx,
                               int coils, const hqs_c64* smaps, int kernel_width, float oversamp,
                               void* stream) {
    return plan_create_internal(out, traj, M, ny, nx, coils, smaps, kernel_width, oversamp, stream, false);
}

int plan_create_internal(hqs_plan* out, const float* traj, int64_t M, int ny, int nx, int coils,
                         const hqs_c64* smaps, int kernel_width, float oversamp, void* stream, bool nufft_only) {
    if (!out) return HQS_ERR_INVALID_ARG;
    *out = nullptr;
    if (ny != nx || ny <= 0 || coils <= 0 || coils > 64 || M < 0 || M > (int64_t)1 << 30)
        return HQS_ERR_INVALID_ARG;
    if (kernel_width < 2 || kernel_width > HQS_MAX_W) return HQS_ERR_INVALID_ARG;
    if (!(oversamp >= 1.0f) || !smaps || (M > 0 && !traj)) return HQS_ERR_INVALID_ARG;
    const double Gd = (double)oversamp * ny;
    const int G = (int)lround(Gd);
    if (fabs(Gd - G) > 1e-6 || !fft_size_supported(G) || !fft_size_supported(2 * ny) ||
        !fft_size_supported(ny) || G < kernel_width + 1)
        return HQS_ERR_INVALID_ARG;
    const double bsq = (double)kernel_width / oversamp * (oversamp - 0.5);
    if (bsq * bsq - 0.8 <= 0.0) return HQS_ERR_INVALID_ARG;
    hqs_plan_s* p = new (std::nothrow) hqs_plan_s();
    if (!p) return HQS_ERR_OOM;
    cudaGetDevice(&p->device);
    p->n = ny;
    p->L = coils;
    p->G = G;
    p->n2 = 2 * ny;
    p->W = kernel_width;
    p->oversamp = oversamp;
    p->beta = M_PI * sqrt(bsq * bsq - 0.8);
    p->M = M;
    p->scale = (float)(1.0 / ny);
    p->nufft_only = nufft_only;
    int rc = plan_build(p, traj, reinterpret_cast<const float2*>(smaps), (cudaStream_t)stream);
    if (rc != HQS_OK) {
        plan_free(p);
        return rc;
    }
    *out = p;
    return HQS_OK;
}

// Re-binning of the already sorted points for another spreading tile size.
__global__ void k_rebin(const int4* __restrict__ pts, int M, int G, int W, int TB, int nbx,
                        int* __restrict__ bin, int* __restrict__ counts) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int4 pt = pts[j];
    int cx = pt.x + W / 2, cy = pt.y + W / 2;
    if (cx >= G) cx -= G;
    if (cy >= G) cy -= G;
    const int b = (cy / TB) * nbx + cx / TB;
    bin[j] = b;
    atomicAdd(&counts[b], 1);
}

__global__ void k_rebin_scatter(const int4* __restrict__ pts, const int* __restrict__ perm,
                                const int* __restrict__ bin, int M, int* __restrict__ cursor,
                                int4* __restrict__ pts_out, int* __restrict__ perm_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int pos = atomicAdd(&cursor[bin[j]], 1);
    pts_out[pos] = pts[j];
    perm_out[pos] = perm[j];
}

extern "C" int hqs_plan_retile(hqs_plan p, int tile, void* stream) {
    if (!p || (tile != 8 && tile != 16 && tile != 32) || p->G % tile != 0 || 2 * tile < p->W)
        return HQS_ERR_INVALID_ARG;
    if (tile == p->tile) return HQS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int M = (int)p->M;
    const int nbx = p->G / tile, nbins = nbx * nbx;
    int *bin = nullptr, *counts = nullptr, *perm2 = nullptr;
    int4* pts2 = nullptr;
    int rc = HQS_OK;
    const int old_tile = p->tile, old_nbx = p->nbx;
    do {
        const int Mp = std::max(M, 1);
        if (cudaMalloc(&bin, Mp * sizeof(int)) || cudaMalloc(&counts, nbins * sizeof(int)) ||
            cudaMalloc(&perm2, Mp * sizeof(int)) || cudaMalloc(&pts2, Mp * sizeof(int4))) {
            rc = HQS_ERR_OOM;
            break;
        }
        if (cudaMemsetAsync(counts, 0, nbins * sizeof(int), s)) { rc = HQS_ERR_CUDA; break; }
        if (M > 0) k_rebin<<<ceil_div(M, 256), 256, 0, s>>>(p->pts, M, p->G, p->W, tile, nbx, bin, counts);
        std::vector<int> hc(nbins), offs(nbins);
        if (cudaMemcpyAsync(hc.data(), counts, nbins * sizeof(int), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { rc = HQS_ERR_CUDA; break; }
        int acc = 0;
        for (int b = 0; b < nbins; ++b) {
            offs[b] = acc;
            acc += hc[b];
        }
        if (cudaMemcpyAsync(counts, offs.data(), nbins * sizeof(int), cudaMemcpyHostToDevice, s)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        // items for the new tile first: if they cannot be built the points stay as they are
        p->tile = tile;
        p->nbx = nbx;
        if ((rc = spread_build(p, hc, s)) != HQS_OK) {
            p->tile = old_tile;
            p->nbx = old_nbx;
            break;
        }
        if (M > 0) k_rebin_scatter<<<ceil_div(M, 256), 256, 0, s>>>(p->pts, p->perm, bin, M, counts, pts2, perm2);
        if (M > 0 && (cudaMemcpyAsync(p->pts, pts2, M * sizeof(int4), cudaMemcpyDeviceToDevice, s) ||
                      cudaMemcpyAsync(p->perm, perm2, M * sizeof(int), cudaMemcpyDeviceToDevice, s))) {
            rc = HQS_ERR_CUDA;
            break;
        }
        if (M > 0) k_invert_perm<<<ceil_div(M, 256), 256, 0, s>>>(p->perm, M, p->invperm);
        if ((rc = launch_point_weights(p, s)) != HQS_OK) break;
        if (cudaStreamSynchronize(s)) { rc = HQS_ERR_CUDA; break; }
    } while (0);
    cudaFree(bin);
    cudaFree(counts);
    cudaFree(perm2);
    cudaFree(pts2);
    return rc;
}

// ------------------------------------------------ tile-owned spreading items
void spread_free(hqs_plan_s* p) {
    cudaFree(p->spread.items);
    cudaFree(p->spread.tile_info);
    cudaFree(p->spread.tile_nb);
    cudaFree(p->spread.tickets);
    cudaFree(p->spread.partial);
    p->spread.items = nullptr;
    p->spread.tile_info = nullptr;
    p->spread.tile_nb = nullptr;
    p->spread.tickets = nullptr;
    p->spread.partial = nullptr;
    p->bytes -= p->spread.bytes;
    p->spread.bytes = 0;
    p->spread.nitems = p->spread.nslots = 0;
}

// Every tile of p->tile x p->tile grid cells gets items of at most
// HQS_SPREAD_CAND candidates: the points of its distinct neighbouring bins
// (3 x 3, fewer when the grid has fewer than 3 bins per axis).  A tile with
// more candidates gets several items, each with a partial slot.
int spread_build(hqs_plan_s* p, const std::vector<int>& hc, cudaStream_t s) {
    const int T = p->tile, nbx = p->G / T, nbins = nbx * nbx, L = p->L;
    if ((int)hc.size() != nbins) return HQS_ERR_INVALID_ARG;
    std::vector<int> off(nbins + 1, 0);
    for (int b = 0; b < nbins; ++b) off[b + 1] = off[b] + hc[b];
    auto distinct = [&](int t, int* out) {
        int c = 0;
        for (int d = -1; d <= 1; ++d) {
            const int v = (t + d + nbx) % nbx;
            bool seen = false;
            for (int k = 0; k < c; ++k) seen |= out[k] == v;
            if (!seen) out[c++] = v;
        }
        return c;
    };
    std::vector<int4> items;
    std::vector<int2> info(nbins), nbt((size_t)nbins * 10, make_int2(0, 0));
    int slots = 0;
    for (int t = 0; t < nbins; ++t) {
        int xs[3], ys[3];
        const int cx = distinct(t % nbx, xs), cy = distinct(t / nbx, ys);
        int cand = 0, k = 0;
        for (int a = 0; a < cy; ++a)
            for (int b = 0; b < cx; ++b, ++k) {
                const int bin = ys[a] * nbx + xs[b];
                nbt[(size_t)t * 10 + k] = make_int2(off[bin], cand);
                cand += hc[bin];
            }
        nbt[(size_t)t * 10 + 9] = make_int2(k, cand);
        const int nch = std::max(1, ceil_div(cand, HQS_SPREAD_CAND));
        const int first = nch > 1 ? slots : -1;
        if (nch > 1) slots += nch;
        info[t] = make_int2(nch, first);
        for (int k = 0; k < nch; ++k)
            items.push_back(make_int4(t, k * HQS_SPREAD_CAND, std::min((k + 1) * HQS_SPREAD_CAND, cand),
                                      nch > 1 ? first + k : -1));
    }
    // heaviest items first: the long ones start at once instead of at the end
    std::stable_sort(items.begin(), items.end(),
                     [](const int4& u, const int4& v) { return u.z - u.y > v.z - v.y; });
    const size_t slot_elems = (size_t)T * T * L;
    if ((size_t)slots * slot_elems * sizeof(float2) > ((size_t)1 << 30)) return HQS_ERR_UNSUPPORTED;
    hqs_plan_s::Spread nw;
    nw.nitems = (int)items.size();
    nw.nslots = slots;
    nw.ysort = p->spread.ysort;
    nw.kbw = p->spread.kbw;
    int rc = HQS_OK;
    if (cudaMalloc(&nw.items, items.size() * sizeof(int4)) ||
        cudaMalloc(&nw.tile_info, nbins * sizeof(int2)) || cudaMalloc(&nw.tickets, nbins * sizeof(unsigned)) ||
        cudaMalloc(&nw.tile_nb, (size_t)nbins * 10 * sizeof(int2)) ||
        (slots > 0 && cudaMalloc(&nw.partial, slots * slot_elems * sizeof(float2)))) {
        rc = HQS_ERR_OOM;
    } else if (cudaMemcpyAsync(nw.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s) ||
               cudaMemcpyAsync(nw.tile_info, info.data(), nbins * sizeof(int2), cudaMemcpyHostToDevice, s) ||
               cudaMemcpyAsync(nw.tile_nb, nbt.data(), (size_t)nbins * 10 * sizeof(int2), cudaMemcpyHostToDevice, s) ||
               cudaMemsetAsync(nw.tickets, 0, nbins * sizeof(unsigned), s) || cudaStreamSynchronize(s)) {
        rc = HQS_ERR_CUDA;
    }
    if (rc != HQS_OK) {
        cudaFree(nw.items);
        cudaFree(nw.tile_info);
        cudaFree(nw.tile_nb);
        cudaFree(nw.tickets);
        cudaFree(nw.partial);
        return rc;
    }
    spread_free(p);
    nw.bytes = items.size() * sizeof(int4) + nbins * (11 * sizeof(int2) + sizeof(unsigned)) +
               slots * slot_elems * sizeof(float2);
    p->spread = nw;
    p->bytes += nw.bytes;
    return HQS_OK;
}

extern "C" void hqs_plan_destroy(hqs_plan plan) { plan_free(plan); }

extern "C" int hqs_plan_get_info(hqs_plan p, hqs_plan_info* info) {
    if (!p || !info) return HQS_ERR_INVALID_ARG;
    info->ny = p->n;
    info->nx = p->n;
    info->coils = p->L;
    info->kernel_width = p->W;
    info->oversamp = p->oversamp;
    info->grid = p->G;
    info->npoints = p->M;
    info->kb_beta = p->beta;
    info->device_bytes = p->bytes;
    info->nsub = p->spread.nitems;
    info->tile = p->tile;
    return HQS_OK;
}
