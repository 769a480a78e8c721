// Flexible CG with the learned preconditioner (a10) and its fallback
// (Notay's truncated flexible CG, one direction kept):
//
//   r = rhs - H x;  z = B(r);  p = z;  rz = Re<r, z>;  pr = rz
//   repeat: q = H p; alpha = pr / Re<p, q>; x += alpha p; r_old = r; r -= alpha q
//           stop on ||r|| <= tol ||rhs|| or max_iter
//           z = B(r); beta = Re<z, r - r_old> / rz (Polak-Ribiere form);
//           pr = Re<z, r> + beta Re<p, r>;  rz = Re<z, r>;  p = z + beta p
// alpha uses <p, r> (exact line search along p), which keeps r orthogonal to
// the previous direction whatever B does.  B(r) = zdc + s net(zdc / s),
// zdc = M_DC^-1 r, s = rms(zdc).  If Re<z, r> <= 0, Re<p, q> <= 0 or ||r||
// drops by less than 10% over 5 iterations, the solve restarts as
// DC-preconditioned CG from the current x for the remaining iterations.
// Scalars are reduced on the host from per-block fp64 partials in a fixed
// order (one synchronisation per iteration).
#include <algorithm>
#include <cmath>
#include <vector>

#include "net.cuh"

namespace {

constexpr int kBlocks = 256;

__global__ void k_rms_partial(const float2* __restrict__ z, int count, double* __restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 v = z[e];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// s = sqrt(sum(part) / count), the same fixed-order sum in every block
__device__ float rms_from_partials(const double* part, int nb, int count) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += part[i];
    return (float)sqrt(t / count);
}

__global__ void k_split_scaled(const float2* __restrict__ z, const double* __restrict__ part, int nb,
                               int count, float* __restrict__ planar) {
    const float s = rms_from_partials(part, nb, count);
    const float inv = s > 0.f ? 1.f / s : 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 v = z[e];
        planar[e] = v.x * inv;
        planar[count + e] = v.y * inv;
    }
}

__global__ void k_combine(const float2* __restrict__ zdc, const float* __restrict__ out,
                          const double* __restrict__ part, int nb, int count, float2* __restrict__ z) {
    const float s = rms_from_partials(part, nb, count);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 d = zdc[e];
        z[e] = make_float2(fmaf(s, out[e], d.x), fmaf(s, out[count + e], d.y));
    }
}

// partials of Re<a, b>, Re<a, c> and Re<d, b> (c, d may be null)
__global__ void k_dot3(const float2* __restrict__ a, const float2* __restrict__ b,
                       const float2* __restrict__ c, const float2* __restrict__ d, int count,
                       double* __restrict__ part) {
    __shared__ double red[3][32];
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 av = a[e], bv = b[e];
        s1 += (double)av.x * bv.x + (double)av.y * bv.y;
        if (c) {
            const float2 cv = c[e];
            s2 += (double)av.x * cv.x + (double)av.y * cv.y;
        }
        if (d) {
            const float2 dv = d[e];
            s3 += (double)dv.x * bv.x + (double)dv.y * bv.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
        red[2][threadIdx.x >> 5] = s3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
            t3 += red[2][w];
        }
        part[blockIdx.x] = t1;
        part[gridDim.x + blockIdx.x] = t2;
        part[2 * gridDim.x + blockIdx.x] = t3;
    }
}

// r_old = r; x += alpha p; r -= alpha q; partial ||r||^2 into part
__global__ void k_fcg_update(float2* __restrict__ x, float2* __restrict__ r, float2* __restrict__ r_old,
                             const float2* __restrict__ p, const float2* __restrict__ q, float alpha,
                             int count, double* __restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 pv = p[e], qv = q[e];
        float2 xv = x[e], rv = r[e];
        r_old[e] = rv;
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        x[e] = xv;
        r[e] = rv;
        acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// p = z + beta p (beta == 0: p = z)
__global__ void k_p_update(const float2* __restrict__ z, float2* __restrict__ p, float beta, int count) {
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

__global__ void k_init_r(const float2* __restrict__ rhs, const float2* __restrict__ q, float2* __restrict__ r,
                         float2* __restrict__ x, int count, double* __restrict__ part) {
    __shared__ double red[2][32];
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
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rr;
        red[1][threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        part[blockIdx.x] = t1;
        part[gridDim.x + blockIdx.x] = t2;
    }
}

__global__ void k_fill_zero(float2* x, int count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        x[e] = make_float2(0.f, 0.f);
}

int host_sums(const double* dev, int n, std::vector<double>& h, cudaStream_t st) {
    h.resize(n);
    HQS_CUDA_TRY(cudaMemcpyAsync(h.data(), dev, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    return HQS_OK;
}

double fixed_sum(const std::vector<double>& h, int off, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += h[off + i];
    return s;
}

}  // namespace

static int ensure_net_buffers(hqs_net_s* net, int n) {
    if (net->cap_img >= n) return HQS_OK;
    cudaFree(net->zdc);
    cudaFree(net->planar);
    cudaFree(net->scal);
    net->zdc = nullptr;
    net->planar = nullptr;
    net->scal = nullptr;
    HQS_CUDA_TRY(cudaMalloc(&net->zdc, (size_t)n * n * sizeof(float2)));
    HQS_CUDA_TRY(cudaMalloc(&net->planar, (size_t)4 * n * n * sizeof(float)));
    HQS_CUDA_TRY(cudaMalloc(&net->scal, (size_t)kBlocks * sizeof(double)));
    net->cap_img = n;
    return HQS_OK;
}

int learned_apply(hqs_plan_s* p, float a, float b, const float2* r, float2* z, cudaStream_t st) {
    hqs_net_s* net = p->net;
    if (!net) return HQS_ERR_UNSUPPORTED;
    const int n = p->n, count = n * n;
    HQS_TRY_RC(ensure_net_buffers(net, n));
    HQS_TRY_RC(launch_precond_ex(p, a, b, r, net->zdc, false, nullptr, nullptr, st));
    k_rms_partial<<<kBlocks, 256, 0, st>>>(net->zdc, count, net->scal);
    k_split_scaled<<<kBlocks, 256, 0, st>>>(net->zdc, net->scal, kBlocks, count, net->planar);
    float* out = net->planar + 2 * (size_t)count;
    HQS_TRY_RC(net_forward(net, net->planar, out, 1, n, n, st));
    k_combine<<<kBlocks, 256, 0, st>>>(net->zdc, out, net->scal, kBlocks, count, z);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

int fcg_learned(hqs_plan_s* p, float a, float b, const float2* rhs, float2* x, int max_iter, double rel_tol,
                bool x0_zero, cudaStream_t st) {
    if (!p->net) return HQS_ERR_UNSUPPORTED;
    const int n = p->n, count = n * n;
    double* part = p->partials;                       // 2 * kBlocks doubles used here
    double* ppq = p->partials + SLOT_PQ * HQS_MAX_BLOCKS;
    float2 *r = p->cg_r, *z = p->cg_z, *pv = p->cg_p, *q = p->cg_q, *r_old = p->img_tmp;
    std::vector<double> h;
    std::vector<double> hist;
    if (!x0_zero) HQS_TRY_RC(launch_toeplitz_ex(p, x, nullptr, 0, q, x, a, b, 1, nullptr, nullptr, st));
    k_init_r<<<kBlocks, 256, 0, st>>>(rhs, x0_zero ? nullptr : q, r, x, count, part);
    HQS_CUDA_TRY(cudaGetLastError());
    HQS_TRY_RC(host_sums(part, 2 * kBlocks, h, st));
    double rr = fixed_sum(h, 0, kBlocks);
    const double bb = fixed_sum(h, kBlocks, kBlocks);
    const double tol2 = rel_tol * rel_tol * bb;
    hist.push_back(rr);
    CgScalars c{};
    c.bnorm = std::sqrt(bb);
    c.max_iter = max_iter;
    c.status = HQS_OK;
    int it = 0;
    bool fallback = false, done = false;
    if (!(bb == bb) || !(rr == rr) || std::isinf(bb) || std::isinf(rr)) {
        c.status = HQS_ERR_BREAKDOWN;
        done = true;
    } else if (bb == 0.0) {
        k_fill_zero<<<kBlocks, 256, 0, st>>>(x, count);
        c.zero_rhs = 1;
        rr = 0.0;
        hist[0] = 0.0;
        done = true;
    } else if (rr <= tol2 || max_iter == 0) {
        done = true;
        if (rr > tol2 && tol2 > 0.0) c.status = HQS_ERR_NOT_CONVERGED;
    }
    double rz = 0.0, pr = 0.0;
    if (!done) {
        HQS_TRY_RC(learned_apply(p, a, b, r, z, st));
        k_dot3<<<kBlocks, 256, 0, st>>>(z, r, nullptr, nullptr, count, part);
        HQS_TRY_RC(host_sums(part, kBlocks, h, st));
        rz = fixed_sum(h, 0, kBlocks);
        pr = rz;
        if (!(rz > 0.0)) fallback = true;
        else k_p_update<<<kBlocks, 256, 0, st>>>(z, pv, 0.f, count);
    }
    while (!done && !fallback) {
        HQS_TRY_RC(launch_toeplitz_ex(p, pv, nullptr, 0, q, pv, a, b, 1, ppq, nullptr, st));
        const int npq = toep_partial_count(p);
        HQS_TRY_RC(host_sums(ppq, npq, h, st));
        const double pq = fixed_sum(h, 0, npq);
        if (!(pq > 0.0) || std::isinf(pq)) {
            fallback = true;
            break;
        }
        const double alpha = pr / pq;
        k_fcg_update<<<kBlocks, 256, 0, st>>>(x, r, r_old, pv, q, (float)alpha, count, part);
        HQS_TRY_RC(host_sums(part, kBlocks, h, st));
        rr = fixed_sum(h, 0, kBlocks);
        ++it;
        hist.push_back(rr);
        if (!(rr == rr) || std::isinf(rr)) {
            c.status = HQS_ERR_BREAKDOWN;
            break;
        }
        if (rr <= tol2) break;
        if (it >= max_iter) {
            if (tol2 > 0.0) c.status = HQS_ERR_NOT_CONVERGED;
            break;
        }
        if (it >= 5 && rr > 0.81 * hist[it - 5]) {   // ||r|| dropped < 10% over 5 iterations
            fallback = true;
            break;
        }
        HQS_TRY_RC(learned_apply(p, a, b, r, z, st));
        k_dot3<<<kBlocks, 256, 0, st>>>(z, r, r_old, pv, count, part);
        HQS_TRY_RC(host_sums(part, 3 * kBlocks, h, st));
        const double rz_new = fixed_sum(h, 0, kBlocks);
        const double z_rold = fixed_sum(h, kBlocks, kBlocks);
        const double p_r = fixed_sum(h, 2 * kBlocks, kBlocks);
        if (!(rz_new > 0.0)) {
            fallback = true;
            break;
        }
        const double beta = (rz_new - z_rold) / rz;
        pr = rz_new + beta * p_r;
        rz = rz_new;
        k_p_update<<<kBlocks, 256, 0, st>>>(z, pv, (float)beta, count);
    }
    if (fallback && it < max_iter) {
        HQS_TRY_RC(pcg_plain(p, a, b, rhs, x, max_iter - it, rel_tol, HQS_PRECOND_DC, false, st));
        CgScalars pc;
        std::vector<double> ph(HQS_MAX_ITERS + 1);
        HQS_CUDA_TRY(cudaMemcpyAsync(&pc, p->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        HQS_CUDA_TRY(cudaMemcpyAsync(ph.data(), p->hist, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 1; i <= pc.it && (int)hist.size() <= HQS_MAX_ITERS; ++i) hist.push_back(ph[i]);
        it += pc.it;
        rr = pc.rr;
        c.status = pc.status;
    }
    c.it = it;
    c.rr = rr;
    c.rz = rz;
    c.tol2 = tol2;
    c.done = 1;
    c.fallback = fallback ? 1 : 0;
    hist.resize(HQS_MAX_ITERS + 1, 0.0);
    HQS_CUDA_TRY(cudaMemcpyAsync(p->cg, &c, sizeof(CgScalars), cudaMemcpyHostToDevice, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(p->hist, hist.data(), hist.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    HQS_CUDA_TRY(cudaMemsetAsync(p->dev_err, 0, sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    return p->net ? net_check(p->net, st) : HQS_OK;
}

extern "C" int hqs_plan_set_net(hqs_plan p, hqs_net net) {
    if (!p) return HQS_ERR_INVALID_ARG;
    p->net = net;
    return HQS_OK;
}

extern "C" int hqs_learned_precond_apply(hqs_plan p, float a, float b, const hqs_c64* r, hqs_c64* z, void* stream) {
    if (!p || !r || !z || !(b > 0.f)) return HQS_ERR_INVALID_ARG;
    if (!p->net) return HQS_ERR_INVALID_ARG;
    return learned_apply(p, a, b, reinterpret_cast<const float2*>(r), reinterpret_cast<float2*>(z),
                         (cudaStream_t)stream);
}

// ------------------------------------------------------------ conv denoiser
// D_sigma(v) = v - sigma net(v / sigma): the network predicts the noise of an
// image whose noise level is normalised to 1, which conditions it on sigma
// (the paper's prior is a sigma-conditioned 2-channel network, Sec. 4.2; this
// is a small stand-in built from the same convolution kernels).
namespace {

__global__ void k_denoise_split(const float2* __restrict__ v, int count, float inv_sigma, float* __restrict__ planar) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 a = v[e];
        planar[e] = a.x * inv_sigma;
        planar[count + e] = a.y * inv_sigma;
    }
}

__global__ void k_denoise_combine(const float2* __restrict__ v, const float* __restrict__ noise, int count,
                                  float sigma, float2* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 a = v[e];
        out[e] = make_float2(fmaf(-sigma, noise[e], a.x), fmaf(-sigma, noise[count + e], a.y));
    }
}

__global__ void k_copy_c64(const float2* __restrict__ a, float2* __restrict__ b, int count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) b[e] = a[e];
}

}  // namespace

extern "C" int hqs_net_denoise(void* user, const hqs_c64* in, hqs_c64* out, int ny, int nx, float sigma,
                               void* stream) {
    hqs_net_s* net = reinterpret_cast<hqs_net_s*>(user);
    if (!net || !in || !out || ny <= 0 || nx <= 0 || !(sigma >= 0.f)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int count = ny * nx;
    const int nb = std::min(ceil_div(count, 256), 1024);
    const float2* v = reinterpret_cast<const float2*>(in);
    float2* o = reinterpret_cast<float2*>(out);
    if (sigma == 0.f) {
        if (v != o) k_copy_c64<<<nb, 256, 0, st>>>(v, o, count);
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    }
    HQS_TRY_RC(ensure_net_buffers(net, std::max(ny, nx)));
    float* x = net->planar;
    float* noise = net->planar + 2 * (size_t)count;
    k_denoise_split<<<nb, 256, 0, st>>>(v, count, 1.f / sigma, x);
    HQS_TRY_RC(net_forward(net, x, noise, 1, ny, nx, st));
    k_denoise_combine<<<nb, 256, 0, st>>>(v, noise, count, sigma, o);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}
