// Coil-sensitivity (S-map) estimation (Sec. 4.1): the k-space centre of every
// coil under a separable 20 x 20 Hamming window (times optional density
// weights) taken to the image domain by the single-coil adjoint NUFFT,
// normalised by the coils' root-sum-of-squares and masked where that is below
// a fraction of its maximum.
#include <cmath>

#include "solve.cuh"

namespace {

// yw[j] = h(u_x) h(u_y) d_j y_l[j], u = k n / (2 pi), h(u) = 0.54 + 0.46 cos(2 pi u / width) on |u| <= width / 2
__global__ void k_smap_window(const float* __restrict__ traj, const float* __restrict__ dcf, int64_t M, int n,
                              double width, const float2* __restrict__ y, float2* __restrict__ yw) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= M) return;
    double w = 1.0;
    for (int ax = 0; ax < 2; ++ax) {
        const double u = (double)traj[2 * j + ax] * n / (2.0 * 3.141592653589793);
        w *= fabs(u) <= 0.5 * width ? 0.54 + 0.46 * cos(2.0 * 3.141592653589793 * u / width) : 0.0;
    }
    if (dcf) w *= (double)dcf[j];
    const float2 v = y[j];
    yw[j] = make_float2((float)(v.x * w), (float)(v.y * w));
}

__global__ void k_fill_one(float2* __restrict__ s, int count) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) s[e] = make_float2(1.f, 0.f);
}

// rss[e] = sqrt(sum_l |c_l[e]|^2) (fp64 sum), running maximum as float bits
__global__ void k_smap_rss(const float2* __restrict__ c, int L, int count, float* __restrict__ rss,
                           unsigned* __restrict__ amax) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.f;
    if (e < count) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) {
            const float2 v = c[(size_t)l * count + e];
            s += (double)v.x * v.x + (double)v.y * v.y;
        }
        r = (float)sqrt(s);
        rss[e] = r;
    }
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0 && r > 0.f) atomicMax(amax, __float_as_uint(r));
}

__global__ void k_smap_normalise(float2* __restrict__ c, int L, int count, const float* __restrict__ rss,
                                 const unsigned* __restrict__ amax, float thresh) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float r = rss[e], m = __uint_as_float(*amax);
    const bool in = m > 0.f && r >= thresh * m;
    const float inv = in ? 1.f / r : 0.f;
    for (int l = 0; l < L; ++l) {
        float2& v = c[(size_t)l * count + e];
        v = in ? make_float2(v.x * inv, v.y * inv) : make_float2(0.f, 0.f);
    }
}

}  // namespace

extern "C" int hqs_estimate_smaps(const float* traj, int64_t M, const hqs_c64* y, const float* dcf, int n, int coils,
                                  int kernel_width, float oversamp, float width, float thresh, hqs_c64* smaps,
                                  void* stream) {
    if (!traj || !y || !smaps || M <= 0 || n <= 0 || coils <= 0 || !(width > 0.f) || !(thresh >= 0.f))
        return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int count = n * n;
    float2 *ones = nullptr, *yw = nullptr;
    float* rss = nullptr;
    unsigned* amax = nullptr;
    hqs_plan plan = nullptr;
    int rc = HQS_OK;
    do {
        if (cudaMalloc(&ones, (size_t)count * sizeof(float2)) || cudaMalloc(&yw, (size_t)M * sizeof(float2)) ||
            cudaMalloc(&rss, (size_t)count * sizeof(float)) || cudaMalloc(&amax, sizeof(unsigned))) {
            rc = HQS_ERR_OOM;
            break;
        }
        k_fill_one<<<ceil_div(count, 256), 256, 0, st>>>(ones, count);
        // a gridding-only plan: the estimate needs the adjoint, not the Toeplitz kernel
        rc = plan_create_internal(&plan, traj, M, n, n, 1, reinterpret_cast<const hqs_c64*>(ones), kernel_width,
                                  oversamp, stream, true);
        if (rc != HQS_OK) break;
        float2* out = reinterpret_cast<float2*>(smaps);
        const float2* yy = reinterpret_cast<const float2*>(y);
        for (int l = 0; l < coils && rc == HQS_OK; ++l) {
            k_smap_window<<<(int)ceil_div64(M, 256), 256, 0, st>>>(traj, dcf, M, n, (double)width,
                                                                    yy + (size_t)l * M, yw);
            rc = hqs_adjoint(plan, reinterpret_cast<const hqs_c64*>(yw), reinterpret_cast<hqs_c64*>(out + (size_t)l * count),
                             stream);
        }
        if (rc != HQS_OK) break;
        if (cudaMemsetAsync(amax, 0, sizeof(unsigned), st)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        k_smap_rss<<<ceil_div(count, 256), 256, 0, st>>>(out, coils, count, rss, amax);
        k_smap_normalise<<<ceil_div(count, 256), 256, 0, st>>>(out, coils, count, rss, amax, thresh);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = HQS_ERR_CUDA;
    } while (0);
    cudaStreamSynchronize(st);
    if (plan) hqs_plan_destroy(plan);
    cudaFree(ones);
    cudaFree(yw);
    cudaFree(rss);
    cudaFree(amax);
    return rc;
}
