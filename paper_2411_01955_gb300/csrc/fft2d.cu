// Single-image 2D FFT passes: in-place transforms used at plan time (the
// Toeplitz kernel spectrum Khat and the density symbol) and the circulant
// density-compensation preconditioner applied once per CG iteration:
//   z = IFFT_N(FFT_N(r) * m),  m = s^-1/2,  s = max(a*max(lam,0) + b, b/4).
#include "fft.cuh"
#include "plan.cuh"

using namespace hqs;

// Q consecutive rows of a [rows][N] image per CTA, in place.
template <int N, bool INV>
__global__ void k_fft_rows(float2* __restrict__ data, int rows, int Q, const float2* __restrict__ twg) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    const int r0 = blockIdx.x * Q;
    const int lines = min(Q, rows - r0);
#pragma unroll 4
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int q = e / N, pos = e % N;
        s[pos * kLines + q] = data[(int64_t)(r0 + q) * N + pos];
    }
    __syncthreads();
    block_fft<N, INV>(s, lines, tw);
#pragma unroll 4
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int q = e / N, pos = e % N;
        data[(int64_t)(r0 + q) * N + pos] = s[pos * kLines + q];
    }
}

// Q adjacent columns of a [N][cols] image per CTA, in place.
template <int N, bool INV>
__global__ void k_fft_cols(float2* __restrict__ data, int cols, int Q, const float2* __restrict__ twg) {
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    const int c0 = blockIdx.x * Q;
    const int lines = min(Q, cols - c0);
#pragma unroll 4
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int pos = e / lines, q = e % lines;
        s[pos * kLines + q] = data[(int64_t)pos * cols + c0 + q];
    }
    __syncthreads();
    block_fft<N, INV>(s, lines, tw);
#pragma unroll 4
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int pos = e / lines, q = e % lines;
        data[(int64_t)pos * cols + c0 + q] = s[pos * kLines + q];
    }
}

template <int N, bool INV>
static int fft2d_impl(const hqs_plan_s* p, float2* data, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, N);
    if (!tw) return HQS_ERR_INVALID_ARG;
    const int Q = 16;
    const int th = fft_threads<N>(Q);
    const size_t sm = (size_t)(N * kLines + N) * sizeof(float2);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fft_rows<N, INV><<<ceil_div(N, Q), th, sm, st>>>(data, N, Q, tw);
    k_fft_cols<N, INV><<<ceil_div(N, Q), th, sm, st>>>(data, N, Q, tw);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

int launch_fft2d(const hqs_plan_s* p, float2* data, int N, bool inverse, cudaStream_t st) {
    return dispatch_fft_size(N, [&]<int NN>() {
        return inverse ? fft2d_impl<NN, true>(p, data, st) : fft2d_impl<NN, false>(p, data, st);
    });
}

// ------------------------------------------------------ preconditioner

// rows: out[row][:] = FFT_N(in[row][:]) for Q rows per CTA
template <int N>
__global__ void k_pc_rows_fwd(const float2* __restrict__ in, float2* __restrict__ out, int Q,
                              const float2* __restrict__ twg, const CgScalars* __restrict__ cg) {
    if (cg && cg->done) return;
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    const int r0 = blockIdx.x * Q;
    const int lines = min(Q, N - r0);
    constexpr int BD = FftSize<N>::TPL * kLines;
    auto ld = [&](int e) {
        const int q = e / N, pos = e % N;
        s[pos * kLines + q] = in[(int64_t)(r0 + q) * N + pos];
    };
    if (lines == kLines && blockDim.x == BD) unrolled<N * kLines / BD, BD>(threadIdx.x, ld);
    else for (int e = threadIdx.x; e < N * lines; e += blockDim.x) ld(e);
    __syncthreads();
    block_fft<N, false>(s, lines, tw);
    auto st = [&](int e) {
        const int q = e / N, pos = e % N;
        out[(int64_t)(r0 + q) * N + pos] = s[pos * kLines + q];
    };
    if (lines == kLines && blockDim.x == BD) unrolled<N * kLines / BD, BD>(threadIdx.x, st);
    else for (int e = threadIdx.x; e < N * lines; e += blockDim.x) st(e);
}

// columns: FFT, multiply by m = s^-1/2, optional partial sum of |R|^2 m
// (Parseval: N^2 <r, z>), inverse FFT; in place on buf.
template <int N>
__global__ void k_pc_cols(float2* __restrict__ buf, int Q, const float* __restrict__ lam, float a,
                          float b, const float2* __restrict__ twg, const CgScalars* __restrict__ cg,
                          double* __restrict__ part) {
    if (cg && cg->done) return;
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    __shared__ double red[32];
    const int c0 = blockIdx.x * Q;
    const int lines = min(Q, N - c0);
    constexpr int BD = FftSize<N>::TPL * kLines;
    const bool full = lines == kLines && blockDim.x == BD;
    if (full) {
        unrolled<N * kLines / BD, BD>(threadIdx.x, [&](int e) {
            s[e] = buf[(int64_t)(e / kLines) * N + c0 + (e % kLines)];
        });
    } else {
        for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
            const int pos = e / lines, q = e % lines;
            s[pos * kLines + q] = buf[(int64_t)pos * N + c0 + q];
        }
    }
    __syncthreads();
    block_fft<N, false>(s, lines, tw);
    double acc = 0.0;
#pragma unroll 4
    for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
        const int pos = e / lines, q = e % lines;
        const float l = lam[(int64_t)pos * N + c0 + q];
        const float sv = fmaxf(fmaf(a, fmaxf(l, 0.f), b), 0.25f * b);
        const float m = rsqrtf(sv);
        const float2 v = s[pos * kLines + q];
        acc += (double)(m * (v.x * v.x + v.y * v.y));
        s[pos * kLines + q] = cscale(v, m);
    }
    if (part) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (part && threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
    block_fft<N, true>(s, lines, tw);
    if (full) {
        unrolled<N * kLines / BD, BD>(threadIdx.x, [&](int e) {
            buf[(int64_t)(e / kLines) * N + c0 + (e % kLines)] = s[e];
        });
    } else {
        for (int e = threadIdx.x; e < N * lines; e += blockDim.x) {
            const int pos = e / lines, q = e % lines;
            buf[(int64_t)pos * N + c0 + q] = s[pos * kLines + q];
        }
    }
}

// rows: z[row][:] = IFFT_N(buf[row][:]) / N^2
template <int N>
__global__ void k_pc_rows_inv(const float2* __restrict__ buf, float2* __restrict__ z, int Q,
                              const float2* __restrict__ twg, const CgScalars* __restrict__ cg) {
    if (cg && cg->done) return;
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    const int r0 = blockIdx.x * Q;
    const int lines = min(Q, N - r0);
    constexpr int BD = FftSize<N>::TPL * kLines;
    const bool full = lines == kLines && blockDim.x == BD;
    auto ld = [&](int e) {
        const int q = e / N, pos = e % N;
        s[pos * kLines + q] = buf[(int64_t)(r0 + q) * N + pos];
    };
    if (full) unrolled<N * kLines / BD, BD>(threadIdx.x, ld);
    else for (int e = threadIdx.x; e < N * lines; e += blockDim.x) ld(e);
    __syncthreads();
    block_fft<N, true>(s, lines, tw);
    const float sc = 1.0f / ((float)N * (float)N);
    auto st = [&](int e) {
        const int q = e / N, pos = e % N;
        z[(int64_t)(r0 + q) * N + pos] = cscale(s[pos * kLines + q], sc);
    };
    if (full) unrolled<N * kLines / BD, BD>(threadIdx.x, st);
    else for (int e = threadIdx.x; e < N * lines; e += blockDim.x) st(e);
}

template <int N>
static int precond_impl(hqs_plan_s* p, float a, float b, const float2* r, float2* z, bool rows_done,
                        const CgScalars* cg, double* part, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, N);
    const int Q = p->q_rows;
    const int th = fft_threads<N>(Q);
    const size_t sm = (size_t)(N * kLines + N) * sizeof(float2);
    const int nb = ceil_div(N, Q);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_rows_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_rows_inv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (!rows_done) k_pc_rows_fwd<N><<<nb, th, sm, st>>>(r, p->pc_buf, Q, tw, cg);
    k_pc_cols<N><<<nb, th, sm, st>>>(p->pc_buf, Q, p->lam, a, b, tw, cg, part);
    k_pc_rows_inv<N><<<nb, th, sm, st>>>(p->pc_buf, z, Q, tw, cg);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// Full preconditioner apply (standalone entry and solver use).  When
// rows_done is set the forward row pass has already written pc_buf.
int launch_precond_ex(hqs_plan_s* p, float a, float b, const float2* r, float2* z, bool rows_done,
                      const CgScalars* cg, double* part, cudaStream_t st) {
    return dispatch_fft_size(p->n, [&]<int NN>() {
        return precond_impl<NN>(p, a, b, r, z, rows_done, cg, part, st);
    });
}

int launch_precond(hqs_plan_s* p, float a, float b, const float2* r, float2* z, cudaStream_t st) {
    return launch_precond_ex(p, a, b, r, z, false, nullptr, nullptr, st);
}

extern "C" int hqs_precond_apply(hqs_plan p, float a, float b, const hqs_c64* r, hqs_c64* z,
                                 void* stream) {
    if (!p || !r || !z || !(b > 0.f)) return HQS_ERR_INVALID_ARG;
    return launch_precond(p, a, b, reinterpret_cast<const float2*>(r), reinterpret_cast<float2*>(z),
                          (cudaStream_t)stream);
}

// ------------------------------------------------ allocation-free variant
// hqs_precond_apply_noalloc: the density-compensation preconditioner apply
// for callers that must not allocate device memory.  Its scratch (the n x n
// spectrum between the row and column passes) and its twiddle tables are
// file-scope device arrays sized for n <= HQS_NOALLOC_MAX_N; every GPU that
// loads this library holds them until the process exits.
#include <mutex>

#define HQS_NOALLOC_MAX_N 384
#define HQS_NOALLOC_MAX_DEVICES 64
#define HQS_NOALLOC_TW_TOTAL 1200   // 16 + 32 + 64 + 128 + 256 + 320 + 384

static __device__ __align__(256) float2 g_noalloc_spectrum[HQS_NOALLOC_MAX_N * HQS_NOALLOC_MAX_N];
static __device__ __align__(256) float2 g_noalloc_twiddles[HQS_NOALLOC_TW_TOTAL];

static const int kNoallocSizes[7] = {16, 32, 64, 128, 256, 320, 384};

static int noalloc_tw_offset(int n) {
    int off = 0;
    for (int s : kNoallocSizes) {
        if (s == n) return off;
        off += s;
    }
    return -1;
}

// exp(-2 pi i m / N) for every supported N, in double precision, rounded to float
__global__ void k_noalloc_twiddles(float2* tw) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= HQS_NOALLOC_TW_TOTAL) return;
    int off = 0;
    const int sizes[7] = {16, 32, 64, 128, 256, 320, 384};
    for (int i = 0; i < 7; ++i) {
        if (e < off + sizes[i]) {
            double sn, cs;
            sincospi(-2.0 * (double)(e - off) / (double)sizes[i], &sn, &cs);
            tw[e] = make_float2((float)cs, (float)sn);
            return;
        }
        off += sizes[i];
    }
}

struct NoallocDevice {
    bool ready = false;
    unsigned long long ctx_id = 0;   // context the addresses below belong to
    float2* spectrum = nullptr;      // device address of g_noalloc_spectrum
    float2* twiddles = nullptr;      // device address of g_noalloc_twiddles
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[HQS_NOALLOC_MAX_DEVICES];

// The current context's process-unique id (the driver's cuCtxGetId, reached
// through the runtime's entry-point query so that no libcuda link is needed).
// A device reset makes a new context with a new id, so a cache entry keyed by
// it is never reused for the reloaded module.
typedef int (*ctx_get_id_fn)(void* ctx, unsigned long long* id);
static int noalloc_context_id(unsigned long long* id) {
    static ctx_get_id_fn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        HQS_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !f) return HQS_ERR_CUDA;
        fn = reinterpret_cast<ctx_get_id_fn>(f);
    }
    return fn(nullptr, id) == 0 ? HQS_OK : HQS_ERR_CUDA;
}

// Loads the three pass kernels for one size and sets their shared-memory
// limit, so that no later call loads code (which may allocate device memory
// under lazy module loading).
template <int N>
static int noalloc_prepare_size() {
    const int sm = (int)((N * kLines + N) * sizeof(float2));
    cudaFuncAttributes fa;
    HQS_CUDA_TRY(cudaFuncGetAttributes(&fa, k_pc_rows_fwd<N>));
    HQS_CUDA_TRY(cudaFuncGetAttributes(&fa, k_pc_cols<N>));
    HQS_CUDA_TRY(cudaFuncGetAttributes(&fa, k_pc_rows_inv<N>));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_rows_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_pc_rows_inv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return HQS_OK;
}

// Once per device and context, with that device current: resolve the arrays'
// device addresses (their names are only host stand-ins in host code), load
// every kernel this entry point launches, and fill the twiddle tables; the
// caller's stream is synchronised once so that later calls on any stream see
// the tables.
static int noalloc_setup(int dev, cudaStream_t st, NoallocDevice** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice& d = g_noalloc_dev[dev];
    void* spec = nullptr;
    void* tw = nullptr;
    // the lookup also makes the runtime's context current (after a device reset: a new one)
    HQS_CUDA_TRY(cudaGetSymbolAddress(&spec, g_noalloc_spectrum));
    unsigned long long ctx = 0;
    int rc = noalloc_context_id(&ctx);
    if (rc != HQS_OK) return rc;
    if (!d.ready || d.ctx_id != ctx) {
        d.ready = false;
        HQS_CUDA_TRY(cudaGetSymbolAddress(&tw, g_noalloc_twiddles));
        if ((rc = noalloc_prepare_size<16>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<32>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<64>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<128>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<256>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<320>()) != HQS_OK) return rc;
        if ((rc = noalloc_prepare_size<384>()) != HQS_OK) return rc;
        k_noalloc_twiddles<<<ceil_div(HQS_NOALLOC_TW_TOTAL, 256), 256, 0, st>>>(static_cast<float2*>(tw));
        HQS_CUDA_TRY(cudaGetLastError());
        HQS_CUDA_TRY(cudaStreamSynchronize(st));
        d.spectrum = static_cast<float2*>(spec);
        d.twiddles = static_cast<float2*>(tw);
        d.ctx_id = ctx;
        d.ready = true;
    }
    *out = &d;
    return HQS_OK;
}

template <int N>
static int precond_noalloc_impl(const NoallocDevice& d, float a, float b, const float2* r, const float* lam,
                                float2* z, cudaStream_t st) {
    const float2* tw = d.twiddles + noalloc_tw_offset(N);
    const int Q = kLines;
    const int th = fft_threads<N>(Q);
    const size_t sm = (size_t)(N * kLines + N) * sizeof(float2);
    const int nb = ceil_div(N, Q);
    k_pc_rows_fwd<N><<<nb, th, sm, st>>>(r, d.spectrum, Q, tw, nullptr);
    k_pc_cols<N><<<nb, th, sm, st>>>(d.spectrum, Q, lam, a, b, tw, nullptr, nullptr);
    k_pc_rows_inv<N><<<nb, th, sm, st>>>(d.spectrum, z, Q, tw, nullptr);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

extern "C" int hqs_precond_apply_noalloc(const hqs_c64* r, const float* lam, int n, float a, float b,
                                         hqs_c64* z, void* stream) {
    if (!r || !lam || !z || !(b > 0.f) || !(a == a)) return HQS_ERR_INVALID_ARG;
    if (n > HQS_NOALLOC_MAX_N || noalloc_tw_offset(n) < 0) return HQS_ERR_INVALID_ARG;
    int dev = 0;
    HQS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= HQS_NOALLOC_MAX_DEVICES) return HQS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    NoallocDevice* d = nullptr;
    const int rc = noalloc_setup(dev, st, &d);
    if (rc != HQS_OK) return rc;
    const float2* rr = reinterpret_cast<const float2*>(r);
    float2* zz = reinterpret_cast<float2*>(z);
    switch (n) {
        case 16: return precond_noalloc_impl<16>(*d, a, b, rr, lam, zz, st);
        case 32: return precond_noalloc_impl<32>(*d, a, b, rr, lam, zz, st);
        case 64: return precond_noalloc_impl<64>(*d, a, b, rr, lam, zz, st);
        case 128: return precond_noalloc_impl<128>(*d, a, b, rr, lam, zz, st);
        case 256: return precond_noalloc_impl<256>(*d, a, b, rr, lam, zz, st);
        case 320: return precond_noalloc_impl<320>(*d, a, b, rr, lam, zz, st);
        case 384: return precond_noalloc_impl<384>(*d, a, b, rr, lam, zz, st);
        default: return HQS_ERR_INVALID_ARG;
    }
}
