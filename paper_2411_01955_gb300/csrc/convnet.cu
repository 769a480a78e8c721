// Learned CG preconditioner (a10): a 4-layer 3x3 conv net (2 -> H -> H -> H -> 2,
// ReLU) with hand-written forward, backward and Adam kernels, used as
//   z = zdc + s * net(zdc / s),  zdc = M_DC^-1 r,  s = rms(zdc)
// inside flexible CG (learned.cu).  Activations are planar [N][C][H][W] float.
//
// Convolution is cross-correlation with one pixel of zero padding:
//   y[n,o,p] = b[o] + sum_i sum_tap W[o,i,tap] x[n,i,p + tap - 1].
// The input gradient is the same stencil on dz with flipped taps and swapped
// channels, fused with the ReLU mask of the layer input; the weight gradient
// is reduced per 16x16 tile and then over tiles in a fixed order.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>

#include "net.cuh"
#include "tc.cuh"

#define CONV_TILE 16

namespace {

enum ConvMode { CONV_FWD = 0, CONV_FWD_RELU = 1, CONV_DGRAD_MASK = 2 };

// CIN input channels -> COUT output channels on a 16x16 pixel tile.
// CONV_FWD*: weights W[COUT][CIN][9], bias b[COUT].
// CONV_DGRAD_MASK: the layer's weights W[CIN][COUT][9] are read flipped and
// transposed, no bias, output multiplied by (mask > 0).
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(256) k_conv3x3(const float* __restrict__ x, const float* __restrict__ W,
                                                 const float* __restrict__ bias,
                                                 const float* __restrict__ mask, float* __restrict__ y,
                                                 int H, int Wd) {
    extern __shared__ float sm[];
    float* xs = sm;                              // [CIN][18][18]
    float* ws = sm + CIN * 18 * 18;              // [CIN][9][COUT]
    const int n = blockIdx.z;
    const int y0 = blockIdx.y * CONV_TILE, x0 = blockIdx.x * CONV_TILE;
    const int tid = threadIdx.x;
    for (int e = tid; e < CIN * 9 * COUT; e += blockDim.x) {
        const int co = e % COUT, rest = e / COUT;
        const int tap = rest % 9, ci = rest / 9;
        float w;
        if (MODE == CONV_DGRAD_MASK)
            w = W[((size_t)ci * COUT + co) * 9 + (8 - tap)];   // layer W[o = ci][i = co]
        else
            w = W[((size_t)co * CIN + ci) * 9 + tap];
        ws[e] = w;
    }
    const float* xn = x + (size_t)n * CIN * H * Wd;
    for (int e = tid; e < CIN * 18 * 18; e += blockDim.x) {
        const int ci = e / 324, r = e - ci * 324;
        const int ty = r / 18, tx = r - ty * 18;
        const int gy = y0 + ty - 1, gx = x0 + tx - 1;
        xs[e] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? xn[((size_t)ci * H + gy) * Wd + gx] : 0.f;
    }
    __syncthreads();
    const int ty = tid / CONV_TILE, tx = tid % CONV_TILE;
    const int gy = y0 + ty, gx = x0 + tx;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = (MODE == CONV_DGRAD_MASK) ? 0.f : bias[co];
    for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const float v = xs[(ci * 18 + ty + tap / 3) * 18 + tx + tap % 3];
            const float* wr = ws + (ci * 9 + tap) * COUT;
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
        }
    }
    if (gy >= H || gx >= Wd) return;
    float* yn = y + (size_t)n * COUT * H * Wd;
    const float* mn = mask ? mask + (size_t)n * COUT * H * Wd : nullptr;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        const size_t idx = ((size_t)co * H + gy) * Wd + gx;
        float v = acc[co];
        if (MODE == CONV_FWD_RELU) v = fmaxf(v, 0.f);
        if (MODE == CONV_DGRAD_MASK) v = mn[idx] > 0.f ? v : 0.f;
        yn[idx] = v;
    }
}

// Weight and bias gradient partials of one 16x16 tile of one sample:
// part[tile][o*CIN*9 + i*9 + tap] and part[tile][COUT*CIN*9 + o].
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv3x3_wgrad(const float* __restrict__ a, const float* __restrict__ dz,
                                                       float* __restrict__ part, int H, int Wd) {
    extern __shared__ float sm[];
    float* as = sm;                        // [CIN][18][18]
    float* ds = sm + CIN * 324;            // [COUT][16][16]
    const int n = blockIdx.z;
    const int y0 = blockIdx.y * CONV_TILE, x0 = blockIdx.x * CONV_TILE;
    const int tile = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const float* an = a + (size_t)n * CIN * H * Wd;
    const float* dn = dz + (size_t)n * COUT * H * Wd;
    for (int e = threadIdx.x; e < CIN * 324; e += blockDim.x) {
        const int ci = e / 324, r = e - ci * 324;
        const int ty = r / 18, tx = r - ty * 18;
        const int gy = y0 + ty - 1, gx = x0 + tx - 1;
        as[e] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? an[((size_t)ci * H + gy) * Wd + gx] : 0.f;
    }
    for (int e = threadIdx.x; e < COUT * 256; e += blockDim.x) {
        const int co = e / 256, r = e - co * 256;
        const int gy = y0 + r / 16, gx = x0 + r % 16;
        ds[e] = (gy < H && gx < Wd) ? dn[((size_t)co * H + gy) * Wd + gx] : 0.f;
    }
    __syncthreads();
    constexpr int NW = COUT * CIN * 9;
    float* out = part + (size_t)tile * (NW + COUT);
    for (int e = threadIdx.x; e < NW + COUT; e += blockDim.x) {
        float acc = 0.f;
        if (e < NW) {
            const int co = e / (CIN * 9), rest = e - co * CIN * 9;
            const int ci = rest / 9, tap = rest - ci * 9;
            const float* d = ds + co * 256;
            const float* av = as + ci * 324 + (tap / 3) * 18 + tap % 3;
            for (int p = 0; p < 256; ++p) acc = fmaf(d[p], av[(p / 16) * 18 + p % 16], acc);
        } else {
            const float* d = ds + (e - NW) * 256;
            for (int p = 0; p < 256; ++p) acc += d[p];
        }
        out[e] = acc;
    }
}

// ------------------------------------------------ tensor-core 3x3 conv, 32 -> 32
// The hidden layers as implicit GEMMs on the tcgen05 tensor cores.  One output
// tile is 128 pixels of one image row (x0..x0+127 of row y), M = 128, with the
// 32 output channels as N and the 9 taps x 32 input channels as K:
//   D[m][o] = sum over taps (dy, dx) and channels i of X[i][y+dy][x0+m+dx] W[o][i][tap].
// Every operand is split into BF16 hi + lo parts, v = hi + lo + r with
// |r| <= 2^-16 |v|, and multiplied as hi*hi + hi*lo + lo*hi with FP32
// accumulation (each product within 3 * 2^-16 of its exact value, relative).
//
// Shared memory holds three staged input rows (y-1, y, y+1) in a ring, each as
// 130 pixel rows (x0-1..x0+128, zero outside the image) of 128 bytes =
// [32 channels hi | 32 channels lo] BF16, K-major with the 128-byte swizzle.
// A tap's A operand is then a view of the ring: the row buffer of y+dy started
// dx+1 pixel rows in, so no im2col copy exists; a CTA walks a vertical run of output
// rows and stages one new input row per tile, fetched into registers while the
// tensor cores work on the previous tile.  The weights are staged once per CTA
// as 5 chunks of two taps: 64 rows (32 output channels hi, then lo) x 128 bytes.
// Per 16-channel K step and tap two MMAs run: A_hi x [W_hi; W_lo] (N = 64) into
// TMEM columns 0..63 and A_lo x W_hi (N = 32) into columns 64..95; the epilogue
// adds the three 32-column blocks.
constexpr int kTcC = 32, kTcM = 128, kTcThreads = 256;
constexpr int kTcRowPx = kTcM + 2;                          // staged pixels of an input row
constexpr uint32_t kTcRowBytes = 17408;                     // 130 rows x 128 B, rounded up to 1 KB
constexpr uint32_t kTcBChunk = 64 * 128;                    // two taps of W: 64 rows x 128 B
constexpr size_t kTcSmem = 3 * (size_t)kTcRowBytes + 5 * (size_t)kTcBChunk + 16 + 1024;
constexpr int kTcRowUnits = 4 * kTcRowPx;                   // (pixel, 8-channel unit) pairs of a row
constexpr int kTcPer = (kTcRowUnits + kTcThreads - 1) / kTcThreads;
constexpr long long kTcWaitCycles = 2000000000ll;

// byte offset of the 16-byte unit `unit` of row `row` in a 128-byte-swizzled,
// K-major operand region that starts on a 1 KB boundary
__device__ __forceinline__ uint32_t sw128_off(int row, int unit) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((unit ^ (row & 7)) << 4));
}

// descriptor of a view starting at any 128-byte row of a region written with
// the swizzle of its absolute shared-memory addresses: the tensor core applies
// the XOR pattern to the absolute address bits, so the base offset field stays
// 0 (measured on sm_103a for every start row phase 0..7; with the phase in that
// field the reads come out permuted)
__device__ __forceinline__ uint64_t sdesc_view(uint32_t saddr) { return tc::sdesc_sw128(saddr); }

// 8 channels of one operand row, split: hi into unit `uh`, lo into unit `ul`
__device__ __forceinline__ void put_split(uint8_t* base, int row, int uh, int ul, const float* v) {
    uint32_t a[4], b[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * t]), h1 = __float2bfloat16_rn(v[2 * t + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * t] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * t + 1] - __bfloat162float(h1));
        a[t] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        b[t] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint4*>(base + sw128_off(row, uh)) = make_uint4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<uint4*>(base + sw128_off(row, ul)) = make_uint4(b[0], b[1], b[2], b[3]);
}

// input row yy of sample plane xn (channel stride HW), pixels x0-1..x0+128:
// this thread's (pixel, 8-channel unit) pairs idx = tid + k * kTcThreads
__device__ __forceinline__ void fetch_row(const float* __restrict__ xn, int HW, int H, int Wd, int yy, int x0,
                                          float (&v)[kTcPer][8]) {
#pragma unroll
    for (int k = 0; k < kTcPer; ++k) {
        const int idx = threadIdx.x + k * kTcThreads;
        const int q = idx / kTcRowPx, pl = idx - q * kTcRowPx;
        const int xx = x0 - 1 + pl;
        const bool ok = idx < kTcRowUnits && yy >= 0 && yy < H && xx >= 0 && xx < Wd;
        const float* src = xn + (ok ? (size_t)8 * q * HW + (size_t)yy * Wd + xx : 0);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[k][e] = ok ? __ldg(src + (size_t)e * HW) : 0.f;
    }
}

__device__ __forceinline__ void put_row(uint8_t* buf, const float (&v)[kTcPer][8]) {
#pragma unroll
    for (int k = 0; k < kTcPer; ++k) {
        const int idx = threadIdx.x + k * kTcThreads;
        if (idx < kTcRowUnits) {
            const int q = idx / kTcRowPx, pl = idx - q * kTcRowPx;
            put_split(buf, pl, q, 4 + q, v[k]);
        }
    }
}

// MODE as k_conv3x3 (CONV_FWD / CONV_FWD_RELU with bias, CONV_DGRAD_MASK with
// the layer's weights flipped and transposed and the ReLU mask of its input).
// Work unit u = (sample, 128-column strip, run of `rows` output rows).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_conv3x3_tc(const float* __restrict__ x, const float* __restrict__ W, const float* __restrict__ bias,
                 const float* __restrict__ mask, float* __restrict__ y, int N, int H, int Wd, int strips,
                 int rows, int runs, unsigned* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* bsm = ring + 3 * kTcRowBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(bsm + 5 * kTcBChunk);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = H * Wd;
    const int units = N * strips * runs;

    if (tid == 0) {
        tc::mbar_init(bar, 1);
        s_fail = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, 128);
    // W: chunk tap / 2, units (tap & 1) * 4 + q of row o (hi) and row 32 + o (lo)
    for (int u = tid; u < kTcC * 9 * 4; u += blockDim.x) {
        const int q = u & 3, tap = (u >> 2) % 9, o = (u >> 2) / 9;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = 8 * q + e;
            v[e] = MODE == CONV_DGRAD_MASK ? W[((size_t)i * kTcC + o) * 9 + (8 - tap)]   // layer W[o = i][i = o]
                                           : W[((size_t)o * kTcC + i) * 9 + tap];
        }
        uint8_t* cb = bsm + (tap >> 1) * kTcBChunk;
        const int un = (tap & 1) * 4 + q;
        // hi into row o, lo into row 32 + o (same unit)
        uint32_t a[4], b[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * t]), h1 = __float2bfloat16_rn(v[2 * t + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * t] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * t + 1] - __bfloat162float(h1));
            a[t] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            b[t] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        *reinterpret_cast<uint4*>(cb + sw128_off(o, un)) = make_uint4(a[0], a[1], a[2], a[3]);
        *reinterpret_cast<uint4*>(cb + sw128_off(32 + o, un)) = make_uint4(b[0], b[1], b[2], b[3]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t ring_s = tc::smem_u32(ring), b_s = tc::smem_u32(bsm);
    const int g = warp & 3, h = warp >> 2;   // TMEM lane quarter, 16-channel half
    uint32_t phase = 0;
    for (int u = blockIdx.x; u < units && !s_fail; u += gridDim.x) {
        const int n = u / (strips * runs);
        const int rest = u - n * strips * runs;
        const int strip = rest / runs, run = rest - strip * runs;
        const int x0 = strip * kTcM, ya = run * rows, yb = min(H, ya + rows);
        const float* xn = x + (size_t)n * kTcC * HW;
        float pre[kTcPer][8];
        for (int r = 0; r < 3; ++r) {
            fetch_row(xn, HW, H, Wd, ya - 1 + r, x0, pre);
            put_row(ring + r * kTcRowBytes, pre);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        for (int yy = ya; yy < yb; ++yy) {
            const int s0 = (yy - ya) % 3;   // ring slot of row yy - 1; yy and yy + 1 follow
            if (tid == 0) {
                const uint32_t id64 = tc::idesc_f16(kTcM, 64, false), id32 = tc::idesc_f16(kTcM, 32, false);
                uint32_t acc = 0;
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int slot = (s0 + tap / 3) % 3, dx = tap % 3;
                    const uint32_t a = ring_s + slot * kTcRowBytes + dx * 128;
                    const uint32_t b = b_s + (tap >> 1) * kTcBChunk + (tap & 1) * 64;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        tc::mma_f16(tmem, sdesc_view(a + ks * 32), sdesc_view(b + ks * 32), id64, acc);
                        tc::mma_f16(tmem + 64, sdesc_view(a + 64 + ks * 32), sdesc_view(b + ks * 32), id32, acc);
                        acc = 1u;
                    }
                }
                tc::mma_commit(bar);
            }
            const bool more = yy + 1 < yb;
            if (more) fetch_row(xn, HW, H, Wd, yy + 2, x0, pre);   // the next tile's new row
            const bool ok = tc::mbar_wait(bar, phase, kTcWaitCycles, &s_fail);
            phase ^= 1u;
            if (!ok) {
                atomicOr(err, HQS_DEVERR_TIMEOUT);
                s_fail = 1;
            }
            __syncthreads();
            if (s_fail) break;
            tc::fence_after();
            // epilogue: pixels x0 + 32 g + lane, channels 16 h..16 h + 15
            float d0[16], d1[16], d2[16];
            const uint32_t tl = tmem + ((uint32_t)(32 * g) << 16) + 16 * h;
            tc::tmem_ld16(tl, d0);
            tc::tmem_ld16(tl + 32, d1);
            tc::tmem_ld16(tl + 64, d2);
            const int xx = x0 + 32 * g + lane;
            if (xx < Wd) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int co = 16 * h + e;
                    const size_t idx = ((size_t)n * kTcC + co) * HW + (size_t)yy * Wd + xx;
                    float v = (d0[e] + d1[e]) + d2[e];
                    if (MODE != CONV_DGRAD_MASK) v += __ldg(bias + co);
                    if (MODE == CONV_FWD_RELU) v = fmaxf(v, 0.f);
                    if (MODE == CONV_DGRAD_MASK) v = mask[idx] > 0.f ? v : 0.f;
                    y[idx] = v;
                }
            }
            if (more) put_row(ring + s0 * kTcRowBytes, pre);   // row yy + 2 replaces row yy - 1
            tc::fence_proxy_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 128);
    }
}

// out[k] = sum over t of part[t][k] (fixed order), accumulated in fp64.
__global__ void k_sum_tiles(const float* __restrict__ part, int ntiles, int count, float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double acc = 0.0;
    for (int t = 0; t < ntiles; ++t) acc += (double)part[(size_t)t * count + k];
    out[k] = (float)acc;
}

// Per sample: tn = ||t||^2, loss_n = ||o - t||^2 / tn, dout = 2 (o - t) / (N tn).
__global__ void k_rel_mse(const float* __restrict__ o, const float* __restrict__ t, int per, int N,
                          float* __restrict__ dout, double* __restrict__ loss_n) {
    __shared__ double red[32];
    const int n = blockIdx.x;
    const float* on = o + (size_t)n * per;
    const float* tn = t + (size_t)n * per;
    double a = 0.0, d = 0.0;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const double tv = tn[e], df = (double)on[e] - tv;
        a += tv * tv;
        d += df * df;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        d += __shfl_xor_sync(0xffffffffu, d, off);
    }
    __shared__ double red2[32];
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = a;
        red2[threadIdx.x >> 5] = d;
    }
    __syncthreads();
    __shared__ double tot[2];
    if (threadIdx.x == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) {
            s1 += red[w];
            s2 += red2[w];
        }
        tot[0] = s1 > 0.0 ? s1 : 1.0;
        tot[1] = s2;
        loss_n[n] = s2 / tot[0];
    }
    __syncthreads();
    const float sc = (float)(2.0 / ((double)N * tot[0]));
    for (int e = threadIdx.x; e < per; e += blockDim.x) dout[(size_t)n * per + e] = sc * (on[e] - tn[e]);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

template <int CIN, int COUT, int MODE>
int conv_launch(const float* x, const float* W, const float* b, const float* mask, float* y, int N, int H,
                int Wd, cudaStream_t st) {
    const size_t sm = (size_t)(CIN * 324 + CIN * 9 * COUT) * sizeof(float);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
    dim3 grid(ceil_div(Wd, CONV_TILE), ceil_div(H, CONV_TILE), N);
    k_conv3x3<CIN, COUT, MODE><<<grid, 256, sm, st>>>(x, W, b, mask, y, H, Wd);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// the 32 -> 32 layers on the tensor cores: units of (sample, 128-column strip,
// run of output rows), the runs sized so that the units fill two CTAs per SM
template <int MODE>
int conv_tc_launch(const float* x, const float* W, const float* b, const float* mask, float* y, int N, int H,
                   int Wd, unsigned* err, cudaStream_t st) {
    static int sms[64] = {0};
    int dev = 0;
    HQS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return HQS_ERR_UNSUPPORTED;
    if (!sms[dev]) HQS_CUDA_TRY(cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kTcSmem));
    const int slots = 2 * sms[dev];
    const int strips = ceil_div(Wd, kTcM);
    const long long row_tiles = (long long)N * strips * H;
    const int rows = (int)std::min<long long>(H, std::max<long long>(1, (row_tiles + slots - 1) / slots));
    const int runs = ceil_div(H, rows);
    const long long units = (long long)N * strips * runs;
    if (units > INT_MAX) return HQS_ERR_UNSUPPORTED;
    const int grid = (int)std::min<long long>(units, slots);
    k_conv3x3_tc<MODE><<<grid, kTcThreads, kTcSmem, st>>>(x, W, b, mask, y, N, H, Wd, strips, rows, runs, err);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int CIN, int COUT>
int wgrad_launch(const float* a, const float* dz, float* part, float* grad, int N, int H, int Wd,
                 cudaStream_t st) {
    const size_t sm = (size_t)(CIN * 324 + COUT * 256) * sizeof(float);
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
    dim3 grid(ceil_div(Wd, CONV_TILE), ceil_div(H, CONV_TILE), N);
    const int ntiles = grid.x * grid.y * grid.z;
    const int count = COUT * CIN * 9 + COUT;
    k_conv3x3_wgrad<CIN, COUT><<<grid, 256, sm, st>>>(a, dz, part, H, Wd);
    k_sum_tiles<<<ceil_div(count, 256), 256, 0, st>>>(part, ntiles, count, grad);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

}  // namespace

// ------------------------------------------------------------ net object
static size_t layer_offset(int layer) {
    size_t off = 0;
    const int ci[4] = {2, HQS_NET_HIDDEN, HQS_NET_HIDDEN, HQS_NET_HIDDEN};
    const int co[4] = {HQS_NET_HIDDEN, HQS_NET_HIDDEN, HQS_NET_HIDDEN, 2};
    for (int l = 0; l < layer; ++l) off += (size_t)co[l] * ci[l] * 9 + co[l];
    return off;
}

int net_num_params() { return (int)layer_offset(4); }

static int net_reserve(hqs_net_s* net, int N, int H, int Wd) {
    const size_t pix = (size_t)N * H * Wd;
    const size_t tiles = (size_t)N * ceil_div(H, CONV_TILE) * ceil_div(Wd, CONV_TILE);
    if (pix <= net->cap_pix && tiles <= net->cap_tiles) return HQS_OK;
    for (float*& b : net->act) {
        cudaFree(b);
        b = nullptr;
    }
    cudaFree(net->dbuf[0]);
    cudaFree(net->dbuf[1]);
    cudaFree(net->part);
    cudaFree(net->loss_n);
    net->dbuf[0] = net->dbuf[1] = net->part = nullptr;
    net->loss_n = nullptr;
    for (int l = 0; l < 3; ++l) HQS_CUDA_TRY(cudaMalloc(&net->act[l], pix * HQS_NET_HIDDEN * sizeof(float)));
    HQS_CUDA_TRY(cudaMalloc(&net->act[3], pix * 2 * sizeof(float)));
    HQS_CUDA_TRY(cudaMalloc(&net->dbuf[0], pix * HQS_NET_HIDDEN * sizeof(float)));
    HQS_CUDA_TRY(cudaMalloc(&net->dbuf[1], pix * HQS_NET_HIDDEN * sizeof(float)));
    const size_t maxw = (size_t)HQS_NET_HIDDEN * HQS_NET_HIDDEN * 9 + HQS_NET_HIDDEN;
    HQS_CUDA_TRY(cudaMalloc(&net->part, tiles * maxw * sizeof(float)));
    HQS_CUDA_TRY(cudaMalloc(&net->loss_n, (size_t)N * sizeof(double)));
    net->cap_pix = pix;
    net->cap_tiles = tiles;
    net->cap_n = N;
    return HQS_OK;
}

// forward; activations kept in net->act[0..3] (act[3] = output)
int net_forward(hqs_net_s* net, const float* x, float* out, int N, int H, int Wd, cudaStream_t st) {
    HQS_TRY_RC(net_reserve(net, N, H, Wd));
    const float* P = net->params;
    const int Hd = HQS_NET_HIDDEN;
    HQS_TRY_RC((conv_launch<2, HQS_NET_HIDDEN, CONV_FWD_RELU>(x, P + layer_offset(0), P + layer_offset(0) + Hd * 2 * 9,
                                                              nullptr, net->act[0], N, H, Wd, st)));
    for (int l = 1; l <= 2; ++l) {
        const float* Wl = P + layer_offset(l);
        if (net->precision == HQS_PREC_BF16X3)
            HQS_TRY_RC((conv_tc_launch<CONV_FWD_RELU>(net->act[l - 1], Wl, Wl + Hd * Hd * 9, nullptr, net->act[l], N,
                                                      H, Wd, net->dev_err, st)));
        else
            HQS_TRY_RC((conv_launch<HQS_NET_HIDDEN, HQS_NET_HIDDEN, CONV_FWD_RELU>(
                net->act[l - 1], Wl, Wl + Hd * Hd * 9, nullptr, net->act[l], N, H, Wd, st)));
    }
    HQS_TRY_RC((conv_launch<HQS_NET_HIDDEN, 2, CONV_FWD>(net->act[2], P + layer_offset(3),
                                                         P + layer_offset(3) + 2 * Hd * 9, nullptr,
                                                         out ? out : net->act[3], N, H, Wd, st)));
    return HQS_OK;
}

// Back-propagation from the output gradient in net->dbuf[0] (activations of
// the last forward in net->act) into net->grads.
static int net_backprop(hqs_net_s* net, const float* x, int N, int H, int Wd, cudaStream_t st) {
    const float* P = net->params;
    float* G = net->grads;
    float* dz = net->dbuf[0];
    float* da = net->dbuf[1];
    // layer 4 (H -> 2)
    HQS_TRY_RC((wgrad_launch<HQS_NET_HIDDEN, 2>(net->act[2], dz, net->part, G + layer_offset(3), N, H, Wd, st)));
    HQS_TRY_RC((conv_launch<2, HQS_NET_HIDDEN, CONV_DGRAD_MASK>(dz, P + layer_offset(3), nullptr, net->act[2], da, N,
                                                                H, Wd, st)));
    std::swap(dz, da);
    // layers 3 and 2 (H -> H)
    for (int l = 2; l >= 1; --l) {
        HQS_TRY_RC((wgrad_launch<HQS_NET_HIDDEN, HQS_NET_HIDDEN>(net->act[l - 1], dz, net->part, G + layer_offset(l),
                                                                 N, H, Wd, st)));
        if (net->precision == HQS_PREC_BF16X3)
            HQS_TRY_RC((conv_tc_launch<CONV_DGRAD_MASK>(dz, P + layer_offset(l), nullptr, net->act[l - 1], da, N, H,
                                                        Wd, net->dev_err, st)));
        else
            HQS_TRY_RC((conv_launch<HQS_NET_HIDDEN, HQS_NET_HIDDEN, CONV_DGRAD_MASK>(
                dz, P + layer_offset(l), nullptr, net->act[l - 1], da, N, H, Wd, st)));
        std::swap(dz, da);
    }
    // layer 1 (2 -> H)
    HQS_TRY_RC((wgrad_launch<2, HQS_NET_HIDDEN>(x, dz, net->part, G + layer_offset(0), N, H, Wd, st)));
    return HQS_OK;
}

// loss and gradient into net->grads; loss per sample into net->loss_n
static int net_backward(hqs_net_s* net, const float* x, const float* target, int N, int H, int Wd,
                        cudaStream_t st) {
    HQS_TRY_RC(net_forward(net, x, nullptr, N, H, Wd, st));
    const int per = 2 * H * Wd;
    k_rel_mse<<<N, 256, 0, st>>>(net->act[3], target, per, N, net->dbuf[0], net->loss_n);
    HQS_CUDA_TRY(cudaGetLastError());
    return net_backprop(net, x, N, H, Wd, st);
}

// gradient into net->grads for a loss whose gradient with respect to the
// network output is dy (N x 2 x H x W)
static int net_backward_dy(hqs_net_s* net, const float* x, const float* dy, int N, int H, int Wd, cudaStream_t st) {
    HQS_TRY_RC(net_forward(net, x, nullptr, N, H, Wd, st));
    HQS_CUDA_TRY(cudaMemcpyAsync(net->dbuf[0], dy, (size_t)N * 2 * H * Wd * sizeof(float), cudaMemcpyDeviceToDevice,
                                 st));
    return net_backprop(net, x, N, H, Wd, st);
}

static int adam_update(hqs_net_s* net, float lr, cudaStream_t st) {
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, net->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, net->adam_t));
    const int np = net_num_params();
    k_adam<<<ceil_div(np, 256), 256, 0, st>>>(net->params, net->grads, net->m, net->v, np, lr, b1, b2, 1e-8f, c1, c2);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// HQS_ERR_TIMEOUT when a tensor-core convolution of this network gave up a wait
// since the last check (the flag is cleared); blocks on the stream
int net_check(hqs_net_s* net, cudaStream_t st) {
    unsigned e = 0;
    HQS_CUDA_TRY(cudaMemcpyAsync(&e, net->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    if (!e) return HQS_OK;
    HQS_CUDA_TRY(cudaMemsetAsync(net->dev_err, 0, sizeof(unsigned), st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    return HQS_ERR_TIMEOUT;
}

static int read_loss(hqs_net_s* net, int N, double* loss, cudaStream_t st) {
    if (!loss) return HQS_OK;
    std::vector<double> h(N);
    HQS_CUDA_TRY(cudaMemcpyAsync(h.data(), net->loss_n, N * sizeof(double), cudaMemcpyDeviceToHost, st));
    HQS_TRY_RC(net_check(net, st));
    double s = 0.0;
    for (double v : h) s += v;
    *loss = s / N;
    return HQS_OK;
}

extern "C" int hqs_net_create(hqs_net* out) {
    if (!out) return HQS_ERR_INVALID_ARG;
    *out = nullptr;
    hqs_net_s* net = new (std::nothrow) hqs_net_s();
    if (!net) return HQS_ERR_OOM;
    const size_t np = net_num_params();
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&net->params, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->grads, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->m, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->v, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->dev_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(net->dev_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(net->params, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, np * sizeof(float));
    if (e != cudaSuccess) {
        hqs_note_cuda_error(e, "hqs_net_create", __FILE__, __LINE__);
        hqs_net_destroy(net);
        return HQS_ERR_OOM;
    }
    *out = net;
    return HQS_OK;
}

extern "C" void hqs_net_destroy(hqs_net net) {
    if (!net) return;
    cudaFree(net->params);
    cudaFree(net->grads);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->dev_err);
    for (float* b : net->act) cudaFree(b);
    cudaFree(net->dbuf[0]);
    cudaFree(net->dbuf[1]);
    cudaFree(net->part);
    cudaFree(net->loss_n);
    cudaFree(net->zdc);
    cudaFree(net->planar);
    cudaFree(net->scal);
    delete net;
}

extern "C" int hqs_net_num_params(void) { return net_num_params(); }

extern "C" int hqs_net_set_precision(hqs_net net, int precision) {
    if (!net) return HQS_ERR_INVALID_ARG;
    if (precision != HQS_PREC_FP32 && precision != HQS_PREC_BF16X3) return HQS_ERR_UNSUPPORTED;
    net->precision = precision;
    return HQS_OK;
}

extern "C" int hqs_net_status(hqs_net net, void* stream) {
    if (!net) return HQS_ERR_INVALID_ARG;
    return net_check(net, (cudaStream_t)stream);
}

extern "C" int hqs_net_set_params(hqs_net net, const float* host, int count) {
    if (!net || !host || count != net_num_params()) return HQS_ERR_INVALID_ARG;
    HQS_CUDA_TRY(cudaMemcpy(net->params, host, count * sizeof(float), cudaMemcpyHostToDevice));
    HQS_CUDA_TRY(cudaMemset(net->m, 0, count * sizeof(float)));
    HQS_CUDA_TRY(cudaMemset(net->v, 0, count * sizeof(float)));
    net->adam_t = 0;
    return HQS_OK;
}

extern "C" int hqs_net_get_params(hqs_net net, float* host, int count) {
    if (!net || !host || count != net_num_params()) return HQS_ERR_INVALID_ARG;
    HQS_CUDA_TRY(cudaMemcpy(host, net->params, count * sizeof(float), cudaMemcpyDeviceToHost));
    return HQS_OK;
}

extern "C" int hqs_net_forward(hqs_net net, const float* x, float* y, int N, int H, int Wd, void* stream) {
    if (!net || !x || !y || N <= 0 || H <= 0 || Wd <= 0) return HQS_ERR_INVALID_ARG;
    return net_forward(net, x, y, N, H, Wd, (cudaStream_t)stream);
}

extern "C" int hqs_net_gradient(hqs_net net, const float* x, const float* target, int N, int H, int Wd,
                                float* grad, double* loss, void* stream) {
    if (!net || !x || !target || N <= 0 || H <= 0 || Wd <= 0) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HQS_TRY_RC(net_backward(net, x, target, N, H, Wd, st));
    if (grad)
        HQS_CUDA_TRY(cudaMemcpyAsync(grad, net->grads, net_num_params() * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return read_loss(net, N, loss, st);
}

extern "C" int hqs_net_train_step(hqs_net net, const float* x, const float* target, int N, int H, int Wd,
                                  float lr, double* loss, void* stream) {
    if (!net || !x || !target || N <= 0 || H <= 0 || Wd <= 0 || !(lr > 0.f)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HQS_TRY_RC(net_backward(net, x, target, N, H, Wd, st));
    HQS_TRY_RC(adam_update(net, lr, st));
    return read_loss(net, N, loss, st);
}

extern "C" int hqs_net_backward(hqs_net net, const float* x, const float* dy, int N, int H, int Wd, float* grad,
                                void* stream) {
    if (!net || !x || !dy || N <= 0 || H <= 0 || Wd <= 0) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HQS_TRY_RC(net_backward_dy(net, x, dy, N, H, Wd, st));
    if (grad)
        HQS_CUDA_TRY(cudaMemcpyAsync(grad, net->grads, net_num_params() * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HQS_OK;
}

extern "C" int hqs_net_train_step_dy(hqs_net net, const float* x, const float* dy, int N, int H, int Wd, float lr,
                                     void* stream) {
    if (!net || !x || !dy || N <= 0 || H <= 0 || Wd <= 0 || !(lr > 0.f)) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HQS_TRY_RC(net_backward_dy(net, x, dy, N, H, Wd, st));
    return adam_update(net, lr, st);
}

extern "C" int hqs_net_save(hqs_net net, const char* path) {
    if (!net || !path) return HQS_ERR_INVALID_ARG;
    const int np = net_num_params();
    std::vector<float> h(np);
    HQS_TRY_RC(hqs_net_get_params(net, h.data(), np));
    FILE* f = fopen(path, "wb");
    if (!f) return HQS_ERR_INVALID_ARG;
    const char magic[8] = {'H', 'Q', 'S', 'N', 'E', 'T', '0', '1'};
    const int hdr[2] = {HQS_NET_HIDDEN, np};
    const bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 2, f) == 2 &&
                    fwrite(h.data(), sizeof(float), np, f) == (size_t)np;
    fclose(f);
    return ok ? HQS_OK : HQS_ERR_INVALID_ARG;
}

extern "C" int hqs_net_load(hqs_net net, const char* path) {
    if (!net || !path) return HQS_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return HQS_ERR_INVALID_ARG;
    char magic[8];
    int hdr[2];
    const int np = net_num_params();
    std::vector<float> h(np);
    const bool ok = fread(magic, 1, 8, f) == 8 && std::equal(magic, magic + 8, "HQSNET01") &&
                    fread(hdr, sizeof(int), 2, f) == 2 && hdr[0] == HQS_NET_HIDDEN && hdr[1] == np &&
                    fread(h.data(), sizeof(float), np, f) == (size_t)np;
    fclose(f);
    if (!ok) return HQS_ERR_INVALID_ARG;
    return hqs_net_set_params(net, h.data(), np);
}
