// Mixed-precision Toeplitz normal operator (a8): the four pruned 2n-point DFT
// passes of A^H A x = sum_l conj(S_l) crop(IFFT(Khat . FFT(pad(S_l x))))
// (Toeplitz embedding of Sec. 3.4's normal operator) run as dense DFT-GEMMs on
// the tcgen05 tensor cores with hi/lo split 16-bit operands (BF16 or FP16) and
// FP32 accumulation in TMEM:
//
//   S1  rows (l,y)  x K=(part,x)   . F   -> (l,kx,part,y)   row DFT of pad(S_l x)
//   S2  rows (l,kx) x K=(part,y)   . F   -> *Khat -> (l,kx,part,ky)   column DFT
//   S3  rows (l,kx) x K=(part,ky)  . G   -> (y,l,part,kx)   column IDFT, rows y < n kept
//   S4  rows (y,l)  x K=(part,kx)  . G   -> sum_l conj(S_l) .  row IDFT, x < n kept
//
// Complex data are planar per row ([Re | Im] along K) so that each pass is a
// real GEMM against the real-block form of the complex DFT matrix
// [[Fr, Fi], [-Fi, Fr]]; the zero padding and the crop are pruned into the
// matrix shapes (F = F_2n[0:n, :], G = conj(F_2n)[:, 0:n], both scaled by
// 1/sqrt(2n)).  Each product is a_hi b_hi + a_lo b_hi + a_hi b_lo (the lo*lo
// term is below the FP32 accumulator's resolution), issued as three MMAs.
// BF16 keeps FP32's exponent range, so all three go into one accumulator.
// FP16 lo parts would sink into subnormals, so they are stored scaled by
// 2^11 and their two products go into a second TMEM accumulator that the
// epilogue adds back with 2^-11.  The epilogue of every pass writes the next pass's operand
// already split, in the layout its TMA loads want, so no transpose kernel runs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solve.cuh"
#include "tc.cuh"

namespace {

constexpr int kBM = 128;           // GEMM rows per tile = TMEM lanes
constexpr int kBK = 64;            // 16-bit elements per k-block (one 128-byte swizzle row)
constexpr int kThreads = 320;      // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2-9 epilogue
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, alternating 16-column chunks
constexpr uint32_t kTmemCols = 512;   // two accumulator buffers of 256 columns
constexpr uint32_t kAccStride = 256;
constexpr int kCorrOff = 128;         // FP16: correction accumulator (tiles of <= 128 columns)
constexpr float kLoScale = 2048.f;       // FP16 lo parts are stored x 2^11
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz
constexpr size_t kSmemLimit = 232448;

enum MixedStage { MX_S1 = 0, MX_S2 = 1, MX_S3 = 2, MX_S4 = 3 };

struct MixedArgs {
    int n, n2, L, Lp;
    int cb;                 // complex columns per N tile; the tile is [Re cb | Im cb]
    int BN;                 // = 2 cb
    int M, KB, stages;
    int MT, NT;             // tiles along M and N (persistent tile loop)
    uint16_t* out_hi;       // next pass's operand
    uint16_t* out_lo;
    const float* khat;      // S2: [n2][n2] (kx-major) scaled by 1/kp
    const float2* smaps;    // S4: [n][n][L]
    float2* out;            // S4: [n][n]
    const unsigned* amax;   // bits of max(|Re|,|Im|) of the input image
    float kp;               // S4: spectrum scale to undo
    unsigned* err;
};

// Power-of-two input scale s with max|x s| < 1 (exact scaling).
HQS_DEV float input_scale(const unsigned* amax) {
    const float m = __uint_as_float(*amax);
    if (!(m > 0.f) || isinf(m)) return 1.f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.f, -e);
}

template <bool F16> HQS_DEV void split16(float v, uint16_t& hi, uint16_t& lo) {
    if constexpr (F16) {
        const __half h = __float2half_rn(v);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn((v - __half2float(h)) * kLoScale));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
    }
}
template <bool F16> HQS_DEV float join16(uint16_t hi, uint16_t lo) {
    if constexpr (F16) return __half2float(__ushort_as_half(hi)) + __half2float(__ushort_as_half(lo)) / kLoScale;
    else return __bfloat162float(__ushort_as_bfloat16(hi)) + __bfloat162float(__ushort_as_bfloat16(lo));
}

// 16 accumulator columns: main (+ correction / 2^11 for FP16)
template <bool F16> HQS_DEV void acc_ld16(uint32_t tl, int col, int corr_off, float* v) {
    tc::tmem_ld16(tl + col, v);
    if constexpr (F16) {
        float c[16];
        tc::tmem_ld16(tl + corr_off + col, c);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaf(c[i], 1.f / kLoScale, v[i]);
    }
}

// Transposing store of 16 accumulator columns: lanes 2k and 2k+1 hold two rows
// that are adjacent elements of the destination, so the pair is written as one
// 32-bit word per column (even lanes take even columns, odd lanes odd ones);
// idx(i) is the element index of column i at the pair's even row.
template <bool F16, class Idx>
HQS_DEV void store_pairs(const float* v, int lane, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, Idx idx) {
    const int odd = lane & 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float send = odd ? v[2 * j] : v[2 * j + 1];
        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
        const float r0 = odd ? recv : v[2 * j];
        const float r1 = odd ? v[2 * j + 1] : recv;
        uint16_t h0, l0, h1, l1;
        split16<F16>(r0, h0, l0);
        split16<F16>(r1, h1, l1);
        const size_t e = idx(2 * j + odd);
        *reinterpret_cast<uint32_t*>(hi + e) = (uint32_t)h0 | ((uint32_t)h1 << 16);
        *reinterpret_cast<uint32_t*>(lo + e) = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
}

// ------------------------------------------------------------ the GEMM pass
template <int STAGE, bool F16>
HQS_DEV void pass_epilogue(const MixedArgs& P, uint32_t tl, int m, int nt, int lane, int h) {
    const int n = P.n, n2 = P.n2, cb = P.cb;
    const bool valid = m < P.M;
    if constexpr (STAGE == MX_S4) {
        const int Lp = P.Lp, y = m / Lp, l = m - y * Lp;
        const float f = P.kp / input_scale(P.amax);
        for (int w = 16 * h; w < cb; w += 32) {
            const int x0 = nt * cb + w;
            // coil-map values first: their latency overlaps the TMEM loads
            float2 sv[16];
            const bool own = valid && l < P.L;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                sv[i] = own ? P.smaps[((size_t)y * n + x0 + i) * P.L + l] : make_float2(0.f, 0.f);
            float re[16], im[16];
            acc_ld16<F16>(tl, w, kCorrOff, re);
            acc_ld16<F16>(tl, cb + w, kCorrOff, im);
            float2 acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = cmulc(sv[i], make_float2(re[i], im[i]));
            for (int off = Lp >> 1; off > 0; off >>= 1) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    acc[i].x += __shfl_xor_sync(0xffffffffu, acc[i].x, off);
                    acc[i].y += __shfl_xor_sync(0xffffffffu, acc[i].y, off);
                }
            }
            if (valid && l == 0) {
                float4* dst = reinterpret_cast<float4*>(P.out + (size_t)y * n + x0);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    dst[i] = make_float4(acc[2 * i].x * f, acc[2 * i].y * f, acc[2 * i + 1].x * f,
                                         acc[2 * i + 1].y * f);
            }
        }
        (void)lane;
    } else {
        for (int w = 16 * h; w < P.BN; w += 32) {
            const int part = w >= cb ? 1 : 0;
            const int c0 = nt * cb + w - part * cb;
            float4 k4[4];
            if constexpr (STAGE == MX_S2) {
                // Khat row values first: their latency overlaps the TMEM loads
                const float4* kr = reinterpret_cast<const float4*>(P.khat + (size_t)(m % n2) * n2 + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) k4[i] = valid ? __ldg(kr + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float v[16];
            acc_ld16<F16>(tl, w, kCorrOff, v);
            if (!valid) continue;   // warp-uniform: M and the warp's 32 rows are multiples of 32
            if constexpr (STAGE == MX_S1) {
                // rows (l, y) -> next operand rows (l, kx), K = (part, y); lanes 2k, 2k+1
                // hold y, y+1 (a warp's 32 rows lie in one coil since 32 | n)
                const int l = m / n, y = m - l * n;
                store_pairs<F16>(v, lane, P.out_hi, P.out_lo,
                                 [&](int i) { return (size_t)(l * n2 + c0 + i) * (2 * n) + part * n + (y & ~1); });
            } else if constexpr (STAGE == MX_S2) {
                // * Khat[kx][ky], same rows (l, kx), K = (part, ky)
                uint16_t hs[16], ls[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    split16<F16>(v[4 * i] * k4[i].x, hs[4 * i], ls[4 * i]);
                    split16<F16>(v[4 * i + 1] * k4[i].y, hs[4 * i + 1], ls[4 * i + 1]);
                    split16<F16>(v[4 * i + 2] * k4[i].z, hs[4 * i + 2], ls[4 * i + 2]);
                    split16<F16>(v[4 * i + 3] * k4[i].w, hs[4 * i + 3], ls[4 * i + 3]);
                }
                const size_t idx = (size_t)m * (4 * n) + part * n2 + c0;
                uint4* dh = reinterpret_cast<uint4*>(P.out_hi + idx);
                uint4* dl = reinterpret_cast<uint4*>(P.out_lo + idx);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint32_t a[4], b[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        a[t] = (uint32_t)hs[8 * j + 2 * t] | ((uint32_t)hs[8 * j + 2 * t + 1] << 16);
                        b[t] = (uint32_t)ls[8 * j + 2 * t] | ((uint32_t)ls[8 * j + 2 * t + 1] << 16);
                    }
                    dh[j] = make_uint4(a[0], a[1], a[2], a[3]);
                    dl[j] = make_uint4(b[0], b[1], b[2], b[3]);
                }
            } else {
                // rows (l, kx) -> next operand rows (y, l) (coil-padded to Lp), K = (part, kx);
                // lanes 2k, 2k+1 hold kx, kx+1
                const int l = m / n2, kx = m - l * n2;
                store_pairs<F16>(v, lane, P.out_hi, P.out_lo, [&](int i) {
                    return (size_t)((c0 + i) * P.Lp + l) * (4 * n) + part * n2 + (kx & ~1);
                });
            }
        }
    }
}

// Persistent: one CTA per SM walks the tiles t = blockIdx.x + i gridDim.x
// (N tile fastest, so CTAs running together share A rows in L2).  The
// shared-memory ring continues across tiles, and the accumulator is double
// buffered in TMEM, so the epilogue of tile i overlaps the MMAs of tile i+1.
template <int STAGE, bool F16>
__global__ void __launch_bounds__(kThreads, 1)
    k_dft_gemm(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
               const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
               const MixedArgs P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t a_bytes = kBM * kBK * 2;
    const uint32_t b_bytes = (uint32_t)P.BN * kBK * 2;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const int ST = P.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + ST * stage_bytes);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;     // [2] accumulator buffer ready for the epilogue
    uint64_t* tempty = tfull + 2;     // [2] accumulator buffer drained by the epilogue
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ int s_fail;
    const volatile int* fail = &s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = P.MT * P.NT;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], kEpiWarps);
        }
        s_fail = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int c = 0;
            for (int t = blockIdx.x; t < tiles && !*fail; t += gridDim.x) {
                const int m0 = (t / P.NT) * kBM, n0 = (t % P.NT) * P.BN;
                for (int kb = 0; kb < P.KB; ++kb, ++c) {
                    const int s = c % ST;
                    if (c >= ST && !tc::mbar_wait(&empty[s], ((c / ST) - 1) & 1, kWaitCycles, fail)) {
                        atomicOr(P.err, HQS_DEVERR_TIMEOUT);
                        s_fail = 1;
                        break;
                    }
                    uint8_t* st = smem + s * stage_bytes;
                    tc::mbar_expect_tx(&full[s], stage_bytes);
                    tc::tma_load_2d(st, &tA_hi, &full[s], kb * kBK, m0);
                    tc::tma_load_2d(st + a_bytes, &tA_lo, &full[s], kb * kBK, m0);
                    tc::tma_load_2d(st + 2 * a_bytes, &tB_hi, &full[s], kb * kBK, n0);
                    tc::tma_load_2d(st + 2 * a_bytes + b_bytes, &tB_lo, &full[s], kb * kBK, n0);
                }
            }
            // on failure, let the copies in flight land before the CTA leaves
            if (*fail)
                for (int k = max(0, c - ST); k < c; ++k) tc::mbar_wait(&full[k % ST], (k / ST) & 1, kWaitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kBM, P.BN, F16);
            int c = 0, i = 0;
            for (int t = blockIdx.x; t < tiles && !*fail; t += gridDim.x, ++i) {
                const int buf = i & 1;
                if (i >= 2 && !tc::mbar_wait(&tempty[buf], ((i >> 1) - 1) & 1, kWaitCycles, fail)) {
                    atomicOr(P.err, HQS_DEVERR_TIMEOUT);
                    s_fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t d = tmem + buf * kAccStride;
                for (int kb = 0; kb < P.KB; ++kb, ++c) {
                    const int s = c % ST;
                    if (!tc::mbar_wait(&full[s], (c / ST) & 1, kWaitCycles, fail)) {
                        atomicOr(P.err, HQS_DEVERR_TIMEOUT);
                        s_fail = 1;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t base = tc::smem_u32(smem + s * stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t ah = tc::sdesc_sw128(base + kk * 32);
                        const uint64_t al = tc::sdesc_sw128(base + a_bytes + kk * 32);
                        const uint64_t bh = tc::sdesc_sw128(base + 2 * a_bytes + kk * 32);
                        const uint64_t bl = tc::sdesc_sw128(base + 2 * a_bytes + b_bytes + kk * 32);
                        const uint32_t acc = (kb | kk) != 0 ? 1u : 0u;
                        tc::mma_f16(d, ah, bh, idesc, acc);
                        if constexpr (F16) {
                            tc::mma_f16(d + kCorrOff, al, bh, idesc, acc);
                            tc::mma_f16(d + kCorrOff, ah, bl, idesc, 1u);
                        } else {
                            tc::mma_f16(d, al, bh, idesc, 1u);
                            tc::mma_f16(d, ah, bl, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&tfull[buf]);
            }
        }
    } else {
        const int q = warp & 3;   // TMEM lane quarter this warp may read
        const int h = (warp - 2) >> 2;   // which half of the 16-column chunks
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int buf = i & 1;
            const bool ok = tc::mbar_wait(&tfull[buf], (i >> 1) & 1, kWaitCycles, fail);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    atomicOr(P.err, HQS_DEVERR_TIMEOUT);
                    s_fail = 1;
                }
                break;
            }
            tc::fence_after();
            const uint32_t tl = tmem + buf * kAccStride + ((uint32_t)(32 * q) << 16);
            pass_epilogue<STAGE, F16>(P, tl, (t / P.NT) * kBM + 32 * q + lane, t % P.NT, lane, h);
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------ helper kernels
// Bt[nn][k] (N rows, K-major) of the real-block DFT matrix, hi/lo split.
// kind 0: F[j][c] = e^{-2 pi i j c / n2} / sqrt(n2), j < n, c < n2
// kind 1: G[j][c] = e^{+2 pi i j c / n2} / sqrt(n2), j < n2, c < n
template <bool F16>
__global__ void k_mx_build_b(uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, int kind, int n, int cb) {
    const int n2 = 2 * n;
    const int Kc = kind == 0 ? n : n2, Nc = kind == 0 ? n2 : n;
    const int Kr = 2 * Kc, Nr = 2 * Nc, BN = 2 * cb;
    const int64_t total = (int64_t)Kr * Nr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int nn = (int)(e / Kr), k = (int)(e - (int64_t)nn * Kr);
        const int t = nn / BN, w = nn - t * BN;
        const int pout = w >= cb ? 1 : 0;
        const int c = t * cb + w - pout * cb;
        const int pin = k >= Kc ? 1 : 0;
        const int j = k - pin * Kc;
        const int r = (int)(((int64_t)j * c) % n2);
        double s, co;
        sincospi((double)r / (double)n, &s, &co);   // angle 2 pi r / n2
        const double inv = 1.0 / sqrt((double)n2);
        const double fr = co * inv, fi = (kind == 0 ? -s : s) * inv;
        double v;
        if (pin == 0) v = pout == 0 ? fr : fi;
        else v = pout == 0 ? -fi : fr;
        float hf;
        if constexpr (F16) {
            const __half h = __double2half(v);
            hf = __half2float(h);
            hi[e] = __half_as_ushort(h);
            lo[e] = __half_as_ushort(__double2half((v - (double)hf) * kLoScale));
        } else {
            const __nv_bfloat16 h = __double2bfloat16(v);
            hf = __bfloat162float(h);
            hi[e] = __bfloat16_as_ushort(h);
            lo[e] = __bfloat16_as_ushort(__double2bfloat16(v - (double)hf));
        }
    }
}

// max(|Re|, |Im|) over a complex array (non-negative float bits compare as unsigned)
__global__ void k_mx_amax(const float2* __restrict__ x, int count, unsigned* __restrict__ amax) {
    float m = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float2 v = x[e];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(amax, __float_as_uint(m));
}

// Khat' = Khat * n2^2 / kp (kx-major, as the plan stores it)
__global__ void k_mx_khat(const float* __restrict__ khat, int count, float f, float* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) out[e] = khat[e] * f;
}

// S1 operand: rows (l, y), K = [Re x | Im x] of s * S_l x, hi/lo split
template <bool F16>
__global__ void k_mx_prologue(const float2* __restrict__ x, const float2* __restrict__ smaps, int n, int L,
                              const unsigned* __restrict__ amax, uint16_t* __restrict__ hi,
                              uint16_t* __restrict__ lo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int y = e / n, xi = e - y * n;
    const float s = input_scale(amax);
    const float2 u = cscale(x[e], s);
    for (int l = 0; l < L; ++l) {
        const float2 v = cmul(smaps[(size_t)e * L + l], u);
        const size_t idx = (size_t)(l * n + y) * (2 * n) + xi;
        uint16_t h, o;
        split16<F16>(v.x, h, o);
        hi[idx] = h;
        lo[idx] = o;
        split16<F16>(v.y, h, o);
        hi[idx + n] = h;
        lo[idx + n] = o;
    }
}

// out = a v + b pmul, partial <pmul, out> (mode 1), or out = v (mode 0)
__global__ void k_mx_hepilogue(const float2* __restrict__ v, float2* __restrict__ out,
                               const float2* __restrict__ pmul, float a, float b, int mode, int count,
                               double* __restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        float2 w = v[e];
        if (mode == 1) {
            const float2 pv = pmul[e];
            w = make_float2(fmaf(a, w.x, b * pv.x), fmaf(a, w.y, b * pv.y));
            acc += (double)pv.x * w.x + (double)pv.y * w.y;
        }
        out[e] = w;
    }
    if (part) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            part[blockIdx.x] = t;
        }
    }
}

// Intermediate of pass `stage` (1..3) back to complex64 in natural layout,
// unscaled: stage 1 -> [l][y][kx], stage 2 -> [l][ky][kx], stage 3 -> [l][y][kx].
template <bool F16>
__global__ void k_mx_dump(const uint16_t* __restrict__ hi, const uint16_t* __restrict__ lo, int stage, int n,
                          int L, int Lp, float base, const unsigned* __restrict__ amax, float2* __restrict__ out) {
    const int n2 = 2 * n;
    const int64_t rows = stage == 2 ? (int64_t)L * n2 : (int64_t)L * n;
    const int64_t total = rows * n2;
    const float f = base / input_scale(amax);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % n2);
        const int64_t r = e / n2;
        size_t ire, iim;
        if (stage == 1) {          // r = (l, y); X2 rows (l, kx), K = (part, y) of length 2n
            const int l = (int)(r / n), y = (int)(r % n);
            ire = (size_t)(l * n2 + kx) * (2 * n) + y;
            iim = ire + n;
        } else if (stage == 2) {   // r = (l, ky); X3 rows (l, kx), K = (part, ky) of length 4n
            const int l = (int)(r / n2), ky = (int)(r % n2);
            ire = (size_t)(l * n2 + kx) * (4 * n) + ky;
            iim = ire + n2;
        } else {                   // r = (l, y); X4 rows (y, l), K = (part, kx) of length 4n
            const int l = (int)(r / n), y = (int)(r % n);
            ire = (size_t)(y * Lp + l) * (4 * n) + kx;
            iim = ire + n2;
        }
        const float re = join16<F16>(hi[ire], lo[ire]);
        const float im = join16<F16>(hi[iim], lo[iim]);
        out[e] = make_float2(re * f, im * f);
    }
}

}  // namespace

// ------------------------------------------------------------ plan workspace
struct MixedPrec {
    bool ready = false;
    int cb = 0, BN = 0;     // complex columns per N tile, tile width (2 cb)
    uint16_t *bf_hi = nullptr, *bf_lo = nullptr;   // F: [4n][2n]
    uint16_t *bg_hi = nullptr, *bg_lo = nullptr;   // G: [2n][4n]
    CUtensorMap maps[4][4];                         // [pass][A_hi, A_lo, B_hi, B_lo]
};

struct hqs_mixed_s {
    int n = 0, n2 = 0, L = 0, Lp = 0;
    uint16_t* x_hi[4] = {nullptr, nullptr, nullptr, nullptr};   // operands of S1..S4
    uint16_t* x_lo[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t x_rows[4] = {0, 0, 0, 0};
    int x_k[4] = {0, 0, 0, 0};
    float* khat = nullptr;      // Khat * n2^2 / kp
    float kp = 1.f;
    unsigned* amax = nullptr;
    float2* tmp = nullptr;      // A^H A x before the H epilogue
    MixedPrec prec[2];          // [bf16, fp16]
};

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// [rows][k] 16-bit row-major matrix, box 64 (k) x box_rows, 128-byte swizzle
int make_map(CUtensorMap* map, const void* base, int64_t rows, int k, int box_rows, bool f16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return HQS_ERR_UNSUPPORTED;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)k * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HQS_OK : HQS_ERR_CUDA;
}

template <class T> int ws_alloc(hqs_plan_s* p, T** ptr, size_t count) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        hqs_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return HQS_ERR_OOM;
    }
    p->allocs.push_back(v);
    p->bytes += count * sizeof(T);
    *ptr = static_cast<T*>(v);
    return HQS_OK;
}

size_t stage_bytes(int BN) { return 2 * (size_t)kBM * kBK * 2 + 2 * (size_t)BN * kBK * 2; }
int pipeline_stages(int BN) {
    return std::min<int>(4, (int)((kSmemLimit - 2048) / stage_bytes(BN)));
}

int mixed_workspace_fill(hqs_plan_s* p, hqs_mixed_s* w, cudaStream_t st);

// Shared workspace (operands, scaled Khat); blocking, once per plan.
int mixed_workspace(hqs_plan_s* p, cudaStream_t st) {
    if (p->mixed) return HQS_OK;
    const int n = p->n, L = p->L;
    if (n % 64 != 0 || n > 512 || L > 32 || L < 1) return HQS_ERR_UNSUPPORTED;
    hqs_mixed_s* w = new hqs_mixed_s();
    const int rc = mixed_workspace_fill(p, w, st);
    if (rc != HQS_OK) {
        delete w;      // its buffers stay on the plan's list and go with the plan
        return rc;
    }
    p->mixed = w;
    return HQS_OK;
}

int mixed_workspace_fill(hqs_plan_s* p, hqs_mixed_s* w, cudaStream_t st) {
    const int n = p->n, L = p->L;
    w->n = n;
    w->n2 = 2 * n;
    w->L = L;
    w->Lp = 1;
    while (w->Lp < L) w->Lp <<= 1;
    const int n2 = w->n2;
    w->x_rows[0] = (int64_t)L * n;       w->x_k[0] = 2 * n;
    w->x_rows[1] = (int64_t)L * n2;      w->x_k[1] = 2 * n;
    w->x_rows[2] = (int64_t)L * n2;      w->x_k[2] = 4 * n;
    w->x_rows[3] = (int64_t)n * w->Lp;   w->x_k[3] = 4 * n;
    for (int s = 0; s < 4; ++s) {
        const size_t cnt = (size_t)w->x_rows[s] * w->x_k[s];
        HQS_TRY_RC(ws_alloc(p, &w->x_hi[s], cnt));
        HQS_TRY_RC(ws_alloc(p, &w->x_lo[s], cnt));
    }
    // padded coil rows of the S4 operand stay zero
    HQS_CUDA_TRY(cudaMemsetAsync(w->x_hi[3], 0, (size_t)w->x_rows[3] * w->x_k[3] * 2, st));
    HQS_CUDA_TRY(cudaMemsetAsync(w->x_lo[3], 0, (size_t)w->x_rows[3] * w->x_k[3] * 2, st));
    HQS_TRY_RC(ws_alloc(p, &w->khat, (size_t)n2 * n2));
    HQS_TRY_RC(ws_alloc(p, &w->amax, 1));
    HQS_TRY_RC(ws_alloc(p, &w->tmp, (size_t)n * n));
    // kp: power of two >= max |Khat n2^2|
    HQS_CUDA_TRY(cudaMemsetAsync(w->amax, 0, sizeof(unsigned), st));
    k_mx_amax<<<256, 256, 0, st>>>(reinterpret_cast<const float2*>(p->khat), n2 * n2 / 2, w->amax);
    unsigned bits = 0;
    HQS_CUDA_TRY(cudaMemcpyAsync(&bits, w->amax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    HQS_CUDA_TRY(cudaStreamSynchronize(st));
    float km;
    memcpy(&km, &bits, sizeof(float));
    km *= (float)n2 * (float)n2;
    int e = 0;
    if (km > 0.f && std::isfinite(km)) frexpf(km, &e);
    w->kp = ldexpf(1.f, e);
    k_mx_khat<<<256, 256, 0, st>>>(p->khat, n2 * n2, (float)n2 * (float)n2 / w->kp, w->khat);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

int mixed_precision_ready(hqs_plan_s* p, int pi, cudaStream_t st) {
    hqs_mixed_s* w = p->mixed;
    MixedPrec& m = w->prec[pi];
    if (m.ready) return HQS_OK;
    const int n = w->n, n2 = w->n2;
    const bool f16 = pi == 1;
    // widest N tile whose half divides n in multiples of 16: two accumulator
    // buffers of 256 TMEM columns hold BN (BF16) or 2 BN (FP16: main + correction)
    const int cbmax = f16 ? kCorrOff / 2 : (int)kAccStride / 2;
    m.cb = 0;
    for (int c = 16; c <= std::min(cbmax, n); c += 16)
        if (n % c == 0) m.cb = c;
    m.BN = 2 * m.cb;
    if (m.cb == 0 || pipeline_stages(m.BN) < 2) return HQS_ERR_UNSUPPORTED;
    HQS_TRY_RC(ws_alloc(p, &m.bf_hi, (size_t)4 * n * 2 * n));
    HQS_TRY_RC(ws_alloc(p, &m.bf_lo, (size_t)4 * n * 2 * n));
    HQS_TRY_RC(ws_alloc(p, &m.bg_hi, (size_t)2 * n * 4 * n));
    HQS_TRY_RC(ws_alloc(p, &m.bg_lo, (size_t)2 * n * 4 * n));
    if (f16) {
        k_mx_build_b<true><<<1024, 256, 0, st>>>(m.bf_hi, m.bf_lo, 0, n, m.cb);
        k_mx_build_b<true><<<1024, 256, 0, st>>>(m.bg_hi, m.bg_lo, 1, n, m.cb);
    } else {
        k_mx_build_b<false><<<1024, 256, 0, st>>>(m.bf_hi, m.bf_lo, 0, n, m.cb);
        k_mx_build_b<false><<<1024, 256, 0, st>>>(m.bg_hi, m.bg_lo, 1, n, m.cb);
    }
    HQS_CUDA_TRY(cudaGetLastError());
    for (int s = 0; s < 4; ++s) {
        HQS_TRY_RC(make_map(&m.maps[s][0], w->x_hi[s], w->x_rows[s], w->x_k[s], kBM, f16));
        HQS_TRY_RC(make_map(&m.maps[s][1], w->x_lo[s], w->x_rows[s], w->x_k[s], kBM, f16));
        const bool fmat = s < 2;
        HQS_TRY_RC(make_map(&m.maps[s][2], fmat ? m.bf_hi : m.bg_hi, fmat ? 4 * n : n2, fmat ? 2 * n : 4 * n,
                            m.BN, f16));
        HQS_TRY_RC(make_map(&m.maps[s][3], fmat ? m.bf_lo : m.bg_lo, fmat ? 4 * n : n2, fmat ? 2 * n : 4 * n,
                            m.BN, f16));
    }
    m.ready = true;
    return HQS_OK;
}

template <int STAGE, bool F16>
int launch_pass(hqs_plan_s* p, const MixedPrec& m, MixedArgs P, int Nreal, cudaStream_t st) {
    const size_t smem = (size_t)P.stages * stage_bytes(P.BN) + 1024 + (2 * P.stages + 4) * 8 + 64;
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_dft_gemm<STAGE, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    P.MT = ceil_div(P.M, kBM);
    P.NT = Nreal / P.BN;
    int nsm = 0;
    HQS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    const int grid = std::min(P.MT * P.NT, nsm);
    k_dft_gemm<STAGE, F16><<<grid, kThreads, smem, st>>>(m.maps[STAGE][0], m.maps[STAGE][1], m.maps[STAGE][2],
                                                          m.maps[STAGE][3], P);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <bool F16>
int run_passes(hqs_plan_s* p, const float2* x, float2* out, int upto, cudaStream_t st) {
    hqs_mixed_s* w = p->mixed;
    const MixedPrec& m = w->prec[F16 ? 1 : 0];
    const int n = w->n, n2 = w->n2, L = w->L;
    HQS_CUDA_TRY(cudaMemsetAsync(w->amax, 0, sizeof(unsigned), st));
    k_mx_amax<<<std::min(ceil_div(n * n, 256), 512), 256, 0, st>>>(x, n * n, w->amax);
    k_mx_prologue<F16><<<ceil_div(n * n, 256), 256, 0, st>>>(x, p->smaps, n, L, w->amax, w->x_hi[0], w->x_lo[0]);
    HQS_CUDA_TRY(cudaGetLastError());
    MixedArgs P{};
    P.n = n;
    P.n2 = n2;
    P.L = L;
    P.Lp = w->Lp;
    P.cb = m.cb;
    P.BN = m.BN;
    P.stages = pipeline_stages(m.BN);
    P.khat = w->khat;
    P.smaps = p->smaps;
    P.out = out;
    P.amax = w->amax;
    P.kp = w->kp;
    P.err = p->dev_err;
    // S1
    P.M = L * n;
    P.KB = 2 * n / kBK;
    P.out_hi = w->x_hi[1];
    P.out_lo = w->x_lo[1];
    HQS_TRY_RC((launch_pass<MX_S1, F16>(p, m, P, 4 * n, st)));
    if (upto == 1) return HQS_OK;
    // S2
    P.M = L * n2;
    P.KB = 2 * n / kBK;
    P.out_hi = w->x_hi[2];
    P.out_lo = w->x_lo[2];
    HQS_TRY_RC((launch_pass<MX_S2, F16>(p, m, P, 4 * n, st)));
    if (upto == 2) return HQS_OK;
    // S3
    P.M = L * n2;
    P.KB = 4 * n / kBK;
    P.out_hi = w->x_hi[3];
    P.out_lo = w->x_lo[3];
    HQS_TRY_RC((launch_pass<MX_S3, F16>(p, m, P, 2 * n, st)));
    if (upto == 3) return HQS_OK;
    // S4
    P.M = n * w->Lp;
    P.KB = 4 * n / kBK;
    P.out_hi = nullptr;
    P.out_lo = nullptr;
    HQS_TRY_RC((launch_pass<MX_S4, F16>(p, m, P, 2 * n, st)));
    return HQS_OK;
}

int mixed_prepare(hqs_plan_s* p, int precision, cudaStream_t st) {
    if (precision != HQS_PREC_BF16X3 && precision != HQS_PREC_FP16X3) return HQS_ERR_INVALID_ARG;
    HQS_TRY_RC(mixed_workspace(p, st));
    return mixed_precision_ready(p, precision == HQS_PREC_FP16X3 ? 1 : 0, st);
}

}  // namespace

void mixed_free(hqs_plan_s* p) {
    delete p->mixed;
    p->mixed = nullptr;
}

int mixed_partial_count(const hqs_plan_s* p) { return std::min(ceil_div(p->n * p->n, 256), 1024); }

// out = A^H A x (mode 0) or a A^H A x + b pmul with partial <pmul, out> (mode 1)
int launch_toeplitz_mixed_ex(hqs_plan_s* p, const float2* x, float2* out, const float2* pmul, float a, float b,
                             int mode, double* part, int precision, cudaStream_t st) {
    HQS_TRY_RC(mixed_prepare(p, precision, st));
    hqs_mixed_s* w = p->mixed;
    float2* dst = mode == 1 ? w->tmp : out;
    if (precision == HQS_PREC_FP16X3) HQS_TRY_RC(run_passes<true>(p, x, dst, 4, st));
    else HQS_TRY_RC(run_passes<false>(p, x, dst, 4, st));
    if (mode == 1) {
        k_mx_hepilogue<<<mixed_partial_count(p), 256, 0, st>>>(w->tmp, out, pmul, a, b, 1, p->n * p->n, part);
        HQS_CUDA_TRY(cudaGetLastError());
    }
    return HQS_OK;
}

int launch_toeplitz_mixed(hqs_plan_s* p, const float2* x, float2* out, int precision, cudaStream_t st) {
    return launch_toeplitz_mixed_ex(p, x, out, nullptr, 1.f, 0.f, 0, nullptr, precision, st);
}

extern "C" int hqs_debug_toeplitz_stage(hqs_plan p, const hqs_c64* x, int precision, int stage, hqs_c64* out,
                                        void* stream) {
    if (!p || !x || !out || stage < 1 || stage > 4) return HQS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const float2* xx = reinterpret_cast<const float2*>(x);
    float2* oo = reinterpret_cast<float2*>(out);
    if (stage == 4) return launch_toeplitz_mixed(p, xx, oo, precision, st);
    HQS_TRY_RC(mixed_prepare(p, precision, st));
    hqs_mixed_s* w = p->mixed;
    const bool f16 = precision == HQS_PREC_FP16X3;
    if (f16) HQS_TRY_RC(run_passes<true>(p, xx, nullptr, stage, st));
    else HQS_TRY_RC(run_passes<false>(p, xx, nullptr, stage, st));
    const float rn = sqrtf((float)w->n2);
    const float base = stage == 1 ? rn : (stage == 2 ? (float)w->n2 * w->kp : rn * w->kp);
    if (f16)
        k_mx_dump<true><<<1024, 256, 0, st>>>(w->x_hi[stage], w->x_lo[stage], stage, w->n, w->L, w->Lp, base,
                                              w->amax, oo);
    else
        k_mx_dump<false><<<1024, 256, 0, st>>>(w->x_hi[stage], w->x_lo[stage], stage, w->n, w->L, w->Lp, base,
                                               w->amax, oo);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}
