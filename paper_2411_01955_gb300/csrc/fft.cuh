// In-house batched FFT on shared memory for the sizes the hot path uses.
//
// A CTA transforms up to kLines lines of length N stored line-innermost in
// shared memory (element (pos, line) at s[pos * kLines + line]), which is the
// coil-innermost layout the grids use in global memory, so loads and stores
// are contiguous over coils.  The transform is a mixed-radix Stockham
// autosort FFT: stage with radix R after a product P of earlier radices reads
// x[i + r*N/R], multiplies by w_{P R}^(r k) (k = i mod P), applies the
// radix-R DFT and writes y[(i - k) R + k + s P].  Each thread owns E elements
// of one line (E divisible by every radix of the size), holds them in
// registers across the barrier, so the transform runs in place in one buffer.
// Forward uses exp(-2 pi i m / N), inverse its conjugate; neither scales.
#pragma once

#include <type_traits>
#include <utility>

#include "common.cuh"

namespace hqs {

constexpr float kSqrtHalf = 0.70710678118654752440f;
// Shared-memory stride between positions of a line: a compile-time constant
// keeps the per-element address arithmetic out of the register budget.  It
// is also the coil-chunk size of the FFT passes (lines per CTA).
#ifndef HQS_KLINES
#define HQS_KLINES 16
#endif
constexpr int kLines = HQS_KLINES;

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    HQS_DEV static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV> struct Dft<3, INV> {
    HQS_DEV static void run(float2* v) {
        // w = exp(-+2 pi i / 3) = -1/2 -+ i sqrt(3)/2
        const float h = 0.86602540378443864676f;
        float2 t = cadd(v[1], v[2]);
        float2 d = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 j = mul_mi<INV>(cscale(d, h));      // -+ i * sqrt(3)/2 * d
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <bool INV> struct Dft<4, INV> {
    HQS_DEV static void run(float2* v) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <bool INV> struct Dft<5, INV> {
    HQS_DEV static void run(float2* v) {
        const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
        const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
        const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
        const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
        float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        float2 x0 = v[0];
        float2 m1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        float2 m2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        // forward: out1 = m1 - i(s1 b1 + s2 b2); out2 = m2 - i(s2 b1 - s1 b2)
        float2 n1 = mul_mi<INV>(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
        float2 n2 = mul_mi<INV>(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
        v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
        v[1] = cadd(m1, n1);
        v[4] = csub(m1, n1);
        v[2] = cadd(m2, n2);
        v[3] = csub(m2, n2);
    }
};

template <bool INV> struct Dft<8, INV> {
    HQS_DEV static void run(float2* v) {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        // w8^1, w8^2, w8^3 with w8 = exp(-+ i pi / 4)
        float2 o1, o2, o3;
        if (!INV) {
            o1 = make_float2((o[1].x + o[1].y) * kSqrtHalf, (o[1].y - o[1].x) * kSqrtHalf);
            o3 = make_float2((o[3].y - o[3].x) * kSqrtHalf, -(o[3].x + o[3].y) * kSqrtHalf);
        } else {
            o1 = make_float2((o[1].x - o[1].y) * kSqrtHalf, (o[1].x + o[1].y) * kSqrtHalf);
            o3 = make_float2(-(o[3].x + o[3].y) * kSqrtHalf, (o[3].x - o[3].y) * kSqrtHalf);
        }
        o2 = mul_mi<INV>(o[2]);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// Radix 16 as 4 x 4 with twiddles: n = n1 + 4 n2, k = k1 + 4 k2,
// X[k1 + 4 k2] = sum_n1 w4^(n1 k2) w16^(n1 k1) sum_n2 w4^(n2 k1) x[n1 + 4 n2].
template <bool INV> struct Dft<16, INV> {
    HQS_DEV static float2 tw(float2 v, float c, float s) {   // v * exp(-+ i theta), (c, s) = (cos, sin) theta
        const float sn = INV ? s : -s;
        return make_float2(v.x * c - v.y * sn, v.x * sn + v.y * c);
    }
    HQS_DEV static void run(float2* v) {
        const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
        float2 y[4][4];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            float2 t[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
            Dft<4, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n1][k1] = t[k1];
        }
        y[1][1] = tw(y[1][1], c1, s1);
        y[1][2] = tw(y[1][2], kSqrtHalf, kSqrtHalf);
        y[1][3] = tw(y[1][3], s1, c1);
        y[2][1] = tw(y[2][1], kSqrtHalf, kSqrtHalf);
        y[2][2] = mul_mi<INV>(y[2][2]);
        y[2][3] = tw(y[2][3], -kSqrtHalf, kSqrtHalf);
        y[3][1] = tw(y[3][1], s1, c1);
        y[3][2] = tw(y[3][2], -kSqrtHalf, kSqrtHalf);
        y[3][3] = tw(y[3][3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<4, INV>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
};

// Composite radix R = R1 R2 with gcd(R1, R2) = 1 by the prime-factor
// (Good-Thomas) mapping: input index n = (R2 n1 + R1 n2) mod R, output index
// k with k = k1 (mod R1), k = k2 (mod R2); then
// X[k] = sum_n1 w_R1^(n1 k1) sum_n2 w_R2^(n2 k2) x[n], with no twiddles
// between the two small DFTs.  All indices are compile-time register names.
template <int R1, int R2> struct Crt {
    // k in [0, R) with k % R1 == k1 and k % R2 == k2
    static constexpr int out(int k1, int k2) {
        for (int k = 0; k < R1 * R2; ++k)
            if (k % R1 == k1 && k % R2 == k2) return k;
        return -1;
    }
};

template <int R1, int R2, bool INV> struct DftPfa {
    HQS_DEV static void run(float2* v) {
        constexpr int R = R1 * R2;
        float2 a[R1][R2];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) a[n1][n2] = v[(R2 * n1 + R1 * n2) % R];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) Dft<R2, INV>::run(a[n1]);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            float2 c[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) c[n1] = a[n1][k2];
            Dft<R1, INV>::run(c);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[Crt<R1, R2>::out(k1, k2)] = c[k1];
        }
    }
};

template <bool INV> struct Dft<6, INV> : DftPfa<2, 3, INV> {};
template <bool INV> struct Dft<10, INV> : DftPfa<2, 5, INV> {};
template <bool INV> struct Dft<12, INV> : DftPfa<4, 3, INV> {};
template <bool INV> struct Dft<40, INV> : DftPfa<8, 5, INV> {};

// First-stage DFT when the upper half of the line is known to be zero
// (zero padding): inputs r >= R/2 are not read and not added.
template <int R, bool INV> struct DftHalfIn {
    HQS_DEV static void run(float2* v) {
#pragma unroll
        for (int r = R / 2; r < R; ++r) v[r] = make_float2(0.f, 0.f);
        Dft<R, INV>::run(v);
    }
};
template <bool INV> struct DftHalfIn<4, INV> {
    HQS_DEV static void run(float2* v) {   // inputs (a, b, 0, 0)
        const float2 a = v[0], b = v[1];
        const float2 jb = mul_mi<INV>(b);
        v[0] = cadd(a, b);
        v[1] = cadd(a, jb);
        v[2] = csub(a, b);
        v[3] = csub(a, jb);
    }
};
template <bool INV> struct DftHalfIn<8, INV> {
    HQS_DEV static void run(float2* v) {   // inputs (v0..v3, 0, 0, 0, 0)
        float2 e[4] = {v[0], v[2], make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float2 o[4] = {v[1], v[3], make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        DftHalfIn<4, INV>::run(e);
        DftHalfIn<4, INV>::run(o);
        float2 o1, o3;
        if (!INV) {
            o1 = make_float2((o[1].x + o[1].y) * kSqrtHalf, (o[1].y - o[1].x) * kSqrtHalf);
            o3 = make_float2((o[3].y - o[3].x) * kSqrtHalf, -(o[3].x + o[3].y) * kSqrtHalf);
        } else {
            o1 = make_float2((o[1].x - o[1].y) * kSqrtHalf, (o[1].x + o[1].y) * kSqrtHalf);
            o3 = make_float2(-(o[3].x + o[3].y) * kSqrtHalf, (o[3].x - o[3].y) * kSqrtHalf);
        }
        const float2 o2 = mul_mi<INV>(o[2]);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// One Stockham stage.  `s` points at element (0, line); consecutive positions
// are kLines float2 apart.  Threads with act == false (given t = 0 and line 0)
// read but do not write.  ZIN (first stage only): the line's upper half is
// zero and is neither read nor added.  HOUT (last stage only): only the lower
// half of the output is wanted and the upper half is not written.
template <int N, int E, int R, int P, bool INV, bool ZIN = false, bool HOUT = false>
HQS_DEV void fft_stage(float2* s, int t, bool act, const float2* __restrict__ tw) {
    constexpr int st = kLines;
    constexpr int TPL = N / E;
    constexpr int NB = N / R;
    constexpr int BPT = E / R;
    static_assert(E % R == 0, "radix must divide elements per thread");
    static_assert(NB == TPL * BPT, "butterfly split");
    static_assert(!ZIN || (P == 1 && R % 2 == 0), "zero-input pruning is for an even first stage");
    static_assert(!HOUT || (P * R == N && R % 2 == 0), "half-output pruning is for an even last stage");
    constexpr int RIN = ZIN ? R / 2 : R;
    constexpr int ROUT = HOUT ? R / 2 : R;
    float2 v[E];
    // Loads are unconditional (inactive threads read line 0 at t = 0, which
    // is in bounds): a predicated load block inside a caller's loop makes the
    // register allocator keep the whole array live and spill.
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int i = t + b * TPL;
#pragma unroll
        for (int r = 0; r < RIN; ++r) v[b * R + r] = s[(i + r * NB) * st];
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int i = t + b * TPL;
            const int k = i % P;
            if (P > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw[r * k * (N / (P * R))];
                    if (INV) w.y = -w.y;
                    v[b * R + r] = cmul(v[b * R + r], w);
                }
            }
            if (ZIN)
                DftHalfIn<R, INV>::run(&v[b * R]);
            else
                Dft<R, INV>::run(&v[b * R]);
            const int j = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < ROUT; ++r) s[(j + r * P) * st] = v[b * R + r];
        }
    }
    __syncthreads();
}

// No-op marker for the I/O hooks of fft_stage_io.
struct NoIO {};

// fft_stage with I/O hooks for the first and last stage of a transform:
//   FIRST and LD != NoIO: the stage reads its inputs through ld(pos) (global
//     memory of this thread's line) instead of shared memory, so the caller's
//     separate load pass and one barrier disappear;
//   LAST and XF != NoIO: outputs pass through xf(pos, v) before the shared
//     memory store (a pointwise multiply fused into the stage);
//   LAST and STF != NoIO: outputs go to stf(pos, v) (global memory) instead of
//     shared memory, with no barrier between the stage's loads and stores.
template <int N, int E, int R, int P, bool INV, bool ZIN, bool HOUT, bool FIRST, bool LAST, class LD, class XF,
          class STF>
HQS_DEV void fft_stage_io(float2* s, int t, bool act, const float2* __restrict__ tw, LD& ld, XF& xf, STF& stf) {
    constexpr int st = kLines;
    constexpr int TPL = N / E;
    constexpr int NB = N / R;
    constexpr int BPT = E / R;
    constexpr bool GIN = FIRST && !std::is_same_v<LD, NoIO>;
    constexpr bool GOUT = LAST && !std::is_same_v<STF, NoIO>;
    constexpr bool XOUT = LAST && !std::is_same_v<XF, NoIO>;
    static_assert(E % R == 0, "radix must divide elements per thread");
    static_assert(NB == TPL * BPT, "butterfly split");
    static_assert(!ZIN || (P == 1 && R % 2 == 0), "zero-input pruning is for an even first stage");
    static_assert(!HOUT || (P * R == N && R % 2 == 0), "half-output pruning is for an even last stage");
    constexpr int RIN = ZIN ? R / 2 : R;
    constexpr int ROUT = HOUT ? R / 2 : R;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int i = t + b * TPL;
#pragma unroll
        for (int r = 0; r < RIN; ++r) {
            if constexpr (GIN) v[b * R + r] = ld(i + r * NB);
            else v[b * R + r] = s[(i + r * NB) * st];
        }
    }
    // in place through shared memory: every read lands before any write
    if constexpr (!GIN && !GOUT) __syncthreads();
    if (act) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int i = t + b * TPL;
            const int k = i % P;
            if (P > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw[r * k * (N / (P * R))];
                    if (INV) w.y = -w.y;
                    v[b * R + r] = cmul(v[b * R + r], w);
                }
            }
            if (ZIN)
                DftHalfIn<R, INV>::run(&v[b * R]);
            else
                Dft<R, INV>::run(&v[b * R]);
            const int j = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < ROUT; ++r) {
                const int pos = j + r * P;
                if constexpr (GOUT) {
                    stf(pos, v[b * R + r]);
                } else if constexpr (XOUT) {
                    s[pos * st] = xf(pos, v[b * R + r]);
                } else {
                    s[pos * st] = v[b * R + r];
                }
            }
        }
    }
    if constexpr (!GOUT) __syncthreads();
}

// Size table: elements per thread and radix sequence.
template <int N> struct FftSize;

#define HQS_FFT_SIZE(NN, EE, ...)                                                     \
    template <> struct FftSize<NN> {                                                  \
        static constexpr int E = EE;                                                  \
        static constexpr int TPL = NN / EE;                                           \
        template <bool INV, bool ZIN, bool HOUT>                                      \
        HQS_DEV static void run(float2* s, int t, bool act, const float2* tw) {        \
            NoIO ld, xf, stf;                                                         \
            __VA_ARGS__                                                               \
        }                                                                             \
        template <bool INV, bool ZIN, bool HOUT, class LD, class XF, class STF>       \
        HQS_DEV static void run_io(float2* s, int t, bool act, const float2* tw, LD& ld, \
                                   XF& xf, STF& stf) {                                \
            __VA_ARGS__                                                               \
        }                                                                             \
    };

#define ST(R, P)                                                                              \
    fft_stage_io<NN_, E_, R, P, INV, ZIN && (P == 1), HOUT && (P * R == NN_), P == 1, P * R == NN_>( \
        s, t, act, tw, ld, xf, stf);

#define NN_ 16
#define E_ 4
HQS_FFT_SIZE(16, 4, ST(4, 1) ST(4, 4))
#undef NN_
#undef E_
#define NN_ 32
#define E_ 8
HQS_FFT_SIZE(32, 8, ST(8, 1) ST(4, 8))
#undef NN_
#undef E_
#define NN_ 64
#define E_ 8
HQS_FFT_SIZE(64, 8, ST(8, 1) ST(8, 8))
#undef NN_
#undef E_
#define NN_ 128
#define E_ 8
HQS_FFT_SIZE(128, 8, ST(8, 1) ST(4, 8) ST(4, 32))
#undef NN_
#undef E_
#define NN_ 256
#define E_ 8
HQS_FFT_SIZE(256, 8, ST(8, 1) ST(8, 8) ST(4, 64))
#undef NN_
#undef E_
#define NN_ 320
#define E_ 40
HQS_FFT_SIZE(320, 40, ST(8, 1) ST(40, 8))
#undef NN_
#undef E_
#define NN_ 384
#define E_ 24
HQS_FFT_SIZE(384, 24, ST(8, 1) ST(8, 8) ST(6, 64))
#undef NN_
#undef E_
#define NN_ 512
#define E_ 16
HQS_FFT_SIZE(512, 16, ST(8, 1) ST(8, 8) ST(8, 64))
#undef NN_
#undef E_
#define NN_ 640
#define E_ 40
HQS_FFT_SIZE(640, 40, ST(8, 1) ST(8, 8) ST(10, 64))
#undef NN_
#undef E_
#define NN_ 768
#define E_ 24
HQS_FFT_SIZE(768, 24, ST(8, 1) ST(8, 8) ST(12, 64))
#undef NN_
#undef E_
// Two-stage factorisations for the volume passes (fewer shared-memory round
// trips per transform, more elements per thread); other sizes as above.
template <int N> struct FftSizeV : FftSize<N> {};
#define HQS_FFT_SIZE_V(NN, EE, ...)                                                   \
    template <> struct FftSizeV<NN> {                                                 \
        static constexpr int E = EE;                                                  \
        static constexpr int TPL = NN / EE;                                           \
        template <bool INV, bool ZIN, bool HOUT, class LD, class XF, class STF>       \
        HQS_DEV static void run_io(float2* s, int t, bool act, const float2* tw, LD& ld, \
                                   XF& xf, STF& stf) {                                \
            __VA_ARGS__                                                               \
        }                                                                             \
    };
#define NN_ 128
#define E_ 16
HQS_FFT_SIZE_V(128, 16, ST(8, 1) ST(16, 8))
#undef NN_
#undef E_
#define NN_ 256
#define E_ 16
HQS_FFT_SIZE_V(256, 16, ST(16, 1) ST(16, 16))
#undef NN_
#undef E_
#undef HQS_FFT_SIZE_V
#undef ST
#undef HQS_FFT_SIZE

// ------------------------------------------------ forward x factor x inverse pair
// A forward transform, a pointwise factor and the inverse transform of the same
// line, with the inverse taking the forward's radices in reverse order.  Then the
// forward's last Stockham stage (radix R after P = N / R) reads and writes the
// positions i + r N/R, i < N/R, and the inverse's first stage (radix R, P = 1) reads
// exactly those positions: the two stages and the factor run on the same registers,
// with no shared-memory round trip and no barrier between them.
template <int N, int E, int R, class XF>
HQS_DEV void fft_mid_stage(float2* s, int t, bool act, const float2* __restrict__ tw, XF& xf) {
    constexpr int st = kLines;
    constexpr int TPL = N / E;
    constexpr int NB = N / R;   // also P, the product of the forward's earlier radices
    constexpr int BPT = E / R;
    static_assert(E % R == 0 && NB == TPL * BPT, "butterfly split");
    float2 v[E];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int i = t + b * TPL;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = s[(i + r * NB) * st];
    }
    // a factor the caller fetched with cp.async before the transform is complete
    // after this thread's wait and the barrier (a no-op when nothing is pending)
    cp_async_wait_all();
    __syncthreads();
    if (act) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int i = t + b * TPL;   // < NB = P, so i mod P = i
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], tw[r * i]);
            Dft<R, false>::run(&v[b * R]);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = xf(i + r * NB, v[b * R + r]);
            Dft<R, true>::run(&v[b * R]);
#pragma unroll
            for (int r = 0; r < R; ++r) s[(i * R + r) * st] = v[b * R + r];
        }
    }
    __syncthreads();
}

// Stage tables of the pair: forward head stages (the first with the loader and,
// with ZIN, the zero upper half), the middle radix, inverse tail stages in reverse
// order (the last through the store hook, keeping the lower half only with HOUT).
template <int N> struct FftPair;

#define HQS_FFT_PAIR(NN, EE, RM, HEAD, TAIL)                                                      \
    template <> struct FftPair<NN> {                                                              \
        static constexpr int E = EE;                                                              \
        static constexpr int TPL = NN / EE;                                                       \
        template <bool ZIN_, bool HOUT_, class LD, class XF, class STF>                           \
        HQS_DEV static void run(float2* s, int t, bool act, const float2* tw, LD& ld, XF& xf,     \
                                STF& stf) {                                                       \
            NoIO nio;                                                                             \
            HEAD                                                                                  \
            fft_mid_stage<NN, EE, RM>(s, t, act, tw, xf);                                         \
            TAIL                                                                                  \
        }                                                                                         \
    };
#define FH(R, P) fft_stage_io<NN_, E_, R, P, false, ZIN_ && P == 1, false, P == 1, false>(s, t, act, tw, ld, nio, nio);
#define FT(R, P) fft_stage_io<NN_, E_, R, P, true, false, HOUT_ && P * R == NN_, false, P * R == NN_>(s, t, act, tw, nio, nio, stf);

#define NN_ 16
#define E_ 4
HQS_FFT_PAIR(16, 4, 4, FH(4, 1), FT(4, 4))
#undef NN_
#undef E_
#define NN_ 32
#define E_ 8
HQS_FFT_PAIR(32, 8, 4, FH(8, 1), FT(8, 4))
#undef NN_
#undef E_
#define NN_ 64
#define E_ 8
HQS_FFT_PAIR(64, 8, 8, FH(8, 1), FT(8, 8))
#undef NN_
#undef E_
#define NN_ 128
#define E_ 8
HQS_FFT_PAIR(128, 8, 4, FH(8, 1) FH(4, 8), FT(4, 4) FT(8, 16))
#undef NN_
#undef E_
#define NN_ 256
#define E_ 8
HQS_FFT_PAIR(256, 8, 4, FH(8, 1) FH(8, 8), FT(8, 4) FT(8, 32))
#undef NN_
#undef E_
#define NN_ 320
#define E_ 40
HQS_FFT_PAIR(320, 40, 40, FH(8, 1), FT(8, 40))
#undef NN_
#undef E_
#define NN_ 384
#define E_ 24
HQS_FFT_PAIR(384, 24, 6, FH(8, 1) FH(8, 8), FT(8, 6) FT(8, 48))
#undef NN_
#undef E_
#define NN_ 512
#define E_ 16
HQS_FFT_PAIR(512, 16, 8, FH(8, 1) FH(8, 8), FT(8, 8) FT(8, 64))
#undef NN_
#undef E_
#define NN_ 640
#define E_ 40
HQS_FFT_PAIR(640, 40, 10, FH(8, 1) FH(8, 8), FT(8, 10) FT(8, 80))
#undef NN_
#undef E_
#define NN_ 768
#define E_ 24
HQS_FFT_PAIR(768, 24, 12, FH(8, 1) FH(8, 8), FT(8, 12) FT(8, 96))
#undef NN_
#undef E_
#undef FH
#undef FT
#undef HQS_FFT_PAIR

// Element (pos, line) of a CTA's line buffer of N-point lines: lines [0, kLines)
// at s[pos * kLines + line], lines [kLines, 2 kLines) in a second block of
// N * kLines elements after the first (same stride), so short lines can fill a
// CTA with up to 2 kLines lines.
template <int N> HQS_DEV int line_elem(int pos, int line) {
    return line < kLines ? pos * kLines + line : N * kLines + pos * kLines + (line - kLines);
}
template <int N> HQS_DEV float2* line_base(float2* s, int line) { return s + line_elem<N>(0, line); }

// Transform `nlines` (<= kLines; <= 2 kLines with WIDE, lines held at
// s[line_elem<N>(pos, line)]) lines held at s[pos * kLines + line] with the
// whole CTA: thread (line = tid % lpg, t = tid / lpg) owns E elements of one
// line, lpg = blockDim.x / TPL >= nlines (launch with fft_threads).  The
// caller synchronises before (after filling s); this routine ends with a
// barrier.  (A loop over line groups here doubles register use, so the launch
// shape covers every line at once instead.)
template <int N, bool INV, bool ZIN = false, bool HOUT = false, bool WIDE = false>
HQS_DEV void block_fft(float2* s, int nlines, const float2* tw) {
    constexpr int TPL = FftSize<N>::TPL;
    const int lpg = blockDim.x / TPL;
    int tid;
    // The thread index is read through a volatile move so that the per-thread
    // address and twiddle-index arithmetic of the stages (a function of the
    // thread index only) is not hoisted out of a caller's loop, which would
    // keep ~2E extra registers live across the loop and spill.
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int ll = tid % lpg;
    const int t = tid / lpg;
    const bool act = (ll < nlines) && (t < TPL);
    float2* base = WIDE ? line_base<N>(s, act ? ll : 0) : s + (act ? ll : 0);
    FftSize<N>::template run<INV, ZIN, HOUT>(base, act ? t : 0, act, tw);
}

// block_fft with I/O hooks (see fft_stage_io).  The hooks receive this
// thread's line (line 0 for threads without a line, which read in-bounds data
// and store nothing) and a position; ld(line, pos, act) feeds the first stage
// (act false: a thread without a line, whose value is discarded, so a loader
// with side effects must skip them),
// xf(line, pos, v) transforms the last stage's outputs before they go to
// shared memory, stf(line, pos, v) takes them instead of shared memory.  With
// a loader the caller need not synchronise before (nothing is read from
// shared memory); with a store hook the routine ends without a barrier.
template <template <int> class TAB, int N, bool INV, bool ZIN, bool HOUT, class LD, class XF, class STF>
HQS_DEV void block_fft_io_tab(float2* s, int nlines, const float2* tw, LD&& ld, XF&& xf, STF&& stf) {
    constexpr int TPL = TAB<N>::TPL;
    const int lpg = blockDim.x / TPL;
    int tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int ll = tid % lpg;
    const int t = tid / lpg;
    const bool act = (ll < nlines) && (t < TPL);
    const int line = act ? ll : 0;
    auto bind_ld = [&]() {
        if constexpr (std::is_same_v<std::decay_t<LD>, NoIO>) return NoIO{};
        else return [&, line, act](int pos) { return ld(line, pos, act); };
    }();
    auto bind_xf = [&]() {
        if constexpr (std::is_same_v<std::decay_t<XF>, NoIO>) return NoIO{};
        else return [&, line](int pos, float2 v) { return xf(line, pos, v); };
    }();
    auto bind_st = [&]() {
        if constexpr (std::is_same_v<std::decay_t<STF>, NoIO>) return NoIO{};
        else return [&, line](int pos, float2 v) { stf(line, pos, v); };
    }();
    TAB<N>::template run_io<INV, ZIN, HOUT>(s + line, act ? t : 0, act, tw, bind_ld, bind_xf, bind_st);
}

// The forward x factor x inverse pair (FftPair) with the same hooks: ld feeds the
// forward's first stage (upper half zero with ZIN), xf(line, pos, v) is the
// factor, stf takes the inverse's output (its lower half only with HOUT).  WIDE:
// up to 2 kLines lines, the buffer laid out as line_elem<N>.
template <int N, bool ZIN, bool HOUT, bool WIDE = false, class LD, class XF, class STF>
HQS_DEV void block_fft_pair(float2* s, int nlines, const float2* tw, LD&& ld, XF&& xf, STF&& stf) {
    constexpr int TPL = FftPair<N>::TPL;
    static_assert(FftPair<N>::E == FftSize<N>::E, "same thread layout as the single transforms");
    const int lpg = blockDim.x / TPL;
    int tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int ll = tid % lpg;
    const int t = tid / lpg;
    const bool act = (ll < nlines) && (t < TPL);
    const int line = act ? ll : 0;
    auto bind_ld = [&, line, act](int pos) { return ld(line, pos, act); };
    auto bind_xf = [&, line](int pos, float2 v) { return xf(line, pos, v); };
    auto bind_st = [&, line](int pos, float2 v) { stf(line, pos, v); };
    FftPair<N>::template run<ZIN, HOUT>(WIDE ? line_base<N>(s, line) : s + line, act ? t : 0, act, tw, bind_ld, bind_xf,
                                        bind_st);
}

template <int N, bool INV, bool ZIN, bool HOUT, class LD, class XF, class STF>
HQS_DEV void block_fft_io(float2* s, int nlines, const float2* tw, LD&& ld, XF&& xf, STF&& stf) {
    block_fft_io_tab<FftSize, N, INV, ZIN, HOUT>(s, nlines, tw, std::forward<LD>(ld), std::forward<XF>(xf),
                                                 std::forward<STF>(stf));
}

// Copies the N-point twiddle table into shared memory; the caller's barrier
// before block_fft publishes it.  Staging it there keeps the stage loops off
// global memory (the streaming grid data would evict it from L1).
template <int N> HQS_DEV const float2* stage_twiddles(float2* dst, const float2* __restrict__ tw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = tw[i];
    return dst;
}

// f(p0 + k * PST) for k = 0..CNT-1, fully unrolled: with compile-time trip
// counts every global load of a pass is in flight at once.
template <int CNT, int PST, class F> HQS_DEV void unrolled(int p0, F&& f) {
#pragma unroll
    for (int k = 0; k < CNT; ++k) f(p0 + k * PST);
}

// Threads per CTA for a pass over `nlines` (<= kLines) lines of size N: every
// line in one group, rounded up to whole warps (TPL is a power of two).
template <int N> inline int fft_threads(int nlines) {
    constexpr int TPL = FftSize<N>::TPL;
    return ((nlines * TPL + 31) / 32) * 32;
}

// Dispatch a functor templated on the FFT size.
template <class F> inline int dispatch_fft_size(int n, F&& f) {
    switch (n) {
        case 16: return f.template operator()<16>();
        case 32: return f.template operator()<32>();
        case 64: return f.template operator()<64>();
        case 128: return f.template operator()<128>();
        case 256: return f.template operator()<256>();
        case 320: return f.template operator()<320>();
        case 384: return f.template operator()<384>();
        case 512: return f.template operator()<512>();
        case 640: return f.template operator()<640>();
        case 768: return f.template operator()<768>();
        default: return HQS_ERR_INVALID_ARG;
    }
}

inline bool fft_size_supported(int n) {
    return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 320 || n == 384 ||
           n == 512 || n == 640 || n == 768;
}

}  // namespace hqs
