// Gridding NUFFT of the multicoil operator of Eq. (1) (Sec. 2.1):
//   forward (a2): apodise + coil-multiply + zero-pad fused into the row FFT,
//                 column FFT, Kaiser-Bessel interpolation (gather);
//   adjoint (a3): tile-owned KB spreading (shared-memory tiles, no atomics),
//                 column IFFT, row IFFT fused with crop + deapodisation +
//                 conj(S_l) coil sum.
// All grids are coil-innermost ([gy][gx][l]) so a grid tap is L contiguous
// complex values.
#include <algorithm>
#include <cstring>

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
    HQS_PDL_ENTRY();
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
    HQS_PDL_ENTRY();
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

// ---- passes with the image in the lower half of each line (G = 2n, 16-coil chunks)
// With G = 2n the centred placement p = (i - n/2) mod G of pixel i is the circular
// shift by n/2 of position q = i, so FFT_G of the centred line is i^k times the FFT of
// the line holding the image in its lower half [0, n), and the centred output pixels
// of an inverse transform are the lower half of the inverse of (-i)^k X[k].  The first
// forward stage then skips the zero half and reads straight from global memory, the
// last inverse stage skips the discarded half, and stores go straight to global
// memory (the I/O hooks of block_fft_io, which need every thread to own a line).
// v * i^k and v * (-i)^k, k >= 0, with selects (k differs from lane to lane: no branches)
HQS_DEV float2 mul_ipow(float2 v, int k) {
    const bool odd = k & 1, neg = k & 2;
    const float re = odd ? -v.y : v.x, im = odd ? v.x : v.y;
    return neg ? make_float2(-re, -im) : make_float2(re, im);
}
HQS_DEV float2 mul_mipow(float2 v, int k) {
    const bool odd = k & 1, neg = k & 2;
    const float re = odd ? v.y : v.x, im = odd ? -v.x : v.y;
    return neg ? make_float2(-re, -im) : make_float2(re, im);
}

// Arguments of the lower-half FFT passes of one plan (G = 2n, chunks of 16 coils),
// for the single-slice launches and, in a table over slices, the batched ones.
struct HalfArgs {
    const float2* x;       // forward: image
    float2* xo;            // adjoint: image (out)
    const float2* z;       // adjoint: xo = A^H y + zc z when z is given
    float zc;
    const float2* smaps;   // [n][n][L]
    const float* apod;     // [n]
    const float2* tw;      // G-point twiddles
    float2* work;          // [n][G][L]
    float2* grid;          // [G][G][L]
    float2* part;          // [nchunk][n][n] coil-chunk sums (nchunk > 1)
    int n, L, nchunk;
    float scale;
};

template <int G> HQS_DEV void fwd_rows_h_item(const HalfArgs& A, int iy, int ch, float2* s) {
    const float2* tw = stage_twiddles<G>(s + G * kLines, A.tw);
    const int n = A.n, L = A.L, l0 = ch * kLines;
    const float ay = A.apod[iy] * A.scale;
    const float2* xr = A.x + (int64_t)iy * n;
    const float2* sm = A.smaps + (int64_t)iy * n * L + l0;
    const float* apod = A.apod;
    float2* dst = A.work + (int64_t)iy * G * L + l0;
    __syncthreads();
    block_fft_io<G, false, true, false>(
        s, kLines, tw,
        [&](int line, int q, bool) { return cscale(cmul(__ldg(sm + (int64_t)q * L + line), __ldg(xr + q)), ay * __ldg(apod + q)); },
        NoIO{}, [&](int line, int k, float2 v) { dst[(int64_t)k * L + line] = mul_ipow(v, k); });
}

template <int G> HQS_DEV void fwd_cols_h_item(const HalfArgs& A, int gx, int ch, float2* s) {
    const float2* tw = stage_twiddles<G>(s + G * kLines, A.tw);
    const int L = A.L, l0 = ch * kLines;
    const int64_t rs = (int64_t)G * L;
    const float2* col = A.work + (int64_t)gx * L + l0;
    float2* dst = A.grid + (int64_t)gx * L + l0;
    __syncthreads();
    block_fft_io<G, false, true, false>(
        s, kLines, tw, [&](int line, int q, bool) { return __ldg(col + q * rs + line); }, NoIO{},
        [&](int line, int k, float2 v) { dst[k * rs + line] = mul_ipow(v, k); });
}

template <int G> HQS_DEV void adj_cols_h_item(const HalfArgs& A, int gx, int ch, float2* s) {
    const float2* tw = stage_twiddles<G>(s + G * kLines, A.tw);
    const int L = A.L, l0 = ch * kLines;
    const int64_t rs = (int64_t)G * L;
    const float2* col = A.grid + (int64_t)gx * L + l0;
    float2* dst = A.work + (int64_t)gx * L + l0;
    __syncthreads();
    block_fft_io<G, true, false, true>(
        s, kLines, tw, [&](int line, int p, bool) { return mul_mipow(__ldg(col + p * rs + line), p); }, NoIO{},
        [&](int line, int q, float2 v) { dst[q * rs + line] = v; });
}

// The row's coil maps go with cp.async to the upper half of the lines buffer once
// the last stage has read it (that stage keeps the lower half only), so their
// latency overlaps the stage instead of following the transform.
template <int G> HQS_DEV void adj_rows_h_item(const HalfArgs& A, int iy, int ch, float2* s) {
    const float2* tw = stage_twiddles<G>(s + G * kLines, A.tw);
    const int n = A.n, L = A.L, l0 = ch * kLines;
    const float2* src = A.work + (int64_t)iy * G * L + l0;
    const float2* sm = A.smaps + (int64_t)iy * n * L + l0;
    float2* msm = s + (int64_t)n * kLines;   // upper half: [n][kLines]
    bool issued = false;
    __syncthreads();
    block_fft_io<G, true, false, true>(
        s, kLines, tw, [&](int line, int p, bool) { return mul_mipow(__ldg(src + (int64_t)p * L + line), p); },
        [&](int, int, float2 v) {
            if (!issued) {   // every thread owns a line position (16 lines, blockDim = 16 TPL)
                issued = true;
                for (int e = threadIdx.x; e < n * (kLines / 2); e += blockDim.x) {
                    const int ix = e / (kLines / 2), h = e - ix * (kLines / 2);
                    cp_async16(msm + ix * kLines + 2 * h, sm + (int64_t)ix * L + 2 * h);
                }
            }
            return v;
        },
        NoIO{});
    cp_async_wait_all();
    __syncthreads();
    const float ay = A.apod[iy] * A.scale;
    for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
        const float4* s4 = reinterpret_cast<const float4*>(msm + ix * kLines);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < kLines / 2; ++h) {
            const float4 sv = s4[h];
            const float2 g0 = s[ix * kLines + 2 * h], g1 = s[ix * kLines + 2 * h + 1];
            a.x += sv.x * g0.x + sv.y * g0.y + sv.z * g1.x + sv.w * g1.y;
            a.y += sv.x * g0.y - sv.y * g0.x + sv.z * g1.y - sv.w * g1.x;
        }
        if (A.nchunk == 1) {
            const int64_t e = (int64_t)iy * n + ix;
            float2 v = cscale(a, ay * A.apod[ix]);
            if (A.z) {
                const float2 zv = A.z[e];
                v.x = fmaf(A.zc, zv.x, v.x);
                v.y = fmaf(A.zc, zv.y, v.y);
            }
            A.xo[e] = v;
        } else {
            A.part[((int64_t)ch * n + iy) * n + ix] = a;
        }
    }
}

// single slice: grid (rows or columns, chunks); batched: grid (rows or columns,
// largest chunk count, slices), the slice's arguments from a device table
#define HQS_HALF_KERNELS(NAME)                                                            \
    template <int G> __global__ void k_##NAME(HalfArgs A) {                               \
        HQS_PDL_ENTRY();                                                                  \
        extern __shared__ __align__(16) float2 s[];                                       \
        NAME##_item<G>(A, blockIdx.x, blockIdx.y, s);                                     \
    }                                                                                     \
    template <int G> __global__ void k_##NAME##_b(const HalfArgs* __restrict__ tab, float zc) { \
        HQS_PDL_ENTRY();                                                                  \
        extern __shared__ __align__(16) float2 s[];                                       \
        HalfArgs A = tab[blockIdx.z];                                                     \
        A.zc = zc;                                                                        \
        if ((int)blockIdx.y >= A.nchunk) return;                                          \
        NAME##_item<G>(A, blockIdx.x, blockIdx.y, s);                                     \
    }
HQS_HALF_KERNELS(fwd_rows_h)
HQS_HALF_KERNELS(fwd_cols_h)
HQS_HALF_KERNELS(adj_cols_h)
HQS_HALF_KERNELS(adj_rows_h)
#undef HQS_HALF_KERNELS

template <int W>
__global__ void __launch_bounds__(256) k_interp(const float2* __restrict__ Gh, const int4* __restrict__ pts,
                                                const int* __restrict__ perm, int M, int G, int L,
                                                float beta, float2* __restrict__ y) {
    HQS_PDL_ENTRY();
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

// Type-2 interpolation for 16-coil chunks: 8 lanes per point, lane q owning coils
// (2q, 2q+1) of a chunk, so one float4 load per lane reads a tap's 16 coils as one
// 128-byte line; the 2W weights come from the plan's table; the result goes to the
// sorted order, coil-innermost (one 128-byte store per point and chunk), and
// k_y_from_sorted puts it in the caller's (coil, point) order.
template <int W>
__global__ void __launch_bounds__(256) k_interp16(const float2* __restrict__ Gh, const int4* __restrict__ pts,
                                                  const float* __restrict__ kbw, int M, int G, int L,
                                                  float2* __restrict__ ys) {
    HQS_PDL_ENTRY();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j = t >> 3;
    const int q = threadIdx.x & 7;
    if (j >= M) return;
    const int4 pt = pts[j];
    float wx[W], wy[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        wx[w] = __ldg(kbw + j * 2 * W + w);
        wy[w] = __ldg(kbw + j * 2 * W + W + w);
    }
    int gxs[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        const int gx = pt.x + b;
        gxs[b] = gx >= G ? gx - G : gx;
    }
    for (int l0 = 0; l0 < L; l0 += 16) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            int gy = pt.y + a;
            if (gy >= G) gy -= G;
            const float4* row = reinterpret_cast<const float4*>(Gh + (int64_t)gy * G * L + l0) + q;
            float4 ra = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float4 g = __ldg(row + (int64_t)gxs[b] * (L / 2));
                ra.x = fmaf(wx[b], g.x, ra.x);
                ra.y = fmaf(wx[b], g.y, ra.y);
                ra.z = fmaf(wx[b], g.z, ra.z);
                ra.w = fmaf(wx[b], g.w, ra.w);
            }
            acc.x = fmaf(wy[a], ra.x, acc.x);
            acc.y = fmaf(wy[a], ra.y, acc.y);
            acc.z = fmaf(wy[a], ra.z, acc.z);
            acc.w = fmaf(wy[a], ra.w, acc.w);
        }
        reinterpret_cast<float4*>(ys + j * L + l0)[q] = acc;
    }
}

// ---------------------------------------------------------------- adjoint
// k-space data to the sorted point order, coil-innermost: ys[invperm[m]][l] =
// y[l][m].  A CTA stages kSortPts caller-order points of every coil (coalesced
// rows of y) in shared memory and writes each point's L-coil line contiguously.
constexpr int kSortPts = 64;
__global__ void __launch_bounds__(256) k_y_to_sorted(const float2* __restrict__ y, const int* __restrict__ invperm,
                                                     int M, int L, float2* __restrict__ ys) {
    HQS_PDL_ENTRY();
    extern __shared__ float2 sy[];   // [kSortPts][L + 1]
    const int m0 = blockIdx.x * kSortPts;
    const int np = min(kSortPts, M - m0);
    for (int e = threadIdx.x; e < L * kSortPts; e += blockDim.x) {
        const int l = e / kSortPts, q = e - l * kSortPts;
        if (q < np) sy[q * (L + 1) + l] = y[(int64_t)l * M + m0 + q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np * L; e += blockDim.x) {
        const int q = e / L, l = e - q * L;
        ys[(int64_t)invperm[m0 + q] * L + l] = sy[q * (L + 1) + l];
    }
}

// The reverse copy for the forward operator: y[l][m] = ys[invperm[m]][l], each
// point's L-coil line read contiguously, each coil's kSortPts points written as one run.
__global__ void __launch_bounds__(256) k_y_from_sorted(const float2* __restrict__ ys, const int* __restrict__ invperm,
                                                       int M, int L, float2* __restrict__ y) {
    HQS_PDL_ENTRY();
    extern __shared__ float2 sy[];   // [kSortPts][L + 1]
    const int m0 = blockIdx.x * kSortPts;
    const int np = min(kSortPts, M - m0);
    for (int e = threadIdx.x; e < np * L; e += blockDim.x) {
        const int q = e / L, l = e - q * L;
        sy[q * (L + 1) + l] = ys[(int64_t)invperm[m0 + q] * L + l];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * kSortPts; e += blockDim.x) {
        const int l = e / kSortPts, q = e - l * kSortPts;
        if (q < np) y[(int64_t)l * M + m0 + q] = sy[q * (L + 1) + l];
    }
}

// Tile-owned type-1 spreading.  One CTA per item of a TT x TT tile of the
// grid: the item's candidates (points [c0, c1) of the tile's 3 x 3
// neighbouring bins, taken in a fixed order; a point's W taps reach at most
// one bin to either side because TT >= W/2) that touch the tile are staged in
// shared memory, in candidate order, with their plan-time Kaiser-Bessel
// weights, their first tap relative to the tile and their k-space values.
// Warp w owns the tile rows w (mod 8); for one row and a chunk of LCS coils a
// lane owns the (cell, coil) pairs p = lane + 32 k of the row and keeps their
// sums in registers while it walks the staged points in order, so no two
// threads ever update one cell and every cell is summed in the same order.
// The row is then written once with plain stores: to the grid when the tile
// has one item, else to the item's partial slot, and the last of the tile's
// items to arrive sums the slots in slot order into the grid.  No atomics on
// data and no memset of the grid.
constexpr int kSpreadWarps = 8;
// FULL16: every coil chunk has exactly 16 coils (L a multiple of 16).  Then lane
// (h, l) = (lane / 16, lane % 16) owns coil l of the cells x = h + 2 k of a row,
// and each staged point's x weights over the tile row are tabulated once
// (wrow[i][h][k], zero outside the footprint), so a cell update is one
// multiply-add pair on registers.
template <int W, int TT, bool FULL16>
__global__ void __launch_bounds__(256) k_spread_tiles(const float2* __restrict__ ys, const int4* __restrict__ pts,
                                                      const float* __restrict__ kbw, const int2* __restrict__ tile_nb,
                                                      const int4* __restrict__ items, const int2* __restrict__ tinfo,
                                                      unsigned* __restrict__ tickets, float2* __restrict__ partial,
                                                      int G, int L, int LCS, int nbx, float2* __restrict__ grid) {
    HQS_PDL_ENTRY();
    constexpr int CAND = HQS_SPREAD_CAND;
    constexpr int NK = (TT * 16 + 31) / 32;   // (cell, coil) pairs of a row per lane, LCS <= 16
    extern __shared__ float4 smem4[];
    float2* sval = reinterpret_cast<float2*>(smem4);              // [CAND][LCS]
    float* swt = reinterpret_cast<float*>(sval + CAND * LCS);      // [CAND][2W]
    int2* soff = reinterpret_cast<int2*>(swt + CAND * 2 * W);      // [CAND]: first tap - tile origin (x, y)
    int* sidx = reinterpret_cast<int*>(soff + CAND);               // [CAND]: sorted point index
    float* wrow = reinterpret_cast<float*>(sidx + CAND);           // FULL16: [CAND][2][TT / 2]
    __shared__ int2 nbs[10];
    __shared__ int npts, wcount[kSpreadWarps], last;
    const int4 it = items[blockIdx.x];
    const int t = it.x, tx = t % nbx, ty = t / nbx;
    const int x0 = tx * TT, y0 = ty * TT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the tile's distinct neighbouring bins from the plan: (first point, candidate
    // prefix) in candidate order, entry 9 = (bins, candidates)
    if (threadIdx.x < 10) nbs[threadIdx.x] = tile_nb[(int64_t)t * 10 + threadIdx.x];
    __syncthreads();
    // stage the candidates that touch the tile, in candidate order (CAND == blockDim)
    {
        const int c = it.y + threadIdx.x;
        bool ov = false;
        int j = 0, ox = 0, oy = 0;
        if (c < it.z) {
            const int nnb = nbs[9].x;
            int k = 0;
            while (k + 1 < nnb && nbs[k + 1].y <= c) ++k;
            j = nbs[k].x + (c - nbs[k].y);
            const int4 pt = pts[j];
            // first tap relative to the tile, on the periodic grid: in [0, TT) when the
            // taps start inside the tile, in [-(W-1), 0) when they start left of it
            ox = pt.x - x0;
            oy = pt.y - y0;
            if (ox < 0) ox += G;
            if (oy < 0) oy += G;
            if (ox >= TT) ox -= G;
            if (oy >= TT) oy -= G;
            ov = ox > -W && oy > -W;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ov);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int base = 0;
        for (int w = 0; w < warp; ++w) base += wcount[w];
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < kSpreadWarps; ++w) tot += wcount[w];
            npts = tot;
        }
        if (ov) {
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            soff[pos] = make_int2(ox, oy);
            sidx[pos] = j;
        }
        __syncthreads();
    }
    const int np = npts;
    for (int e = threadIdx.x; e < np * 2 * W; e += blockDim.x) {
        const int i = e / (2 * W), h = e - i * (2 * W);
        swt[e] = __ldg(kbw + (int64_t)sidx[i] * 2 * W + h);
    }
    if constexpr (FULL16) {
        // the first chunk's values load together with the weights (one latency round)
        for (int e = threadIdx.x; e < np * 16; e += blockDim.x) {
            const int i = e >> 4, ll = e & 15;
            sval[i * 16 + ll] = __ldg(ys + (int64_t)sidx[i] * L + ll);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < np * TT; e += blockDim.x) {
            const int i = e / TT, x = e - i * TT;
            int b = x - soff[i].x;
            b += b < 0 ? G : 0;
            wrow[i * TT + (x & 1) * (TT / 2) + (x >> 1)] = (unsigned)b < (unsigned)W ? swt[i * 2 * W + b] : 0.f;
        }
        const int h = lane >> 4, l = lane & 15;
        for (int l0 = 0; l0 < L; l0 += 16) {
            if (l0 > 0) {   // later 16-coil chunks
                for (int e = threadIdx.x; e < np * 16; e += blockDim.x) {
                    const int i = e >> 4, ll = e & 15;
                    sval[i * 16 + ll] = __ldg(ys + (int64_t)sidx[i] * L + l0 + ll);
                }
            }
            __syncthreads();
            float2* dst = it.w < 0 ? grid : partial + (int64_t)it.w * TT * TT * L;
            for (int r = warp; r < TT; r += kSpreadWarps) {
                float2 acc[TT / 2];
#pragma unroll
                for (int k = 0; k < TT / 2; ++k) acc[k] = make_float2(0.f, 0.f);
                for (int i = 0; i < np; ++i) {
                    int a = r - soff[i].y;
                    a += a < 0 ? G : 0;
                    if ((unsigned)a >= (unsigned)W) continue;
                    const float wy = swt[i * 2 * W + W + a];
                    float2 v = sval[i * 16 + l];
                    v.x *= wy;
                    v.y *= wy;
                    const float4* wr = reinterpret_cast<const float4*>(wrow + i * TT + h * (TT / 2));
#pragma unroll
                    for (int k4 = 0; k4 < TT / 8; ++k4) {
                        const float4 w4 = wr[k4];
                        const float wk[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            acc[4 * k4 + q].x = fmaf(wk[q], v.x, acc[4 * k4 + q].x);
                            acc[4 * k4 + q].y = fmaf(wk[q], v.y, acc[4 * k4 + q].y);
                        }
                    }
                }
                const int64_t rowo = it.w < 0 ? ((int64_t)(y0 + r) * G + x0) * L : (int64_t)r * TT * L;
#pragma unroll
                for (int k = 0; k < TT / 2; ++k) dst[rowo + (int64_t)(h + 2 * k) * L + l0 + l] = acc[k];
            }
            __syncthreads();
        }
    }
    for (int l0 = 0; !FULL16 && l0 < L; l0 += LCS) {
        const int lc = min(LCS, L - l0);
        for (int e = threadIdx.x; e < np * lc; e += blockDim.x) {
            const int i = e / lc, l = e - i * lc;
            sval[i * LCS + l] = __ldg(ys + (int64_t)sidx[i] * L + l0 + l);
        }
        __syncthreads();
        const int npair = TT * lc;
        int px[NK], pl[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int pp = lane + 32 * k;
            px[k] = pp / lc;
            pl[k] = pp - px[k] * lc;
        }
        float2* dst = it.w < 0 ? grid : partial + (int64_t)it.w * TT * TT * L;
        for (int r = warp; r < TT; r += kSpreadWarps) {
            float2 acc[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) acc[k] = make_float2(0.f, 0.f);
            for (int i = 0; i < np; ++i) {
                const int2 o = soff[i];
                // the point's row tap for this row (the wrap matters only when the tile is
                // the whole grid: there a footprint can leave its right edge and re-enter)
                int a = r - o.y;
                a += a < 0 ? G : 0;
                if ((unsigned)a >= (unsigned)W) continue;
                const float wy = swt[i * 2 * W + W + a];
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    int b = px[k] - o.x;
                    b += b < 0 ? G : 0;
                    const int bc = min(max(b, 0), W - 1);
                    float w = swt[i * 2 * W + bc];
                    w = ((unsigned)b < (unsigned)W) ? w * wy : 0.f;
                    const float2 v = sval[i * LCS + pl[k]];
                    acc[k].x = fmaf(w, v.x, acc[k].x);
                    acc[k].y = fmaf(w, v.y, acc[k].y);
                }
            }
            const int64_t rowo = it.w < 0 ? ((int64_t)(y0 + r) * G + x0) * L : (int64_t)r * TT * L;
#pragma unroll
            for (int k = 0; k < NK; ++k)
                if (lane + 32 * k < npair) dst[rowo + (int64_t)px[k] * L + l0 + pl[k]] = acc[k];
        }
        __syncthreads();
    }
    if (it.w >= 0) {
        // the last item of the tile to arrive sums the partial slots in order
        __threadfence();
        __syncthreads();
        const int2 ti = tinfo[t];
        if (threadIdx.x == 0) last = atomicAdd(&tickets[t], 1u) == (unsigned)(ti.x - 1);
        __syncthreads();
        if (last) {
            __threadfence();
            const int64_t slot = (int64_t)TT * TT * L;
            const float2* p0 = partial + (int64_t)ti.y * slot;
            for (int e = threadIdx.x; e < TT * TT * L; e += blockDim.x) {
                float2 acc = __ldcg(p0 + e);
                for (int c = 1; c < ti.x; ++c) {
                    const float2 v = __ldcg(p0 + c * slot + e);
                    acc.x += v.x;
                    acc.y += v.y;
                }
                const int l = e % L, cell = e / L;
                const int r = cell / TT, cx = cell - r * TT;
                grid[((int64_t)(y0 + r) * G + x0 + cx) * L + l] = acc;
            }
            if (threadIdx.x == 0) tickets[t] = 0u;
        }
    }
}

// Column gx: IFFT along y of the spread grid, keep the image rows -> V[iy][gx][l].
template <int G>
__global__ void k_adj_cols(const float2* __restrict__ Hg, int n, int L, int LC, int nchunk,
                           const float2* __restrict__ twg, float2* __restrict__ V) {
    HQS_PDL_ENTRY();
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
    HQS_PDL_ENTRY();
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
    HQS_PDL_ENTRY();
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
// the lower-half passes apply when G = 2n and every coil chunk has 16 coils
inline bool half_passes(const hqs_plan_s* p) { return p->G == 2 * p->n && p->LC == kLines && p->L % kLines == 0; }

static HalfArgs half_args(const hqs_plan_s* p, const float2* x, float2* xo, float zc, const float2* z) {
    HalfArgs A;
    A.x = x;
    A.xo = xo;
    A.z = z;
    A.zc = zc;
    A.smaps = p->smaps;
    A.apod = p->apod;
    A.tw = plan_twiddles(p, p->G);
    A.work = p->work;
    A.grid = p->grid;
    A.part = p->chunk_buf;
    A.n = p->n;
    A.L = p->L;
    A.nchunk = p->nchunk;
    A.scale = p->scale;
    return A;
}

template <int G>
static int fwd_fft_impl(hqs_plan_s* p, const float2* x, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, G);
    const int th = fft_threads<G>(p->LC);
    const size_t sm = nufft_smem_floats2<G>() * sizeof(float2);
    if (half_passes(p)) {
        HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows_h<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_cols_h<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const HalfArgs A = half_args(p, x, nullptr, 0.f, nullptr);
        HQS_CUDA_TRY(launch_pdl(k_fwd_rows_h<G>, dim3(p->n, p->nchunk), th, sm, st, A));
        HQS_CUDA_TRY(launch_pdl(k_fwd_cols_h<G>, dim3(G, p->nchunk), th, sm, st, A));
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    }
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(launch_pdl(k_fwd_rows<G>, dim3(p->n, p->nchunk), th, sm, st, x, p->smaps, p->apod, p->n, p->L, p->LC,
                            p->nchunk, p->scale, tw, p->work));
    HQS_CUDA_TRY(launch_pdl(k_fwd_cols<G>, dim3(G, p->nchunk), th, sm, st, p->work, p->n, p->L, p->LC, p->nchunk, tw,
                            p->grid));
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int G>
static int adj_fft_impl(hqs_plan_s* p, float2* x, float zc, const float2* z, cudaStream_t st) {
    const float2* tw = plan_twiddles(p, G);
    const int th = fft_threads<G>(p->LC);
    const size_t sm = nufft_smem_floats2<G>() * sizeof(float2);
    if (half_passes(p)) {
        HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_cols_h<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_rows_h<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const HalfArgs A = half_args(p, nullptr, x, zc, z);
        HQS_CUDA_TRY(launch_pdl(k_adj_cols_h<G>, dim3(G, p->nchunk), th, sm, st, A));
        HQS_CUDA_TRY(launch_pdl(k_adj_rows_h<G>, dim3(p->n, p->nchunk), th, sm, st, A));
        if (p->nchunk > 1)
            HQS_CUDA_TRY(launch_pdl(k_adj_chunk_sum, dim3(std::min(ceil_div(p->n * p->n, 256), 1024)), dim3(256), 0, st,
                                    p->chunk_buf, p->apod, p->n, p->nchunk, p->scale, x, zc, z));
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    }
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HQS_CUDA_TRY(launch_pdl(k_adj_cols<G>, dim3(G, p->nchunk), th, sm, st, p->grid, p->n, p->L, p->LC, p->nchunk, tw,
                            p->work));
    HQS_CUDA_TRY(launch_pdl(k_adj_rows<G>, dim3(p->n, p->nchunk), th, sm, st, p->work, p->smaps, p->apod, p->n, p->L,
                            p->LC, p->nchunk, p->scale, tw, x, p->chunk_buf, zc, z));
    if (p->nchunk > 1)
        HQS_CUDA_TRY(launch_pdl(k_adj_chunk_sum, dim3(std::min(ceil_div(p->n * p->n, 256), 1024)), dim3(256), 0, st,
                                p->chunk_buf, p->apod, p->n, p->nchunk, p->scale, x, zc, z));
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int W>
static int interp_impl(hqs_plan_s* p, float2* y, cudaStream_t st) {
    if (p->M == 0) return HQS_OK;
    if (p->L % 16 == 0) {
        const int64_t threads8 = p->M * 8;
        HQS_CUDA_TRY(launch_pdl(k_interp16<W>, dim3((unsigned)ceil_div64(threads8, 256)), dim3(256), 0, st, p->grid,
                                p->pts, p->spread.kbw, (int)p->M, p->G, p->L, p->spread.ysort));
        const size_t smy = (size_t)kSortPts * (p->L + 1) * sizeof(float2);
        HQS_CUDA_TRY(launch_pdl(k_y_from_sorted, dim3((unsigned)ceil_div64(p->M, kSortPts)), dim3(256), smy, st,
                                p->spread.ysort, p->invperm, (int)p->M, p->L, y));
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    }
    const int64_t threads = p->M * 16;
    HQS_CUDA_TRY(launch_pdl(k_interp<W>, dim3((unsigned)ceil_div64(threads, 256)), dim3(256), 0, st, p->grid, p->pts,
                            p->perm, (int)p->M, p->G, p->L, (float)p->beta, y));
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// Kaiser-Bessel weights of every sorted point: kbw[j][h] = phi(dx_j - h),
// kbw[j][W + h] = phi(dy_j - h), h < W (a plan-time table of the spreading).
__global__ void k_point_weights(const int4* __restrict__ pts, int M, int W, float beta, float* __restrict__ kbw) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * 2 * W) return;
    const int j = (int)(e / (2 * W)), h = (int)(e - (int64_t)j * 2 * W);
    const int4 pt = pts[j];
    const float t = h < W ? __int_as_float(pt.z) - (float)h : __int_as_float(pt.w) - (float)(h - W);
    kbw[e] = kb_phi(t, (float)W, beta);
}

int launch_point_weights(hqs_plan_s* p, cudaStream_t st) {
    if (p->M == 0) return HQS_OK;
    const int64_t cnt = p->M * 2 * p->W;
    k_point_weights<<<(unsigned)ceil_div64(cnt, 256), 256, 0, st>>>(p->pts, (int)p->M, p->W, (float)p->beta,
                                                                     p->spread.kbw);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// coils per chunk of the tile-owned spreading (shared tile TT^2 x LCS)
inline int spread_lcs(int tile, int L) {
    (void)tile;
    const int nch = ceil_div(L, 16);
    return ceil_div(L, nch);
}

inline size_t spread_smem(int W, int lcs, int tile) {
    return (size_t)HQS_SPREAD_CAND * lcs * sizeof(float2) + (size_t)HQS_SPREAD_CAND * 2 * W * sizeof(float) +
           (size_t)HQS_SPREAD_CAND * (sizeof(int2) + sizeof(int)) + (size_t)HQS_SPREAD_CAND * tile * sizeof(float);
}

template <int W, int TT>
static int spread_tiles_impl(hqs_plan_s* p, const float2* y, cudaStream_t st) {
    const int lcs = spread_lcs(TT, p->L);
    const bool full16 = p->L % 16 == 0;
    const size_t sm = spread_smem(W, lcs, full16 ? TT : 0);
    auto kern = full16 ? k_spread_tiles<W, TT, true> : k_spread_tiles<W, TT, false>;
    HQS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (p->M > 0) {
        const size_t smy = (size_t)kSortPts * (p->L + 1) * sizeof(float2);
        HQS_CUDA_TRY(launch_pdl(k_y_to_sorted, dim3((unsigned)ceil_div64(p->M, kSortPts)), dim3(256), smy, st, y,
                                p->invperm, (int)p->M, p->L, p->spread.ysort));
    }
    HQS_CUDA_TRY(launch_pdl(kern, dim3(p->spread.nitems), dim3(256), sm, st, p->spread.ysort, p->pts, p->spread.kbw,
                            p->spread.tile_nb, p->spread.items, p->spread.tile_info, p->spread.tickets,
                            p->spread.partial, p->G, p->L, lcs, p->nbx, p->grid));
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

template <int W>
static int spread_impl(hqs_plan_s* p, const float2* y, cudaStream_t st) {
    switch (p->tile) {
        case 8: return spread_tiles_impl<W, 8>(p, y, st);
        case 16: return spread_tiles_impl<W, 16>(p, y, st);
        case 32: return spread_tiles_impl<W, 32>(p, y, st);
        default: return HQS_ERR_INVALID_ARG;
    }
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
    // every grid cell is written by the tile-owned spreading: no memset
    int rc = dispatch_w(p->W, [&]<int WW>() { return spread_impl<WW>(p, y, st); });
    if (rc != HQS_OK) return rc;
    return dispatch_fft_size(p->G, [&]<int GG>() { return adj_fft_impl<GG>(p, x, zc, z, st); });
}

// ---- the passes of several plans in one launch per pass (batched operators)
bool plan_half_passes(const hqs_plan_s* p) { return half_passes(p); }
size_t half_args_bytes() { return sizeof(HalfArgs); }
void fill_half_args(const hqs_plan_s* p, const float2* x, float2* xo, const float2* z, void* dst) {
    const HalfArgs A = half_args(p, x, xo, 0.f, z);
    std::memcpy(dst, &A, sizeof(HalfArgs));
}

// `count` plans with grid G = 2n and 16-coil chunks whose arguments are the
// consecutive HalfArgs at d_tab: the forward's row and column passes (adjoint 0)
// or the adjoint's column and row passes (adjoint 1), grid (lines, chunks, plans)
int launch_half_group(int G, int n, int maxchunk, int count, const void* d_tab, int adjoint, float zc,
                      cudaStream_t st) {
    return dispatch_fft_size(G, [&]<int GG>() -> int {
        if constexpr (GG % 2 != 0 || GG < 32) {
            return HQS_ERR_UNSUPPORTED;
        } else {
            const int th = fft_threads<GG>(kLines);
            const size_t sm = nufft_smem_floats2<GG>() * sizeof(float2);
            const HalfArgs* tab = static_cast<const HalfArgs*>(d_tab);
            if (adjoint) {
                HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_cols_h_b<GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                HQS_CUDA_TRY(cudaFuncSetAttribute(k_adj_rows_h_b<GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                HQS_CUDA_TRY(launch_pdl(k_adj_cols_h_b<GG>, dim3(GG, maxchunk, count), th, sm, st, tab, zc));
                HQS_CUDA_TRY(launch_pdl(k_adj_rows_h_b<GG>, dim3(n, maxchunk, count), th, sm, st, tab, zc));
            } else {
                HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows_h_b<GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                HQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_cols_h_b<GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                HQS_CUDA_TRY(launch_pdl(k_fwd_rows_h_b<GG>, dim3(n, maxchunk, count), th, sm, st, tab, zc));
                HQS_CUDA_TRY(launch_pdl(k_fwd_cols_h_b<GG>, dim3(GG, maxchunk, count), th, sm, st, tab, zc));
            }
            HQS_CUDA_TRY(cudaGetLastError());
            return HQS_OK;
        }
    });
}

// the parts of the operators outside the lower-half passes, per plan
int launch_spread(hqs_plan_s* p, const float2* y, cudaStream_t st) {
    return dispatch_w(p->W, [&]<int WW>() { return spread_impl<WW>(p, y, st); });
}
int launch_interp(hqs_plan_s* p, float2* y, cudaStream_t st) {
    return dispatch_w(p->W, [&]<int WW>() { return interp_impl<WW>(p, y, st); });
}
int launch_adj_chunks(hqs_plan_s* p, float2* x, float zc, const float2* z, cudaStream_t st) {
    if (p->nchunk <= 1) return HQS_OK;
    HQS_CUDA_TRY(launch_pdl(k_adj_chunk_sum, dim3(std::min(ceil_div(p->n * p->n, 256), 1024)), dim3(256), 0, st,
                            p->chunk_buf, p->apod, p->n, p->nchunk, p->scale, x, zc, z));
    return HQS_OK;
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
