// Volumetric (3D) multicoil operator of Eq. (1): the paper's conclusion
// (Sec. 5) names 3D data as the next target, and the operator changes only
// by one more axis.
//
//   forward : apodise + coil-multiply fused into the x-axis FFT of the
//             centred, sigma-oversampled grid, then the y and z FFTs, then
//             W^3-tap Kaiser-Bessel interpolation (gather, one half-warp per
//             point, lanes over coils);
//   adjoint : shared-memory tiled spreading (TB^3 bins), z / y / x inverse
//             FFTs with crop, conj(S_l) per coil, coil sum + deapodisation;
//   A^H A   : the 2N^3 circulant embedding (Sec. 3.4 form of the normal
//             operator): pad(S_l x) -> FFT_x, FFT_y, FFT_z * Khat * IFFT_z,
//             IFFT_y, IFFT_x -> crop, conj(S_l) sum.  Zero-padded inputs use
//             the pruned first stage, cropped outputs the pruned last stage.
//   kernel  : t(d) = Nvox^-1 sum_j exp(+i k_j . d) on d in [-N, N)^3 by the
//             adjoint gridding of unit data onto a 4N grid with an 8-wide
//             kernel (an M-independent cost; the exact sum costs M (2N)^3),
//             then Khat = Re FFT_2N(t) / (2N)^3.
//   DC solve: CG on (a A^H A + b I) x = rhs with fp64 inner products.
//
// Grids and per-coil volumes are coil-innermost ([z][y][x][l]); every FFT
// pass is one kernel over lines (a, p, b) at base + a*sA + p*sP + b with b
// the contiguous index, 16 lines per CTA, so loads and stores are coalesced
// over b.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <vector>

#include "fft.cuh"
#include "plan.cuh"

using namespace hqs;

#define HQS3_TILE 8           // spreading bin edge on the grid
#define HQS3_MAXPTS 256       // points per spreading sub-problem
#define HQS3_KERNEL_W 8       // KB width used to grid the Toeplitz kernel

struct Cg3 {
    double rr, rz, pq, alpha, beta, bnorm2, tol2;
    int it, done, status, max_iter;
};

struct hqs_plan3d_s {
    int device = 0;
    int n[3] = {0, 0, 0};     // nx, ny, nz
    int G[3] = {0, 0, 0};     // oversampled NUFFT grid (= 2n: also the Toeplitz grid)
    int L = 0, W = 0;
    double beta = 0.0;
    int64_t M = 0;
    float scale = 1.f;        // Nvox^-1/2
    int nb[3] = {0, 0, 0};
    int nsub = 0;
    float2* smaps = nullptr;  // [nz][ny][nx][L]
    float* apod[3] = {nullptr, nullptr, nullptr};
    int4* pti = nullptr;      // sorted points: (i0x, i0y, i0z, caller index)
    float4* ptd = nullptr;    // (dx, dy, dz, 0)
    int4* subs = nullptr;     // (bin, start, count, 0)
    float* khat = nullptr;    // [2nz][2ny][2nx], includes 1 / (8 Nvox)
    float2* tw = nullptr;     // twiddle bank
    int tw_sizes[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int tw_offs[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool pc_ok = false;       // every axis has an n-point transform: DC preconditioner available
    float* lam = nullptr;     // [nz][ny][nx] Chan symbol of the density preconditioner
    float2* bufA = nullptr;   // 8 Nvox L
    float2* bufB = nullptr;   // 4 Nvox L
    float2* bufC = nullptr;   // Nvox L
    float2* cg_r = nullptr;
    float2* cg_p = nullptr;
    float2* cg_q = nullptr;
    float2* cg_z = nullptr;
    float2* hqs_b0 = nullptr;   // A^H y of the outer loop
    float2* hqs_rhs = nullptr;
    float2* hqs_u = nullptr;
    float2* hqs_w = nullptr;    // A^H A x for the P-metric prox (c1 != 0)
    double* partials = nullptr;
    Cg3* cg = nullptr;
    Cg3* h_cg = nullptr;
    double* hist = nullptr;
    const int* stop = nullptr;          // device flag: passes launched while set return at once
    cudaStream_t cap_stream = nullptr;  // private stream the PCG iteration is captured on
    cudaGraphExec_t iter_graph = nullptr;
    float g_a = 0.f, g_b = 0.f;         // what the captured iteration was built for
    int g_dc = -1;
    const void* g_x = nullptr;
    size_t bytes = 0;
    std::vector<void*> allocs;
};

namespace {

// ---------------------------------------------------------------- helpers
HQS_DEV float kb_phi3(float t, float W, float beta) {
    const float z = 2.0f * t / W;
    const float s = 1.0f - z * z;
    return s >= 0.f ? cyl_bessel_i0f(beta * sqrtf(s)) : 0.f;
}
HQS_DEV int wrap(int i, int G) { return i < 0 ? i + G : (i >= G ? i - G : i); }
// ------------------------------------------------------------ point setup
__global__ void k_points3(const float* __restrict__ traj, int M, int Gx, int Gy, int Gz, int W, int TB,
                          int nbx, int nby, int4* __restrict__ rawi, float4* __restrict__ rawd,
                          int* __restrict__ bin, int* __restrict__ counts) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int Gs[3] = {Gx, Gy, Gz};
    int i0v[3], cb[3];
    float dv[3];
    for (int ax = 0; ax < 3; ++ax) {
        const double G = (double)Gs[ax];
        double u = ((double)traj[3 * (int64_t)j + ax] * G) / (2.0 * 3.141592653589793);
        u -= G * floor(u / G);
        const double i0 = ceil(u - 0.5 * (double)W);
        dv[ax] = (float)(u - i0);
        int ii = (int)i0;
        if (ii < 0) ii += Gs[ax];
        if (ii >= Gs[ax]) ii -= Gs[ax];
        i0v[ax] = ii;
        int c = ii + W / 2;
        if (c >= Gs[ax]) c -= Gs[ax];
        cb[ax] = c / TB;
    }
    rawi[j] = make_int4(i0v[0], i0v[1], i0v[2], j);
    rawd[j] = make_float4(dv[0], dv[1], dv[2], 0.f);
    const int b = (cb[2] * nby + cb[1]) * nbx + cb[0];
    bin[j] = b;
    atomicAdd(&counts[b], 1);
}

__global__ void k_points3_scatter(const int4* __restrict__ rawi, const float4* __restrict__ rawd,
                                  const int* __restrict__ bin, int M, int* __restrict__ cursor,
                                  int4* __restrict__ pti, float4* __restrict__ ptd) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int pos = atomicAdd(&cursor[bin[j]], 1);
    pti[pos] = rawi[j];
    ptd[pos] = rawd[j];
}

__global__ void k_smaps3_coil_inner(const float2* __restrict__ in, float2* __restrict__ out, int64_t nvox,
                                    int L) {
    const int64_t total = nvox * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / L;
        const int l = (int)(e - v * L);
        out[e] = in[(int64_t)l * nvox + v];
    }
}

// ------------------------------------------------------ interpolation
// Type-2 interpolation: a half-warp per point, lane = coil (looping beyond
// 16 coils).  The 3W separable weights are computed once per point by the
// lanes (index q on lane q and q - 16) and broadcast with shuffles.
template <int W>
__global__ void __launch_bounds__(256) k_interp3(const float2* __restrict__ Gh, const int4* __restrict__ pti,
                                                 const float4* __restrict__ ptd, int M, int Gx, int Gy,
                                                 int Gz, int L, float beta, float2* __restrict__ y) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4;
    const int h = threadIdx.x & 15;
    const int base = threadIdx.x & 16;
    const bool valid = j < M;
    const int4 pi = valid ? pti[j] : make_int4(0, 0, 0, 0);
    const float4 pd = valid ? ptd[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    float w0 = 0.f, w1 = 0.f;
    if (valid) {
        const float dd[3] = {pd.x, pd.y, pd.z};
        if (h < 3 * W) w0 = kb_phi3(dd[h / W] - (float)(h % W), (float)W, beta);
        const int q = h + 16;
        if (q < 3 * W) w1 = kb_phi3(dd[q / W] - (float)(q % W), (float)W, beta);
    }
    float wx[W], wy[W], wz[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int qx = w, qy = W + w, qz = 2 * W + w;
        wx[w] = qx < 16 ? __shfl_sync(0xffffffffu, w0, base + qx) : __shfl_sync(0xffffffffu, w1, base + qx - 16);
        wy[w] = qy < 16 ? __shfl_sync(0xffffffffu, w0, base + qy) : __shfl_sync(0xffffffffu, w1, base + qy - 16);
        wz[w] = qz < 16 ? __shfl_sync(0xffffffffu, w0, base + qz) : __shfl_sync(0xffffffffu, w1, base + qz - 16);
    }
    if (!valid) return;
    int gx[W];
#pragma unroll
    for (int b = 0; b < W; ++b) gx[b] = wrap(pi.x + b, Gx);
    for (int l = h; l < L; l += 16) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int c = 0; c < W; ++c) {
            const int gz = wrap(pi.z + c, Gz);
            float2 az = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const int gy = wrap(pi.y + a, Gy);
                const float2* row = Gh + ((int64_t)gz * Gy + gy) * Gx * L + l;
                float2 ra = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float2 g = __ldg(row + (int64_t)gx[b] * L);
                    ra.x = fmaf(wx[b], g.x, ra.x);
                    ra.y = fmaf(wx[b], g.y, ra.y);
                }
                az.x = fmaf(wy[a], ra.x, az.x);
                az.y = fmaf(wy[a], ra.y, az.y);
            }
            acc.x = fmaf(wz[c], az.x, acc.x);
            acc.y = fmaf(wz[c], az.y, acc.y);
        }
        y[(int64_t)l * M + pi.w] = acc;
    }
}

// ------------------------------------------------------------ spreading
// One sub-problem (<= HQS3_MAXPTS points of one TB^3 bin) is spread into a
// (TB+W-1)^3 patch of LC coils (a power of two) in shared memory, then added
// to the global grid with one float2 atomic per nonzero patch cell.  The
// patch has no shared atomics: warp w owns the patch planes z = w (mod 8), so
// for each point the (at most one) footprint plane of a warp is updated by
// that warp alone, lanes over (cell, coil) entries of the plane, with a warp
// barrier between points.  `unit` spreads the value 1 for every point (the
// Toeplitz-kernel gridding).
#define HQS3_SPREAD_WARPS 8
template <int W>
__global__ void __launch_bounds__(HQS3_SPREAD_WARPS * 32)
    k_spread3(const float2* __restrict__ y, const int4* __restrict__ pti, const float4* __restrict__ ptd,
              const int4* __restrict__ subs, int64_t M, int Gx, int Gy, int Gz, int L, int lcs, int nchunk,
              int TB, int nbx, int nby, float beta, int unit, float2* __restrict__ grid) {
    static_assert(W <= HQS3_SPREAD_WARPS, "one footprint plane per warp and point");
    extern __shared__ float4 smem4[];
    const int LC = 1 << lcs;
    const int P = TB + W - 1;
    const int P3 = P * P * P;
    int4* loc = reinterpret_cast<int4*>(smem4);
    float* wts = reinterpret_cast<float*>(loc + HQS3_MAXPTS);
    float2* vals = reinterpret_cast<float2*>(wts + HQS3_MAXPTS * 3 * W);
    float2* patch = vals + HQS3_MAXPTS * LC;
    const int4 sb = subs[blockIdx.x];
    const int bin = sb.x, start = sb.y, cnt = sb.z;
    const int bx = bin % nbx, by = (bin / nbx) % nby, bz = bin / (nbx * nby);
    for (int i = threadIdx.x; i < cnt * 3 * W; i += blockDim.x) {
        const int q = i / (3 * W), hh = i - q * 3 * W;
        const float4 pd = ptd[start + q];
        const int ax = hh / W;
        const float d = ax == 0 ? pd.x : (ax == 1 ? pd.y : pd.z);
        wts[i] = kb_phi3(d - (float)(hh - ax * W), (float)W, beta);
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int4 pi = pti[start + i];
        const int cx = wrap(pi.x + W / 2, Gx), cy = wrap(pi.y + W / 2, Gy), cz = wrap(pi.z + W / 2, Gz);
        loc[i] = make_int4(cx - bx * TB, cy - by * TB, cz - bz * TB, pi.w);
    }
    __syncthreads();   // loc and wts are read by other threads below
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ox = bx * TB - W / 2, oy = by * TB - W / 2, oz = bz * TB - W / 2;
    // lane -> (x tap b, coil l) of a footprint row; W * LC <= 32 (LC = 4 needs W <= 6,
    // the launcher uses LC <= 2 above that)
    const bool has_tap = lane < (W << lcs);
    const int lb = lane >> lcs, ll = lane & ((1 << lcs) - 1);
    for (int ch = blockIdx.y; ch < nchunk; ch += gridDim.y) {
        const int l0 = ch * LC;
        const int lines = min(LC, L - l0);
        for (int e = threadIdx.x; e < P3 * LC; e += blockDim.x) patch[e] = make_float2(0.f, 0.f);
        for (int e = threadIdx.x; e < cnt * LC; e += blockDim.x) {
            const int i = e >> lcs, l = e & (LC - 1);
            float2 v = make_float2(0.f, 0.f);
            if (l < lines) v = unit ? make_float2(1.f, 0.f) : y[(int64_t)(l0 + l) * M + loc[i].w];
            vals[e] = v;
        }
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            const int4 c0 = loc[i];
            const int c = ((warp - c0.z) % HQS3_SPREAD_WARPS + HQS3_SPREAD_WARPS) % HQS3_SPREAD_WARPS;
            if (c < W && has_tap) {
                // this lane's (b, l): the value times the z and x weights once, then down
                // the W rows of the plane
                const float* wv = wts + i * 3 * W;
                const float wzx = wv[2 * W + c] * wv[lb];
                const float2 v = vals[(i << lcs) + ll];
                const float2 t = make_float2(v.x * wzx, v.y * wzx);
                float2* col = patch + ((((c0.z + c) * P + c0.y) * P + c0.x + lb) << lcs) + ll;
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const float wy = wv[W + a];
                    float2* dst = col + ((a * P) << lcs);
                    float2 acc = *dst;
                    acc.x = fmaf(wy, t.x, acc.x);
                    acc.y = fmaf(wy, t.y, acc.y);
                    *dst = acc;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P3 * LC; e += blockDim.x) {
            const int l = e & (LC - 1);
            if (l >= lines) continue;
            const float2 v = patch[e];
            if (v.x == 0.f && v.y == 0.f) continue;
            const int cell = e >> lcs;
            const int cx = cell % P, cy = (cell / P) % P, cz = cell / (P * P);
            const int gx = wrap(ox + cx, Gx), gy = wrap(oy + cy, Gy), gz = wrap(oz + cz, Gz);
            atomicAdd(&grid[(((int64_t)gz * Gy + gy) * Gx + gx) * L + l0 + l], v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ FFT passes
// Line (a, b) of a pass: element p at base + a*sA + p*sP + b.  Every
// functor resolves its line once per thread (prepare(a, b) -> a small state,
// in practice base pointers), so the per-element work is base + p*stride.
struct Lines {
    int64_t sA, sP;
};

// plain line load: positions < count read, the rest zero
struct LdLine {
    const float2* src;
    Lines g;
    int count;
    struct St { const float2* p; };
    HQS_DEV St prepare(int64_t a, int64_t b) const { return {src + a * g.sA + b}; }
    HQS_DEV float2 operator()(const St& t, int p) const {
        return p < count ? t.p[(int64_t)p * g.sP] : make_float2(0.f, 0.f);
    }
};
// centred placement: grid position p holds image index p + n/2 (p < n/2) or p - G + n/2
struct LdCentred {
    const float2* src;
    Lines g;
    int n, G;
    struct St { const float2* p; };
    HQS_DEV St prepare(int64_t a, int64_t b) const { return {src + a * g.sA + b}; }
    HQS_DEV float2 operator()(const St& t, int p) const {
        const int h = n >> 1;
        const int i = p < h ? p + h : (p >= G - h ? p - G + h : -1);
        return i >= 0 ? t.p[(int64_t)i * g.sP] : make_float2(0.f, 0.f);
    }
};
// first forward pass of the NUFFT: S_l x / (phihat^3) at centred positions,
// a = z * ny + y, b = coil
struct LdImageX {
    const float2* x;
    const float2* S;
    const float *apx, *apy, *apz;
    int nx, ny, G, L;
    float scale;
    struct St { const float2* xr; const float2* sr; float f; };
    HQS_DEV St prepare(int64_t a, int64_t b) const {
        const int z = (int)(a / ny), yy = (int)(a - (int64_t)z * ny);
        return {x + a * nx, S + a * nx * L + b, scale * apz[z] * apy[yy]};
    }
    HQS_DEV float2 operator()(const St& t, int p) const {
        const int h = nx >> 1;
        const int ix = p < h ? p + h : (p >= G - h ? p - G + h : -1);
        if (ix < 0) return make_float2(0.f, 0.f);
        return cscale(cmul(t.sr[(int64_t)ix * L], t.xr[ix]), t.f * apx[ix]);
    }
};
// first pass of the Toeplitz product: S_l x in [0, n) (the upper half is zero)
struct LdToepX {
    const float2* x;
    const float2* S;
    int nx, L;
    struct St { const float2* xr; const float2* sr; };
    HQS_DEV St prepare(int64_t a, int64_t b) const { return {x + a * nx, S + a * nx * L + b}; }
    HQS_DEV float2 operator()(const St& t, int p) const { return cmul(t.sr[(int64_t)p * L], t.xr[p]); }
};

// Output of the last stage, position pos of line (a, b): stored at
// dst[a*sA + o*sP + b] for the output index o of pos, if o < count.
// mode 0: o = pos; mode 1: centred crop (image n = count on grid G, pos =
// i - n/2 mod G); mode 2: circulant crop (count = 2h, pos = o or o - 2h mod G).
HQS_DEV int out_index(int pos, int count, int mode, int G) {
    if (mode == 0) return pos < count ? pos : -1;
    const int h = count >> 1;
    if (mode == 1) return pos < h ? pos + h : (pos >= G - h ? pos - G + h : -1);
    return pos < h ? pos : (pos >= G - h ? pos - G + 2 * h : -1);
}
struct StLine {
    static constexpr bool kReduce = false;
    float2* dst;
    Lines g;
    int count, mode, G;
    struct St { float2* p; };
    HQS_DEV St prepare(int64_t a, int64_t b) const { return {dst + a * g.sA + b}; }
    HQS_DEV void put(const St& t, int pos, float2 v) const {
        const int o = out_index(pos, count, mode, G);
        if (o >= 0) t.p[(int64_t)o * g.sP] = v;
    }
};
// last pass with coil weighting: P[(a*nx + o)*L + b] = conj(S) * v
struct StCoil {
    static constexpr bool kReduce = false;
    float2* dst;
    const float2* S;
    int nx, L, centred, G;
    struct St { float2* d; const float2* s; };
    HQS_DEV St prepare(int64_t a, int64_t b) const {
        const int64_t e0 = a * nx * L + b;
        return {dst + e0, S + e0};
    }
    HQS_DEV void put(const St& t, int pos, float2 v) const {
        const int o = out_index(pos, nx, centred ? 1 : 0, G);
        if (o < 0) return;
        const int64_t e = (int64_t)o * L;
        t.d[e] = cmulc(t.s[e], v);
    }
};

// Last x pass with the coil sum fused: the CTA's kLines lines are kLines / L
// whole rows (a = z*ny + y) of all L coils (L divides kLines), so after the
// transform the row's output is reduced over the coils from shared memory:
// out[a*nx + o] = ca * f(a, o) * sum_l conj(S_l) line_l[pos(o)] + cb * z[a*nx + o],
// f the deapodisation (apx etc., or 1 without), pos(o) = o or the centred crop.
// A half-warp per output column, lane j = (row j / L, coil j % L), shuffles
// over the coil lanes.
struct StCoilSum {
    static constexpr bool kReduce = true;
    float2* out;
    const float2* S;
    const float2* z;
    const float *apx, *apy, *apz;
    int nx, ny, L, centred, G;
    float ca, cb;
    HQS_DEV void reduce(int64_t l0, const float2* s) const {
        const int hw = threadIdx.x >> 4, nhw = blockDim.x >> 4;
        const int j = threadIdx.x & 15;
        const int r = j / L, l = j - r * L;
        const int64_t a = l0 / L + r;
        for (int base = 0; base < nx; base += nhw) {
            const int o = base + hw;
            float2 v = make_float2(0.f, 0.f);
            if (o < nx) {
                const int pos = centred ? (o - (nx >> 1) >= 0 ? o - (nx >> 1) : o - (nx >> 1) + G) : o;
                v = cmulc(S[(a * nx + o) * L + l], s[pos * kLines + j]);
            }
            for (int m = L >> 1; m > 0; m >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
            }
            if (o < nx && l == 0) {
                float f = ca;
                if (apx) {
                    const int zz = (int)(a / ny), yy = (int)(a - (int64_t)zz * ny);
                    f *= apz[zz] * apy[yy] * apx[o];
                }
                float2 w = cscale(v, f);
                if (z) {
                    const float2 zv = z[a * nx + o];
                    w.x = fmaf(cb, zv.x, w.x);
                    w.y = fmaf(cb, zv.y, w.y);
                }
                out[a * nx + o] = w;
            }
        }
    }
};

struct NoMid {};
// Khat multiply between the forward and inverse z transforms: b = (ky*Tx + kx)*L + l
struct MidKhat {
    const float* khat;
    int64_t plane;   // Ty * Tx
    int L;
    struct St { const float* k; };
    HQS_DEV St prepare(int64_t, int64_t b) const { return {khat + b / L}; }
    HQS_DEV float2 operator()(const St& t, int p, float2 v) const { return cscale(v, t.k[(int64_t)p * plane]); }
};

// density-preconditioner multiply s^-1/2 / Nvox between the forward and
// inverse z transforms of a single volume: b = ky*nx + kx
struct MidPrecond {
    const float* lam;
    int64_t plane;   // ny * nx
    float a, b, inv_nvox;
    struct St { const float* l; };
    HQS_DEV St prepare(int64_t, int64_t bb) const { return {lam + bb}; }
    HQS_DEV float2 operator()(const St& t, int p, float2 v) const {
        const float sv = fmaxf(fmaf(a, fmaxf(t.l[(int64_t)p * plane], 0.f), b), 0.25f * b);
        return cscale(v, rsqrtf(sv) * inv_nvox);
    }
};

template <int N> constexpr size_t pass_smem() { return ((size_t)N * kLines + N) * sizeof(float2); }
template <int N> constexpr int pass_threads() { return ((kLines * FftSizeV<N>::TPL + 31) / 32) * 32; }

// One FFT pass over `nlines` lines (a = line / B, b = line % B), kLines per
// CTA, with the two-stage volume transforms: the first stage loads through
// ld (global memory), the last stage stores through st.put (global memory),
// so shared memory holds only the data between stages.  INV, ZIN, HOUT as in
// block_fft.  With a MID functor the pass is FFT -> mid (fused into the last
// forward stage) -> inverse FFT, HOUT applying to the inverse.
template <int N, bool INV, bool ZIN, bool HOUT, class LD, class ST, class MID>
__global__ void k_pass3(LD ld, ST st, MID mid, int64_t nlines, int64_t B, const float2* __restrict__ twg,
                        const int* stop) {
    if (stop && *stop) return;
    extern __shared__ float2 s[];
    const float2* tw = stage_twiddles<N>(s + N * kLines, twg);
    constexpr int TPL = FftSizeV<N>::TPL;
    const int64_t l0 = (int64_t)blockIdx.x * kLines;
    const int lines = (int)min((int64_t)kLines, nlines - l0);
    const int ll = (int)(threadIdx.x % (blockDim.x / TPL));
    const int64_t mine = l0 + (ll < lines ? ll : 0);
    const int64_t a = mine / B, b = mine - a * B;
    // threads without a line (ll >= lines) were given line l0 above: they read
    // it (in bounds) and store nothing
    const auto lds = ld.prepare(a, b);
    auto load = [&](int, int pos, bool) { return ld(lds, pos); };
    if constexpr (ST::kReduce) {
        static_assert(std::is_same_v<MID, NoMid>, "the coil-sum store ends a plain pass");
        block_fft_io_tab<FftSizeV, N, INV, ZIN, HOUT>(s, lines, tw, load, NoIO{}, NoIO{});   // ends with a barrier
        st.reduce(l0, s);
        return;
    } else {
    const auto sts = st.prepare(a, b);
    auto store = [&](int, int pos, float2 v) { st.put(sts, pos, v); };
    if constexpr (std::is_same_v<MID, NoMid>) {
        block_fft_io_tab<FftSizeV, N, INV, ZIN, HOUT>(s, lines, tw, load, NoIO{}, store);
    } else {
        const auto mds = mid.prepare(a, b);
        auto xf = [&](int, int pos, float2 v) { return mid(mds, pos, v); };
        block_fft_io_tab<FftSizeV, N, false, ZIN, false>(s, lines, tw, load, xf, NoIO{});
        block_fft_io_tab<FftSizeV, N, true, false, HOUT>(s, lines, tw, NoIO{}, NoIO{}, store);
    }
    }
}

template <class F> int dispatch3(int n, F&& f) { return dispatch_fft_size(n, std::forward<F>(f)); }

const float2* tw3(const hqs_plan3d_s* p, int N) {
    for (int i = 0; i < 9; ++i)
        if (p->tw_sizes[i] == N) return p->tw + p->tw_offs[i];
    return nullptr;
}

template <bool INV, bool ZIN, bool HOUT, class LD, class ST, class MID = NoMid>
int run_pass(const hqs_plan3d_s* p, int N, LD ld, ST st, int64_t nlines, int64_t B, cudaStream_t s,
             MID mid = MID{}) {
    if (nlines <= 0) return HQS_OK;
    const float2* tw = tw3(p, N);
    if (!tw) return HQS_ERR_INVALID_ARG;
    return dispatch3(N, [&]<int NN>() {
        auto kern = k_pass3<NN, INV, ZIN, HOUT, LD, ST, MID>;
        const size_t sm = pass_smem<NN>();
        HQS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int64_t nblk = ceil_div64(nlines, kLines);
        if (nblk > 0x7fffffff) return HQS_ERR_INVALID_ARG;
        kern<<<(unsigned)nblk, pass_threads<NN>(), sm, s>>>(ld, st, mid, nlines, B, tw, p->stop);
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    });
}

// out[v] = ca * apod(v) * sum_l P[v*L + l] + cb * z[v]   (apod optional, z optional)
__global__ void k_coil_sum3(const float2* __restrict__ P, int L, int nx, int ny, int64_t nvox,
                            const float* __restrict__ apx, const float* __restrict__ apy,
                            const float* __restrict__ apz, float ca, float cb, const float2* z,
                            float2* out, const int* stop) {
    if (stop && *stop) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (int64_t)gridDim.x * blockDim.x) {
        float2 a = make_float2(0.f, 0.f);
        const float2* pv = P + v * L;
        for (int l = 0; l < L; ++l) a = cadd(a, pv[l]);
        float f = ca;
        if (apx) {
            const int ix = (int)(v % nx);
            const int64_t r = v / nx;
            const int iy = (int)(r % ny), iz = (int)(r / ny);
            f *= apx[ix] * apy[iy] * apz[iz];
        }
        float2 o = cscale(a, f);
        if (z) {
            const float2 zv = z[v];
            o.x = fmaf(cb, zv.x, o.x);
            o.y = fmaf(cb, zv.y, o.y);
        }
        out[v] = o;
    }
}

// circulant column: c[p] *= prod_axis 1/phihat(d/G') / Nvox, zero on every d = -N plane
__global__ void k_kernel_deapod(float2* __restrict__ c, int Tx, int Ty, int Tz, const float* __restrict__ ax,
                                const float* __restrict__ ay, const float* __restrict__ az, float inv_nvox) {
    const int64_t total = (int64_t)Tx * Ty * Tz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(e % Tx);
        const int64_t r = e / Tx;
        const int py = (int)(r % Ty), pz = (int)(r / Ty);
        const bool zero = px == Tx / 2 || py == Ty / 2 || pz == Tz / 2;
        c[e] = zero ? make_float2(0.f, 0.f) : cscale(c[e], ax[px] * ay[py] * az[pz] * inv_nvox);
    }
}

// Chan circulant column of the N^3 Toeplitz part (per axis d in {q, q - N},
// weights (N - q)/N and q/N) from the 2N circulant column c.
__global__ void k_chan3(const float2* __restrict__ c, int nx, int ny, int nz, float2* __restrict__ out) {
    const int64_t total = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int qx = (int)(e % nx);
        const int64_t r = e / nx;
        const int qy = (int)(r % ny), qz = (int)(r / ny);
        float2 acc = make_float2(0.f, 0.f);
        for (int sz = 0; sz < 2; ++sz) {
            const int pz = sz ? qz + nz : qz;
            const float wz = sz ? (float)qz / nz : (float)(nz - qz) / nz;
            for (int sy = 0; sy < 2; ++sy) {
                const int py = sy ? qy + ny : qy;
                const float wy = sy ? (float)qy / ny : (float)(ny - qy) / ny;
                for (int sx = 0; sx < 2; ++sx) {
                    const int px = sx ? qx + nx : qx;
                    const float wx = sx ? (float)qx / nx : (float)(nx - qx) / nx;
                    const float2 v = c[((int64_t)pz * 2 * ny + py) * 2 * nx + px];
                    const float w = wz * wy * wx;
                    acc.x = fmaf(w, v.x, acc.x);
                    acc.y = fmaf(w, v.y, acc.y);
                }
            }
        }
        out[e] = acc;
    }
}

__global__ void k_real_part3(const float2* __restrict__ in, float* __restrict__ out, int64_t count, float s) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in[e].x * s;
}

// ------------------------------------------------------------ Gaussian smoothing
#define HQS3_BLUR_MAXR 24
struct Taps3 {
    int r;
    float g[2 * HQS3_BLUR_MAXR + 1];
};

// One axis of the separable periodic blur: out[.., c, ..] = sum_i g[i] in[.., (c + i - r) mod n, ..],
// the axis of length n with element stride `stride`; taps in order i = 0..2r.
__global__ void k_blur3(const float2* __restrict__ in, float2* __restrict__ out, int n, int64_t stride,
                        int64_t nvox, Taps3 t) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)((v / stride) % n);
        const float2* base = in + (v - (int64_t)c * stride);
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i <= 2 * t.r; ++i) {
            int q = (c + i - t.r) % n;
            if (q < 0) q += n;
            const float2 w = base[(int64_t)q * stride];
            acc.x = fmaf(t.g[i], w.x, acc.x);
            acc.y = fmaf(t.g[i], w.y, acc.y);
        }
        out[v] = acc;
    }
}

// out = u + cb v (+ cc w)
__global__ void k_axpbypcz3(float2* __restrict__ out, const float2* __restrict__ u, const float2* __restrict__ v,
                            float cb, const float2* __restrict__ w, float cc, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        float2 o = u[e];
        const float2 vv = v[e];
        o.x = fmaf(cb, vv.x, o.x);
        o.y = fmaf(cb, vv.y, o.y);
        if (w) {
            const float2 ww = w[e];
            o.x = fmaf(cc, ww.x, o.x);
            o.y = fmaf(cc, ww.y, o.y);
        }
        out[e] = o;
    }
}

// ------------------------------------------------------------ CG kernels
#define CG3_BLOCKS 1024
enum { CG3_INIT = 0, CG3_ALPHA = 1, CG3_RES = 2, CG3_RZ = 3, CG3_RZ_RR = 4 };

HQS_DEV double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// partials[blk] = Re <a, b> over this block's grid-stride share (fp64)
__global__ void k_dot3(const float2* __restrict__ a, const float2* __restrict__ b, int64_t count,
                       double* __restrict__ part, const int* stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 u = a[e], v = b[e];
        acc += (double)u.x * v.x + (double)u.y * v.y;
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// r = rhs - q; partials: <r, r> (slot 0) and <rhs, rhs> (slot 1)
__global__ void k_cg3_init(const float2* __restrict__ rhs, const float2* __restrict__ q, float2* __restrict__ r,
                           int64_t count, double* __restrict__ part) {
    __shared__ double sh[32];
    double rr = 0.0, bb = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 b = rhs[e];
        const float2 v = csub(b, q[e]);
        r[e] = v;
        rr += (double)v.x * v.x + (double)v.y * v.y;
        bb += (double)b.x * b.x + (double)b.y * b.y;
    }
    const double t0 = block_sum(rr, sh);
    const double t1 = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t0;
        part[CG3_BLOCKS + blockIdx.x] = t1;
    }
}

// CG scalars from fixed-order sums of the per-block partials:
//   INIT  rr, ||rhs||^2, tolerance, done if converged at the start
//   ALPHA alpha = rz / <p, q> (breakdown if <p, q> <= 0)
//   RES   one more iteration: rr, history, convergence / iteration limit
//   RZ    rz = <r, z>, beta = rz_new / rz_old (after the first)
//   RZ_RR the same with z = r (no preconditioner): rz = rr
// One warp: lane i sums partials i, i + 32, ... in order, then a butterfly
// of shuffles (every lane ends with the same, run-to-run identical value).
HQS_DEV double warp_fixed_sum(const double* part, int n) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += part[i];
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

__global__ void k_cg3_scalar(Cg3* cg, const double* __restrict__ part, int nparts, int mode, double* hist,
                             double rel_tol, int max_iter) {
    const double s = mode != CG3_RZ_RR ? warp_fixed_sum(part, nparts) : 0.0;
    const double bb = mode == CG3_INIT ? warp_fixed_sum(part + CG3_BLOCKS, nparts) : 0.0;
    if (threadIdx.x != 0) return;
    if (mode == CG3_INIT) {
        cg->rr = s;
        cg->bnorm2 = bb;
        cg->tol2 = rel_tol * rel_tol * bb;
        cg->it = 0;
        cg->max_iter = max_iter;
        cg->status = HQS_OK;
        cg->beta = 0.0;
        cg->done = (bb == 0.0 || s <= cg->tol2) ? 1 : 0;
        if (!cg->done && max_iter <= 0) {
            cg->done = 1;
            cg->status = HQS_ERR_NOT_CONVERGED;
        }
        hist[0] = s;
        return;
    }
    if (cg->done) return;
    if (mode == CG3_ALPHA) {
        cg->pq = s;
        if (!(s > 0.0) || !isfinite(s)) {
            cg->done = 1;
            cg->status = HQS_ERR_BREAKDOWN;
            cg->alpha = 0.0;
            return;
        }
        cg->alpha = cg->rz / s;
    } else if (mode == CG3_RES) {
        cg->it += 1;
        cg->rr = s;
        if (cg->it <= HQS_MAX_ITERS) hist[cg->it] = s;
        if (!isfinite(s)) {
            cg->done = 1;
            cg->status = HQS_ERR_BREAKDOWN;
        } else if (s <= cg->tol2) {
            cg->done = 1;
        } else if (cg->it >= cg->max_iter) {
            cg->done = 1;
            cg->status = HQS_ERR_NOT_CONVERGED;
        }
    } else {
        const double rz = mode == CG3_RZ_RR ? cg->rr : s;
        if (!(rz > 0.0) || !isfinite(rz)) {
            cg->done = 1;
            cg->status = HQS_ERR_BREAKDOWN;
            return;
        }
        cg->beta = cg->it > 0 ? rz / cg->rz : 0.0;
        cg->rz = rz;
    }
}

// x += alpha p, r -= alpha q; partials <r, r>
__global__ void k_cg3_update(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                             const float2* __restrict__ q, int64_t count, const Cg3* __restrict__ cg,
                             double* __restrict__ part) {
    __shared__ double sh[32];
    const bool skip = cg->done != 0;
    const float al = (float)cg->alpha;
    double rr = 0.0;
    if (!skip) {
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
             e += (int64_t)gridDim.x * blockDim.x) {
            const float2 pv = p[e], qv = q[e];
            float2 xv = x[e], rv = r[e];
            xv.x = fmaf(al, pv.x, xv.x);
            xv.y = fmaf(al, pv.y, xv.y);
            rv.x = fmaf(-al, qv.x, rv.x);
            rv.y = fmaf(-al, qv.y, rv.y);
            x[e] = xv;
            r[e] = rv;
            rr += (double)rv.x * rv.x + (double)rv.y * rv.y;
        }
    }
    const double t = block_sum(rr, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z (first) or z + beta p; skipped once done
__global__ void k_cg3_pupdate(float2* __restrict__ p, const float2* __restrict__ z, int64_t count,
                              const Cg3* __restrict__ cg) {
    if (cg->done) return;
    const bool first = cg->it == 0;
    const float be = (float)cg->beta;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 zv = z[e];
        if (first) {
            p[e] = zv;
        } else {
            const float2 pv = p[e];
            p[e] = make_float2(fmaf(be, pv.x, zv.x), fmaf(be, pv.y, zv.y));
        }
    }
}

// ------------------------------------------------------------ host side
double kb_phihat3(double nu, int W, double beta) {
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
double kb_beta3(int W, double sigma) {
    return M_PI * sqrt((double)W * W / (sigma * sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
}

template <class T> int alloc3(hqs_plan3d_s* p, T** ptr, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        hqs_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return HQS_ERR_OOM;
    }
    p->allocs.push_back(v);
    p->bytes += count * sizeof(T);
    *ptr = static_cast<T*>(v);
    return HQS_OK;
}

void plan3d_free(hqs_plan3d_s* p) {
    if (!p) return;
    if (p->iter_graph) cudaGraphExecDestroy(p->iter_graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (void* v : p->allocs) cudaFree(v);
    if (p->h_cg) cudaFreeHost(p->h_cg);
    delete p;
}

#define TRY3(expr)                   \
    do {                             \
        const int rc_ = (expr);      \
        if (rc_ != HQS_OK) return rc_; \
    } while (0)

bool size3_ok(int n) {
    // n even, 2n and 4n transform sizes of the library
    return n >= 8 && n % 2 == 0 && fft_size_supported(2 * n) && fft_size_supported(4 * n);
}

// Sorted points and spreading sub-problems for grid G with kernel width W.
struct Points3 {
    int4* pti = nullptr;
    float4* ptd = nullptr;
    int4* subs = nullptr;
    int nsub = 0;
    int nb[3] = {0, 0, 0};
};

int build_points(hqs_plan3d_s* p, const float* traj, int64_t M, const int G[3], int W, Points3* out,
                 bool owned, cudaStream_t s) {
    for (int a = 0; a < 3; ++a) out->nb[a] = G[a] / HQS3_TILE;
    const int nbins = out->nb[0] * out->nb[1] * out->nb[2];
    int4* rawi = nullptr;
    float4* rawd = nullptr;
    int* bin = nullptr;
    int* counts = nullptr;
    auto cleanup = [&]() {
        cudaFree(rawi);
        cudaFree(rawd);
        cudaFree(bin);
        cudaFree(counts);
    };
    const int64_t Mp = std::max<int64_t>(M, 1);
    if (cudaMalloc(&rawi, Mp * sizeof(int4)) || cudaMalloc(&rawd, Mp * sizeof(float4)) ||
        cudaMalloc(&bin, Mp * sizeof(int)) || cudaMalloc(&counts, nbins * sizeof(int))) {
        cleanup();
        return HQS_ERR_OOM;
    }
    int rc = HQS_OK;
    do {
        if (owned) {
            if ((rc = alloc3(p, &out->pti, (size_t)Mp)) != HQS_OK) break;
            if ((rc = alloc3(p, &out->ptd, (size_t)Mp)) != HQS_OK) break;
        } else if (cudaMalloc(&out->pti, Mp * sizeof(int4)) || cudaMalloc(&out->ptd, Mp * sizeof(float4))) {
            rc = HQS_ERR_OOM;
            break;
        }
        if (cudaMemsetAsync(counts, 0, nbins * sizeof(int), s)) { rc = HQS_ERR_CUDA; break; }
        if (M > 0)
            k_points3<<<(unsigned)ceil_div64(M, 256), 256, 0, s>>>(traj, (int)M, G[0], G[1], G[2], W, HQS3_TILE,
                                                                  out->nb[0], out->nb[1], rawi, rawd, bin, counts);
        std::vector<int> hc(nbins);
        if (cudaMemcpyAsync(hc.data(), counts, nbins * sizeof(int), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s)) { rc = HQS_ERR_CUDA; break; }
        std::vector<int> offs(nbins);
        std::vector<int4> subs;
        int acc = 0;
        for (int b = 0; b < nbins; ++b) {
            offs[b] = acc;
            for (int st = 0; st < hc[b]; st += HQS3_MAXPTS)
                subs.push_back(make_int4(b, acc + st, std::min(HQS3_MAXPTS, hc[b] - st), 0));
            acc += hc[b];
        }
        out->nsub = (int)subs.size();
        if (owned) {
            if ((rc = alloc3(p, &out->subs, subs.size())) != HQS_OK) break;
        } else if (cudaMalloc(&out->subs, std::max<size_t>(subs.size(), 1) * sizeof(int4))) {
            rc = HQS_ERR_OOM;
            break;
        }
        if (!subs.empty() &&
            cudaMemcpyAsync(out->subs, subs.data(), subs.size() * sizeof(int4), cudaMemcpyHostToDevice, s)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(counts, offs.data(), nbins * sizeof(int), cudaMemcpyHostToDevice, s)) {
            rc = HQS_ERR_CUDA;
            break;
        }
        if (M > 0)
            k_points3_scatter<<<(unsigned)ceil_div64(M, 256), 256, 0, s>>>(rawi, rawd, bin, (int)M, counts,
                                                                          out->pti, out->ptd);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = HQS_ERR_CUDA;
    } while (0);
    cleanup();
    return rc;
}

template <class F> int dispatch_w3(int W, F&& f) {
    switch (W) {
        case 4: return f.template operator()<4>();
        case 5: return f.template operator()<5>();
        case 6: return f.template operator()<6>();
        case 7: return f.template operator()<7>();
        case 8: return f.template operator()<8>();
        default: return HQS_ERR_INVALID_ARG;
    }
}

// Spread y (or unit data) onto `grid` (zeroed here) of size G with L coils.
int spread3(const Points3& pts, const float2* y, int64_t M, const int G[3], int L, int W, double beta,
            bool unit, float2* grid, cudaStream_t s) {
    const size_t cells = (size_t)G[0] * G[1] * G[2] * L;
    HQS_CUDA_TRY(cudaMemsetAsync(grid, 0, cells * sizeof(float2), s));
    if (pts.nsub == 0) return HQS_OK;
    return dispatch_w3(W, [&]<int WW>() {
        const int P = HQS3_TILE + WW - 1;
        const size_t cell_bytes = (size_t)P * P * P * sizeof(float2);
        // coils per chunk: 4, or 2 where a 4-coil patch would exceed 72 KB or the
        // W x 4 (tap, coil) lanes a warp (W > 6), or 1 for one coil
        int lcs = (cell_bytes * 4 <= 72 * 1024 && WW <= 6) ? 2 : 1;
        while (lcs > 0 && (1 << (lcs - 1)) >= L) --lcs;
        const int nch = ceil_div(L, 1 << lcs);
        const size_t sm = HQS3_MAXPTS * sizeof(int4) + HQS3_MAXPTS * 3 * WW * sizeof(float) +
                          (size_t)HQS3_MAXPTS * (1 << lcs) * sizeof(float2) + cell_bytes * (1 << lcs);
        HQS_CUDA_TRY(cudaFuncSetAttribute(k_spread3<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_spread3<WW><<<dim3(pts.nsub, nch), HQS3_SPREAD_WARPS * 32, sm, s>>>(
            y, pts.pti, pts.ptd, pts.subs, M, G[0], G[1], G[2], L, lcs, nch, HQS3_TILE, pts.nb[0], pts.nb[1],
            (float)beta, unit ? 1 : 0, grid);
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    });
}

int vec_blocks(int64_t count) { return (int)std::min<int64_t>(ceil_div64(count, 256), CG3_BLOCKS); }

// -------- operators
int fwd3(hqs_plan3d_s* p, const float2* x, float2* y, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int Gx = p->G[0], Gy = p->G[1], Gz = p->G[2], L = p->L;
    // x pass: [nz][ny][Gx][L] in bufA
    TRY3((run_pass<false, false, false>(
        p, Gx, LdImageX{x, p->smaps, p->apod[0], p->apod[1], p->apod[2], nx, ny, Gx, L, p->scale},
        StLine{p->bufA, {(int64_t)Gx * L, L}, Gx, 0, Gx}, (int64_t)nz * ny * L, L, s)));
    // y pass: [nz][Gy][Gx][L] in bufB
    const int64_t row = (int64_t)Gx * L;
    TRY3((run_pass<false, false, false>(p, Gy, LdCentred{p->bufA, {(int64_t)ny * row, row}, ny, Gy},
                                        StLine{p->bufB, {(int64_t)Gy * row, row}, Gy, 0, Gy},
                                        (int64_t)nz * row, row, s)));
    // z pass: [Gz][Gy][Gx][L] in bufA
    const int64_t plane = (int64_t)Gy * row;
    TRY3((run_pass<false, false, false>(p, Gz, LdCentred{p->bufB, {0, plane}, nz, Gz},
                                        StLine{p->bufA, {0, plane}, Gz, 0, Gz}, plane, plane, s)));
    if (p->M == 0) return HQS_OK;
    return dispatch_w3(p->W, [&]<int WW>() {
        const int64_t threads = p->M * 16;
        k_interp3<WW><<<(unsigned)ceil_div64(threads, 256), 256, 0, s>>>(p->bufA, p->pti, p->ptd, (int)p->M, Gx,
                                                                        Gy, Gz, L, (float)p->beta, y);
        HQS_CUDA_TRY(cudaGetLastError());
        return HQS_OK;
    });
}

int adj3(hqs_plan3d_s* p, const float2* y, float2* x, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int Gx = p->G[0], Gy = p->G[1], Gz = p->G[2], L = p->L;
    Points3 pts;
    pts.pti = p->pti;
    pts.ptd = p->ptd;
    pts.subs = p->subs;
    pts.nsub = p->nsub;
    for (int a = 0; a < 3; ++a) pts.nb[a] = p->nb[a];
    TRY3(spread3(pts, y, p->M, p->G, L, p->W, p->beta, false, p->bufA, s));
    const int64_t row = (int64_t)Gx * L, plane = (int64_t)Gy * row;
    // z: [nz][Gy][Gx][L] in bufB
    TRY3((run_pass<true, false, false>(p, Gz, LdLine{p->bufA, {0, plane}, Gz},
                                       StLine{p->bufB, {0, plane}, nz, 1, Gz}, plane, plane, s)));
    // y: [nz][ny][Gx][L] in bufA
    TRY3((run_pass<true, false, false>(p, Gy, LdLine{p->bufB, {plane, row}, Gy},
                                       StLine{p->bufA, {(int64_t)ny * row, row}, ny, 1, Gy}, (int64_t)nz * row,
                                       row, s)));
    // x: conj(S_l) coil sum and deapodisation fused where the CTA holds whole rows,
    // else per coil into bufC and a separate sum
    if (kLines % L == 0) {
        TRY3((run_pass<true, false, false>(
            p, Gx, LdLine{p->bufA, {row, L}, Gx},
            StCoilSum{x, p->smaps, nullptr, p->apod[0], p->apod[1], p->apod[2], nx, ny, L, 1, Gx, p->scale, 0.f},
            (int64_t)nz * ny * L, L, s)));
        return HQS_OK;
    }
    TRY3((run_pass<true, false, false>(p, Gx, LdLine{p->bufA, {row, L}, Gx},
                                       StCoil{p->bufC, p->smaps, nx, L, 1, Gx}, (int64_t)nz * ny * L, L, s)));
    const int64_t nvox = (int64_t)nx * ny * nz;
    k_coil_sum3<<<vec_blocks(nvox), 256, 0, s>>>(p->bufC, L, nx, ny, nvox, p->apod[0], p->apod[1], p->apod[2],
                                                 p->scale, 0.f, nullptr, x, p->stop);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// out = ca * A^H A x + cb * z (z optional)
int toep3(hqs_plan3d_s* p, const float2* x, float2* out, float ca, float cb, const float2* z, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int Tx = p->G[0], Ty = p->G[1], Tz = p->G[2], L = p->L;
    const int64_t row = (int64_t)Tx * L, plane = (int64_t)Ty * row;
    // x: [nz][ny][Tx][L] in bufA
    TRY3((run_pass<false, true, false>(p, Tx, LdToepX{x, p->smaps, nx, L}, StLine{p->bufA, {row, L}, Tx, 0, Tx},
                                       (int64_t)nz * ny * L, L, s)));
    // y: [nz][Ty][Tx][L] in bufB
    TRY3((run_pass<false, true, false>(p, Ty, LdLine{p->bufA, {(int64_t)ny * row, row}, ny},
                                       StLine{p->bufB, {plane, row}, Ty, 0, Ty}, (int64_t)nz * row, row, s)));
    // z: FFT, Khat, IFFT, rows z < nz, in place in bufB
    TRY3((run_pass<true, true, true>(p, Tz, LdLine{p->bufB, {0, plane}, nz}, StLine{p->bufB, {0, plane}, nz, 0, Tz},
                                     plane, plane, s, MidKhat{p->khat, (int64_t)Ty * Tx, L})));
    // y inverse: [nz][ny][Tx][L] in bufA
    TRY3((run_pass<true, false, true>(p, Ty, LdLine{p->bufB, {plane, row}, Ty},
                                      StLine{p->bufA, {(int64_t)ny * row, row}, ny, 0, Ty}, (int64_t)nz * row, row,
                                      s)));
    // x inverse with the conj(S_l) coil sum fused (whole rows per CTA), else per coil in bufC + sum
    if (kLines % L == 0) {
        TRY3((run_pass<true, false, true>(
            p, Tx, LdLine{p->bufA, {row, L}, Tx},
            StCoilSum{out, p->smaps, z, nullptr, nullptr, nullptr, nx, ny, L, 0, Tx, ca, cb},
            (int64_t)nz * ny * L, L, s)));
        return HQS_OK;
    }
    TRY3((run_pass<true, false, true>(p, Tx, LdLine{p->bufA, {row, L}, Tx}, StCoil{p->bufC, p->smaps, nx, L, 0, Tx},
                                      (int64_t)nz * ny * L, L, s)));
    const int64_t nvox = (int64_t)nx * ny * nz;
    k_coil_sum3<<<vec_blocks(nvox), 256, 0, s>>>(p->bufC, L, nx, ny, nvox, nullptr, nullptr, nullptr, ca, cb, z,
                                                 out, p->stop);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// Chan symbol of the density preconditioner from the 2N circulant column c:
// column on the N grid, FFT_N (x, y, z in place), real part.
int build_lambda(hqs_plan3d_s* p, const float2* c, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int64_t nvox = (int64_t)nx * ny * nz;
    float2* col = p->cg_z;   // scratch volume (free until the first solve)
    k_chan3<<<vec_blocks(nvox), 256, 0, s>>>(c, nx, ny, nz, col);
    HQS_CUDA_TRY(cudaGetLastError());
    const int64_t plane = (int64_t)ny * nx;
    TRY3((run_pass<false, false, false>(p, nx, LdLine{col, {nx, 1}, nx}, StLine{col, {nx, 1}, nx, 0, nx},
                                        (int64_t)nz * ny, 1, s)));
    TRY3((run_pass<false, false, false>(p, ny, LdLine{col, {plane, nx}, ny}, StLine{col, {plane, nx}, ny, 0, ny},
                                        (int64_t)nz * nx, nx, s)));
    TRY3((run_pass<false, false, false>(p, nz, LdLine{col, {0, plane}, nz}, StLine{col, {0, plane}, nz, 0, nz},
                                        plane, plane, s)));
    k_real_part3<<<vec_blocks(nvox), 256, 0, s>>>(col, p->lam, nvox, 1.f);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// z = M^-1 r = IFFT_N(FFT_N(r) s^-1/2) for H = a A^H A + b I: x transform
// into z, then y, z (with the symbol multiply and the inverse z), inverse y,
// inverse x in place.
int precond3(hqs_plan3d_s* p, float a, float b, const float2* r, float2* z, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int64_t plane = (int64_t)ny * nx;
    const int64_t nvox = plane * nz;
    TRY3((run_pass<false, false, false>(p, nx, LdLine{r, {nx, 1}, nx}, StLine{z, {nx, 1}, nx, 0, nx},
                                        (int64_t)nz * ny, 1, s)));
    TRY3((run_pass<false, false, false>(p, ny, LdLine{z, {plane, nx}, ny}, StLine{z, {plane, nx}, ny, 0, ny},
                                        (int64_t)nz * nx, nx, s)));
    TRY3((run_pass<true, false, false>(p, nz, LdLine{z, {0, plane}, nz}, StLine{z, {0, plane}, nz, 0, nz}, plane,
                                       plane, s, MidPrecond{p->lam, plane, a, b, (float)(1.0 / (double)nvox)})));
    TRY3((run_pass<true, false, false>(p, ny, LdLine{z, {plane, nx}, ny}, StLine{z, {plane, nx}, ny, 0, ny},
                                       (int64_t)nz * nx, nx, s)));
    TRY3((run_pass<true, false, false>(p, nx, LdLine{z, {nx, 1}, nx}, StLine{z, {nx, 1}, nx, 0, nx},
                                       (int64_t)nz * ny, 1, s)));
    return HQS_OK;
}

// Khat from the gridded kernel: unit data spread on the 4N grid (width 8),
// inverse transforms cropped to the 2N circulant, deapodised, FFT_2N.
int build_khat(hqs_plan3d_s* p, const float* traj, cudaStream_t s) {
    const int T[3] = {p->G[0], p->G[1], p->G[2]};
    const int G4[3] = {2 * T[0], 2 * T[1], 2 * T[2]};
    const int Wk = HQS3_KERNEL_W;
    const double bk = kb_beta3(Wk, 2.0);
    Points3 pts;
    float2* grid = nullptr;
    float2* mid = nullptr;
    float* ap[3] = {nullptr, nullptr, nullptr};
    auto cleanup = [&]() {
        cudaFree(pts.pti);
        cudaFree(pts.ptd);
        cudaFree(pts.subs);
        cudaFree(grid);
        cudaFree(mid);
        for (int a = 0; a < 3; ++a) cudaFree(ap[a]);
    };
    int rc = HQS_OK;
    do {
        const size_t g4 = (size_t)G4[0] * G4[1] * G4[2];
        const size_t m2 = (size_t)T[2] * G4[1] * G4[0];   // [2nz][4ny][4nx]
        if (cudaMalloc(&grid, g4 * sizeof(float2)) || cudaMalloc(&mid, m2 * sizeof(float2))) {
            rc = HQS_ERR_OOM;
            break;
        }
        for (int a = 0; a < 3; ++a) {
            std::vector<float> h(T[a]);
            const int hn = T[a] / 2;
            for (int q = 0; q < T[a]; ++q) {
                const int d = q < hn ? q : q - T[a];
                h[q] = (float)(1.0 / kb_phihat3((double)d / G4[a], Wk, bk));
            }
            if (cudaMalloc(&ap[a], T[a] * sizeof(float)) ||
                cudaMemcpyAsync(ap[a], h.data(), T[a] * sizeof(float), cudaMemcpyHostToDevice, s) ||
                cudaStreamSynchronize(s)) {
                rc = HQS_ERR_CUDA;
                break;
            }
        }
        if (rc != HQS_OK) break;
        if ((rc = build_points(p, traj, p->M, G4, Wk, &pts, false, s)) != HQS_OK) break;
        if ((rc = spread3(pts, nullptr, p->M, G4, 1, Wk, bk, true, grid, s)) != HQS_OK) break;
        // z: [2nz][4ny][4nx] in mid (circulant crop)
        const int64_t row4 = G4[0], plane4 = (int64_t)G4[1] * G4[0];
        if ((rc = run_pass<true, false, false>(p, G4[2], LdLine{grid, {0, plane4}, G4[2]},
                                               StLine{mid, {0, plane4}, T[2], 2, G4[2]}, plane4, plane4, s)))
            break;
        // y: [2nz][2ny][4nx] in grid
        if ((rc = run_pass<true, false, false>(p, G4[1], LdLine{mid, {plane4, row4}, G4[1]},
                                               StLine{grid, {(int64_t)T[1] * row4, row4}, T[1], 2, G4[1]},
                                               (int64_t)T[2] * row4, row4, s)))
            break;
        // x: [2nz][2ny][2nx] in mid
        if ((rc = run_pass<true, false, false>(p, G4[0], LdLine{grid, {row4, 1}, G4[0]},
                                               StLine{mid, {T[0], 1}, T[0], 2, G4[0]}, (int64_t)T[2] * T[1], 1, s)))
            break;
        const int64_t t3 = (int64_t)T[0] * T[1] * T[2];
        const double nvox = (double)p->n[0] * p->n[1] * p->n[2];
        k_kernel_deapod<<<vec_blocks(t3), 256, 0, s>>>(mid, T[0], T[1], T[2], ap[0], ap[1], ap[2],
                                                        (float)(1.0 / nvox));
        if (p->pc_ok && (rc = build_lambda(p, mid, s)) != HQS_OK) break;
        // forward FFT of the circulant column, in place (x, y, z)
        const int64_t rowT = T[0], planeT = (int64_t)T[1] * T[0];
        if ((rc = run_pass<false, false, false>(p, T[0], LdLine{mid, {rowT, 1}, T[0]}, StLine{mid, {rowT, 1}, T[0], 0, T[0]},
                                                (int64_t)T[2] * T[1], 1, s)))
            break;
        if ((rc = run_pass<false, false, false>(p, T[1], LdLine{mid, {planeT, rowT}, T[1]},
                                                StLine{mid, {planeT, rowT}, T[1], 0, T[1]}, (int64_t)T[2] * rowT,
                                                rowT, s)))
            break;
        if ((rc = run_pass<false, false, false>(p, T[2], LdLine{mid, {0, planeT}, T[2]},
                                                StLine{mid, {0, planeT}, T[2], 0, T[2]}, planeT, planeT, s)))
            break;
        k_real_part3<<<vec_blocks(t3), 256, 0, s>>>(mid, p->khat, t3, (float)(1.0 / (double)t3));
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = HQS_ERR_CUDA;
    } while (0);
    cleanup();
    return rc;
}

int plan3d_build(hqs_plan3d_s* p, const float* traj, const float2* smaps_user, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2], L = p->L;
    const int64_t nvox = (int64_t)nx * ny * nz;
    const int64_t gvox = (int64_t)p->G[0] * p->G[1] * p->G[2];
    TRY3(alloc3(p, &p->smaps, (size_t)(nvox * L)));
    for (int a = 0; a < 3; ++a) TRY3(alloc3(p, &p->apod[a], (size_t)p->n[a]));
    TRY3(alloc3(p, &p->khat, (size_t)gvox));
    TRY3(alloc3(p, &p->bufA, (size_t)(gvox * L)));
    TRY3(alloc3(p, &p->bufB, (size_t)(gvox / 2 * L)));
    TRY3(alloc3(p, &p->bufC, (size_t)(nvox * L)));
    TRY3(alloc3(p, &p->cg_r, (size_t)nvox));
    TRY3(alloc3(p, &p->cg_p, (size_t)nvox));
    TRY3(alloc3(p, &p->cg_q, (size_t)nvox));
    TRY3(alloc3(p, &p->cg_z, (size_t)nvox));
    TRY3(alloc3(p, &p->hqs_b0, (size_t)nvox));
    TRY3(alloc3(p, &p->hqs_rhs, (size_t)nvox));
    TRY3(alloc3(p, &p->hqs_u, (size_t)nvox));
    TRY3(alloc3(p, &p->hqs_w, (size_t)nvox));
    p->pc_ok = fft_size_supported(nx) && fft_size_supported(ny) && fft_size_supported(nz);
    if (p->pc_ok) TRY3(alloc3(p, &p->lam, (size_t)nvox));
    TRY3(alloc3(p, &p->partials, (size_t)2 * CG3_BLOCKS));
    TRY3(alloc3(p, &p->cg, 1));
    TRY3(alloc3(p, &p->hist, HQS_MAX_ITERS + 1));
    HQS_CUDA_TRY(cudaMallocHost(&p->h_cg, sizeof(Cg3)));
    // twiddles for 2n and 4n per axis
    {
        int ns = 0, total = 0;
        for (int a = 0; a < 3; ++a)
            for (int m = 1; m <= 4; m *= 2) {
                const int N = m * p->n[a];
                if (!fft_size_supported(N)) continue;
                bool seen = false;
                for (int k = 0; k < ns; ++k) seen |= p->tw_sizes[k] == N;
                if (!seen) {
                    p->tw_sizes[ns] = N;
                    p->tw_offs[ns] = total;
                    total += N;
                    ++ns;
                }
            }
        std::vector<float2> h(total);
        for (int k = 0; k < ns; ++k)
            for (int m = 0; m < p->tw_sizes[k]; ++m) {
                const double ang = -2.0 * M_PI * (double)m / (double)p->tw_sizes[k];
                h[p->tw_offs[k] + m] = make_float2((float)cos(ang), (float)sin(ang));
            }
        TRY3(alloc3(p, &p->tw, (size_t)total));
        HQS_CUDA_TRY(cudaMemcpyAsync(p->tw, h.data(), total * sizeof(float2), cudaMemcpyHostToDevice, s));
        HQS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    for (int a = 0; a < 3; ++a) {
        std::vector<float> h(p->n[a]);
        for (int i = 0; i < p->n[a]; ++i)
            h[i] = (float)(1.0 / kb_phihat3((double)(i - p->n[a] / 2) / p->G[a], p->W, p->beta));
        HQS_CUDA_TRY(cudaMemcpyAsync(p->apod[a], h.data(), p->n[a] * sizeof(float), cudaMemcpyHostToDevice, s));
        HQS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    k_smaps3_coil_inner<<<(unsigned)std::min<int64_t>(ceil_div64(nvox * L, 256), 8192), 256, 0, s>>>(
        smaps_user, p->smaps, nvox, L);
    HQS_CUDA_TRY(cudaGetLastError());
    Points3 pts;
    TRY3(build_points(p, traj, p->M, p->G, p->W, &pts, true, s));
    p->pti = pts.pti;
    p->ptd = pts.ptd;
    p->subs = pts.subs;
    p->nsub = pts.nsub;
    for (int a = 0; a < 3; ++a) p->nb[a] = pts.nb[a];
    if (p->M > 0) {
        TRY3(build_khat(p, traj, s));
    } else {
        HQS_CUDA_TRY(cudaMemsetAsync(p->khat, 0, gvox * sizeof(float), s));
    }
    HQS_CUDA_TRY(cudaStreamSynchronize(s));
    return HQS_OK;
}

}  // namespace

// ================================================================ C ABI
extern "C" int hqs_plan3d_create(hqs_plan3d* out, const float* traj, int64_t M, int nz, int ny, int nx, int coils,
                                 const hqs_c64* smaps, int kernel_width, float oversamp, void* stream) {
    if (!out) return HQS_ERR_INVALID_ARG;
    *out = nullptr;
    if (M < 0 || M > 0x7fffffffLL || (M > 0 && !traj) || !smaps || coils < 1 || coils > 64) return HQS_ERR_INVALID_ARG;
    if (kernel_width < 4 || kernel_width > 8 || oversamp != 2.0f) return HQS_ERR_INVALID_ARG;
    if (!size3_ok(nx) || !size3_ok(ny) || !size3_ok(nz)) return HQS_ERR_INVALID_ARG;
    auto* p = new (std::nothrow) hqs_plan3d_s;
    if (!p) return HQS_ERR_OOM;
    cudaGetDevice(&p->device);
    p->n[0] = nx;
    p->n[1] = ny;
    p->n[2] = nz;
    for (int a = 0; a < 3; ++a) p->G[a] = 2 * p->n[a];
    p->L = coils;
    p->W = kernel_width;
    p->beta = kb_beta3(kernel_width, 2.0);
    p->M = M;
    p->scale = (float)(1.0 / sqrt((double)nx * ny * nz));
    const int rc = plan3d_build(p, traj, reinterpret_cast<const float2*>(smaps), (cudaStream_t)stream);
    if (rc != HQS_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        plan3d_free(p);
        return rc;
    }
    *out = p;
    return HQS_OK;
}

extern "C" void hqs_plan3d_destroy(hqs_plan3d plan) {
    if (plan) cudaDeviceSynchronize();
    plan3d_free(plan);
}

extern "C" int hqs_plan3d_get_khat(hqs_plan3d p, float* out, void* stream) {
    if (!p || !out) return HQS_ERR_INVALID_ARG;
    const size_t n = (size_t)p->G[0] * p->G[1] * p->G[2];
    HQS_CUDA_TRY(cudaMemcpyAsync(out, p->khat, n * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return HQS_OK;
}

extern "C" int hqs_forward3d(hqs_plan3d p, const hqs_c64* x, hqs_c64* y, void* stream) {
    if (!p || !x || (!y && p->M > 0)) return HQS_ERR_INVALID_ARG;
    return fwd3(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y), (cudaStream_t)stream);
}

extern "C" int hqs_adjoint3d(hqs_plan3d p, const hqs_c64* y, hqs_c64* x, void* stream) {
    if (!p || !x || (!y && p->M > 0)) return HQS_ERR_INVALID_ARG;
    return adj3(p, reinterpret_cast<const float2*>(y), reinterpret_cast<float2*>(x), (cudaStream_t)stream);
}

extern "C" int hqs_toeplitz_normal3d(hqs_plan3d p, const hqs_c64* x, hqs_c64* out, void* stream) {
    if (!p || !x || !out || x == out) return HQS_ERR_INVALID_ARG;
    return toep3(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(out), 1.f, 0.f, nullptr,
                 (cudaStream_t)stream);
}


namespace {

const int* done_flag(const hqs_plan3d_s* p) {
    return reinterpret_cast<const int*>(reinterpret_cast<const char*>(p->cg) + offsetof(Cg3, done));
}

// z = M^-1 r (or r), rz = <r, z>, beta; p = z + beta p
int pcg_precond_step(hqs_plan3d_s* p, float a, float b, bool dc, int nb, int64_t nvox, cudaStream_t s) {
    if (dc) {
        TRY3(precond3(p, a, b, p->cg_r, p->cg_z, s));
        k_dot3<<<nb, 256, 0, s>>>(p->cg_r, p->cg_z, nvox, p->partials, p->stop);
        k_cg3_scalar<<<1, 32, 0, s>>>(p->cg, p->partials, nb, CG3_RZ, p->hist, 0.0, 0);
    } else {
        k_cg3_scalar<<<1, 32, 0, s>>>(p->cg, p->partials, nb, CG3_RZ_RR, p->hist, 0.0, 0);
    }
    k_cg3_pupdate<<<nb, 256, 0, s>>>(p->cg_p, dc ? p->cg_z : p->cg_r, nvox, p->cg);
    HQS_CUDA_TRY(cudaGetLastError());
    return HQS_OK;
}

// one PCG iteration: q = H p, alpha, x and r updates, residual, preconditioner step
int pcg_iteration(hqs_plan3d_s* p, float a, float b, bool dc, float2* x, int nb, int64_t nvox, cudaStream_t s) {
    TRY3(toep3(p, p->cg_p, p->cg_q, a, b, p->cg_p, s));
    k_dot3<<<nb, 256, 0, s>>>(p->cg_p, p->cg_q, nvox, p->partials, p->stop);
    k_cg3_scalar<<<1, 32, 0, s>>>(p->cg, p->partials, nb, CG3_ALPHA, p->hist, 0.0, 0);
    k_cg3_update<<<nb, 256, 0, s>>>(x, p->cg_r, p->cg_p, p->cg_q, nvox, p->cg, p->partials);
    k_cg3_scalar<<<1, 32, 0, s>>>(p->cg, p->partials, nb, CG3_RES, p->hist, 0.0, 0);
    HQS_CUDA_TRY(cudaGetLastError());
    return pcg_precond_step(p, a, b, dc, nb, nvox, s);
}

// The iteration as a CUDA graph on the plan's capture stream, rebuilt when
// (a, b, preconditioner, x) change.  Every kernel of it reads alpha, beta and
// the done flag from the device, and returns at once once the solve is done,
// so replays past convergence cost only their launches.
int ensure_iteration_graph(hqs_plan3d_s* p, float a, float b, bool dc, float2* x, int nb, int64_t nvox) {
    if (p->iter_graph && p->g_a == a && p->g_b == b && p->g_dc == (int)dc && p->g_x == x) return HQS_OK;
    if (p->iter_graph) {
        cudaGraphExecDestroy(p->iter_graph);
        p->iter_graph = nullptr;
    }
    if (!p->cap_stream) HQS_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    HQS_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    const int rc = pcg_iteration(p, a, b, dc, x, nb, nvox, p->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (rc != HQS_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) hqs_note_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        return rc != HQS_OK ? rc : HQS_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&p->iter_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        p->iter_graph = nullptr;
        hqs_note_cuda_error(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        return HQS_ERR_CUDA;
    }
    p->g_a = a;
    p->g_b = b;
    p->g_dc = (int)dc;
    p->g_x = x;
    return HQS_OK;
}

#define HQS3_GRAPH_CHUNK 4   // iterations replayed between host checks of the done flag

}  // namespace

extern "C" int hqs_precond_apply3d(hqs_plan3d p, float a, float b, const hqs_c64* r, hqs_c64* z, void* stream) {
    if (!p || !r || !z || !(b > 0.f)) return HQS_ERR_INVALID_ARG;
    if (!p->pc_ok) return HQS_ERR_UNSUPPORTED;
    return precond3(p, a, b, reinterpret_cast<const float2*>(r), reinterpret_cast<float2*>(z), (cudaStream_t)stream);
}

extern "C" int hqs_dc_solve3d(hqs_plan3d p, float a, float b, const hqs_c64* rhs_c, hqs_c64* x_c, int max_iter,
                              double rel_tol, int precond, hqs_solve_info* info, void* stream) {
    if (!p || !rhs_c || !x_c || max_iter < 0 || max_iter > HQS_MAX_ITERS || !(rel_tol >= 0.0) ||
        reinterpret_cast<const void*>(rhs_c) == reinterpret_cast<const void*>(x_c))
        return HQS_ERR_INVALID_ARG;
    if (precond != HQS_PRECOND_NONE && precond != HQS_PRECOND_DC) return HQS_ERR_INVALID_ARG;
    const bool dc = precond == HQS_PRECOND_DC;
    if (dc && (!p->pc_ok || !(b > 0.f))) return dc && !p->pc_ok ? HQS_ERR_UNSUPPORTED : HQS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float2* rhs = reinterpret_cast<const float2*>(rhs_c);
    float2* x = reinterpret_cast<float2*>(x_c);
    const int64_t nvox = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const int nb = vec_blocks(nvox);
    // r = rhs - H x: launched without the stop flag, which still holds the last solve's state
    p->stop = nullptr;
    TRY3(toep3(p, x, p->cg_q, a, b, x, s));
    k_cg3_init<<<nb, 256, 0, s>>>(rhs, p->cg_q, p->cg_r, nvox, p->partials);
    k_cg3_scalar<<<1, 32, 0, s>>>(p->cg, p->partials, nb, CG3_INIT, p->hist, rel_tol, max_iter);
    HQS_CUDA_TRY(cudaGetLastError());
    p->stop = done_flag(p);
    int rc = pcg_precond_step(p, a, b, dc, nb, nvox, s);
    if (rc == HQS_OK) rc = ensure_iteration_graph(p, a, b, dc, x, nb, nvox);
    p->stop = nullptr;
    if (rc != HQS_OK) return rc;
    for (int it = 0; it < max_iter;) {
        HQS_CUDA_TRY(cudaMemcpyAsync(p->h_cg, p->cg, sizeof(Cg3), cudaMemcpyDeviceToHost, s));
        HQS_CUDA_TRY(cudaStreamSynchronize(s));
        if (p->h_cg->done) break;
        const int chunk = std::min(HQS3_GRAPH_CHUNK, max_iter - it);
        for (int k = 0; k < chunk; ++k) HQS_CUDA_TRY(cudaGraphLaunch(p->iter_graph, s));
        it += chunk;
    }
    HQS_CUDA_TRY(cudaMemcpyAsync(p->h_cg, p->cg, sizeof(Cg3), cudaMemcpyDeviceToHost, s));
    HQS_CUDA_TRY(cudaStreamSynchronize(s));
    const Cg3 c = *p->h_cg;
    if (info) {
        std::vector<double> h(HQS_MAX_ITERS + 1);
        HQS_CUDA_TRY(cudaMemcpy(h.data(), p->hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        info->iterations = c.it;
        info->status = c.status;
        info->fallback = 0;
        info->reserved = 0;
        info->rhs_norm = sqrt(c.bnorm2);
        const double bn = c.bnorm2 > 0.0 ? sqrt(c.bnorm2) : 1.0;
        info->rel_residual = c.bnorm2 > 0.0 ? sqrt(std::max(c.rr, 0.0)) / bn : 0.0;
        for (int i = 0; i <= HQS_MAX_ITERS; ++i)
            info->res_history[i] = i <= c.it ? sqrt(std::max(h[i], 0.0)) / bn : 0.0;
    }
    if (c.bnorm2 == 0.0) HQS_CUDA_TRY(cudaMemsetAsync(x, 0, nvox * sizeof(float2), s));
    return c.status;
}

extern "C" int hqs_plan3d_get_info(hqs_plan3d p, int64_t* npoints, int* nsub, size_t* device_bytes) {
    if (!p) return HQS_ERR_INVALID_ARG;
    if (npoints) *npoints = p->M;
    if (nsub) *nsub = p->nsub;
    if (device_bytes) *device_bytes = p->bytes;
    return HQS_OK;
}

extern "C" int hqs_gaussian_denoise3d(void* user, const hqs_c64* in_c, hqs_c64* out_c, int nz, int ny, int nx,
                                      float sigma, void* stream) {
    if (!in_c || !out_c || nz <= 0 || ny <= 0 || nx <= 0 || !(sigma >= 0.f)) return HQS_ERR_INVALID_ARG;
    float sd = sigma;
    if (user) {
        const hqs_gauss_params* gp = static_cast<const hqs_gauss_params*>(user);
        if (gp->sigma0 > 0.f) sd = gp->kappa * sigma / gp->sigma0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const float2* in = reinterpret_cast<const float2*>(in_c);
    float2* out = reinterpret_cast<float2*>(out_c);
    if (sd < 0.1f) {
        if (in != out) HQS_CUDA_TRY(cudaMemcpyAsync(out, in, nvox * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        return HQS_OK;
    }
    Taps3 t;
    t.r = (int)std::ceil(3.0 * (double)sd);
    if (t.r > HQS3_BLUR_MAXR) return HQS_ERR_INVALID_ARG;
    std::vector<double> g(2 * t.r + 1);
    double sum = 0.0;
    for (int i = -t.r; i <= t.r; ++i) {
        g[i + t.r] = std::exp(-(double)i * i / (2.0 * (double)sd * (double)sd));
        sum += g[i + t.r];
    }
    for (int i = 0; i <= 2 * t.r; ++i) t.g[i] = (float)(g[i] / sum);
    // x, y, z passes through two stream-ordered scratch volumes
    float2* tmp = nullptr;
    HQS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tmp), 2 * nvox * sizeof(float2), st));
    const int nb = vec_blocks(nvox);
    k_blur3<<<nb, 256, 0, st>>>(in, tmp, nx, 1, nvox, t);
    k_blur3<<<nb, 256, 0, st>>>(tmp, tmp + nvox, ny, nx, nvox, t);
    k_blur3<<<nb, 256, 0, st>>>(tmp + nvox, out, nz, (int64_t)ny * nx, nvox, t);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    HQS_CUDA_TRY(e);
    return HQS_OK;
}

extern "C" int hqs_run3d(hqs_plan3d p, const hqs_c64* y, hqs_c64* x_c, const float* mu, const float* sigma, int K,
                         int k0, int cg_iters, float c0, float c1, hqs_denoiser3d_fn denoiser, void* user,
                         void* stream) {
    if (!p || !x_c || (!y && p->M > 0) || !mu || !sigma || K < 0 || k0 < 0 || k0 > K || cg_iters < 0 ||
        cg_iters > HQS_MAX_ITERS || !(c0 > 0.f))
        return HQS_ERR_INVALID_ARG;
    for (int k = k0; k < K; ++k)
        if (!(mu[k] > 0.f) || !(sigma[k] >= 0.f) || !(1.f + c1 * mu[k] > 0.f)) return HQS_ERR_INVALID_ARG;
    if (!denoiser) denoiser = hqs_gaussian_denoise3d;
    cudaStream_t st = (cudaStream_t)stream;
    float2* x = reinterpret_cast<float2*>(x_c);
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int64_t nvox = (int64_t)nx * ny * nz;
    const int nb = vec_blocks(nvox);
    TRY3(adj3(p, reinterpret_cast<const float2*>(y), p->hqs_b0, st));
    const int precond = p->pc_ok ? HQS_PRECOND_DC : HQS_PRECOND_NONE;
    for (int k = k0; k < K; ++k) {
        const float m = mu[k];
        const float a = 1.f + c1 * m, b = c0 * m;
        // rhs = A^H y + mu (c0 x + c1 A^H A x); u starts at x
        const float2* w = nullptr;
        if (c1 != 0.f) {
            TRY3(toep3(p, x, p->hqs_w, 1.f, 0.f, nullptr, st));
            w = p->hqs_w;
        }
        k_axpbypcz3<<<nb, 256, 0, st>>>(p->hqs_rhs, p->hqs_b0, x, m * c0, w, m * c1, nvox);
        HQS_CUDA_TRY(cudaMemcpyAsync(p->hqs_u, x, nvox * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        const int rc = hqs_dc_solve3d(p, a, b, reinterpret_cast<const hqs_c64*>(p->hqs_rhs),
                                      reinterpret_cast<hqs_c64*>(p->hqs_u), cg_iters, 0.0, precond, nullptr, stream);
        if (rc != HQS_OK && rc != HQS_ERR_NOT_CONVERGED) return rc;
        if (denoiser(user, reinterpret_cast<const hqs_c64*>(p->hqs_u), x_c, nz, ny, nx, sigma[k], stream) != 0)
            return HQS_ERR_CALLBACK;
    }
    return HQS_OK;
}
