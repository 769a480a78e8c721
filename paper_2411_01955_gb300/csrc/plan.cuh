// Internal plan layout shared by the translation units of the library.
#pragma once

#include <vector>

#include "common.cuh"

#define HQS_MAX_W 8
#ifndef HQS_KLINES
#define HQS_KLINES 16
#endif
#define HQS_MAX_LC HQS_KLINES  // coils per chunk in the FFT passes
#define HQS_MAX_BLOCKS 2048    // partial-sum slots per reduction (and >= 3 x 256 for the FCG dots)
#define HQS_SPREAD_CAND 256    // candidate points per tile-owned spreading item
#define HQS_TRACE_MAX 4096     // phase-trace stamps kept per persistent solve

// CG scalars kept on the device so that the solve never needs the host
// between iterations.
struct CgScalars {
    double rz;          // <r, z> of the current iterate
    double pq;          // <p, H p>
    double alpha, beta;
    double bnorm;       // ||rhs||
    double rr;          // ||r||^2
    double tol2;        // (rel_tol * ||rhs||)^2
    int it;             // completed iterations
    int done;           // 1 once converged, failed or out of iterations
    int status;         // HQS_OK / HQS_ERR_NOT_CONVERGED / HQS_ERR_BREAKDOWN
    int zero_rhs;       // rhs == 0: solution is exactly 0
    int max_iter;
    int fallback;
};

enum PartialSlot { SLOT_PQ = 0, SLOT_RR = 1, SLOT_BB = 2, SLOT_RZ = 3, SLOT_AUX = 4, NSLOTS = 6 };

struct hqs_plan_s {
    int device = 0;
    int n = 0;          // ny == nx
    int L = 0;          // coils
    int G = 0;          // NUFFT grid
    int n2 = 0;         // Toeplitz grid (2n)
    int W = 0;
    float oversamp = 2.f;
    double beta = 0.0;
    int64_t M = 0;
    float scale = 1.f;  // Npix^-1/2
    int LC = 1, nchunk = 1;
    int tile = 8, nbx = 0;
    int q_rows = 8;     // lines per CTA in the single-image FFT passes
    int fused_grid = 0; // cap on the persistent solver's CTAs (0: occupancy limit)
    bool nufft_only = false; // internal plans that only grid (no Toeplitz kernel, density symbol zero)
    int pc_lines = 4;   // preconditioner lines per item in the persistent solver (1..16)
    int debug_barrier_skip = 0;  // test hook for the next persistent solve (HQS_TUNE_DEBUG_BARRIER_SKIP)

    // constant tables and plan data (device)
    float2* smaps = nullptr;    // [n][n][L]
    float* apod = nullptr;      // [n] 1/phihat((i - n/2)/G)
    int4* pts = nullptr;        // sorted points: (i0x, i0y, bits(dx), bits(dy)), i0 in [0, G)
    int* perm = nullptr;        // sorted -> caller index
    int* invperm = nullptr;     // caller index -> sorted position
    // tile-owned spreading (adjoint): every grid tile of tile x tile cells is
    // written by the CTAs of its items; candidates are the points of the 3 x 3
    // neighbouring bins, taken in chunks of <= HQS_SPREAD_CAND
    struct Spread {
        int4* items = nullptr;         // (tile, first candidate, end candidate, partial slot or -1)
        int2* tile_info = nullptr;     // [nbins] (chunks, first partial slot)
        int2* tile_nb = nullptr;       // [nbins][10]: (first point, candidate prefix) of each distinct
                                       // neighbouring bin in candidate order, entry 9 = (bins, candidates)
        unsigned* tickets = nullptr;   // [nbins] arrival counts of multi-chunk tiles (reset by the last)
        float2* partial = nullptr;     // [slots][tile * tile * L] partial tiles of multi-chunk tiles
        float2* ysort = nullptr;       // [M][L] k-space data in sorted order, coil-innermost
        float* kbw = nullptr;          // [M][2W] Kaiser-Bessel weights of the sorted points (x taps, y taps)
        int nitems = 0, nslots = 0;
        size_t bytes = 0;              // device bytes of the arrays above but ysort
    } spread;
    float* khat = nullptr;      // [n2][n2] transposed (khat[kx][ky]), includes 1/n2^2
    float* lam = nullptr;       // [n][n] density symbol
    float2* tw = nullptr;       // twiddle bank
    int tw_sizes[4] = {0, 0, 0, 0};
    int tw_offs[4] = {0, 0, 0, 0};

    // workspace
    float2* grid = nullptr;     // [G][G][L]
    float2* work = nullptr;     // [n][max(G, n2)][L]
    float2* cg_r = nullptr;     // CG vectors, [n][n] each
    float2* cg_z = nullptr;
    float2* cg_p = nullptr;
    float2* cg_q = nullptr;
    float2* img_tmp = nullptr;  // [n][n] scratch image
    float2* img_tmp2 = nullptr; // [n][n] scratch image
    float2* pc_buf = nullptr;   // [n][n] preconditioner spectrum
    float2* img_b0 = nullptr;   // [n][n] A^H y of the outer loop
    float2* img_rhs = nullptr;  // [n][n] right-hand side of the outer loop
    float2* img_u = nullptr;    // [n][n] prox output of the outer loop
    float2* chunk_buf = nullptr; // [nchunk][n][n] per-coil-chunk partial sums (nchunk > 1)
    double* partials = nullptr; // [NSLOTS][HQS_MAX_BLOCKS]
    CgScalars* cg = nullptr;
    double* hist = nullptr;     // [HQS_MAX_ITERS + 1] ||r_i||^2
    CgScalars* h_cg = nullptr;  // pinned host mirror
    double* h_hist = nullptr;
    unsigned* h_err = nullptr;  // pinned mirror of dev_err
    unsigned* dev_err = nullptr;
    unsigned* barrier = nullptr; // grid barrier words for the persistent solve
    unsigned long long* trace = nullptr;  // optional phase trace of the persistent solve
    struct hqs_net_s* net = nullptr;      // learned preconditioner (not owned)
    struct hqs_mixed_s* mixed = nullptr;  // tensor-core Toeplitz workspace (built on first use)

    size_t bytes = 0;
    std::vector<void*> allocs;
};

const float2* plan_twiddles(const hqs_plan_s* p, int N);
// hqs_plan_create; with nufft_only the plan serves hqs_forward / hqs_adjoint only:
// its Toeplitz kernel and density symbol are left zero (for internal helpers such as
// the S-map estimation, which grids one coil at a time)
int plan_create_internal(hqs_plan* out, const float* traj, int64_t M, int ny, int nx, int coils,
                         const hqs_c64* smaps, int kernel_width, float oversamp, void* stream, bool nufft_only);
void mixed_free(hqs_plan_s* p);

// launchers implemented in the kernel translation units
int launch_fwd(hqs_plan_s* p, const float2* x, float2* y, cudaStream_t s);
int launch_adj(hqs_plan_s* p, const float2* y, float2* x, cudaStream_t s);
int launch_adj_axpy(hqs_plan_s* p, const float2* y, float zc, const float2* z, float2* x, cudaStream_t s);
// batched operators (csrc/nufft.cu): per-plan pieces and the lower-half passes of
// a group of plans (G = 2n, 16-coil chunks) in one launch per pass
bool plan_half_passes(const hqs_plan_s* p);
size_t half_args_bytes();
void fill_half_args(const hqs_plan_s* p, const float2* x, float2* xo, const float2* z, void* dst);
int launch_half_group(int G, int n, int maxchunk, int count, const void* d_tab, int adjoint, float zc,
                      cudaStream_t s);
int launch_spread(hqs_plan_s* p, const float2* y, cudaStream_t s);
int launch_interp(hqs_plan_s* p, float2* y, cudaStream_t s);
int launch_adj_chunks(hqs_plan_s* p, float2* x, float zc, const float2* z, cudaStream_t s);
int launch_toeplitz(hqs_plan_s* p, const float2* x, float2* out, cudaStream_t s);
int launch_fft2d(const hqs_plan_s* p, float2* data, int N, bool inverse, cudaStream_t s);
int launch_precond(hqs_plan_s* p, float a, float b, const float2* r, float2* z, cudaStream_t s);
// (re)builds the tile-owned spreading items for p->tile from the per-bin point
// counts (host) and the sorted points; blocking
int spread_build(hqs_plan_s* p, const std::vector<int>& counts, cudaStream_t s);
int launch_point_weights(hqs_plan_s* p, cudaStream_t s);   // spread.kbw from the sorted points
void spread_free(hqs_plan_s* p);
