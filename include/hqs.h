/*
 * hqs.h - C ABI of the GB300 (sm_103a) multicoil non-Cartesian MRI hot path
 * of annealed plug-and-play HQS reconstruction (Comby, Lapostolle, Terris,
 * Ciuciu, "Robust Plug-and-Play Methods for Highly Accelerated Non-Cartesian
 * MRI Reconstruction", arXiv 2411.01955).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex arrays are interleaved float32 pairs (re, im) = hqs_c64.
 * - Images are (ny, nx) row-major; pixel (iy, ix) has the centred coordinate
 *   n = (ix - nx/2, iy - ny/2).  Only square images (ny == nx) are accepted
 *   (the volumetric entry points below take (nz, ny, nx) volumes).
 * - Coil maps at the boundary are (L, ny, nx); k-space data are (L, M) in the
 *   caller's point order; trajectories are (M, 2) float32 (kx, ky) in radians
 *   per pixel (any real value; the grid is periodic in 2*pi).
 * - Unless stated otherwise every array argument is a DEVICE pointer owned by
 *   the caller, valid for the duration of the work the call enqueues.  The
 *   plan copies what it keeps.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  Calls enqueue work asynchronously on it unless documented as
 *   blocking.
 * - Every call returns an int status: HQS_OK (0) or a negative HQS_ERR_*
 *   code.  No C++ exception and no abort crosses this boundary.  A plan must
 *   not be used from two host threads at once (it owns its workspace).
 */
#ifndef HQS_GB300_H
#define HQS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HQS_API __attribute__((visibility("default")))
#else
#define HQS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HQS_OK                  0
#define HQS_ERR_INVALID_ARG    (-1)  /* bad size, NULL pointer, unsupported shape */
#define HQS_ERR_OOM            (-2)  /* device allocation failed */
#define HQS_ERR_NOT_CONVERGED  (-3)  /* max_iter reached above rel_tol */
#define HQS_ERR_BREAKDOWN      (-4)  /* CG curvature <= 0 or non-finite value */
#define HQS_ERR_TIMEOUT        (-5)  /* a device-side wait exceeded its limit */
#define HQS_ERR_CALLBACK       (-6)  /* the denoiser callback returned non-zero */
#define HQS_ERR_CUDA           (-7)  /* a CUDA runtime call failed */
#define HQS_ERR_UNSUPPORTED    (-8)  /* valid request this build does not implement */

/* operator precision for hqs_toeplitz_normal / dc_solve */
#define HQS_PREC_FP32    0
#define HQS_PREC_BF16X3  1   /* DFT-GEMM FFT, bf16 hi/lo split operands, fp32 accumulate */
#define HQS_PREC_FP16X3  2   /* same with fp16 hi/lo split operands */

/* preconditioners for hqs_dc_solve */
#define HQS_PRECOND_NONE     0
#define HQS_PRECOND_DC       1   /* circulant density-compensation preconditioner */
#define HQS_PRECOND_LEARNED  2   /* conv-net preconditioner in flexible CG */

/* execution modes for hqs_dc_solve */
#define HQS_SOLVE_PLAIN      0   /* one launch per stage, host checks the residual each iteration */
#define HQS_SOLVE_FUSED      1   /* one persistent cooperative launch for the whole solve */
#define HQS_SOLVE_X0_ZERO    16  /* flag (OR with the mode): start from x = 0, ignoring x on entry;
                                    saves the initial A^H A apply */

#define HQS_MAX_ITERS 512

typedef struct hqs_plan_s* hqs_plan;
typedef struct hqs_net_s* hqs_net;
typedef struct hqs_batch_s* hqs_batch;
typedef struct hqs_plan3d_s* hqs_plan3d;
typedef struct { float re, im; } hqs_c64;

typedef struct {
    int     ny, nx, coils, kernel_width;
    float   oversamp;
    int     grid;             /* NUFFT grid size G = oversamp * n */
    int64_t npoints;          /* M */
    double  kb_beta;          /* Kaiser-Bessel shape parameter */
    size_t  device_bytes;     /* device memory held by the plan */
    int     nsub;             /* spreading work items (tile-owned spreading) */
    int     tile;             /* spreading tile edge on the grid */
} hqs_plan_info;

typedef struct {
    int    iterations;        /* H applications inside the loop */
    int    status;            /* HQS_OK, HQS_ERR_NOT_CONVERGED or HQS_ERR_BREAKDOWN */
    int    fallback;          /* 1 if the learned preconditioner fell back to DC-PCG */
    int    reserved;
    double rhs_norm;          /* ||rhs|| (fp64) */
    double rel_residual;      /* final ||r|| / ||rhs|| of the CG recursion */
    double res_history[HQS_MAX_ITERS + 1];  /* ||r_i|| / ||rhs||, i = 0..iterations */
} hqs_solve_info;

/* Denoiser callback for hqs_run: D_sigma of the PnP-HQS update (Sec. 3.3).
 * `in` and `out` are device (ny, nx) images borrowed for the call; the
 * callback must only enqueue work on `stream` (or finish it) and return 0,
 * any other value aborts hqs_run with HQS_ERR_CALLBACK. */
typedef int (*hqs_denoiser_fn)(void* user, const hqs_c64* in, hqs_c64* out,
                               int ny, int nx, float sigma, void* stream);

/* Parameters of the built-in Gaussian-smoothing denoiser: blur std
 * s = kappa * sigma / sigma0 pixels (sigma0 <= 0 means s = sigma). */
typedef struct { float kappa; float sigma0; } hqs_gauss_params;

/* ------------------------------------------------------------ plan (a1) */
/* Builds the operator A = sampling o NUFFT o coil sensitivities of Eq. (1)
 * (Sec. 2.1) for one trajectory: sorts the M points into grid tiles and
 * spreading sub-problems, tabulates the Kaiser-Bessel deapodisation, copies
 * the coil maps into the plan (coil-innermost), computes the Toeplitz kernel
 * t(d) = Npix^-1 sum_j exp(i k_j.d) of A^H A on the 2N grid with its FFT, and
 * the density symbol of the circulant CG preconditioner.
 *   traj         (M, 2) float32 device, radians per pixel
 *   smaps        (coils, ny, nx) complex device; Sum_l |S_l|^2 need not be 1
 *   kernel_width W in [2, 8]; oversamp * ny must be a supported FFT size
 *   (supported n: 16, 32, 64, 128, 256, 320, 384 with oversamp 2; any
 *   oversamp giving G in {32, 64, 128, 256, 320, 384, 512, 640, 768}).
 * BLOCKING: returns after the plan is ready.  On error *out is NULL. */
HQS_API int hqs_plan_create(hqs_plan* out, const float* traj, int64_t M, int ny, int nx,
                    int coils, const hqs_c64* smaps, int kernel_width,
                    float oversamp, void* stream);
HQS_API void hqs_plan_destroy(hqs_plan plan);
HQS_API int hqs_plan_get_info(hqs_plan plan, hqs_plan_info* info);   /* host struct */

/* --------------------------------------------------------- forward (a2) */
/* y = A x, Eq. (1): y_l[j] = Npix^-1/2 sum_n S_l[n] x[n] exp(-i k_j.n),
 * by gridding (apodised, zero-padded FFT on the oversampled grid, KB
 * interpolation).  x: (ny, nx); y: (L, M). */
HQS_API int hqs_forward(hqs_plan plan, const hqs_c64* x, hqs_c64* y, void* stream);

/* --------------------------------------------------------- adjoint (a3) */
/* x = A^H y (Sec. 3.4 uses A^H), the exact transpose of hqs_forward:
 * KB spreading (each grid tile accumulated in shared memory by the CTAs
 * that own it and written once: no atomics, a fixed summation order, so the
 * result is bitwise repeatable), inverse FFT, deapodisation, coil
 * combination with conj(S_l).  y: (L, M); x: (ny, nx). */
HQS_API int hqs_adjoint(hqs_plan plan, const hqs_c64* y, hqs_c64* x, void* stream);

/* x = A^H y + c z: the data-consistency right-hand side of the HQS step
 * (Sec. 3.3/3.4, rhs = A^H y + mu_k z_k for P = Id), with the axpy fused into
 * the adjoint's last pass.  z: (ny, nx) device; z may be the same buffer as
 * x (each pixel is read before it is written). */
HQS_API int hqs_adjoint_axpy(hqs_plan plan, const hqs_c64* y, float c, const hqs_c64* z,
                             hqs_c64* x, void* stream);

/* S-map estimation (Sec. 4.1): c_l = A_1^H (w d y_l), the single-coil adjoint
 * NUFFT of coil l's samples under the separable Hamming window
 * w = h(u_x) h(u_y), h(u) = 0.54 + 0.46 cos(2 pi u / width) for |u| <= width/2
 * (u = k n / 2 pi, Cartesian grid units; width 20 in the paper), times the
 * optional per-sample density weights d (dcf, device M floats, or NULL);
 * then S_l = c_l / sqrt(sum_l |c_l|^2) where that root-sum-of-squares is at
 * least thresh times its maximum, S_l = 0 elsewhere.  traj: device M x 2
 * (radians), y: device (coils, M), smaps: device (coils, n, n) out.  Builds
 * and frees a one-coil plan and scratch: BLOCKING on `stream`. */
HQS_API int hqs_estimate_smaps(const float* traj, int64_t M, const hqs_c64* y, const float* dcf, int n,
                               int coils, int kernel_width, float oversamp, float width, float thresh,
                               hqs_c64* smaps, void* stream);

/* ------------------------------------------------- Toeplitz normal (a4) */
/* out = A^H A x (Sec. 3.4, A = F_Omega (x) S_l) through the exact 2N
 * circulant embedding of F^H F; never touches the trajectory.
 * precision: HQS_PREC_FP32 (in-house FFTs) or HQS_PREC_BF16X3 / _FP16X3
 * (the four pruned 2N-point DFT passes as tcgen05 GEMMs on split hi/lo
 * 16-bit operands, fp32 accumulation; needs n % 64 == 0, n <= 512, coils
 * <= 32, else HQS_ERR_UNSUPPORTED).  The first mixed-precision call of a plan
 * allocates its workspace and synchronises `stream`. */
HQS_API int hqs_toeplitz_normal(hqs_plan plan, const hqs_c64* x, hqs_c64* out,
                        int precision, void* stream);

/* ------------------------------------------- preconditioner apply (a5) */
/* z = M^-1 r for H = a A^H A + b I: z = IFFT_N(FFT_N(r) * s^-1/2),
 * s = max(a*max(lam,0) + b, b/4), lam the gridded sampling density
 * (eigenvalues of T. Chan's circulant approximation of F^H F). b > 0. */
HQS_API int hqs_precond_apply(hqs_plan plan, float a, float b, const hqs_c64* r,
                      hqs_c64* z, void* stream);

/* Allocation-free preconditioner apply.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, such
 * as a reconstruction service that reserves all GPU memory at start-up and
 * forbids allocation on its serving path, or a host framework whose memory
 * pool owns the device.  It needs no plan (a plan allocates tens of MB of
 * workspace) and calls no cudaMalloc/cudaFree or allocating routine: its
 * scratch (the n x n spectrum, 1.125 MiB at the maximum) and twiddle tables
 * are file-scope device arrays that every GPU loading this library holds
 * until the process exits.
 *   z = IFFT_N(FFT_N(r) * s^-1/2), s = max(a*max(lam,0) + b, b/4), as
 *   hqs_precond_apply, with the density symbol lam given by the caller.
 *   r, z: (n, n) complex device; lam: (n, n) float device; b > 0;
 *   n in {16, 32, 64, 128, 256, 320, 384}: larger n returns HQS_ERR_INVALID_ARG.
 * The first call on a device sets up: it looks up the arrays' device
 * addresses, loads the kernels of every supported n (so that no later call,
 * for any n, loads code), fills the twiddle tables and synchronises `stream`
 * once.  Make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) makes a new context; the next call detects it by the
 * context's id and sets up again, so that call too must come before any
 * capture.  All calls on a device share the scratch
 * array and it keeps the last call's contents: calls that overlap on the GPU
 * (for instance on two streams) race on it.  Nothing in it needs to start at
 * zero: the row pass overwrites the whole n x n region before it is read. */
HQS_API int hqs_precond_apply_noalloc(const hqs_c64* r, const float* lam, int n, float a, float b,
                                      hqs_c64* z, void* stream);

/* --------------------------------------------------- DC solve (a5, a7) */
/* Solves (a A^H A + b I) x = rhs by preconditioned CG with fp64 inner
 * products: the P-metric proximal step of Sec. 3.4 ("subiteration solver").
 * For the HQS data-consistency step with P = Id: a = 1, b = mu_k,
 * rhs = A^H y + mu_k z_k.  x holds the initial guess on entry and the
 * solution on exit.  Stops when ||r|| <= rel_tol ||rhs|| or after max_iter
 * (<= HQS_MAX_ITERS) iterations; rel_tol = 0 runs exactly max_iter.
 * b must be > 0.  precond: HQS_PRECOND_*; mode: HQS_SOLVE_*; precision:
 * HQS_PREC_* (the mixed precisions run with HQS_SOLVE_PLAIN and the DC or no
 * preconditioner; inner products and norms stay fp64).  If info != NULL the call synchronises `stream` and fills it,
 * returning HQS_ERR_NOT_CONVERGED / HQS_ERR_BREAKDOWN when applicable; with
 * info == NULL it only enqueues (capturable in a CUDA graph when mode is
 * HQS_SOLVE_FUSED) and the outcome is read later with hqs_last_solve_info. */
HQS_API int hqs_dc_solve(hqs_plan plan, float a, float b, const hqs_c64* rhs, hqs_c64* x,
                 int max_iter, double rel_tol, int precond, int mode, int precision,
                 hqs_solve_info* info, void* stream);
/* Synchronises `stream` and reports the last solve enqueued on this plan. */
HQS_API int hqs_last_solve_info(hqs_plan plan, hqs_solve_info* info, void* stream);

/* ------------------------------------- learned preconditioner (a10) */
/* A 4-layer 3x3 convolutional network (2 -> 32 -> 32 -> 32 -> 2 channels,
 * ReLU, 19,682 float parameters; no counterpart in the paper, whose networks
 * are its denoisers) used as a nonlinear CG preconditioner:
 *   z = zdc + s * net(zdc / s),  zdc = M_DC^-1 r (hqs_precond_apply),
 *   s = root-mean-square of zdc, channels = (Re, Im).
 * With a zero last layer it equals the DC preconditioner.  Activations are
 * planar float [N][C][H][W] device arrays; the parameter vector is
 * [W1 b1 W2 b2 W3 b3 W4 b4], W[out][in][3][3] (cross-correlation, one pixel
 * of zero padding).  Training minimises the mean over samples of
 * ||net(x_n) - t_n||^2 / ||t_n||^2 with Adam (0.9, 0.999, 1e-8). */
HQS_API int hqs_net_create(hqs_net* out);                  /* parameters zero */
HQS_API void hqs_net_destroy(hqs_net net);
HQS_API int hqs_net_num_params(void);
/* Arithmetic of the two 32 -> 32 layers (their forward and input-gradient
 * convolutions; the other layers and every weight gradient stay FP32):
 * HQS_PREC_BF16X3 (the default) runs them as implicit GEMMs on the tcgen05
 * tensor cores with BF16 hi/lo split operands (hi*hi + lo*hi + hi*lo, FP32
 * accumulation; each product within 3 * 2^-16 of its exact value, relative),
 * HQS_PREC_FP32 on the FP32 cores.  HQS_PREC_FP16X3: HQS_ERR_UNSUPPORTED. */
HQS_API int hqs_net_set_precision(hqs_net net, int precision);
/* Blocks on `stream`; HQS_ERR_TIMEOUT when a tensor-core convolution of this
 * network gave up waiting for its MMAs (a bounded wait; the output of that
 * launch is incomplete) since the last check, which clears the flag.  The loss
 * of hqs_net_gradient / hqs_net_train_step and the learned solve check it too. */
HQS_API int hqs_net_status(hqs_net net, void* stream);
HQS_API int hqs_net_set_params(hqs_net net, const float* host, int count);  /* resets Adam */
HQS_API int hqs_net_get_params(hqs_net net, float* host, int count);
HQS_API int hqs_net_forward(hqs_net net, const float* x, float* y, int N, int H, int W, void* stream);
/* loss (host, blocking) and gradient (device, num_params floats; may be NULL) */
HQS_API int hqs_net_gradient(hqs_net net, const float* x, const float* target, int N, int H, int W,
                             float* grad, double* loss, void* stream);
/* one Adam step on a batch; loss before the step (host, blocking) */
HQS_API int hqs_net_train_step(hqs_net net, const float* x, const float* target, int N, int H, int W,
                               float lr, double* loss, void* stream);
/* Gradient for a loss given through its gradient dy = dL/dy with respect to
 * the network output (N x 2 x H x W, device): the preconditioner is trained on
 * the residual r - H z it leaves, whose gradient needs the operator H (A^H A
 * applies done by the caller).  hqs_net_backward writes the parameter
 * gradient to grad (device, optional); hqs_net_train_step_dy also takes one
 * Adam step (same rule as hqs_net_train_step). */
HQS_API int hqs_net_backward(hqs_net net, const float* x, const float* dy, int N, int H, int W,
                             float* grad, void* stream);
HQS_API int hqs_net_train_step_dy(hqs_net net, const float* x, const float* dy, int N, int H, int W,
                                  float lr, void* stream);
/* Conv-net denoiser with the hqs_denoiser_fn signature (user = the hqs_net):
 * out = in - sigma net(in / sigma), the network predicting the noise of an
 * image whose noise standard deviation (per real / imaginary part) is
 * normalised to 1; sigma = 0 copies.  A sigma-conditioned stand-in for the
 * paper's trained prior (Sec. 4.2) that hqs_run can call directly. */
HQS_API int hqs_net_denoise(void* user, const hqs_c64* in, hqs_c64* out, int ny, int nx, float sigma,
                            void* stream);
HQS_API int hqs_net_save(hqs_net net, const char* path);
HQS_API int hqs_net_load(hqs_net net, const char* path);
/* attach (or detach with NULL) the network used by HQS_PRECOND_LEARNED; the
 * plan does not own it.  The solve is Notay's flexible CG (alpha =
 * <p,r>/<p,Hp>, Polak-Ribiere beta); when Re<z, r> <= 0 or ||r|| fails to
 * drop 10% over 5 iterations it restarts as DC-preconditioned CG from the
 * current iterate (info->fallback = 1). */
HQS_API int hqs_plan_set_net(hqs_plan plan, hqs_net net);
/* z = learned preconditioner applied to r (n x n complex device arrays). */
HQS_API int hqs_learned_precond_apply(hqs_plan plan, float a, float b, const hqs_c64* r, hqs_c64* z,
                                      void* stream);

/* ------------------------------------------------ HQS outer loop (a6) */
/* Annealed PnP-HQS (Sec. 3.3): for k = k0..K-1
 *   u_k = prox^P_{gamma_k f}(x_k), P = c0 I + c1 A^H A (Sec. 3.4),
 *         i.e. ((1 + c1 mu_k) A^H A + c0 mu_k I) u = A^H y + mu_k (c0 x_k + c1 A^H A x_k),
 *         cg_iters DC-preconditioned CG iterations warm-started at x_k;
 *   x_{k+1} = D_{sigma_k}(u_k).
 * mu, sigma: HOST arrays of K floats (mu_k = 1/gamma_k).  y: (L, M) device;
 * x: (ny, nx) device, x_{k0} on entry, x_K on exit.  denoiser NULL selects
 * the built-in Gaussian smoothing with `user` pointing to hqs_gauss_params
 * (NULL: kappa 1.5, sigma0 = sigma[0]).  Resuming from k0 with x_{k0} gives
 * the same x_K as an uninterrupted run: the Toeplitz/CG iterations have no
 * atomics and fixed-order reductions; only A^H y (float atomics in the
 * spreading) may differ in the last bits between calls.
 * The loop enqueues on `stream` and
 * calls the callback from the calling thread between outer iterations; each
 * DC step synchronises `stream` once per CG iteration (plain mode). */
HQS_API int hqs_run(hqs_plan plan, const hqs_c64* y, hqs_c64* x, const float* mu,
            const float* sigma, int K, int k0, int cg_iters, float c0, float c1,
            hqs_denoiser_fn denoiser, void* user, void* stream);

/* --------------------------------------- batched persistent HQS (a9) */
/* PnP-PGD (Sec. 3.3) with the gradient step in the metric P = c0 I + c1 A^H A
 * of Sec. 3.4: for k = 0..K-1,
 *     g = A^H A x - A^H y,  u = x - gamma[k] (c0 g + c1 A^H A g),  x = D_{sigma[k]}(u);
 * x (device, n x n) is x_0 in, x_K out; gamma[k] > 0 and sigma[k] >= 0 are host
 * arrays; denoiser / user as in hqs_run (NULL: the built-in Gaussian smoothing).
 * One A^H A per step for P = Id, two otherwise; enqueued on `stream`. */
HQS_API int hqs_pgd_run(hqs_plan plan, const hqs_c64* y, hqs_c64* x, const float* gamma,
                        const float* sigma, int K, float c0, float c1, hqs_denoiser_fn denoiser,
                        void* user, void* stream);

/* Annealed PnP-HQS (Sec. 3.3, P = Id) for many slices of uneven size at once:
 * one persistent cooperative launch runs, for every slice and k = k0..K-1,
 * rhs = A^H y + mu_k c0 x_k, cg_iters DC-preconditioned CG iterations on
 * (A^H A + c0 mu_k I) u = rhs from u = x_k, then x_{k+1} = Gaussian
 * smoothing of u (std kappa sigma_k / sigma0 px; the built-in denoiser).
 * Work items of all slices share every phase.  Plans: n in {64, 128, 256,
 * 320, 384}, any coil count, <= 64 slices; each plan may belong to one batch
 * at a time (its workspace is used).  hqs_batch_create allocates;
 * hqs_batch_run enqueues on `stream` the per-slice adjoints and the
 * persistent kernel, recorded once into a CUDA graph and replayed when
 * use_graph != 0 (re-recorded when y/x pointers, K, k0, cg_iters, c0 or c1
 * change; mu, sigma may change freely); it synchronises `stream` first.
 * y[i]: (L_i, M_i) device; x[i]: (n_i, n_i) device, x_{k0} in, x_K out.
 * c0, c1: the metric P = c0 I + c1 A^H A of Sec. 3.4, shared by every slice
 * (as in hqs_run: each step solves ((1 + c1 mu_k) A^H A + c0 mu_k I) u =
 * A^H y + mu_k (c0 x_k + c1 A^H A x_k)); for the F-1 and Chebyshev metrics
 * take alpha from the slice with the largest ||A^H A|| (hqs_power_iteration),
 * which keeps P positive definite for every slice.  hqs_batch_status
 * synchronises and reports, per slice, the relative CG residual of the last
 * data-consistency step. */
HQS_API int hqs_batch_create(hqs_batch* out, hqs_plan* plans, int n, int max_outer);
/* Caps the CTAs of the batch's cooperative launches (0, the default: every CTA
 * the kernel keeps resident, two per SM).  With a cap of one CTA per SM, two
 * batches launched on two streams can run side by side, each CTA's grid
 * barriers independent of the other batch's.  Results are unchanged up to the
 * order of the per-CTA fp64 partial sums.  No counterpart in the paper: a
 * launch-shape setting.  ctas < 0 or a NULL batch: HQS_ERR_INVALID_ARG. */
HQS_API int hqs_batch_set_grid(hqs_batch batch, int ctas);
HQS_API void hqs_batch_destroy(hqs_batch batch);
HQS_API int hqs_batch_run(hqs_batch batch, const hqs_c64* const* y, hqs_c64* const* x,
                          const float* mu, const float* sigma, int K, int k0, int cg_iters,
                          float c0, float c1, const hqs_gauss_params* gauss, int use_graph,
                          void* stream);
HQS_API int hqs_batch_status(hqs_batch batch, double* rel_residual, void* stream);
/* Batched data-consistency solve (Sec. 3.4's system, P = Id form): for every
 * slice i of the batch, DC-preconditioned CG on (a A^H A + b I) x[i] = rhs[i]
 * from x[i] = 0 until ||r|| <= rel_tol ||rhs[i]|| or max_iter iterations, all
 * slices in one cooperative launch (a slice that converges drops out).
 * rhs[i], x[i]: device (n_i x n_i) of the i-th plan; b > 0.  Enqueued on
 * `stream`; synchronises it first when the pointers differ from the last
 * call.  hqs_batch_dc_info (blocking) returns per slice the iterations, the
 * relative residual of the CG recursion and the status (HQS_OK,
 * HQS_ERR_NOT_CONVERGED, HQS_ERR_BREAKDOWN); NULL outputs are skipped. */
HQS_API int hqs_batch_dc_solve(hqs_batch batch, const hqs_c64* const* rhs, hqs_c64* const* x, float a, float b,
                               int max_iter, double rel_tol, void* stream);
HQS_API int hqs_batch_dc_info(hqs_batch batch, int* iterations, double* rel_residual, int* status,
                              void* stream);
/* Batched normal operator (Sec. 3.4's A^H A, A = F_Omega (x) S_l): out[i] =
 * A_i^H A_i x[i] for every slice i of the batch in one cooperative launch, by
 * the same exact 2N Toeplitz passes as hqs_toeplitz_normal (FP32), each pass
 * dealing the work items of all slices to all CTAs.  x[i], out[i]: device
 * (n_i x n_i) complex64 of the i-th plan, caller-owned; out[i] may equal x[i].
 * Enqueued on `stream`; synchronises it first when the pointers differ from the
 * last call.  Uses the plans' workspaces: calls on one batch (and on its plans)
 * run in stream order.  A grid barrier that runs out of time is reported by the
 * next hqs_batch_status / hqs_batch_dc_info (HQS_ERR_TIMEOUT).  A NULL batch,
 * array or pointer: HQS_ERR_INVALID_ARG, nothing enqueued. */
HQS_API int hqs_batch_toeplitz_normal(hqs_batch batch, const hqs_c64* const* x, hqs_c64* const* out,
                                      void* stream);
/* Batched NUFFT operators (Eq. (1) and its adjoint, the same gridding as
 * hqs_forward / hqs_adjoint_axpy): y[i] = A_i x[i], and x[i] = A_i^H y[i] +
 * zc z[i] (z NULL, or z[i] NULL: no axpy term), for every slice i.  The
 * slices whose grid is 2n with 16-coil chunks run their row and column FFT
 * passes together, one launch per pass and grid size; spreading,
 * interpolation and the other slices' passes run per slice.  y[i]: (L_i, M_i),
 * x[i], z[i]: (n_i, n_i), device complex64, caller-owned.  Enqueued on
 * `stream`; synchronises it first when the image pointers differ from the last
 * call.  Uses the plans' workspaces: calls on one batch (and on its plans) run
 * in stream order.  A NULL batch, array or image pointer (or a NULL y[i] of a
 * plan with points): HQS_ERR_INVALID_ARG, nothing enqueued. */
HQS_API int hqs_batch_forward(hqs_batch batch, const hqs_c64* const* x, hqs_c64* const* y, void* stream);
HQS_API int hqs_batch_adjoint_axpy(hqs_batch batch, const hqs_c64* const* y, float zc, const hqs_c64* const* z,
                                   hqs_c64* const* x, void* stream);

/* Built-in denoiser (stand-in for the trained prior of Sec. 4.2): separable
 * Gaussian blur of real and imaginary parts, std s pixels (see
 * hqs_gauss_params), radius ceil(3 s), taps normalised to sum 1, periodic
 * boundary; copies in to out when s < 0.1.  Matches hqs_denoiser_fn. */
HQS_API int hqs_gaussian_denoise(void* user, const hqs_c64* in, hqs_c64* out,
                         int ny, int nx, float sigma, void* stream);

/* --------------------------------------------------- power iteration */
/* Largest eigenvalue of A^H A by `iters` power iterations from a fixed seed
 * (alpha = 1/||A^H A|| for the F-1 and Chebyshev metrics of Sec. 3.4).
 * BLOCKING; result in *lam_max (host). */
HQS_API int hqs_power_iteration(hqs_plan plan, int iters, double* lam_max, void* stream);

HQS_API const char* hqs_status_string(int status);


/* Tuning knobs (no counterpart in the paper), set per plan by the autotuner:
 *   HQS_TUNE_FUSED_GRID  cap on the persistent solve's CTAs (0 = all resident)
 *   HQS_TUNE_PC_LINES    preconditioner rows/columns per work item (1..16)
 *   HQS_TUNE_SPREAD_TILE spreading tile edge (8, 16 or 32): re-bins the
 *                        plan's points (hqs_plan_retile on the default stream)
 * and one test hook for the failure path of the persistent solve:
 *   HQS_TUNE_DEBUG_BARRIER_SKIP  1 arms it for the next HQS_SOLVE_FUSED solve
 *                        only: that solve's last CTA leaves before the first
 *                        grid barrier and the barrier waits are cut to about
 *                        10 ms, so the others' waits run out and the solve
 *                        returns HQS_ERR_TIMEOUT (no result); the barrier
 *                        words are reset at every launch, so the next solve
 *                        on the plan runs normally. */
#define HQS_TUNE_FUSED_GRID   1
#define HQS_TUNE_PC_LINES     2
#define HQS_TUNE_SPREAD_TILE  3
#define HQS_TUNE_DEBUG_BARRIER_SKIP 4
HQS_API int hqs_plan_set_tuning(hqs_plan plan, int key, int value);
/* Re-sorts the plan's points into tile x tile spreading bins (8, 16, 32);
 * BLOCKING on `stream`.  The result of hqs_adjoint does not depend on the tile
 * beyond float rounding order. */
HQS_API int hqs_plan_retile(hqs_plan plan, int tile, void* stream);

/* Per-pass view of the mixed-precision A^H A (HQS_PREC_BF16X3 / _FP16X3):
 * runs the DFT-GEMM passes 1..stage on x (device, n x n) and writes the
 * intermediate, unscaled, as complex64 to out (device):
 *   stage 1: [L][n][2n]   row DFT of pad(S_l x)             (y, kx)
 *   stage 2: [L][2n][2n]  Khat . 2D DFT of pad(S_l x)        (ky, kx)
 *   stage 3: [L][n][2n]   column IDFT of stage 2, rows y < n (y, kx)
 *   stage 4: [n][n]       A^H A x (same as hqs_toeplitz_normal)
 * DFTs unnormalised with e^{-i} forward; the inverse carries 1/(2n) per axis.
 * The first mixed-precision call of a plan allocates its workspace and
 * synchronises `stream`.  HQS_ERR_UNSUPPORTED unless n % 64 == 0, n <= 512
 * and coils <= 32. */
HQS_API int hqs_debug_toeplitz_stage(hqs_plan plan, const hqs_c64* x, int precision, int stage,
                                     hqs_c64* out, void* stream);

/* ------------------------------------------------ volumetric operator (3D) */
/* Eq. (1) on volumes, the extension Sec. 5 names as future work: voxel
 * (iz, iy, ix) of an (nz, ny, nx) row-major volume has the centred coordinate
 * n = (ix - nx/2, iy - ny/2, iz - nz/2); trajectories are (M, 3) float32
 * (kx, ky, kz) in radians per voxel (any real value, periodic in 2*pi); coil
 * maps are (L, nz, ny, nx); k-space data (L, M) in the caller's point order.
 *
 * hqs_plan3d_create copies the maps, sorts the points into 8^3 spreading bins
 * and builds the Toeplitz kernel of A^H A on the 2N^3 grid (blocking: it
 * synchronises `stream`).  Each of nz, ny, nx must be one of
 * {8, 16, 32, 64, 128, 160, 192}; coils 1..64; kernel_width 4..8; oversamp
 * must be 2 (the NUFFT grid is then also the 2N Toeplitz grid).  Invalid
 * arguments return HQS_ERR_INVALID_ARG with *out = NULL.  The plan holds
 * about (14 L + 13) * 8 * nz*ny*nx bytes of device memory. */
HQS_API int hqs_plan3d_create(hqs_plan3d* out, const float* traj, int64_t M, int nz, int ny, int nx,
                              int coils, const hqs_c64* smaps, int kernel_width, float oversamp,
                              void* stream);
HQS_API void hqs_plan3d_destroy(hqs_plan3d plan);
/* Host outputs (NULL skipped): point count, spreading sub-problems, device bytes held. */
HQS_API int hqs_plan3d_get_info(hqs_plan3d plan, int64_t* npoints, int* nsub, size_t* device_bytes);

/* y = A x by 3D gridding: apodise, zero-pad to the 2N grid, 3D FFT, W^3
 * Kaiser-Bessel interpolation.  x: (nz, ny, nx); y: (L, M). */
HQS_API int hqs_forward3d(hqs_plan3d plan, const hqs_c64* x, hqs_c64* y, void* stream);
/* x = A^H y, the exact transpose of hqs_forward3d (tiled spreading, inverse
 * 3D FFT, crop, deapodisation, conj(S_l) coil sum). */
HQS_API int hqs_adjoint3d(hqs_plan3d plan, const hqs_c64* y, hqs_c64* x, void* stream);
/* out = A^H A x by the 2N^3 circulant embedding (the normal operator of
 * Sec. 3.4 in 3D): out = sum_l conj(S_l) crop(IFFT(Khat * FFT(pad(S_l x)))).
 * The kernel t(d) = Nvox^-1 sum_j exp(+i k_j . d) is gridded with an
 * 8-wide Kaiser-Bessel kernel on a 4N grid (relative error ~1e-7).
 * x and out: (nz, ny, nx), distinct buffers. */
HQS_API int hqs_toeplitz_normal3d(hqs_plan3d plan, const hqs_c64* x, hqs_c64* out, void* stream);
/* Khat (2nz, 2ny, 2nx) float32 = Re FFT_2N(t) / (8 nz ny nx), copied to out (device). */
HQS_API int hqs_plan3d_get_khat(hqs_plan3d plan, float* out, void* stream);
/* Density-compensation preconditioner of Sec. 3.4 on volumes: z = M^-1 r =
 * IFFT_N(FFT_N(r) s^-1/2), s = max(a max(lam, 0) + b, b/4), lam the
 * eigenvalues of T. Chan's optimal circulant of the N^3 Toeplitz part of
 * A^H A / S (built with the plan).  b > 0.  HQS_ERR_UNSUPPORTED unless each
 * of nz, ny, nx is also a transform size (16, 32, 64, 128). */
HQS_API int hqs_precond_apply3d(hqs_plan3d plan, float a, float b, const hqs_c64* r, hqs_c64* z,
                                void* stream);
/* Data-consistency solve of the HQS step on a volume: CG on
 * (a A^H A + b I) x = rhs (precond HQS_PRECOND_NONE) or PCG with the
 * density preconditioner above (HQS_PRECOND_DC), starting from x on entry,
 * fp64 inner products, stopping at ||r|| <= rel_tol ||rhs|| or after
 * max_iter (<= HQS_MAX_ITERS) iterations; the host checks the residual each
 * iteration (blocking).  Returns HQS_OK, HQS_ERR_NOT_CONVERGED or
 * HQS_ERR_BREAKDOWN (HQS_ERR_UNSUPPORTED for HQS_PRECOND_DC where
 * hqs_precond_apply3d is); info (host, optional) as for hqs_dc_solve.
 * rhs and x distinct (nz, ny, nx). */
HQS_API int hqs_dc_solve3d(hqs_plan3d plan, float a, float b, const hqs_c64* rhs, hqs_c64* x,
                           int max_iter, double rel_tol, int precond, hqs_solve_info* info,
                           void* stream);

/* Denoiser callback of hqs_run3d: D_sigma on a device (nz, ny, nx) volume,
 * same contract as hqs_denoiser_fn. */
typedef int (*hqs_denoiser3d_fn)(void* user, const hqs_c64* in, hqs_c64* out,
                                 int nz, int ny, int nx, float sigma, void* stream);
/* Built-in volume denoiser (stand-in for the trained prior of Sec. 4.2): the
 * Gaussian smoothing of hqs_gaussian_denoise along x, then y, then z (std s
 * voxels from hqs_gauss_params as there, radius ceil(3 s) <= 24, periodic);
 * copies in to out when s < 0.1.  Uses stream-ordered scratch
 * (cudaMallocAsync of 2 volumes).  Matches hqs_denoiser3d_fn. */
HQS_API int hqs_gaussian_denoise3d(void* user, const hqs_c64* in, hqs_c64* out,
                                   int nz, int ny, int nx, float sigma, void* stream);
/* Annealed PnP-HQS of Sec. 3.3 on a volume, the steps of hqs_run: for
 * k = k0..K-1, u_k from ((1 + c1 mu_k) A^H A + c0 mu_k I) u = A^H y +
 * mu_k (c0 x_k + c1 A^H A x_k) by cg_iters PCG iterations (density
 * preconditioner where hqs_precond_apply3d exists, plain CG otherwise)
 * warm-started at x_k, then x_{k+1} = D_{sigma_k}(u_k).  mu, sigma: host
 * arrays (mu_k > 0); y: (L, M) device; x: (nz, ny, nx) device, x_{k0} in,
 * x_K out.  denoiser NULL: hqs_gaussian_denoise3d with `user` pointing to
 * hqs_gauss_params (NULL: s = sigma).  Blocking (each CG iteration chunk is
 * checked on the host); the callback runs on the calling thread. */
HQS_API int hqs_run3d(hqs_plan3d plan, const hqs_c64* y, hqs_c64* x, const float* mu, const float* sigma,
                      int K, int k0, int cg_iters, float c0, float c1, hqs_denoiser3d_fn denoiser,
                      void* user, void* stream);

/* Diagnostics (no counterpart in the paper): phase trace of the batched
 * solve (hqs_batch_dc_solve), same protocol as hqs_debug_phase_trace below:
 * enable = 1 allocates the buffer (returns 0); enable = 0 synchronises
 * `stream` and copies up to max_out globaltimer stamps (ns) of the last
 * batched solve to out (host): the start, one stamp after every grid
 * barrier, and the end.  Returns the number of stamps. */
HQS_API int hqs_batch_debug_trace(hqs_batch batch, int enable, unsigned long long* out, int max_out,
                                  void* stream);

/* Diagnostics (no counterpart in the paper): phase trace of the persistent
 * solve.  enable = 1 allocates a trace buffer on the plan (returns 0); later
 * calls with enable = 0 synchronise `stream` and copy up to max_out
 * globaltimer stamps (ns) of the last fused solve into out (host): the start,
 * one stamp after every grid barrier, and the end.  Returns the number of
 * stamps (or a negative status). */
HQS_API int hqs_debug_phase_trace(hqs_plan plan, int enable, unsigned long long* out, int max_out,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HQS_GB300_H */
