"""ctypes binding of include/hqs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

HQS_OK = 0
HQS_ERR_INVALID_ARG = -1
HQS_ERR_OOM = -2
HQS_ERR_NOT_CONVERGED = -3
HQS_ERR_BREAKDOWN = -4
HQS_ERR_TIMEOUT = -5
HQS_ERR_CALLBACK = -6
HQS_ERR_CUDA = -7
HQS_ERR_UNSUPPORTED = -8

HQS_PREC_FP32, HQS_PREC_BF16X3, HQS_PREC_FP16X3 = 0, 1, 2
HQS_PRECOND_NONE, HQS_PRECOND_DC, HQS_PRECOND_LEARNED = 0, 1, 2
HQS_SOLVE_PLAIN, HQS_SOLVE_FUSED = 0, 1
HQS_SOLVE_X0_ZERO = 16
HQS_TUNE_FUSED_GRID, HQS_TUNE_PC_LINES, HQS_TUNE_SPREAD_TILE = 1, 2, 3
HQS_TUNE_DEBUG_BARRIER_SKIP = 4
HQS_MAX_ITERS = 512

_PKG = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_PKG, "libhqs_gb300.so")


class PlanInfo(C.Structure):
    _fields_ = [("ny", C.c_int), ("nx", C.c_int), ("coils", C.c_int), ("kernel_width", C.c_int),
                ("oversamp", C.c_float), ("grid", C.c_int), ("npoints", C.c_int64),
                ("kb_beta", C.c_double), ("device_bytes", C.c_size_t), ("nsub", C.c_int),
                ("tile", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("fallback", C.c_int),
                ("reserved", C.c_int), ("rhs_norm", C.c_double), ("rel_residual", C.c_double),
                ("res_history", C.c_double * (HQS_MAX_ITERS + 1))]

    def history(self):
        return [self.res_history[i] for i in range(self.iterations + 1)]


class GaussParams(C.Structure):
    _fields_ = [("kappa", C.c_float), ("sigma0", C.c_float)]


DENOISER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                          C.c_float, C.c_void_p)
DENOISER3_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                           C.c_float, C.c_void_p)

_lock = threading.Lock()
_lib = None

_SIGS = {
    "hqs_plan_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_int64, C.c_int, C.c_int,
                                  C.c_int, C.c_void_p, C.c_int, C.c_float, C.c_void_p]),
    "hqs_plan_destroy": (None, [C.c_void_p]),
    "hqs_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    "hqs_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_adjoint_axpy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "hqs_toeplitz_normal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "hqs_precond_apply": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "hqs_dc_solve": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_int,
                               C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(SolveInfo),
                               C.c_void_p]),
    "hqs_last_solve_info": (C.c_int, [C.c_void_p, C.POINTER(SolveInfo), C.c_void_p]),
    "hqs_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                          C.POINTER(C.c_float), C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_pgd_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                          C.POINTER(C.c_float), C.c_int, C.c_float, C.c_float,
                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_gaussian_denoise": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                       C.c_float, C.c_void_p]),
    "hqs_power_iteration": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "hqs_status_string": (C.c_char_p, [C.c_int]),
    "hqs_estimate_smaps": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                     C.c_float, C.c_float, C.c_float, C.c_void_p, C.c_void_p]),
    "hqs_plan_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "hqs_plan_retile": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "hqs_debug_toeplitz_stage": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "hqs_net_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "hqs_net_destroy": (None, [C.c_void_p]),
    "hqs_net_num_params": (C.c_int, []),
    "hqs_net_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "hqs_net_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "hqs_net_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "hqs_net_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "hqs_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                  C.c_void_p]),
    "hqs_net_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                   C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "hqs_net_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                     C.c_float, C.POINTER(C.c_double), C.c_void_p]),
    "hqs_net_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                   C.c_void_p, C.c_void_p]),
    "hqs_net_train_step_dy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                        C.c_float, C.c_void_p]),
    "hqs_net_denoise": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_void_p]),
    "hqs_net_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "hqs_net_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "hqs_plan_set_net": (C.c_int, [C.c_void_p, C.c_void_p]),
    "hqs_learned_precond_apply": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_void_p,
                                            C.c_void_p, C.c_void_p]),
    "hqs_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "hqs_batch_destroy": (None, [C.c_void_p]),
    "hqs_batch_run": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int, C.c_int, C.c_int,
                                C.c_float, C.c_float, C.c_void_p, C.c_int, C.c_void_p]),
    "hqs_batch_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "hqs_batch_dc_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_float,
                                     C.c_float, C.c_int, C.c_double, C.c_void_p]),
    "hqs_batch_dc_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                    C.c_void_p]),
    "hqs_batch_toeplitz_normal": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "hqs_batch_set_grid": (C.c_int, [C.c_void_p, C.c_int]),
    "hqs_batch_forward": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "hqs_batch_adjoint_axpy": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_float, C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.c_void_p]),
    "hqs_precond_apply_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_float,
                                            C.c_void_p, C.c_void_p]),
    "hqs_debug_phase_trace": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_ulonglong), C.c_int,
                                        C.c_void_p]),
    "hqs_batch_debug_trace": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_ulonglong), C.c_int, C.c_void_p]),
    "hqs_plan3d_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_void_p, C.c_int, C.c_float, C.c_void_p]),
    "hqs_plan3d_destroy": (None, [C.c_void_p]),
    "hqs_plan3d_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                      C.POINTER(C.c_size_t)]),
    "hqs_plan3d_get_khat": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_forward3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_adjoint3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_toeplitz_normal3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_dc_solve3d": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_double, C.c_int, C.POINTER(SolveInfo), C.c_void_p]),
    "hqs_precond_apply3d": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hqs_gaussian_denoise3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                         C.c_float, C.c_void_p]),
    "hqs_run3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                            C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_void_p, C.c_void_p,
                            C.c_void_p]),
}


def library():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build it with paper_2411_01955_gb300.build.build() "
                    "(there is no CPU fallback)")
            lib = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class HqsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def estimate_smaps(traj, y, n, out, dcf=None, kernel_width=6, oversamp=2.0, width=20.0, thresh=0.05,
                   stream=None):
    """S-maps (coils, n, n) from the windowed k-space centre of y (coils, M)."""
    coils, M = y.shape
    _check(library().hqs_estimate_smaps(_ptr(traj, torch.float32, "traj"), int(M), _ptr(y, torch.complex64, "y"),
                                        _ptr(dcf, torch.float32, "dcf") if dcf is not None else None, int(n),
                                        int(coils), int(kernel_width), float(oversamp), float(width),
                                        float(thresh), _ptr(out, torch.complex64, "smaps"), _stream(stream)),
           "hqs_estimate_smaps")
    return out


def status_string(status: int) -> str:
    return library().hqs_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != HQS_OK:
        raise HqsError(rc, what)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _need(t, n, name):
    # the C entry points size every buffer from the plan, so a tensor holding fewer
    # (or more) elements than the plan implies is rejected here, before any launch
    if t is not None and t.numel() != n:
        raise ValueError(f"{name} must hold {n} elements, got {t.numel()} (shape {tuple(t.shape)})")


def _image_elems(plan):
    if hasattr(plan, "ny"):
        return plan.ny * plan.nx
    nz, ny, nx = plan.shape
    return nz * ny * nx


def _need_image(plan, **named):
    for name, t in named.items():
        _need(t, _image_elems(plan), name)


def _need_kspace(plan, **named):
    for name, t in named.items():
        _need(t, plan.coils * plan.npoints, name)


def _need_schedule(K, **named):
    for name, v in named.items():
        if len(v) < K:
            raise ValueError(f"{name} needs K = {K} entries, got {len(v)}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Plan:
    """Owns an hqs_plan (hqs_plan_create / hqs_plan_destroy)."""

    def __init__(self, handle, ny, nx, coils, npoints):
        self.handle = handle
        self.ny, self.nx, self.coils, self.npoints = ny, nx, coils, npoints

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(library().hqs_plan_get_info(self.handle, C.byref(inf)), "hqs_plan_get_info")
        return inf

    def close(self):
        if self.handle:
            library().hqs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_create(traj, ny, nx, smaps, kernel_width=6, oversamp=2.0, stream=None) -> Plan:
    """traj (M, 2) float32 CUDA; smaps (L, ny, nx) complex64 CUDA."""
    M = int(traj.shape[0])
    _need(traj, 2 * M, "traj")
    _need(smaps, int(smaps.shape[0]) * int(ny) * int(nx), "smaps")
    lib = library()
    h = C.c_void_p()
    rc = lib.hqs_plan_create(C.byref(h), _ptr(traj, torch.float32, "traj"), M, int(ny), int(nx),
                             int(smaps.shape[0]), _ptr(smaps, torch.complex64, "smaps"),
                             int(kernel_width), float(oversamp), _stream(stream))
    _check(rc, "hqs_plan_create")
    return Plan(h, int(ny), int(nx), int(smaps.shape[0]), M)


def forward(plan: Plan, x, y, stream=None):
    _need_image(plan, x=x)
    _need_kspace(plan, y=y)
    _check(library().hqs_forward(plan.handle, _ptr(x, torch.complex64, "x"),
                                 _ptr(y, torch.complex64, "y"), _stream(stream)), "hqs_forward")
    return y


def adjoint(plan: Plan, y, x, stream=None):
    _need_kspace(plan, y=y)
    _need_image(plan, x=x)
    _check(library().hqs_adjoint(plan.handle, _ptr(y, torch.complex64, "y"),
                                 _ptr(x, torch.complex64, "x"), _stream(stream)), "hqs_adjoint")
    return x


def adjoint_axpy(plan: Plan, y, c, z, x, stream=None):
    """x = A^H y + c z (the HQS data-consistency right-hand side)."""
    _need_kspace(plan, y=y)
    _need_image(plan, z=z, x=x)
    _check(library().hqs_adjoint_axpy(plan.handle, _ptr(y, torch.complex64, "y"), float(c),
                                      _ptr(z, torch.complex64, "z"), _ptr(x, torch.complex64, "x"),
                                      _stream(stream)), "hqs_adjoint_axpy")
    return x


def toeplitz_normal(plan: Plan, x, out, precision=HQS_PREC_FP32, stream=None):
    _need_image(plan, x=x, out=out)
    _check(library().hqs_toeplitz_normal(plan.handle, _ptr(x, torch.complex64, "x"),
                                         _ptr(out, torch.complex64, "out"), int(precision),
                                         _stream(stream)), "hqs_toeplitz_normal")
    return out


def precond_apply(plan: Plan, a, b, r, z, stream=None):
    _need_image(plan, r=r, z=z)
    _check(library().hqs_precond_apply(plan.handle, float(a), float(b), _ptr(r, torch.complex64, "r"),
                                       _ptr(z, torch.complex64, "z"), _stream(stream)),
           "hqs_precond_apply")
    return z


def dc_solve(plan: Plan, a, b, rhs, x, max_iter=30, rel_tol=1e-4, precond=HQS_PRECOND_DC,
             mode=HQS_SOLVE_PLAIN, precision=HQS_PREC_FP32, want_info=True, stream=None,
             check=True):
    """Solves (a A^H A + b I) x = rhs in place; returns SolveInfo (or None)."""
    _need_image(plan, rhs=rhs, x=x)
    info = SolveInfo() if want_info else None
    rc = library().hqs_dc_solve(plan.handle, float(a), float(b), _ptr(rhs, torch.complex64, "rhs"),
                                _ptr(x, torch.complex64, "x"), int(max_iter), float(rel_tol),
                                int(precond), int(mode), int(precision),
                                C.byref(info) if info is not None else None, _stream(stream))
    if check and rc not in (HQS_OK, HQS_ERR_NOT_CONVERGED):
        raise HqsError(rc, "hqs_dc_solve")
    if info is not None:
        info.rc = rc
    return info


def last_solve_info(plan: Plan, stream=None) -> SolveInfo:
    info = SolveInfo()
    _check(library().hqs_last_solve_info(plan.handle, C.byref(info), _stream(stream)),
           "hqs_last_solve_info")
    return info


def _wrap_device(ptr, shape):
    class _Arr:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<c8", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Arr(), device="cuda")


def hqs_run(plan: Plan, y, x, mu, sigma, K=None, k0=0, cg_iters=5, c0=1.0, c1=0.0,
            denoiser=None, gauss=None, stream=None):
    """Annealed PnP-HQS; `denoiser` is None (built-in Gaussian smoothing, with
    optional gauss=(kappa, sigma0)) or a callable(in_tensor, out_tensor, sigma)
    that enqueues work on the current stream and returns 0 on success."""
    _need_kspace(plan, y=y)
    _need_image(plan, x=x)
    lib = library()
    K = len(mu) if K is None else int(K)
    _need_schedule(K, mu=mu, sigma=sigma)
    mu_c = (C.c_float * K)(*[float(v) for v in mu[:K]])
    sg_c = (C.c_float * K)(*[float(v) for v in sigma[:K]])
    user = None
    cb = None
    keep = []
    if isinstance(denoiser, Net):
        # the library's conv-net denoiser, called natively with the network as user data
        cb = C.cast(lib.hqs_net_denoise, DENOISER_FN)
        user = denoiser.handle
        keep.append(denoiser)
    elif denoiser is None:
        if gauss is not None:
            gp = GaussParams(float(gauss[0]), float(gauss[1]))
            keep.append(gp)
            user = C.cast(C.pointer(gp), C.c_void_p)
    else:
        ny, nx = plan.ny, plan.nx

        def _cb(_user, pin, pout, h, w, s, _stream_ptr):
            try:
                tin = _wrap_device(pin, (h, w))
                tout = _wrap_device(pout, (h, w))
                return int(denoiser(tin, tout, float(s)) or 0)
            except Exception:
                return 1
        cb = DENOISER_FN(_cb)
        keep.append(cb)
    rc = lib.hqs_run(plan.handle, _ptr(y, torch.complex64, "y"), _ptr(x, torch.complex64, "x"),
                     mu_c, sg_c, K, int(k0), int(cg_iters), float(c0), float(c1),
                     C.cast(cb, C.c_void_p) if cb is not None else None, user, _stream(stream))
    _check(rc, "hqs_run")
    return x


def pgd_run(plan: Plan, y, x, gamma, sigma, K=None, c0=1.0, c1=0.0, gauss=None, stream=None):
    """PnP-PGD with the gradient step in the metric P = c0 I + c1 A^H A and the
    built-in Gaussian smoothing denoiser (optional gauss=(kappa, sigma0))."""
    _need_kspace(plan, y=y)
    _need_image(plan, x=x)
    K = len(gamma) if K is None else int(K)
    _need_schedule(K, gamma=gamma, sigma=sigma)
    g_c = (C.c_float * max(K, 1))(*[float(v) for v in gamma[:K]])
    s_c = (C.c_float * max(K, 1))(*[float(v) for v in sigma[:K]])
    user, keep = None, []
    if gauss is not None:
        gp = GaussParams(float(gauss[0]), float(gauss[1]))
        keep.append(gp)
        user = C.cast(C.pointer(gp), C.c_void_p)
    _check(library().hqs_pgd_run(plan.handle, _ptr(y, torch.complex64, "y"), _ptr(x, torch.complex64, "x"),
                                 g_c, s_c, K, float(c0), float(c1), None, user, _stream(stream)), "hqs_pgd_run")
    return x


def gaussian_denoise(x, out, sigma, gauss=None, stream=None):
    gp = None
    if gauss is not None:
        gp = GaussParams(float(gauss[0]), float(gauss[1]))
    ny, nx = x.shape[-2], x.shape[-1]
    _need(x, int(ny) * int(nx), "x")
    _need(out, int(ny) * int(nx), "out")
    _check(library().hqs_gaussian_denoise(C.cast(C.pointer(gp), C.c_void_p) if gp else None,
                                          _ptr(x, torch.complex64, "x"),
                                          _ptr(out, torch.complex64, "out"), int(ny), int(nx),
                                          float(sigma), _stream(stream)), "hqs_gaussian_denoise")
    return out


def power_iteration(plan: Plan, iters=50, stream=None) -> float:
    lam = C.c_double()
    _check(library().hqs_power_iteration(plan.handle, int(iters), C.byref(lam), _stream(stream)),
           "hqs_power_iteration")
    return lam.value


def debug_phase_trace(plan: Plan, enable=False, stream=None):
    """enable=True arms the persistent solve's phase trace; enable=False
    returns the globaltimer stamps (ns) of the last fused solve."""
    buf = (C.c_ulonglong * 4096)()
    rc = library().hqs_debug_phase_trace(plan.handle, 1 if enable else 0, buf, 4096, _stream(stream))
    if rc < 0:
        raise HqsError(rc, "hqs_debug_phase_trace")
    return [buf[i] for i in range(rc)]


def toeplitz_stage(plan: Plan, x, precision: int, stage: int, out, stream=None):
    """Intermediate of the mixed-precision A^H A after DFT-GEMM pass `stage`
    (1..3, complex64, natural layout; 4 = the result)."""
    _need_image(plan, x=x)
    _check(library().hqs_debug_toeplitz_stage(plan.handle, _ptr(x, torch.complex64, "x"), int(precision),
                                              int(stage), _ptr(out, torch.complex64, "out"),
                                              _stream(stream)), "hqs_debug_toeplitz_stage")
    return out


def plan_retile(plan: Plan, tile: int, stream=None):
    _check(library().hqs_plan_retile(plan.handle, int(tile), _stream(stream)), "hqs_plan_retile")


def plan_set_tuning(plan: Plan, key: int, value: int):
    _check(library().hqs_plan_set_tuning(plan.handle, int(key), int(value)), "hqs_plan_set_tuning")


NOALLOC_SIZES = (16, 32, 64, 128, 256, 320, 384)


def _noalloc_check(r, lam, z) -> int:
    """Shapes and types of hqs_precond_apply_noalloc's arguments, checked before
    any launch: the C entry point takes n alone and cannot check the buffers."""
    if r.dim() != 2 or r.shape[0] != r.shape[1]:
        raise ValueError(f"r must be (n, n), got {tuple(r.shape)}")
    n = int(r.shape[0])
    if n not in NOALLOC_SIZES:
        raise ValueError(f"n = {n} is not one of {NOALLOC_SIZES}")
    for t, name, dt in ((r, "r", torch.complex64), (lam, "lam", torch.float32), (z, "z", torch.complex64)):
        if tuple(t.shape) != (n, n):
            raise ValueError(f"{name} must be ({n}, {n}), got {tuple(t.shape)}")
        if t.dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    return n


def precond_apply_noalloc(r, lam, a, b, z, stream=None):
    """Preconditioner apply without any device allocation (no plan): scratch
    lives in a static device array, n <= 384; the density symbol lam is given."""
    n = _noalloc_check(r, lam, z)
    _check(library().hqs_precond_apply_noalloc(_ptr(r, torch.complex64, "r"),
                                               _ptr(lam, torch.float32, "lam"), n, float(a),
                                               float(b), _ptr(z, torch.complex64, "z"),
                                               _stream(stream)), "hqs_precond_apply_noalloc")
    return z


class Net:
    """The conv-net preconditioner (hqs_net_*); activations are planar float
    CUDA tensors (N, 2, H, W)."""

    def __init__(self):
        h = C.c_void_p()
        _check(library().hqs_net_create(C.byref(h)), "hqs_net_create")
        self.handle = h
        self.num_params = library().hqs_net_num_params()

    def set_precision(self, precision):
        """HQS_PREC_BF16X3 (default: the 32 -> 32 layers on the tensor cores) or
        HQS_PREC_FP32."""
        _check(library().hqs_net_set_precision(self.handle, int(precision)), "hqs_net_set_precision")

    def status(self, stream=None):
        """Raises HqsError(HQS_ERR_TIMEOUT) if a tensor-core convolution gave up a
        wait since the last check."""
        _check(library().hqs_net_status(self.handle, _stream(stream)), "hqs_net_status")

    def set_params(self, vec):
        import numpy as np
        v = np.ascontiguousarray(np.asarray(vec, dtype=np.float32))
        _check(library().hqs_net_set_params(self.handle, v.ctypes.data_as(C.c_void_p), v.size),
               "hqs_net_set_params")

    def get_params(self):
        import numpy as np
        v = np.empty(self.num_params, dtype=np.float32)
        _check(library().hqs_net_get_params(self.handle, v.ctypes.data_as(C.c_void_p), v.size),
               "hqs_net_get_params")
        return v

    def forward(self, x, y=None, stream=None):
        y = torch.empty_like(x) if y is None else y
        N, _, H, W = x.shape
        _check(library().hqs_net_forward(self.handle, _ptr(x, torch.float32, "x"),
                                         _ptr(y, torch.float32, "y"), N, H, W, _stream(stream)),
               "hqs_net_forward")
        return y

    def gradient(self, x, t, stream=None):
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        loss = C.c_double()
        N, _, H, W = x.shape
        _check(library().hqs_net_gradient(self.handle, _ptr(x, torch.float32, "x"),
                                          _ptr(t, torch.float32, "t"), N, H, W,
                                          _ptr(g, torch.float32, "grad"), C.byref(loss),
                                          _stream(stream)), "hqs_net_gradient")
        return g, loss.value

    def train_step(self, x, t, lr, stream=None):
        loss = C.c_double()
        N, _, H, W = x.shape
        _check(library().hqs_net_train_step(self.handle, _ptr(x, torch.float32, "x"),
                                            _ptr(t, torch.float32, "t"), N, H, W, float(lr),
                                            C.byref(loss), _stream(stream)), "hqs_net_train_step")
        return loss.value

    def backward(self, x, dy, stream=None):
        """Parameter gradient for a loss with output gradient dy."""
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        N, _, H, W = x.shape
        _check(library().hqs_net_backward(self.handle, _ptr(x, torch.float32, "x"), _ptr(dy, torch.float32, "dy"),
                                          N, H, W, _ptr(g, torch.float32, "grad"), _stream(stream)),
               "hqs_net_backward")
        return g

    def train_step_dy(self, x, dy, lr, stream=None):
        N, _, H, W = x.shape
        _check(library().hqs_net_train_step_dy(self.handle, _ptr(x, torch.float32, "x"),
                                               _ptr(dy, torch.float32, "dy"), N, H, W, float(lr),
                                               _stream(stream)), "hqs_net_train_step_dy")

    def denoise(self, v, out, sigma, stream=None):
        """out = v - sigma net(v / sigma) (complex64 image)."""
        ny, nx = v.shape[-2], v.shape[-1]
        _check(library().hqs_net_denoise(self.handle, _ptr(v, torch.complex64, "v"), _ptr(out, torch.complex64, "out"),
                                         int(ny), int(nx), float(sigma), _stream(stream)), "hqs_net_denoise")
        return out

    def save(self, path):
        _check(library().hqs_net_save(self.handle, str(path).encode()), "hqs_net_save")

    def load(self, path):
        _check(library().hqs_net_load(self.handle, str(path).encode()), "hqs_net_load")

    def close(self):
        if self.handle:
            library().hqs_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_set_net(plan: Plan, net):
    _check(library().hqs_plan_set_net(plan.handle, net.handle if net is not None else None),
           "hqs_plan_set_net")
    plan._net = net


def learned_precond_apply(plan: Plan, a, b, r, z, stream=None):
    _need_image(plan, r=r, z=z)
    _check(library().hqs_learned_precond_apply(plan.handle, float(a), float(b),
                                               _ptr(r, torch.complex64, "r"),
                                               _ptr(z, torch.complex64, "z"), _stream(stream)),
           "hqs_learned_precond_apply")
    return z


class Batch:
    """Batched annealed HQS over plans of uneven size (hqs_batch_*)."""

    def __init__(self, plans, max_outer=64):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = C.c_void_p()
        _check(library().hqs_batch_create(C.byref(h), arr, len(self.plans), int(max_outer)),
               "hqs_batch_create")
        self.handle = h

    def run(self, ys, xs, mu, sigma, K=None, k0=0, cg_iters=5, c0=1.0, c1=0.0, gauss=None,
            use_graph=True, stream=None):
        K = len(mu) if K is None else int(K)
        if K > min(len(mu), len(sigma)):
            raise ValueError("mu and sigma need K entries")
        self._check_kspace(ys)
        self._check_images(xs, "x")
        n = len(self.plans)
        yp = (C.c_void_p * n)(*[_ptr(y, torch.complex64, "y") for y in ys])
        xp = (C.c_void_p * n)(*[_ptr(x, torch.complex64, "x") for x in xs])
        mu_c = (C.c_float * K)(*[float(v) for v in mu[:K]])
        sg_c = (C.c_float * K)(*[float(v) for v in sigma[:K]])
        gp = GaussParams(float(gauss[0]), float(gauss[1])) if gauss is not None else None
        _check(library().hqs_batch_run(self.handle, yp, xp, mu_c, sg_c, K, int(k0), int(cg_iters),
                                       float(c0), float(c1),
                                       C.cast(C.pointer(gp), C.c_void_p) if gp else None,
                                       1 if use_graph else 0, _stream(stream)), "hqs_batch_run")
        return xs

    def dc_solve(self, rhs, xs, a, b, max_iter=200, rel_tol=1e-4, stream=None):
        """Solves (a A^H A + b I) x_i = rhs_i for every slice from x_i = 0 in one launch."""
        self._check_images(rhs, "rhs")
        self._check_images(xs, "x")
        n = len(self.plans)
        rp = (C.c_void_p * n)(*[_ptr(r, torch.complex64, "rhs") for r in rhs])
        xp = (C.c_void_p * n)(*[_ptr(x, torch.complex64, "x") for x in xs])
        _check(library().hqs_batch_dc_solve(self.handle, rp, xp, float(a), float(b), int(max_iter),
                                            float(rel_tol), _stream(stream)), "hqs_batch_dc_solve")
        return xs

    def set_grid(self, ctas):
        """Caps the CTAs of the batch's cooperative launches (0: all resident)."""
        _check(library().hqs_batch_set_grid(self.handle, int(ctas)), "hqs_batch_set_grid")

    def toeplitz_normal(self, xs, outs, stream=None):
        """out_i = A_i^H A_i x_i for every slice in one launch."""
        n = len(self.plans)
        if len(xs) != n or len(outs) != n:
            raise ValueError("one x and one out per slice")
        for p, x, o in zip(self.plans, xs, outs):
            if tuple(x.shape) != (p.ny, p.nx) or tuple(o.shape) != (p.ny, p.nx):
                raise ValueError(f"x and out must be ({p.ny}, {p.nx})")
        xp = (C.c_void_p * n)(*[_ptr(x, torch.complex64, "x") for x in xs])
        op = (C.c_void_p * n)(*[_ptr(o, torch.complex64, "out") for o in outs])
        _check(library().hqs_batch_toeplitz_normal(self.handle, xp, op, _stream(stream)),
               "hqs_batch_toeplitz_normal")
        return outs

    def _check_images(self, xs, what):
        if len(xs) != len(self.plans):
            raise ValueError(f"one {what} per slice")
        for p, x in zip(self.plans, xs):
            if tuple(x.shape) != (p.ny, p.nx):
                raise ValueError(f"{what} must be ({p.ny}, {p.nx})")

    def _check_kspace(self, ys):
        if len(ys) != len(self.plans):
            raise ValueError("one y per slice")
        for p, y in zip(self.plans, ys):
            if tuple(y.shape) != (p.coils, p.npoints):
                raise ValueError(f"y must be ({p.coils}, {p.npoints})")

    def forward(self, xs, ys, stream=None):
        """y_i = A_i x_i for every slice (the FFT passes of like slices batched)."""
        self._check_images(xs, "x")
        self._check_kspace(ys)
        n = len(self.plans)
        xp = (C.c_void_p * n)(*[_ptr(x, torch.complex64, "x") for x in xs])
        yp = (C.c_void_p * n)(*[_ptr(y, torch.complex64, "y") for y in ys])
        _check(library().hqs_batch_forward(self.handle, xp, yp, _stream(stream)), "hqs_batch_forward")
        return ys

    def adjoint_axpy(self, ys, zc, zs, xs, stream=None):
        """x_i = A_i^H y_i + zc z_i for every slice (zs None: no axpy term)."""
        self._check_kspace(ys)
        self._check_images(xs, "x")
        if zs is not None:
            self._check_images(zs, "z")
        n = len(self.plans)
        yp = (C.c_void_p * n)(*[_ptr(y, torch.complex64, "y") for y in ys])
        xp = (C.c_void_p * n)(*[_ptr(x, torch.complex64, "x") for x in xs])
        zp = None
        if zs is not None:
            zp = (C.c_void_p * n)(*[_ptr(z, torch.complex64, "z") for z in zs])
        _check(library().hqs_batch_adjoint_axpy(self.handle, yp, float(zc), zp, xp, _stream(stream)),
               "hqs_batch_adjoint_axpy")
        return xs

    def debug_trace(self, enable=False, stream=None):
        """enable=True arms the batched solve's phase trace; enable=False
        returns the globaltimer stamps (ns) of the last batched solve."""
        buf = (C.c_ulonglong * 4096)()
        rc = library().hqs_batch_debug_trace(self.handle, 1 if enable else 0, buf, 4096, _stream(stream))
        if rc < 0:
            raise HqsError(rc, "hqs_batch_debug_trace")
        return [buf[i] for i in range(rc)]

    def dc_info(self, stream=None):
        """Per slice (iterations, relative residual, status) of the last batched solve."""
        n = len(self.plans)
        it = (C.c_int * n)()
        rr = (C.c_double * n)()
        st = (C.c_int * n)()
        _check(library().hqs_batch_dc_info(self.handle, it, rr, st, _stream(stream)), "hqs_batch_dc_info")
        return [(it[i], rr[i], st[i]) for i in range(n)]

    def status(self, stream=None):
        res = (C.c_double * len(self.plans))()
        _check(library().hqs_batch_status(self.handle, res, _stream(stream)), "hqs_batch_status")
        return [res[i] for i in range(len(self.plans))]

    def close(self):
        if self.handle:
            library().hqs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ volumes
class Plan3d:
    """Owns an hqs_plan3d (hqs_plan3d_create / hqs_plan3d_destroy)."""

    def __init__(self, handle, shape, coils, npoints):
        self.handle = handle
        self.shape, self.coils, self.npoints = tuple(shape), coils, npoints

    def info(self):
        M, nsub, nbytes = C.c_int64(), C.c_int(), C.c_size_t()
        _check(library().hqs_plan3d_get_info(self.handle, C.byref(M), C.byref(nsub), C.byref(nbytes)),
               "hqs_plan3d_get_info")
        return {"npoints": M.value, "nsub": nsub.value, "device_bytes": nbytes.value}

    def close(self):
        if self.handle:
            library().hqs_plan3d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan3d_create(traj, shape, smaps, kernel_width=6, oversamp=2.0, stream=None) -> Plan3d:
    """traj (M, 3) float32 CUDA; shape (nz, ny, nx); smaps (L, nz, ny, nx) complex64 CUDA."""
    nz, ny, nx = (int(v) for v in shape)
    M = int(traj.shape[0])
    _need(traj, 3 * M, "traj")
    _need(smaps, int(smaps.shape[0]) * nz * ny * nx, "smaps")
    h = C.c_void_p()
    rc = library().hqs_plan3d_create(C.byref(h), _ptr(traj, torch.float32, "traj"), M, nz, ny, nx,
                                     int(smaps.shape[0]), _ptr(smaps, torch.complex64, "smaps"),
                                     int(kernel_width), float(oversamp), _stream(stream))
    _check(rc, "hqs_plan3d_create")
    return Plan3d(h, (nz, ny, nx), int(smaps.shape[0]), M)


def forward3d(plan: Plan3d, x, y, stream=None):
    _need_image(plan, x=x)
    _need_kspace(plan, y=y)
    _check(library().hqs_forward3d(plan.handle, _ptr(x, torch.complex64, "x"), _ptr(y, torch.complex64, "y"),
                                   _stream(stream)), "hqs_forward3d")
    return y


def adjoint3d(plan: Plan3d, y, x, stream=None):
    _need_kspace(plan, y=y)
    _need_image(plan, x=x)
    _check(library().hqs_adjoint3d(plan.handle, _ptr(y, torch.complex64, "y"), _ptr(x, torch.complex64, "x"),
                                   _stream(stream)), "hqs_adjoint3d")
    return x


def toeplitz_normal3d(plan: Plan3d, x, out, stream=None):
    _need_image(plan, x=x, out=out)
    _check(library().hqs_toeplitz_normal3d(plan.handle, _ptr(x, torch.complex64, "x"),
                                           _ptr(out, torch.complex64, "out"), _stream(stream)),
           "hqs_toeplitz_normal3d")
    return out


def plan3d_khat(plan: Plan3d, out, stream=None):
    """Khat (2nz, 2ny, 2nx) float32, scaled by 1 / (8 nz ny nx)."""
    _need(out, 8 * _image_elems(plan), "out")
    _check(library().hqs_plan3d_get_khat(plan.handle, _ptr(out, torch.float32, "out"), _stream(stream)),
           "hqs_plan3d_get_khat")
    return out


def precond_apply3d(plan: Plan3d, a, b, r, z, stream=None):
    _need_image(plan, r=r, z=z)
    _check(library().hqs_precond_apply3d(plan.handle, float(a), float(b), _ptr(r, torch.complex64, "r"),
                                         _ptr(z, torch.complex64, "z"), _stream(stream)), "hqs_precond_apply3d")
    return z


def dc_solve3d(plan: Plan3d, a, b, rhs, x, max_iter=30, rel_tol=1e-4, precond=HQS_PRECOND_DC, stream=None,
               check=True) -> SolveInfo:
    """Solves (a A^H A + b I) x = rhs in place (PCG, blocking); returns SolveInfo."""
    _need_image(plan, rhs=rhs, x=x)
    info = SolveInfo()
    rc = library().hqs_dc_solve3d(plan.handle, float(a), float(b), _ptr(rhs, torch.complex64, "rhs"),
                                  _ptr(x, torch.complex64, "x"), int(max_iter), float(rel_tol), int(precond),
                                  C.byref(info), _stream(stream))
    if check and rc not in (HQS_OK, HQS_ERR_NOT_CONVERGED):
        raise HqsError(rc, "hqs_dc_solve3d")
    info.rc = rc
    return info


def gaussian_denoise3d(x, out, sigma, gauss=None, stream=None):
    """Built-in volume denoiser; gauss=(kappa, sigma0) or None (s = sigma)."""
    gp = GaussParams(float(gauss[0]), float(gauss[1])) if gauss is not None else None
    nz, ny, nx = (int(v) for v in x.shape)
    _need(out, nz * ny * nx, "out")
    _check(library().hqs_gaussian_denoise3d(C.cast(C.pointer(gp), C.c_void_p) if gp is not None else None,
                                            _ptr(x, torch.complex64, "x"), _ptr(out, torch.complex64, "out"),
                                            nz, ny, nx, float(sigma), _stream(stream)), "hqs_gaussian_denoise3d")
    return out


def hqs_run3d(plan: Plan3d, y, x, mu, sigma, K=None, k0=0, cg_iters=5, c0=1.0, c1=0.0, denoiser=None,
              gauss=None, stream=None):
    """Annealed PnP-HQS on a volume; `denoiser` is None (built-in Gaussian
    smoothing, optional gauss=(kappa, sigma0)) or a callable(in_tensor,
    out_tensor, sigma) that enqueues work on the current stream and returns 0."""
    _need_kspace(plan, y=y)
    _need_image(plan, x=x)
    lib = library()
    K = len(mu) if K is None else int(K)
    _need_schedule(K, mu=mu, sigma=sigma)
    mu_c = (C.c_float * K)(*[float(v) for v in mu[:K]])
    sg_c = (C.c_float * K)(*[float(v) for v in sigma[:K]])
    user, cb, keep = None, None, []
    if denoiser is None:
        if gauss is not None:
            gp = GaussParams(float(gauss[0]), float(gauss[1]))
            keep.append(gp)
            user = C.cast(C.pointer(gp), C.c_void_p)
    else:
        def _cb(_user, pin, pout, d, h, w, s, _stream_ptr):
            try:
                tin = _wrap_device(pin, (d, h, w))
                tout = _wrap_device(pout, (d, h, w))
                return int(denoiser(tin, tout, float(s)) or 0)
            except Exception:
                return 1
        cb = DENOISER3_FN(_cb)
        keep.append(cb)
    rc = lib.hqs_run3d(plan.handle, _ptr(y, torch.complex64, "y"), _ptr(x, torch.complex64, "x"), mu_c, sg_c, K,
                       int(k0), int(cg_iters), float(c0), float(c1),
                       C.cast(cb, C.c_void_p) if cb is not None else None, user, _stream(stream))
    _check(rc, "hqs_run3d")
    return x
