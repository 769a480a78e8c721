"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hqs.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hqs.h")).read()
    return sorted(set(re.findall(r"HQS_API\s+[\w\s\*]+?\b(hqs_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["hqs_plan_create", "hqs_plan_destroy", "hqs_forward", "hqs_adjoint",
                 "hqs_toeplitz_normal", "hqs_dc_solve", "hqs_run", "hqs_precond_apply",
                 "hqs_gaussian_denoise", "hqs_power_iteration", "hqs_status_string"]:
        assert name in syms


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2411_01955_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    lib.hqs_status_string.restype = ctypes.c_char_p
    assert lib.hqs_status_string(0) == b"ok"
    assert lib.hqs_status_string(-1) == b"invalid argument"


def test_invalid_arguments_are_rejected_without_a_gpu():
    from paper_2411_01955_gb300 import build
    lib = ctypes.CDLL(build.build())
    h = ctypes.c_void_p()
    # non-square image, bad width, bad oversampling: rejected before any CUDA call
    assert lib.hqs_plan_create(ctypes.byref(h), None, ctypes.c_int64(0), 32, 64, 4, None, 4,
                               ctypes.c_float(2.0), None) == -1
    assert lib.hqs_plan_create(ctypes.byref(h), None, ctypes.c_int64(0), 32, 32, 4, None, 1,
                               ctypes.c_float(2.0), None) == -1
    assert lib.hqs_plan_create(None, None, ctypes.c_int64(0), 32, 32, 4, None, 4, ctypes.c_float(2.0), None) == -1
    assert lib.hqs_forward(None, None, None, None) == -1


def test_volume_arguments_are_rejected_without_a_gpu():
    """The volumetric plan validates sizes, widths, oversampling and pointers
    before any CUDA call; the operators reject a null plan."""
    from paper_2411_01955_gb300 import build
    lib = ctypes.CDLL(build.build())
    h = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    two = ctypes.c_float(2.0)
    # sizes: 24 (48 is no transform size), 4 (too small), odd; width 3 and 9; oversampling 1.5; coils 0
    for nz, ny, nx in [(8, 16, 24), (4, 16, 16), (8, 15, 16)]:
        assert lib.hqs_plan3d_create(ctypes.byref(h), None, ctypes.c_int64(0), nz, ny, nx, 2, fake, 6, two,
                                     None) == -1
        assert h.value is None
        h = ctypes.c_void_p(123)
    for L, W, sg in [(2, 3, 2.0), (2, 9, 2.0), (2, 6, 1.5), (0, 6, 2.0)]:
        assert lib.hqs_plan3d_create(ctypes.byref(h), None, ctypes.c_int64(0), 8, 16, 16, L, fake, W,
                                     ctypes.c_float(sg), None) == -1
    # points without a trajectory, maps missing, no output handle
    assert lib.hqs_plan3d_create(ctypes.byref(h), None, ctypes.c_int64(10), 8, 16, 16, 2, fake, 6, two, None) == -1
    assert lib.hqs_plan3d_create(ctypes.byref(h), None, ctypes.c_int64(0), 8, 16, 16, 2, None, 6, two, None) == -1
    assert lib.hqs_plan3d_create(None, None, ctypes.c_int64(0), 8, 16, 16, 2, fake, 6, two, None) == -1
    for fn in ("hqs_forward3d", "hqs_adjoint3d", "hqs_toeplitz_normal3d"):
        assert getattr(lib, fn)(None, fake, fake, None) == -1
    assert lib.hqs_precond_apply3d(None, ctypes.c_float(1.0), ctypes.c_float(0.1), fake, fake, None) == -1


def test_noalloc_wrapper_checks_shapes_before_any_launch():
    """hqs_precond_apply_noalloc takes n alone, so the binding is the only
    guard of the buffers' sizes: a non-square r, or a symbol or output of
    another size or type, is rejected before the library is called (CPU
    tensors here: the check runs before the device-pointer check).  The C
    entry point itself rejects unsupported n before any CUDA call."""
    import pytest
    torch = pytest.importorskip("torch")
    import paper_2411_01955_gb300 as hq
    from paper_2411_01955_gb300 import build
    c64, f32 = torch.complex64, torch.float32
    ok_r, ok_l = torch.zeros((64, 64), dtype=c64), torch.zeros((64, 64), dtype=f32)
    bad = [
        (torch.zeros((64, 128), dtype=c64), ok_l, ok_r.clone()),       # non-square r
        (torch.zeros((2, 64, 64), dtype=c64), ok_l, ok_r.clone()),     # batched r
        (torch.zeros((48, 48), dtype=c64), torch.zeros((48, 48), dtype=f32), torch.zeros((48, 48), dtype=c64)),
        (ok_r, torch.zeros((32, 32), dtype=f32), ok_r.clone()),        # smaller symbol
        (ok_r, ok_l, torch.zeros((32, 64), dtype=c64)),                # smaller output
        (ok_r, ok_l.to(torch.float64), ok_r.clone()),                  # symbol of another type
        (ok_r, ok_l, torch.zeros((64, 64), dtype=torch.complex128)),   # output of another type
    ]
    for r, lam, z in bad:
        with pytest.raises((ValueError, TypeError)):
            hq.precond_apply_noalloc(r, lam, 1.0, 0.1, z)
    lib = ctypes.CDLL(build.build())
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    for n in (0, 8, 48, 512, 1024):
        assert lib.hqs_precond_apply_noalloc(fake, fake, n, ctypes.c_float(1.0), ctypes.c_float(0.1),
                                             fake, None) == -1
    assert lib.hqs_precond_apply_noalloc(fake, fake, 64, ctypes.c_float(1.0), ctypes.c_float(0.0),
                                         fake, None) == -1


def test_batch_wrappers_check_counts_and_shapes_before_any_launch():
    # the C side cannot see tensor sizes, so the binding rejects a missing slice or a
    # wrongly sized image / k-space array before it touches a pointer (CPU tensors
    # reach the check; a launch would need CUDA ones)
    import pytest
    torch = pytest.importorskip("torch")
    import types
    import paper_2411_01955_gb300 as hq
    c64 = torch.complex64
    plans = [types.SimpleNamespace(ny=32, nx=32, coils=4, npoints=100),
             types.SimpleNamespace(ny=64, nx=64, coils=2, npoints=300)]
    bt = object.__new__(hq.Batch)
    bt.plans, bt.handle = plans, None
    img = [torch.zeros((32, 32), dtype=c64), torch.zeros((64, 64), dtype=c64)]
    ksp = [torch.zeros((4, 100), dtype=c64), torch.zeros((2, 300), dtype=c64)]
    small = [img[0], torch.zeros((32, 32), dtype=c64)]
    calls = [
        lambda: bt.dc_solve(img[:1], img, 1.0, 0.1),
        lambda: bt.dc_solve(img, small, 1.0, 0.1),
        lambda: bt.run(ksp, small, [0.1], [0.1]),
        lambda: bt.run([ksp[0], torch.zeros((2, 200), dtype=c64)], img, [0.1], [0.1]),
        lambda: bt.run(ksp, img, [0.1, 0.1], [0.1], K=2),
        lambda: bt.toeplitz_normal(img, small),
        lambda: bt.forward(img, ksp[:1]),
        lambda: bt.adjoint_axpy(ksp, 0.1, small, img),
    ]
    for call in calls:
        with pytest.raises(ValueError):
            call()


def test_plan_wrappers_check_element_counts_before_any_launch():
    # every single-plan entry point sizes its buffers from the plan: a tensor holding
    # another number of elements, or a schedule shorter than K, is rejected before a
    # pointer reaches the library
    import types
    import pytest
    torch = pytest.importorskip("torch")
    import paper_2411_01955_gb300 as hq
    c64 = torch.complex64
    p2 = types.SimpleNamespace(ny=16, nx=16, coils=3, npoints=50, handle=None)
    p3 = types.SimpleNamespace(shape=(4, 8, 8), coils=2, npoints=40, handle=None)
    img, ksp = torch.zeros((16, 16), dtype=c64), torch.zeros((3, 50), dtype=c64)
    vol, ksp3 = torch.zeros((4, 8, 8), dtype=c64), torch.zeros((2, 40), dtype=c64)
    small, big = torch.zeros((16, 8), dtype=c64), torch.zeros((3, 51), dtype=c64)
    calls = [
        lambda: hq.forward(p2, small, ksp),
        lambda: hq.forward(p2, img, big),
        lambda: hq.adjoint(p2, big, img),
        lambda: hq.adjoint_axpy(p2, ksp, 0.1, small, img),
        lambda: hq.toeplitz_normal(p2, img, small),
        lambda: hq.precond_apply(p2, 1.0, 0.1, small, img),
        lambda: hq.dc_solve(p2, 1.0, 0.1, img, small),
        lambda: hq.hqs_run(p2, big, img, [0.1], [0.1]),
        lambda: hq.hqs_run(p2, ksp, img, [0.1, 0.1], [0.1]),
        lambda: hq.pgd_run(p2, ksp, small, [0.1], [0.1]),
        lambda: hq.learned_precond_apply(p2, 1.0, 0.1, img, small),
        lambda: hq.gaussian_denoise(img, small, 1.0),
        lambda: hq.plan_create(torch.zeros((50, 3)), 16, 16, torch.zeros((3, 16, 16), dtype=c64)),
        lambda: hq.forward3d(p3, vol[:2], ksp3),
        lambda: hq.adjoint3d(p3, ksp, vol),
        lambda: hq.toeplitz_normal3d(p3, vol, small),
        lambda: hq.plan3d_khat(p3, torch.zeros((4, 8, 8))),
        lambda: hq.precond_apply3d(p3, 1.0, 0.1, vol, vol[1:]),
        lambda: hq.dc_solve3d(p3, 1.0, 0.1, vol[:, :4], vol),
        lambda: hq.hqs_run3d(p3, ksp3, vol, [0.1, 0.1], [0.1], K=2),
        lambda: hq.gaussian_denoise3d(vol, vol[:3], 1.0),
    ]
    for call in calls:
        with pytest.raises(ValueError):
            call()
