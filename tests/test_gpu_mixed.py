"""Mixed-precision A^H A (BF16x3 / FP16x3 tensor-core DFT-GEMM passes) against
the FP64 oracle: the relative L2 error of every pass's intermediate and of
the operator, the mixed-precision DC solve, and the unsupported shapes.

Error model (the bound each check derives from).  A value split as
hi + lo with p-bit significands (p = 8 for BF16, 11 for FP16; FP16 lo parts
are kept scaled by 2^11 so they do not sink into subnormals) is represented
to |x - hi - lo| <= 2^-2p |x|, and the dropped lo*lo product is <= 2^-2p of
the product, so one pass adds a relative error of about 3 * 2^-2p on top of
the FP32 accumulation (2^-24 sqrt(K)); the passes add up.  The checks allow
four times that per pass: BF16x3 (2^-16 = 1.5e-5) x 4 / pass, FP16x3
(2^-22 = 2.4e-7) x 4 / pass plus the FP32 floor of 2e-6.
"""
import numpy as np
import pytest

import synth
from helpers import make_plan, quantised, rel, to_dev, to_host
from oracle import nufft, solvers, toeplitz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def hq():
    import paper_2411_01955_gb300 as m
    return m


CASES = {
    "tiny": lambda: quantised(synth.tiny_case(0)),
    # coil count padded 5 -> 8 in the last pass, 640 GEMM rows (5 tiles)
    "n128_l5": lambda: quantised(dict(n=128, L=5, W=6, sigma=2.0, x=synth.phantom(11, 128),
                                      smaps=synth.coil_maps(11, 128, 5), traj=synth.traj_spiral(8, 900, 128))),
    "brain": lambda: quantised(dict(n=320, L=16, W=6, sigma=2.0, x=synth.phantom(3, 320),
                                    smaps=synth.coil_maps(3, 320, 16), traj=synth.traj_spiral(16, 2048, 320))),
}


def pass_bound(precision, passes):
    per = 4 * 2.0 ** -16 if precision == 1 else 4 * 2.0 ** -22 + 2e-6
    return per * passes


def oracle_stages(case):
    n, L = case["n"], case["L"]
    K0 = toeplitz.khat(toeplitz.kernel(case["traj"], n, n))
    pad = np.zeros((L, 2 * n, 2 * n), dtype=np.complex128)
    pad[:, :n, :n] = case["smaps"] * case["x"]
    s1 = np.fft.fft(pad[:, :n, :], axis=-1)
    s2 = K0 * np.fft.fft2(pad)
    s3 = np.fft.ifft(s2, axis=-2)[:, :n, :]
    s4 = toeplitz.normal(case["x"], case["smaps"], K0)
    return [s1, s2, s3, s4]


@pytest.mark.parametrize("precision", [1, 2], ids=["bf16x3", "fp16x3"])
@pytest.mark.parametrize("name", ["tiny", "n128_l5", "brain"])
def test_mixed_passes_match_oracle(name, precision):
    case = CASES[name]()
    n, L = case["n"], case["L"]
    plan, _, _ = make_plan(case)
    want = oracle_stages(case)
    x = to_dev(case["x"])
    shapes = [(L, n, 2 * n), (L, 2 * n, 2 * n), (L, n, 2 * n), (n, n)]
    errs = []
    for stage in (1, 2, 3, 4):
        out = torch.empty(shapes[stage - 1], dtype=torch.complex64, device="cuda")
        hq().toeplitz_stage(plan, x, precision, stage, out)
        errs.append(rel(to_host(out), want[stage - 1]))
    # the public operator gives the stage-4 result
    y = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal(plan, x, y, precision=precision)
    fp32 = torch.empty_like(y)
    hq().toeplitz_normal(plan, x, fp32)
    e32 = rel(to_host(fp32), want[3])
    print(f"{name} prec={precision}: per-pass rel L2 error {['%.2e' % e for e in errs]}, "
          f"operator {rel(to_host(y), want[3]):.2e} (FP32 path {e32:.2e})")
    for s, e in enumerate(errs, start=1):
        assert e <= pass_bound(precision, s), (s, e)
    # the FP32 in-house FFT path at the same size (640-point lines at 320^2)
    assert e32 <= 1e-5
    assert rel(to_host(y), want[3]) <= pass_bound(precision, 4)


@pytest.mark.parametrize("precision", [1, 2], ids=["bf16x3", "fp16x3"])
def test_mixed_dc_solve_converges(precision):
    case = CASES["n128_l5"]()
    n, L, mu = case["n"], case["L"], 1e-2
    plan, _, _ = make_plan(case)
    K0 = toeplitz.khat(toeplitz.kernel(case["traj"], n, n))
    y = nufft.forward(case["x"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = nufft.adjoint(y, case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: toeplitz.normal(v, case["smaps"], K0) + mu * v
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=200, rel_tol=1e-4, precision=precision)
    x32 = torch.zeros_like(x)
    i32 = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x32, max_iter=200, rel_tol=1e-4)
    got = to_host(x)
    true_res = float(np.linalg.norm(rhs - H(got)) / np.linalg.norm(rhs))
    print(f"prec={precision}: {info.iterations} iterations (FP32 {i32.iterations}), recursion residual "
          f"{info.rel_residual:.2e}, true residual {true_res:.2e}, vs FP32 solution "
          f"{rel(got, to_host(x32)):.2e}")
    assert info.status == 0 and info.rel_residual <= 1e-4
    # the recursion drifts from the true residual by at most the operator error times ||x|| ||H||/||rhs||
    assert true_res <= 1e-4 + 50 * pass_bound(precision, 4)
    assert abs(info.iterations - i32.iterations) <= max(3, i32.iterations // 5)


def test_mixed_unsupported_shapes():
    case = quantised(synth.odd_case(0))        # n = 16: not a multiple of 64
    plan, _, _ = make_plan(case)
    x = to_dev(case["x"])
    y = torch.empty_like(x)
    with pytest.raises(hq().HqsError) as e:
        hq().toeplitz_normal(plan, x, y, precision=1)
    assert e.value.status == hq().HQS_ERR_UNSUPPORTED
