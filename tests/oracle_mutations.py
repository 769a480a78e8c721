"""Mutation scan of the FP64 oracle (test infrastructure, run by hand).

Plants one plausible mistake at a time (a wrong sign, scale, index or axis, a
transposed operand, a dropped term or clamp) in a scratch copy of `oracle/`
and runs the CPU pin suites (`test_oracle_pins.py`, `test_oracle_pins_3d.py`)
on that copy; a mistake the pins do not catch is reported as NOT CAUGHT.  The
repository's own files are never modified.

    python tests/oracle_mutations.py [--scratch DIR] [--jobs J] [index ...]

Expected: every mutation caught except two conventions that no fact fixes,
the Strang symbol's choice of the d = -N/2 offset (the first reading of the
preconditioner, not on the path) and the 0.1-pixel identity threshold of the
smoothing denoiser.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file under oracle/, exact text, replacement, label); each text occurs once
M = [
    # kb
    ("kb.py", "term = term * q / (m * m)", "term = term * q / m", "i0 series term"),
    ("kb.py", "s = 1.0 - (2.0 * t / W) ** 2", "s = 1.0 - (t / W) ** 2", "phi support"),
    ("kb.py", "r2 = b * b - (math.pi * W * nu) ** 2", "r2 = b * b - (2 * math.pi * W * nu) ** 2", "phihat freq scale"),
    ("kb.py", "out[pos] = W * np.sinh(r) / r", "out[pos] = np.sinh(r) / r", "phihat dropped W"),
    ("kb.py", "(sigma - 0.5) ** 2 - 0.8", "(sigma - 0.5) ** 2 - 0.9", "beta constant"),
    # nudft
    ("nudft.py", "return np.arange(n, dtype=np.float64) - n // 2", "return np.arange(n, dtype=np.float64) - (n - 1) // 2", "centring"),
    ("nudft.py", "return y / np.sqrt(ny * nx)", "return y / (ny * nx)", "forward scale"),
    ("nudft.py", "Ex, Ey = _axis_matrices(traj, ny, nx, +1.0)", "Ex, Ey = _axis_matrices(traj, ny, nx, -1.0)", "adjoint sign"),
    ("nudft.py", "Ex = np.exp(sign * 1j * np.outer(k[:, 0], centred(nx)))", "Ex = np.exp(sign * 1j * np.outer(k[:, 1], centred(nx)))", "kx/ky swap"),
    ("nudft.py", "x += np.conj(smaps[l]) * img", "x += smaps[l] * img", "nudft adjoint conj"),
    ("nudft.py", "    Ex, Ey = _axis_matrices(traj, ny, nx, -1.0)\n", "    Ex, Ey = _axis_matrices(traj, nx, ny, -1.0)\n", "forward axes swapped"),
    # nufft
    ("nufft.py", "i0 = np.ceil(u - W / 2.0)", "i0 = np.floor(u - W / 2.0)", "tap origin"),
    ("nufft.py", "return 1.0 / kb.phihat(centred(n) / G, W, b)", "return 1.0 / kb.phihat(centred(n) / n, W, b)", "apodisation scale"),
    ("nufft.py", "acc += wy[:, a] * wx[:, c] * Ghat[iy[:, a], ix[:, c]]", "acc += wy[:, a] * wx[:, c] * Ghat[ix[:, c], iy[:, a]]", "interp transposed"),
    ("nufft.py", "x += np.conj(smaps[l]) * V[np.ix_(py, px)]", "x += smaps[l] * V[np.ix_(py, px)]", "adjoint conj"),
    ("nufft.py", "V = np.fft.ifft2(H) * (Gy * Gx)", "V = np.fft.ifft2(H)", "adjoint scale"),
    ("nufft.py", "flat = iy[:, a] * Gx + ix[:, c]", "flat = ix[:, c] * Gy + iy[:, a]", "spread transposed"),
    ("nufft.py", "wx = kb.phi(dx[:, None] - w[None, :], W, b)", "wx = kb.phi(dx[:, None] + w[None, :], W, b)", "tap weight sign"),
    ("nufft.py", "grid[np.ix_(py, px)] = smaps[l] * x * apy[:, None] * apx[None, :]", "grid[np.ix_(py, px)] = smaps[l] * x * apy[None, :] * apx[:, None]", "apod axes swapped"),
    # toeplitz
    ("toeplitz.py", "Ey = np.exp(1j * np.outer(k[:, 1], dy))", "Ey = np.exp(-1j * np.outer(k[:, 1], dy))", "kernel sign y"),
    ("toeplitz.py", "c = (Ey.T @ Ex) / (ny * nx)", "c = (Ey.T @ Ex) / np.sqrt(ny * nx)", "kernel scale"),
    ("toeplitz.py", "    c[ny, :] = 0.0\n    c[:, nx] = 0.0\n", "", "kernel -N zeroing dropped"),
    ("toeplitz.py", "    return K.real", "    return np.abs(K)", "khat abs"),
    ("toeplitz.py", "w = np.fft.ifft2(Kh * np.fft.fft2(pad))[:ny, :nx]", "w = np.fft.fft2(Kh * np.fft.ifft2(pad))[:ny, :nx]", "normal fft order"),
    ("toeplitz.py", "out += np.conj(smaps[l]) * w", "out += smaps[l] * w", "normal conj"),
    ("toeplitz.py", "for dy, wy in ((qy, (ny - qy) / ny), (qy - ny, qy / ny)):", "for dy, wy in ((qy, (ny - qy) / ny), (qy - ny, (ny - qy) / ny)):", "chan weight"),
    ("toeplitz.py", "return np.fft.fft2(chan_column(c, ny, nx)).real", "return np.fft.ifft2(chan_column(c, ny, nx)).real", "chan symbol fft"),
    ("toeplitz.py", "dy = np.arange(ny) - ny // 2", "dy = np.arange(ny) - (ny - 1) // 2", "strang centring"),
    ("toeplitz.py", "return 1.0 / np.sqrt(np.maximum(s, 0.25 * b))", "return 1.0 / np.sqrt(np.maximum(s, 0.5 * b))", "precond floor"),
    ("toeplitz.py", "    c[ny, :] = 0.0\n", "    c[ny - 1, :] = 0.0\n", "kernel zeroed row off by one"),
    # solvers
    ("solvers.py", "        beta = rz_new / rz\n", "        beta = rz / rz_new\n", "pcg beta inverted"),
    ("solvers.py", "        r = r - alpha * q\n        it += 1\n        hist.append(float(np.linalg.norm(r)) / bnorm)\n        if hist[-1] <= tol:\n            status = \"ok\"",
     "        r = r + alpha * q\n        it += 1\n        hist.append(float(np.linalg.norm(r)) / bnorm)\n        if hist[-1] <= tol:\n            status = \"ok\"", "pcg residual sign"),
    ("solvers.py", "        p = z + beta * p\n    if tol == 0.0", "        p = r + beta * p\n    if tol == 0.0", "pcg direction unpreconditioned"),
    ("solvers.py", "    p = z.copy()\n    rz = vdot_re(r, z)\n    it = 0\n    status", "    p = r.copy()\n    rz = vdot_re(r, z)\n    it = 0\n    status", "pcg first direction"),
    ("solvers.py", "alpha = vdot_re(p, r) / pq", "alpha = vdot_re(p, q) / pq", "fcg alpha"),
    ("solvers.py", "if it >= stall_window and hist[-1] > stall_factor", "if it >= stall_window and hist[-1] < stall_factor", "fcg stall sign"),
    ("solvers.py", "            beta = vdot_re(z, r - r_old) / rz", "            beta = vdot_re(z, r + r_old) / rz", "fcg beta PR sign"),
    ("solvers.py", "        x, inf2 = pcg(apply_H, rhs, x, apply_Minv, max_iter - it, tol)", "        x, inf2 = pcg(apply_H, rhs, np.zeros_like(x), apply_Minv, max_iter - it, tol)", "fcg fallback cold start"),
    ("solvers.py", "    return 0.5 * vdot_re(x, apply_H(x)) - vdot_re(rhs, x)", "    return vdot_re(x, apply_H(x)) - vdot_re(rhs, x)", "cg energy factor"),
    ("solvers.py", "        lam_new = vdot_re(v, w)", "        lam_new = float(np.linalg.norm(w)) ** 0.5", "power iteration rayleigh"),
    # hqs
    ("hqs.py", "return 1.0 + c1 * mu, c0 * mu", "return 1.0 - c1 * mu, c0 * mu", "prox a sign"),
    ("hqs.py", "return 1.0 + c1 * mu, c0 * mu", "return 1.0 + c1 * mu, mu", "prox b drops c0"),
    ("hqs.py", "        rhs = b0 + mu[k] * c0 * x\n", "        rhs = b0 + mu[k] * x\n", "hqs rhs drops c0"),
    ("hqs.py", "            rhs = rhs + mu[k] * c1 * apply_AHA(x)", "            rhs = rhs - mu[k] * c1 * apply_AHA(x)", "hqs rhs c1 sign"),
    ("hqs.py", "        u, _ = solvers.pcg(H, rhs, x, Minv, max_iter=cg_iters, tol=0.0)", "        u, _ = solvers.pcg(H, rhs, np.zeros_like(x), Minv, max_iter=cg_iters, tol=0.0)", "hqs cold start"),
    ("hqs.py", "        x = denoiser(u, float(sigma[k]))\n        hist.append", "        x = denoiser(u, float(sigma[0]))\n        hist.append", "hqs sigma index"),
    ("hqs.py", "    return g / g.sum()", "    return g", "gauss taps unnormalised"),
    ("hqs.py", "    g = np.exp(-(i * i) / (2.0 * s * s))", "    g = np.exp(-(i * i) / (s * s))", "gauss width"),
    ("hqs.py", "    r = int(math.ceil(3.0 * s))", "    r = int(math.ceil(2.0 * s))", "gauss radius"),
    ("hqs.py", "    if s < 0.1:", "    if s < 0.01:", "gauss identity threshold"),
    ("hqs.py", "    return kappa * sigma_k / sigma_0", "    return kappa * sigma_0 / sigma_k", "denoiser std inverted"),
    ("hqs.py", "        Pg = c0 * g + (c1 * apply_AHA(g) if c1 != 0.0 else 0.0)", "        Pg = g + (c1 * apply_AHA(g) if c1 != 0.0 else 0.0)", "pgd drops c0"),
    ("hqs.py", "        x = denoiser(x - gamma[k] * Pg, float(sigma[k]))", "        x = denoiser(x + gamma[k] * Pg, float(sigma[k]))", "pgd step sign"),
    ("hqs.py", "        g = apply_AHA(x) - b0", "        g = apply_AHA(x) + b0", "pgd grad sign"),
    # convnet
    ("convnet.py", "patch = xp[:, :, dy:dy + H, dx:dx + Wd]", "patch = xp[:, :, dx:dx + H, dy:dy + Wd]", "conv taps transposed"),
    ("convnet.py", "dxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum(\"oi,nohw->nihw\", W[:, :, dy, dx], dz)", "dxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum(\"oi,nohw->nihw\", W[:, :, 2 - dy, 2 - dx], dz)", "input grad flipped"),
    ("convnet.py", "            dz = da * (acts[li] > 0.0)", "            dz = da", "relu grad dropped"),
    ("convnet.py", "    dz = 2.0 * diff / (N * tn[:, None, None, None])", "    dz = diff / (N * tn[:, None, None, None])", "loss grad factor"),
    ("convnet.py", "    mh = m / (1 - b1 ** t)", "    mh = m", "adam bias correction"),
    ("convnet.py", "    return zdc + s * (out[0, 0] + 1j * out[0, 1])", "    return zdc + (out[0, 0] + 1j * out[0, 1])", "learned scale"),
    ("convnet.py", "        h = z if li == len(params) - 1 else np.maximum(z, 0.0)", "        h = np.maximum(z, 0.0)", "relu on last layer"),
    ("convnet.py", "    s = math.sqrt(float(np.mean(np.abs(zdc) ** 2)))", "    s = float(np.mean(np.abs(zdc)))", "learned scale mean abs"),
    ("convnet.py", "    v = b2 * v + (1 - b2) * grad * grad", "    v = b2 * v + (1 - b2) * np.abs(grad)", "adam second moment"),
    ("convnet.py", "    return vec - lr * mh / (np.sqrt(vh) + eps), m, v", "    return vec - lr * mh / np.sqrt(vh + eps), m, v", "adam eps placement"),
    ("convnet.py", "    return dW, dz.sum(axis=(0, 2, 3))", "    return dW, dz.sum(axis=(0, 2, 3)) / dz.shape[0]", "bias grad scale"),
    # smaps
    ("smaps.py", "0.54 + 0.46 * np.cos(2.0 * np.pi * u / width)", "0.54 + 0.46 * np.cos(np.pi * u / width)", "hamming period"),
    ("smaps.py", "    return h[:, 0] * h[:, 1]", "    return h[:, 0]", "hamming separable"),
    ("smaps.py", "    rss = np.sqrt(np.sum(np.abs(c) ** 2, axis=0))", "    rss = np.sum(np.abs(c), axis=0)", "rss norm"),
    ("smaps.py", "        w = w * np.asarray(dcf, dtype=np.float64)", "        w = w / np.asarray(dcf, dtype=np.float64)", "dcf inverted"),
    ("smaps.py", "    u = np.asarray(traj, dtype=np.float64) * n / (2.0 * np.pi)", "    u = np.asarray(traj, dtype=np.float64) * n / np.pi", "window units"),
    ("smaps.py", "    mask = rss >= thresh * rss.max()", "    mask = rss >= thresh", "mask threshold absolute"),
    # nufft3d
    ("nufft3d.py", "    Ez = np.exp(sign * 1j * np.outer(k[:, 2], centred(nz)))   # (M, nz)", "    Ez = np.exp(sign * 1j * np.outer(k[:, 2], centred(nx)))   # (M, nz)", "3d nudft z uses nx"),
    ("nufft3d.py", "        sy = np.einsum(\"zyj,jy->zj\", sx, Ey)           # sum over n_y", "        sy = np.einsum(\"zyj,jy->zj\", sx, np.conj(Ey))           # sum over n_y", "3d nudft y sign"),
    ("nufft3d.py", "    return y / math.sqrt(nz * ny * nx)\n\n\ndef nudft_adjoint", "    return y / (nz * ny * nx)\n\n\ndef nudft_adjoint", "3d nudft scale"),
    ("nufft3d.py", "    return (apodisation(nz, G[2], W, b)[:, None, None] * apodisation(ny, G[1], W, b)[None, :, None]", "    return (apodisation(nz, G[0], W, b)[:, None, None] * apodisation(ny, G[1], W, b)[None, :, None]", "3d apod z grid"),
    ("nufft3d.py", "                    acc += wz[:, c] * wy[:, a] * wx[:, e] * Gh[iz[:, c], iy[:, a], ix[:, e]]", "                    acc += wz[:, c] * wy[:, a] * wx[:, e] * Gh[ix[:, e], iy[:, a], iz[:, c]]", "3d interp transposed"),
    ("nufft3d.py", "                flat = (iz[:, c] * G[1] + iy[:, a]) * G[0] + ix[:, e]", "                flat = (iz[:, c] * G[0] + iy[:, a]) * G[1] + ix[:, e]", "3d spread strides"),
    ("nufft3d.py", "        V = np.fft.ifftn(H) * H.size ", "        V = np.fft.ifftn(H) ", "3d adjoint scale"),
    ("nufft3d.py", "    Ez = np.exp(1j * np.outer(k[:, 2], _circ_offsets(nz)))   # (M, 2nz)", "    Ez = np.exp(-1j * np.outer(k[:, 2], _circ_offsets(nz)))   # (M, 2nz)", "3d kernel z sign"),
    ("nufft3d.py", "    c[:, :, nx] = 0.0\n", "", "3d kernel x plane kept"),
    ("nufft3d.py", "        w = np.fft.ifftn(Kh * np.fft.fftn(pad))[:nz, :ny, :nx]", "        w = np.fft.ifftn(Kh * np.fft.fftn(pad))[nz:, :ny, :nx]", "3d normal crop"),
    ("nufft3d.py", "        choices.append(((np.mod(q, 2 * n), (n - q) / n), (np.mod(q - n, 2 * n), q / n)))", "        choices.append(((np.mod(q, 2 * n), (n - q) / n), (np.mod(q - n, 2 * n), (n - q) / n)))", "3d chan weight"),
    ("nufft3d.py", "    return np.fft.fftn(chan_column(c, shape)).real", "    return np.fft.ifftn(chan_column(c, shape)).real", "3d chan fft"),
    ("nufft3d.py", "    return np.fft.ifftn(np.fft.fftn(v) / np.sqrt(np.maximum(s, 0.25 * b)))", "    return np.fft.ifftn(np.fft.fftn(v) / np.maximum(s, 0.25 * b))", "3d precond full inverse"),
    ("nufft3d.py", "    s = a * np.maximum(lam, 0.0) + b\n    return np.fft.ifftn", "    s = a * lam + b\n    return np.fft.ifftn", "3d precond no clamp"),
]


def run_one(i, scratch):
    f, old, new, label = M[i]
    d = os.path.join(scratch, str(i))
    if os.path.exists(d):
        shutil.rmtree(d)
    os.makedirs(d)
    for sub in ("oracle", "synth"):
        shutil.copytree(os.path.join(REPO, sub), os.path.join(d, sub), ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(d, "tests"))
    for t in ("conftest.py", "helpers.py", "test_oracle_pins.py", "test_oracle_pins_3d.py"):
        shutil.copy(os.path.join(REPO, "tests", t), os.path.join(d, "tests", t))
    shutil.copy(os.path.join(REPO, "pytest.ini"), os.path.join(d, "pytest.ini"))
    p = os.path.join(d, "oracle", f)
    with open(p) as fh:
        s = fh.read()
    if s.count(old) != 1:
        shutil.rmtree(d)
        return f"pattern found {s.count(old)} times (table out of date)"
    with open(p, "w") as fh:
        fh.write(s.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_pins_3d.py"],
                       cwd=d, capture_output=True, text=True, timeout=900)
    shutil.rmtree(d)
    if r.returncode == 0:
        return "NOT CAUGHT"
    failed = [l for l in r.stdout.splitlines() if l.startswith(("FAILED", "ERROR"))]
    return "caught by " + (failed[0].split("::")[-1].split(" ")[0] if failed else "an error")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scratch", default=None, help="directory for the scratch copies (default: a new temporary one)")
    ap.add_argument("--jobs", type=int, default=6)
    ap.add_argument("index", type=int, nargs="*")
    args = ap.parse_args()
    scratch = args.scratch or tempfile.mkdtemp(prefix="oracle_mutations_")
    os.makedirs(scratch, exist_ok=True)
    sel = args.index or list(range(len(M)))
    caught = 0
    with ThreadPoolExecutor(args.jobs) as ex:
        for i, res in zip(sel, ex.map(lambda j: run_one(j, scratch), sel)):
            caught += res.startswith("caught")
            print(f"{i:3d} {M[i][0]:12s} {M[i][3]:32s} {res}", flush=True)
    print(f"{caught} of {len(sel)} caught")
    if not args.scratch:
        shutil.rmtree(scratch, ignore_errors=True)


if __name__ == "__main__":
    main()
