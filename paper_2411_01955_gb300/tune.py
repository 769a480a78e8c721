"""Autotuner for the per-plan launch shapes, with a JSON cache.

Three knobs change how work is cut into launches, never what is computed
(beyond float rounding order of atomics and sums):

  spread_tile  edge of the shared-memory spreading tile of the adjoint (8, 16, 32)
  pc_lines     rows/columns of the preconditioner FFT per work item of the
               persistent solve (1..16)
  fused_grid   cap on the persistent solve's CTAs (0 = every resident CTA)

`autotune(plan)` times each candidate with CUDA events on the plan's own
operators (hqs_adjoint for the tile, a fixed-iteration persistent DC solve
for the other two), keeps the fastest, applies it and stores it in the cache
under a key made of the device name and the problem shape, so the next plan of
the same shape gets the winners without timing anything.
"""
from __future__ import annotations

import json
import os
from dataclasses import asdict, dataclass

from . import _lib as L

SPREAD_TILES = (8, 16, 32)
PC_LINES = (2, 4, 8)
FUSED_GRIDS = (0, 152, 228)


@dataclass
class Tuning:
    spread_tile: int = 16
    pc_lines: int = 4
    fused_grid: int = 0


def default_cache_path() -> str:
    return os.environ.get("HQS_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hqs_gb300", "tune.json"))


def cache_key(device: str, n: int, coils: int, points: int, width: int, sigma: float) -> str:
    return f"{device}|n{n}|L{coils}|M{points}|W{width}|s{sigma:g}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, t: Tuning) -> None:
    data = load_cache(path)
    data[key] = asdict(t)
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def valid_tiles(G: int, W: int) -> list[int]:
    """Spreading tiles that divide the grid and are at least half the kernel
    width (so a point's taps reach at most one neighbouring tile per side)."""
    return [t for t in SPREAD_TILES if G % t == 0 and 2 * t >= W]


def pick(timings: dict) -> object:
    """Fastest candidate; ties go to the first listed (deterministic)."""
    best, best_t = None, float("inf")
    for cand, t in timings.items():
        if t < best_t:
            best, best_t = cand, t
    return best


def apply(plan: L.Plan, t: Tuning) -> None:
    L.plan_set_tuning(plan, L.HQS_TUNE_SPREAD_TILE, t.spread_tile)
    L.plan_set_tuning(plan, L.HQS_TUNE_PC_LINES, t.pc_lines)
    L.plan_set_tuning(plan, L.HQS_TUNE_FUSED_GRID, t.fused_grid)


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps


def autotune(plan: L.Plan, cache_path: str | None = None, use_cache: bool = True,
             reps: int = 5, solve_iters: int = 10, solve_shapes: bool = True) -> Tuning:
    """Times the candidates on `plan` (or reads them from the cache), applies
    the winners to the plan and returns them.  solve_shapes=False tunes the
    spreading tile only (for plans whose solves run in the batched kernel,
    which has its own work decomposition)."""
    import torch
    info = plan.info()
    dev = torch.cuda.get_device_name()
    n, Lc, M, G, W = info.nx, info.coils, int(info.npoints), info.grid, info.kernel_width
    key = cache_key(dev, n, Lc, M, W, info.oversamp) + ("" if solve_shapes else "|tile")
    path = cache_path or default_cache_path()
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            t = Tuning(**hit)
            apply(plan, t)
            return t
    g = torch.Generator(device="cuda").manual_seed(0)
    y = torch.randn((Lc, max(M, 1)), dtype=torch.complex64, device="cuda", generator=g)[:, :M].contiguous()
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    tile_t = {}
    for tile in valid_tiles(G, W):
        L.plan_set_tuning(plan, L.HQS_TUNE_SPREAD_TILE, tile)
        tile_t[tile] = _time(lambda: L.adjoint(plan, y, x), reps)
    best = Tuning(spread_tile=pick(tile_t))
    L.plan_set_tuning(plan, L.HQS_TUNE_SPREAD_TILE, best.spread_tile)
    if not solve_shapes:
        if use_cache:
            store_cache(path, key, best)
        return best
    rhs = torch.randn((n, n), dtype=torch.complex64, device="cuda", generator=g)
    u = torch.zeros_like(rhs)

    def solve():
        L.dc_solve(plan, 1.0, 1e-2, rhs, u, max_iter=solve_iters, rel_tol=0.0,
                   mode=L.HQS_SOLVE_FUSED | L.HQS_SOLVE_X0_ZERO, want_info=False)

    shape_t = {}
    for lines in PC_LINES:
        for grid in FUSED_GRIDS:
            L.plan_set_tuning(plan, L.HQS_TUNE_PC_LINES, lines)
            L.plan_set_tuning(plan, L.HQS_TUNE_FUSED_GRID, grid)
            shape_t[(lines, grid)] = _time(solve, reps)
    best.pc_lines, best.fused_grid = pick(shape_t)
    apply(plan, best)
    if use_cache:
        store_cache(path, key, best)
    return best
