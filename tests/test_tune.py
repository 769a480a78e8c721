"""Autotuner: cache and selection logic on the CPU; on the GPU, every
candidate launch shape gives the same operator (to float rounding order) and
the tuner applies and caches its winners."""
import numpy as np
import pytest

from paper_2411_01955_gb300 import tune


def test_cache_roundtrip_and_key(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tune.load_cache(path) == {}
    k1 = tune.cache_key("GB300", 320, 16, 32768, 6, 2.0)
    k2 = tune.cache_key("GB300", 320, 16, 32768, 4, 2.0)
    assert k1 != k2
    tune.store_cache(path, k1, tune.Tuning(32, 8, 152))
    tune.store_cache(path, k2, tune.Tuning(8, 2, 0))
    data = tune.load_cache(path)
    assert tune.Tuning(**data[k1]) == tune.Tuning(32, 8, 152)
    assert tune.Tuning(**data[k2]) == tune.Tuning(8, 2, 0)
    with open(path, "w") as f:
        f.write("{not json")
    assert tune.load_cache(path) == {}


def test_valid_tiles_and_pick():
    assert tune.valid_tiles(640, 6) == [8, 16, 32]
    assert tune.valid_tiles(40, 6) == [8]           # 40 is not a multiple of 16 or 32
    assert tune.valid_tiles(16, 6) == [8, 16]       # one 16 tile covers the whole grid
    assert tune.valid_tiles(64, 8) == [8, 16, 32]
    assert tune.pick({8: 2.0, 16: 1.0, 32: 1.5}) == 16
    assert tune.pick({(2, 0): 1.0, (4, 0): 1.0}) == (2, 0)   # ties: first listed


@pytest.mark.gpu
def test_retile_keeps_adjoint_and_autotune_applies(tmp_path):
    import torch
    import synth
    from helpers import make_plan, quantised, rel, to_dev, to_host
    from oracle import nufft
    import paper_2411_01955_gb300 as hq
    case = quantised(dict(n=128, L=5, W=6, sigma=2.0, x=synth.phantom(3, 128),
                          smaps=synth.coil_maps(3, 128, 5), traj=synth.traj_spiral(6, 700, 128)))
    plan, _, _ = make_plan(case)
    rng = np.random.default_rng(4)
    M = case["traj"].shape[0]
    y = (rng.normal(size=(5, M)) + 1j * rng.normal(size=(5, M))).astype(np.complex64)
    want = nufft.adjoint(y.astype(np.complex128), case["smaps"], case["traj"], 6, 2.0)
    x = torch.empty((128, 128), dtype=torch.complex64, device="cuda")
    yd = to_dev(y)
    for tile in (8, 16, 32, 8):
        hq.plan_set_tuning(plan, hq.HQS_TUNE_SPREAD_TILE, tile)
        assert plan.info().tile == tile
        hq.adjoint(plan, yd, x)
        assert rel(to_host(x), want) <= 1e-5, tile
    with pytest.raises(hq.HqsError):
        hq.plan_set_tuning(plan, hq.HQS_TUNE_SPREAD_TILE, 12)
    path = str(tmp_path / "tune.json")
    t = tune.autotune(plan, cache_path=path, reps=2, solve_iters=3)
    assert plan.info().tile == t.spread_tile
    assert len(tune.load_cache(path)) == 1
    # a fresh plan of the same shape takes the cached winners without timing
    plan2, _, _ = make_plan(case)
    assert tune.autotune(plan2, cache_path=path) == t
    assert plan2.info().tile == t.spread_tile
    hq.adjoint(plan2, yd, x)
    assert rel(to_host(x), want) <= 1e-5
