"""The allocation-free preconditioner apply (for callers that may not allocate
device memory, e.g. a service that reserves all GPU memory at start-up) must
give what the plan-based entry point gives, on two calls in a row.  This file
is collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import synth
from helpers import make_plan, quantised, rel, to_dev, to_host
from oracle import toeplitz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def hq():
    import paper_2411_01955_gb300 as m
    return m


@pytest.mark.parametrize("n,L,spokes", [(64, 4, 16), (320, 8, 64)])
def test_noalloc_precond_matches_plan_entry_point(n, L, spokes):
    case = dict(n=n, L=L, W=4, sigma=2.0, x=synth.phantom(3, n),
                smaps=synth.coil_maps(3, n, L), traj=synth.traj_radial(spokes, 2 * n))
    case = quantised(case)
    plan, _, _ = make_plan(case)
    # the caller supplies the density symbol (here from the FP64 oracle, in float32)
    lam = toeplitz.chan_symbol(toeplitz.kernel(case["traj"], n, n), n, n)
    lam_d = torch.from_numpy(lam.astype(np.float32)).cuda()
    r = to_dev(case["x"])
    for a, b in [(1.0, 1e-2), (0.9, 0.2)]:
        z_ref = torch.empty_like(r)
        hq().precond_apply(plan, a, b, r, z_ref)
        outs = []
        for _ in range(2):   # two calls in a row share the static scratch
            z = torch.full_like(r, complex(3.0, -1.0))
            hq().precond_apply_noalloc(r, lam_d, a, b, z)
            outs.append(to_host(z))
        for z in outs:
            assert rel(z, to_host(z_ref)) <= TOL
        assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    r = torch.zeros((512, 512), dtype=torch.complex64, device="cuda")
    lam = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(hq().HqsError) as ei:
        hq().precond_apply_noalloc(r, lam, 1.0, 0.1, r.clone())
    assert ei.value.status == hq().HQS_ERR_INVALID_ARG
