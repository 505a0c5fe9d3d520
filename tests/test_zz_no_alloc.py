"""The allocation-free entry point (celeste_elbo_grad_hess_noalloc).

It serves callers that must not allocate device memory (a locked or
defragmenting memory pool, a host program that owns every allocation), so
it keeps its intermediates in one fixed device array shared by all calls.
This file is collected last: the entry point must give the same results as
celeste_elbo_grad_hess whether it runs alone in a fresh process or after
every other test, and on consecutive calls that reuse the shared array.
"""
import numpy as np
import pytest
import torch

import fields

pytestmark = pytest.mark.gpu

TOL_ELBO = 1e-5      # the parity tests' tolerances
TOL_DERIV = 1e-4


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _outputs(n, dev):
    return (torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n, 27), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n, 27, 27), float("nan"), dtype=torch.float64, device=dev))


def _close(a, b):
    e, er, g, H = (t.cpu().numpy() for t in a)
    re, rer, rg, rH = (t.cpu().numpy() for t in b)
    assert np.all(np.abs(e - re) <= TOL_ELBO * np.abs(re))
    assert np.all(np.abs(er - rer) <= TOL_ELBO * np.maximum(np.abs(rer), 1.0))
    gs = np.abs(rg).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - rg) <= TOL_DERIV * (np.abs(rg) + 1e-3 * gs))
    hs = np.abs(rH).reshape(len(rH), -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(H - rH) <= TOL_DERIV * (np.abs(rH) + 1e-3 * hs))


def test_noalloc_matches_existing_entry_point_on_consecutive_calls(cel):
    p = fields.batched(seed=61, n_sources=9, min_side=15, max_side=45, max_images_per_band=2,
                       max_neighbours=4)
    dev = torch.device("cuda")
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    model = p.model
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    for sources in (list(range(p.n_sources)), [7, 2, 5]):
        plan = cel.Plan(ctx, dp, sources)
        ref = cel.elbo_grad_hess(plan)
        ctx.synchronize()
        out = _outputs(len(sources), dev)
        cel.elbo_grad_hess_noalloc(model, dp, sources, out, device_error=err)
        torch.cuda.synchronize()
        assert int(err[0]) == 0
        _close(out, ref)


def test_noalloc_rejects_requests_beyond_its_limits(cel):
    p = fields.plain_source(side=15)
    dp = cel.DeviceProblem(p)
    dev = torch.device("cuda")
    too_many = list(range(1025))      # more sources than CELESTE_NOALLOC_MAX_SOURCES
    with pytest.raises(cel.CelesteError, match="-8"):
        cel.elbo_grad_hess_noalloc(p.model, dp, too_many, _outputs(1025, dev))
