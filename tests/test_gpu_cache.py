"""The render cache: neighbour backgrounds gathered from cached renders must
be the very values the recompute path produces (same functions, same order),
through evaluation, Newton steps and the region fit."""
import numpy as np
import pytest
import torch

import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _blend():
    return fields.batched(seed=61, n_sources=24, min_side=15, max_side=41, max_images_per_band=2,
                          max_neighbours=5)


def _setup(cel, p, cache):
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p, render_cache=cache)
    plans = [cel.Plan(ctx, dp, c) for c in cel.color_classes(p)]
    if cache:
        for pl in plans:
            cel.render_cache(pl)
    return ctx, dp, plans


def test_cached_background_and_derivatives_are_identical(cel):
    p = _blend()
    assert p.nbr_ptr[-1] > 0
    out = {}
    for cache in (False, True):
        ctx, dp, plans = _setup(cel, p, cache)
        res = []
        for pl in plans:
            bgE, bgV = cel.background(pl)
            e, er, g, H = cel.elbo_grad_hess(pl)
            res.append([t.cpu().numpy() for t in (bgE, bgV, e, er, g, H)])
        ctx.synchronize()
        out[cache] = res
    for a, b in zip(out[False], out[True]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_newton_steps_over_classes_are_identical(cel):
    p = _blend()
    thetas = {}
    for cache in (False, True):
        ctx, dp, plans = _setup(cel, p, cache)
        delta, status = cel.newton_state(dp)
        for _ in range(3):
            for pl in plans:
                cel.newton_step(pl, delta, status)
        ctx.synchronize()
        thetas[cache] = (dp.theta.cpu().numpy(), delta.cpu().numpy(), status.cpu().numpy())
    for x, y in zip(thetas[False], thetas[True]):
        assert np.array_equal(x, y)


def test_region_fit_with_cache_is_identical(cel):
    p = _blend()
    region = list(range(0, p.n_sources, 2)) + [1]        # neighbours outside the region too
    out = {}
    for cache in (False, True):
        ctx = cel.Context(p.model)
        dp = cel.DeviceProblem(p, render_cache=cache)
        fit = cel.Fit(ctx, dp, region)
        passes, gains = fit.run(max_passes=3, max_iter=50, pass_tol=0.0)
        ctx.synchronize()
        # per-source results are specified for region sources only
        out[cache] = (passes, gains, dp.theta.cpu().numpy(),
                      *[t.cpu().numpy()[sorted(region)] for t in fit.results()])
    for x, y in zip(out[False], out[True]):
        assert np.array_equal(np.asarray(x), np.asarray(y))
