"""GPU parity at the full shape of the batched workload.

The batched field (Sec. 4.4's parallel block updates over blended sources)
has patches of 15..101 px, 1..6 exposures per band and 0..10 neighbours per
source, runs with the render cache and with tile shapes picked by the
autotuner.  Here a smaller field of that shape is set up exactly that way,
one colour class takes a Newton step (so that accepted sources' trial
renders are committed into the cache), and then the ELBO, gradient and
Hessian of the most-neighboured source, a source with six exposures in a
band and the source with the largest patch are compared with the FP64
oracle element by element, at the parity tolerances (ELBO 1e-5 relative,
gradient and Hessian entries 1e-4 of their magnitude scales).
"""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu

TOL_ELBO = 1e-5
TOL_DERIV = 1e-4


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _max_exposures(p, s):
    bands = p.img_band[p.patch_img[p.patch_ptr[s]:p.patch_ptr[s + 1]]]
    return int(np.bincount(bands, minlength=5).max())


def _largest_area(p, s):
    sl = slice(p.patch_ptr[s], p.patch_ptr[s + 1])
    return int((p.patch_w[sl].astype(np.int64) * p.patch_h[sl]).max())


def test_batched_shape_after_a_cached_newton_step_matches_the_oracle(cel):
    from paper_1803_00113_gb300.autotune import autotune
    p = fields.batched(seed=1803_00113 + 33, n_sources=160)
    nn = np.diff(p.nbr_ptr)
    assert nn.max() == 10 and max(_max_exposures(p, s) for s in range(p.n_sources)) == 6
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p, render_cache=True)
    classes = cel.color_classes(p)
    tiles, _ = autotune(ctx, dp, range(p.n_sources), reps=1, groups=classes)
    dp.set_theta(p.theta)
    plans = [cel.Plan(ctx, dp, c, ppi_bucket=tiles) for c in classes]
    for pl in plans:
        cel.render_cache(pl)
    delta, status = cel.newton_state(dp)
    cel.newton_step(plans[0], delta, status)
    ctx.synchronize()
    st = status.cpu().numpy()
    moved = [int(s) for s in classes[0] if st[s] == cel.ST_ACCEPTED]
    assert moved, "no source of the first class accepted its step"
    p.theta = dp.theta.cpu().numpy().copy()

    vis = np.array([p.visits([s]) for s in range(p.n_sources)])
    # sources outside the first class with an accepted neighbour read the
    # committed renders through the cache
    moved_set = set(moved)
    reads_commit = np.array([any(int(t) in moved_set for t in p.nbr_idx[p.nbr_ptr[s]:p.nbr_ptr[s + 1]])
                             and s not in set(int(x) for x in classes[0])
                             for s in range(p.n_sources)])
    most_nbrs = int(np.argmax(np.where(reads_commit, nn * 1e7 - vis, -1e18)))
    six = int(np.argmin(np.where([_max_exposures(p, s) == 6 for s in range(p.n_sources)], vis, 1e18)))
    largest = int(np.argmax([_largest_area(p, s) * 1e3 - vis[s] / 1e6 for s in range(p.n_sources)]))
    picks = sorted({most_nbrs, six, largest, moved[0]})
    assert reads_commit[most_nbrs] and nn[most_nbrs] >= 8
    assert _largest_area(p, largest) == 101 * 101

    plan = cel.Plan(ctx, dp, picks, ppi_bucket=tiles)
    e, er, g, H = (t.cpu().numpy() for t in cel.elbo_grad_hess(plan))
    ctx.synchronize()
    for k, s in enumerate(picks):
        ref = oracle.elbo_grad_hess(p, s)
        sc = oracle.abs_sum_scales(p, s)
        label = f"source {s}: {nn[s]} neighbours, {_max_exposures(p, s)} exposures, {vis[s]} visits"
        assert abs(e[k] - ref["elbo"]) <= TOL_ELBO * abs(ref["elbo"]), (label, e[k], ref["elbo"])
        assert abs(er[k] - ref["elbo_rel"]) <= TOL_ELBO * max(abs(ref["elbo_rel"]), sc["elbo"]), \
            (label, er[k], ref["elbo_rel"])
        gs = np.maximum(np.abs(ref["grad"]), sc["grad"])
        bad = np.abs(g[k] - ref["grad"]) > TOL_DERIV * gs
        assert not bad.any(), (label, np.flatnonzero(bad), g[k][bad], ref["grad"][bad])
        hs = np.maximum(np.abs(ref["hess"]), sc["hess"])
        bad = np.abs(H[k] - ref["hess"]) > TOL_DERIV * hs
        assert not bad.any(), (label, np.argwhere(bad)[:10], H[k][bad][:10], ref["hess"][bad][:10])
