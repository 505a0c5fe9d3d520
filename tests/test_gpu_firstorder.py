"""The first-order (L-BFGS) comparison subsolver reaches the optimum the
Newton trust-region subsolver finds, climbing monotonically."""
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


def _newton(cel, plan, dp, iters=50):
    delta, status = cel.newton_state(dp)
    for _ in range(iters):
        cel.newton_step(plan, delta, status)
        st = status.cpu().numpy()[plan.sources]
        if not np.any(np.isin(st, (cel.ST_ACCEPTED, cel.ST_REJECTED))):
            break
    return cel.elbo(plan)[1].cpu().numpy()


def test_lbfgs_reaches_the_newton_optimum(cel):
    p = fields.batched(seed=81, n_sources=4, min_side=15, max_side=25, max_images_per_band=1,
                       max_neighbours=0)
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, list(range(p.n_sources)))
    best = _newton(cel, plan, dp)
    dp.set_theta(p.theta)
    lb = cel.Lbfgs(plan, m=10)
    target = torch.tensor(best - 1e-6 * (1 + np.abs(best)), dtype=torch.float64, device="cuda")
    status = torch.zeros(p.n_sources, dtype=torch.int32, device="cuda")
    prev = cel.elbo(plan)[1].cpu().numpy()
    for it in range(4000):
        lb.step(status, target)
        if it % 25 == 24:
            now = cel.elbo(plan)[1].cpu().numpy()
            # Armijo: never descends beyond the FP32 noise of the value
            assert np.all(now >= prev - 1e-6 * (1 + np.abs(prev)))
            prev = now
            if np.all(status.cpu().numpy() == cel.ST_CONVERGED):
                break
    ctx.synchronize()
    final = cel.elbo(plan)[1].cpu().numpy()
    iters, fevals, reached = [t.cpu().numpy() for t in lb.counts()]
    assert np.all(final <= best + 1e-6 * (1 + np.abs(best)))
    assert np.all(reached > 0), (reached, final - best, best)
    assert np.all(fevals >= iters) and np.all(iters >= reached)
