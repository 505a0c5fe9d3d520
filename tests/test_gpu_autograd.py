"""Differentiation: the gradient-only pass, the autograd wrapper and
Hessian-vector products against the FP64 oracle and its finite differences."""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _field_subset(n=16, seed=4):
    p = fields.single_field(seed=seed, n_sources=200, height=600, width=500)
    # keep sources with neighbours first so that backgrounds are exercised
    nb = [s for s in range(p.n_sources) if p.nbr_ptr[s + 1] > p.nbr_ptr[s]]
    rest = [s for s in range(p.n_sources) if s not in nb]
    keep = sorted((nb + rest)[:n])
    return p, keep


def test_gradient_only_pass_matches_oracle_and_full_pass(cel):
    p = fields.batched(seed=33, n_sources=6, min_side=15, max_side=41, max_images_per_band=2,
                       max_neighbours=3)
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, list(range(p.n_sources)))
    e1, er1, g1 = cel.elbo_grad(plan)
    e2, er2, g2, H2 = cel.elbo_grad_hess(plan)
    ctx.synchronize()
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.allclose(e1.cpu().numpy(), e2.cpu().numpy(), rtol=1e-9, atol=0)
    for s in range(p.n_sources):
        ref = oracle.elbo_grad_hess(p, s)
        sc = oracle.abs_sum_scales(p, s)
        scale = np.maximum(np.abs(ref["grad"]), sc["grad"])
        assert np.all(np.abs(g1[s] - ref["grad"]) <= TOL * scale), s
        # the two passes share every formula up to FP32 summation order
        assert np.all(np.abs(g1[s] - g2[s]) <= 1e-5 * scale), s


def test_autograd_gradient_against_oracle_and_finite_differences(cel):
    p, keep = _field_subset()
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, keep)
    from paper_1803_00113_gb300.autograd import SourceObjective
    obj = SourceObjective(plan)
    theta = torch.tensor(p.theta[keep], dtype=torch.float64, device="cuda", requires_grad=True)
    L = obj(theta)
    L.sum().backward()
    g = theta.grad.cpu().numpy()
    j = 0
    s = keep[j]
    ref = oracle.elbo_grad_hess(p, s)
    sc = oracle.abs_sum_scales(p, s)
    scale = np.maximum(np.abs(ref["grad"]), sc["grad"])
    assert np.all(np.abs(g[j] - ref["grad"]) <= TOL * scale)
    # central differences of the FP64 oracle, h = 1e-4
    h = 1e-4
    fd = np.zeros(27)
    for k in range(27):
        tp, tm = p.theta[s].copy(), p.theta[s].copy()
        tp[k] += h
        tm[k] -= h
        Lp = oracle.source_elbo(p, s, tp)
        Lm = oracle.source_elbo(p, s, tm)
        fd[k] = ((Lp[0] - Lp[1]) - (Lm[0] - Lm[1])) / (2 * h)
    assert np.all(np.abs(g[j] - fd) <= TOL * scale + 1e-6 * np.abs(fd).max())


def test_hessian_vector_products(cel):
    p, keep = _field_subset(n=8, seed=6)
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, keep)
    from paper_1803_00113_gb300.autograd import SourceObjective
    obj = SourceObjective(plan)
    theta = torch.tensor(p.theta[keep], dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(0)
    v = torch.tensor(rng.choice([-1.0, 1.0], size=theta.shape), dtype=torch.float64, device="cuda")
    _, hv = torch.autograd.functional.hvp(lambda t: obj(t).sum(), theta, v)
    hv = hv.cpu().numpy()
    vv = v.cpu().numpy()
    for j in (0, len(keep) - 1):
        s = keep[j]
        ref = oracle.elbo_grad_hess(p, s)
        sc = oracle.abs_sum_scales(p, s)
        scale = np.maximum(np.abs(ref["hess"]), sc["hess"]) @ np.abs(vv[j])
        assert np.all(np.abs(hv[j] - ref["hess"] @ vv[j]) <= TOL * scale), j


def test_kernel_timing_by_kind(cel):
    p = fields.batched(seed=34, n_sources=5, min_side=15, max_side=31, max_images_per_band=2,
                       max_neighbours=2)
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, list(range(p.n_sources)))
    ctx.profile(True, kinds="all")
    cel.elbo_grad_hess(plan)
    cel.elbo_grad(plan)
    cel.elbo(plan)
    t = ctx.profile_kernels(reset=True)
    assert t["background"][1] == 3 and t["derivs"][1] == 1 and t["grad"][1] == 1
    assert t["value"][1] == 1 and t["epilogue"][1] == 3 and t["tr_step"][1] == 0
    for k in ("derivs", "grad", "value", "background"):
        assert t[k][0] > 0 and t[k][2] == t[k][1] * plan.visits
    # derivative kernel only: the other kinds run untimed
    ctx.profile(True)
    delta, status = cel.newton_state(dp)
    cel.newton_step(plan, delta, status)
    t = ctx.profile_kernels(reset=True)
    assert t["derivs"][1] == 1 and sum(v[1] for v in t.values()) == 1
    assert ctx.profile_read(reset=True)[1] == 0
    ctx.profile(False)
