"""GPU parity: the CUDA library against the FP64 oracle on the same inputs.

Tolerances (from the targets of this path, FP32 arithmetic with FP32
accumulation on the device):
  * ELBO: |L_gpu - L| <= 1e-5 |L|; the source's own part L_rel (the ELBO
    minus its value with the source absent) within 1e-5 of its magnitude
    scale sum_pix |term - term_absent| + |KL|;
  * gradient and Hessian entries: |d| <= 1e-4 max(|ref|, scale), the scale
    being the sum over pixels of the absolute per-pixel derivative (plus the
    KL's), so entries that cancel to ~0 over the patch are compared with
    the magnitudes that were summed.
"""
import math

import numpy as np
import pytest
import torch

import fields
import oracle
from oracle import elbo as OE
from oracle import newton as ON

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


def _ctx(cel, problem):
    return cel.Context(problem.model)


def _check_source(problem, s, e, er, g, H, label=""):
    ref = oracle.elbo_grad_hess(problem, s)
    sc = oracle.abs_sum_scales(problem, s)
    assert abs(e - ref["elbo"]) <= TOL_ELBO * abs(ref["elbo"]), (label, e, ref["elbo"])
    assert abs(er - ref["elbo_rel"]) <= TOL_ELBO * max(abs(ref["elbo_rel"]), sc["elbo"]), \
        (label, er, ref["elbo_rel"], sc["elbo"])
    gs = np.maximum(np.abs(ref["grad"]), sc["grad"])
    bad = np.abs(g - ref["grad"]) > TOL_DERIV * gs
    assert not bad.any(), (label, np.flatnonzero(bad), g[bad], ref["grad"][bad], gs[bad])
    hs = np.maximum(np.abs(ref["hess"]), sc["hess"])
    bad = np.abs(H - ref["hess"]) > TOL_DERIV * hs
    assert not bad.any(), (label, np.argwhere(bad)[:10], H[bad][:10], ref["hess"][bad][:10])


def _eval(cel, problem, sources, ppi=0):
    ctx = _ctx(cel, problem)
    dp = cel.DeviceProblem(problem)
    plan = cel.Plan(ctx, dp, sources, pixels_per_item=ppi)
    e, er, g, H = cel.elbo_grad_hess(plan)
    ctx.synchronize()
    return (e.cpu().numpy(), er.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy()), (ctx, dp, plan)


@pytest.mark.parametrize("star", [None, True, False])
def test_plain_source_elbo_grad_hess(cel, star):
    p = fields.plain_source(star=star, psf_offsets=True)
    (e, er, g, H), _ = _eval(cel, p, [0])
    _check_source(p, 0, e[0], er[0], g[0], H[0], f"plain star={star}")


def test_blend_with_neighbours_sky_grid_and_ragged_tiles(cel):
    p = fields.batched(seed=33, n_sources=7, min_side=15, max_side=41, max_images_per_band=2,
                       max_neighbours=3)
    # a sloped sky on every image and PSF offsets exercise every input path
    rng = np.random.default_rng(0)
    p.img_psf[:, :, 1:3] = rng.uniform(-0.2, 0.2, p.img_psf[:, :, 1:3].shape)
    srcs = list(range(p.n_sources))
    (e, er, g, H), _ = _eval(cel, p, srcs, ppi=96)     # 96-pixel tiles: ragged tails
    with_nbrs = [s for s in srcs if p.nbr_ptr[s + 1] > p.nbr_ptr[s]]
    assert with_nbrs
    for s in with_nbrs[:3] + [srcs[-1]]:
        _check_source(p, s, e[s], er[s], g[s], H[s], f"blend s={s}")


def test_sky_grid_interpolation(cel):
    p = fields.plain_source(sky_grid=(3, 4), seed=77)
    (e, er, g, H), _ = _eval(cel, p, [0])
    _check_source(p, 0, e[0], er[0], g[0], H[0], "sky grid")


def test_render_and_background_match_oracle(cel):
    p = fields.batched(seed=5, n_sources=5, min_side=15, max_side=31, max_images_per_band=1,
                       max_neighbours=4)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, list(range(p.n_sources)))
    E, V = cel.render(plan)
    bE, bV = cel.background(plan)
    ctx.synchronize()
    E, V, bE, bV = (t.cpu().numpy().astype(np.float64) for t in (E, V, bE, bV))
    for s in range(p.n_sources):
        pds = OE.gather_patches(p, s)
        own = oracle.render_source_patch(p, s)
        for q, pd, (Es, Vs) in zip(range(p.patch_ptr[s], p.patch_ptr[s + 1]), pds, own):
            off = int(dp.pool_offset[q])
            n = pd.px.shape[0]
            np.testing.assert_allclose(E[off:off + n], Es.numpy(), rtol=2e-5, atol=1e-6 * Es.abs().max().item())
            np.testing.assert_allclose(V[off:off + n], Vs.numpy(), rtol=2e-5, atol=1e-6 * Vs.abs().max().item())
            rbE, rbV = OE.background_patch(p, s, pd)
            np.testing.assert_allclose(bE[off:off + n], rbE.numpy(), rtol=2e-6)
            np.testing.assert_allclose(bV[off:off + n], rbV.numpy(), rtol=2e-5, atol=1e-6 * max(rbV.abs().max().item(), 1.0))


def test_alone_equals_in_batch_bitwise(cel):
    p = fields.batched(seed=8, n_sources=12, min_side=15, max_side=51, max_images_per_band=2)
    (e, er, g, H), _ = _eval(cel, p, list(range(p.n_sources)))
    for s in (0, 5, 11):
        (e1, er1, g1, H1), _ = _eval(cel, p, [s])
        assert e1[0] == e[s] and er1[0] == er[s]
        assert np.array_equal(g1[0], g[s]) and np.array_equal(H1[0], H[s])


def test_tr_subproblem_matches_oracle(cel):
    ctx = cel.Context(fields.make_model())
    rng = np.random.default_rng(3)
    gs, Hs, ds, kinds = [], [], [], []
    for shift, delta in ((-6.0, 0.5), (-6.0, 50.0), (0.0, 0.3), (4.0, 1.0), (9.0, 0.05), (9.0, 1e3)):
        for _ in range(3):
            M = rng.normal(size=(27, 27))
            Hm = -(0.5 * (M + M.T) + shift * np.eye(27))
            gs.append(rng.normal(size=27))
            Hs.append(Hm)
            ds.append(delta)
    # an exact hard case
    Q, _ = np.linalg.qr(rng.normal(size=(27, 27)))
    lam = np.sort(rng.uniform(0.5, 5.0, 27))
    lam[0] = -2.0
    Hs.append(-(Q @ np.diag(lam) @ Q.T))
    gs.append(Q[:, 1:] @ rng.normal(size=26))
    ds.append(50.0)
    dev = torch.device("cuda")
    p, pred = cel.tr_subproblem(ctx, torch.tensor(np.array(gs), device=dev),
                                torch.tensor(np.array(Hs), device=dev),
                                torch.tensor(np.array(ds), device=dev))
    ctx.synchronize()
    p, pred = p.cpu().numpy(), pred.cpu().numpy()
    for k in range(len(gs)):
        rp, rpred, rl, hard = ON.tr_subproblem(gs[k], Hs[k], ds[k])
        np.testing.assert_allclose(p[k], rp, rtol=1e-7, atol=1e-9 * np.linalg.norm(rp))
        assert abs(pred[k] - rpred) <= 1e-9 * max(1.0, abs(rpred))


def test_newton_iteration_matches_oracle(cel):
    p = fields.plain_source(seed=41)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, [0])
    delta, status = cel.newton_state(dp)
    theta, d = p.theta[0].copy(), 1.0
    for it in range(4):
        L0 = oracle.source_elbo(p, 0, theta)
        cel.newton_step(plan, delta, status)
        ctx.synchronize()
        theta_ref, d_ref, st, info = ON.newton_iteration(p, 0, theta, d)
        gth = dp.theta[0].cpu().numpy()
        assert int(status[0]) == st, (it, int(status[0]), st, info.get("rho"))
        assert abs(float(delta[0]) - d_ref) <= 1e-3 * d_ref, (it, float(delta[0]), d_ref)
        # FP32 sums move the step a little along flat directions; both steps
        # must buy the same gain in the objective
        gain_gpu = oracle.source_elbo(p, 0, gth)[0] - L0[0]
        gain_ref = oracle.source_elbo(p, 0, theta_ref)[0] - L0[0]
        assert abs(gain_gpu - gain_ref) <= 1e-3 * abs(gain_ref) + 1e-6, (it, gain_gpu, gain_ref)
        theta, d = gth.copy(), float(delta[0])   # continue both from the device iterate


def test_newton_fit_converges_to_oracle_optimum(cel):
    p = fields.plain_source(seed=17, side=25)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, [0])
    delta, status = cel.newton_state(dp)
    for it in range(50):
        cel.newton_step(plan, delta, status)
        if int(status[0]) in (cel.ST_CONVERGED, cel.ST_FAILED):
            break
    ctx.synchronize()
    assert int(status[0]) in (cel.ST_CONVERGED, cel.ST_ACCEPTED, cel.ST_REJECTED)
    th_gpu = dp.theta[0].cpu().numpy()
    th_ref, _, st, _ = oracle.newton_fit(p, 0)
    assert st == ON.ST_CONVERGED
    L_gpu = oracle.source_elbo(p, 0, th_gpu)[0]
    L_ref = oracle.source_elbo(p, 0, th_ref)[0]
    # both sit at the same maximum: equal objective to within FP32 noise
    r = oracle.elbo_grad_hess(p, 0, th_ref)
    assert abs(L_gpu - L_ref) <= 1e-6 * abs(r["elbo_rel"]) + 1e-4
    # and the same point, measured in posterior standard deviations
    sd = np.sqrt(np.maximum(np.diag(np.linalg.inv(-r["hess"])), 1e-30))
    assert np.max(np.abs(th_gpu - th_ref) / sd) < 0.05


def test_full_field_sampled_sources(cel):
    """600-source field, one colour class plan per class (the bench layout)."""
    p = fields.single_field()
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    classes = cel.color_classes(p)
    results = {}
    for cls in classes:
        plan = cel.Plan(ctx, dp, cls)
        e, er, g, H = cel.elbo_grad_hess(plan)
        ctx.synchronize()
        for k, s in enumerate(cls):
            results[int(s)] = (float(e[k]), float(er[k]), g[k].cpu().numpy(), H[k].cpu().numpy())
    assert len(results) == p.n_sources
    rng = np.random.default_rng(0)
    nb = [s for s in range(p.n_sources) if p.nbr_ptr[s + 1] > p.nbr_ptr[s]]
    big = int(np.argmax([p.patch_w[p.patch_ptr[s]] for s in range(p.n_sources)]))
    for s in sorted(set([int(rng.integers(p.n_sources)), nb[0], big])):
        _check_source(p, s, *results[s], f"field s={s}")


def test_edge_cases(cel):
    p = fields.plain_source(side=15)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    # empty plan
    plan0 = cel.Plan(ctx, dp, [])
    e, er, g, H = cel.elbo_grad_hess(plan0)
    ctx.synchronize()
    assert e.numel() == 0
    # duplicate and out-of-range sources are rejected on the host
    with pytest.raises(cel.CelesteError):
        cel.Plan(ctx, dp, [0, 0])
    with pytest.raises(cel.CelesteError):
        cel.Plan(ctx, dp, [1])
    # a patch outside its image is rejected
    bad = fields.plain_source(side=15)
    bad.patch_x0[0] = 3
    dbad = cel.DeviceProblem(bad)
    with pytest.raises(cel.CelesteError):
        cel.Plan(ctx, dbad, [0])
    # all-zero counts: the pixel term reduces to -E
    z = fields.plain_source(side=15, seed=4)
    z.pixels[:] = 0.0
    (e, er, g, H), _ = _eval(cel, z, [0])
    _check_source(z, 0, e[0], er[0], g[0], H[0], "zero counts")
    # non-positive sky sets the device error bit
    s0 = fields.plain_source(side=15, seed=6)
    s0.sky[0] = 0.0
    ctx2 = _ctx(cel, s0)
    d2 = cel.DeviceProblem(s0)
    pl = cel.Plan(ctx2, d2, [0])
    cel.elbo_grad_hess(pl)
    with pytest.raises(cel.CelesteError):
        ctx2.synchronize()


def test_largest_patch_101(cel):
    """The largest patch of the workloads (101 x 101 px, five bands)."""
    p = fields.plain_source(side=101, seed=19)
    (e, er, g, H), _ = _eval(cel, p, [0])
    _check_source(p, 0, e[0], er[0], g[0], H[0], "101x101")


def test_autotuned_tiles_give_the_same_results(cel):
    p = fields.batched(seed=12, n_sources=20, min_side=15, max_side=101, max_images_per_band=2)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p)
    from paper_1803_00113_gb300.autotune import autotune
    tiles, report = autotune(ctx, dp, range(p.n_sources), candidates=(64, 256, 1024), reps=1)
    assert all(t in (0, 64, 256, 1024) for t in tiles) and report
    ref = cel.elbo_grad_hess(cel.Plan(ctx, dp, list(range(p.n_sources))))
    got = cel.elbo_grad_hess(cel.Plan(ctx, dp, list(range(p.n_sources)), ppi_bucket=tiles))
    ctx.synchronize()
    for a, b in zip(got, ref):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        # only the FP32 summation order differs between tilings
        assert np.all(np.abs(a - b) <= 1e-5 * np.abs(b) + 1e-6 * np.abs(b).max())


def test_composed_autotune_over_colour_classes(cel):
    """The composed mode times the step's own plans (the colour classes) and
    only touches buckets that hold sources."""
    p = fields.batched(seed=13, n_sources=24, min_side=15, max_side=101, max_images_per_band=2,
                       max_neighbours=3)
    ctx = _ctx(cel, p)
    dp = cel.DeviceProblem(p, render_cache=True)
    classes = cel.color_classes(p)
    from paper_1803_00113_gb300.autotune import autotune, source_bucket
    tiles, report = autotune(ctx, dp, range(p.n_sources), candidates=(64, 256), reps=1,
                             groups=classes)
    used = {source_bucket(p, s) for s in range(p.n_sources)}
    for b in range(4):
        assert tiles[b] in ((64, 256) if b in used else (0,))
    assert all(v > 0 for v in report["composed_ms"].values())
    ref = cel.elbo_grad_hess(cel.Plan(ctx, dp, list(range(p.n_sources))))
    got = cel.elbo_grad_hess(cel.Plan(ctx, dp, list(range(p.n_sources)), ppi_bucket=tiles))
    ctx.synchronize()
    for a, b in zip(got, ref):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-5 * np.abs(b) + 1e-6 * np.abs(b).max())
