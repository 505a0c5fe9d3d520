"""The MCMC consumer on the GPU: the batched point-value log-likelihood
against the FP64 oracle, and AIS type probabilities on bright sources."""
import numpy as np
import pytest
import torch

import fields
from oracle import mcmc as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import mcmc
    return mcmc


def test_batched_loglik_matches_oracle(mc):
    p = fields.batched(seed=91, n_sources=6, min_side=15, max_side=31, max_images_per_band=2,
                       max_neighbours=3)
    s = int(np.argmax(np.diff(p.nbr_ptr)))
    assert p.nbr_ptr[s + 1] > p.nbr_ptr[s]
    rng = np.random.default_rng(0)
    u0 = p.theta[s, fields.I_U:fields.I_U + 2]
    n = 6
    thetas = []
    for kind in (mc.STAR, mc.GALAXY):
        W = mc.Prior(p.model, kind, u0, box=1.0).sample(rng, n // 2)
        W[:, 2] = p.theta[s, fields.I_LOGR_MEAN[0]] + rng.normal(0, 0.2, n // 2)
        thetas.append(mc.point_theta(W, kind, p.theta[s]))
    thetas = np.concatenate(thetas)
    ev = mc.GpuLogLik(p, s, n)
    got = ev(thetas)
    again = ev(thetas)
    assert np.array_equal(got, again)
    for k in range(n):
        ref, scale = OM.point_loglik(p, s, thetas[k])
        assert abs(got[k] - ref) <= 1e-5 * scale + 1e-6, (k, got[k], ref, scale)


@pytest.mark.parametrize("seed,star", [(102, True), (119, False)])
def test_ais_picks_the_true_type_of_a_bright_source(mc, seed, star):
    p = fields.plain_source(seed=seed, side=31, star=star)
    r = mc.type_posterior(p, 0, n_chains=12, T=40, B=4, seed=1)
    assert np.isfinite(r["star"]["log_evidence"]) and np.isfinite(r["galaxy"]["log_evidence"])
    if star:
        assert r["p_star"] > 0.9, r["p_star"]
    else:
        assert r["p_star"] < 0.1, r["p_star"]
    # the position samples concentrate near the truth
    post = r["star" if star else "galaxy"]["samples"][:, 0:2].mean(0)
    assert np.all(np.abs(post - p.truth["pos"][0]) < 0.5), (post, p.truth["pos"][0])


def test_several_sources_in_one_call_equal_one_at_a_time(mc):
    p = fields.batched(seed=92, n_sources=8, min_side=15, max_side=31, max_images_per_band=2,
                       max_neighbours=3)
    srcs = [0, 3, 5]
    rng = np.random.default_rng(3)
    n = 4
    rows = []
    for s in srcs:
        u0 = p.theta[s, fields.I_U:fields.I_U + 2]
        W = mc.Prior(p.model, mc.GALAXY, u0, box=1.0).sample(rng, n)
        rows.append(mc.point_theta(W, mc.GALAXY, p.theta[s]))
    together = mc.GpuLogLik(p, srcs, n)(np.concatenate(rows))
    for i, s in enumerate(srcs):
        alone = mc.GpuLogLik(p, s, n)(rows[i])
        assert np.array_equal(together[i * n:(i + 1) * n], alone), s
