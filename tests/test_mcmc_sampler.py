"""Pins of the MCMC consumer (Sec. 3): the point-value log-likelihood
against SciPy's Poisson pmf, and the batched slice sampler and AIS against
targets whose answers are known in closed form (host code, no GPU)."""
import math

import numpy as np
import pytest
import torch

import fields
from oracle import elbo as OE
from oracle import mcmc as OM


def _point_theta(theta, star):
    from paper_1803_00113_gb300 import mcmc
    W = np.zeros(7 if star else 11)
    W[0:2] = theta[fields.I_U:fields.I_U + 2]
    W[2] = theta[fields.I_LOGR_MEAN[0]]
    W[3:7] = theta[fields.I_COLOR_MEAN[0]:fields.I_COLOR_MEAN[0] + 4]
    if not star:
        W[7] = theta[fields.I_ANGLE] % math.pi
        W[8] = theta[fields.I_LOGRADIUS]
        W[9] = 1 / (1 + math.exp(-theta[fields.I_AXIS]))
        W[10] = 1 / (1 + math.exp(-theta[fields.I_PROFILE]))
    return mcmc.point_theta(W, mcmc.STAR if star else mcmc.GALAXY, theta)[0]


@pytest.mark.parametrize("star", [True, False])
def test_point_loglik_is_the_poisson_likelihood_ratio(star):
    from scipy.stats import poisson
    p = fields.plain_source(seed=31, side=21, star=star)
    th = _point_theta(p.theta[0], star)
    value, scale = OM.point_loglik(p, 0, th)
    tht = OE.Theta.from_vector(torch.as_tensor(th, dtype=OE.DT))
    ref = 0.0
    for pd in OE.gather_patches(p, 0):
        E, V = OE.source_moments(tht, pd, p.model)
        assert float(V.abs().max()) <= 1e-12 * float(E.max()) ** 2
        lam = (pd.sky + E).numpy()
        x = pd.x.numpy()
        ref += float(np.sum(poisson.logpmf(x, lam) - poisson.logpmf(x, pd.sky.numpy())))
    assert abs(value - ref) <= 1e-9 * scale, (value, ref)


class _Gaussian:
    """prior N(0, I_d), likelihood N(x; w, s2 I): evidence and posterior known."""

    def __init__(self, d, x, s2, n):
        self.d, self.x, self.s2 = d, np.asarray(x), s2
        self.lo = np.full((n, d), -np.inf)
        self.hi = np.full((n, d), np.inf)
        self.movable = np.ones((n, d), dtype=bool)
        self.n = n

    def sample(self, rng):
        return rng.standard_normal((self.n, self.d))

    def logprior(self, W):
        return -0.5 * np.sum(W ** 2, axis=1) - 0.5 * self.d * math.log(2 * math.pi)

    def loglik(self, W):
        return (-0.5 * np.sum((W - self.x) ** 2, axis=1) / self.s2
                - 0.5 * self.d * math.log(2 * math.pi * self.s2))


def test_slice_sweeps_leave_the_target_invariant():
    from paper_1803_00113_gb300 import mcmc
    rng = np.random.default_rng(0)
    n = 4000
    W = rng.standard_normal((n, 2)) * np.array([1.0, 3.0]) + np.array([0.5, -1.0])

    def logp(P):
        return -0.5 * ((P[:, 0] - 0.5) ** 2 + ((P[:, 1] + 1.0) / 3.0) ** 2)

    lp = logp(W)
    for _ in range(5):
        W, lp = mcmc.slice_sweep(logp, W, lp, rng, np.array([1.0, 1.0]), -np.inf, np.inf)
    se = 4 * np.array([1.0, 3.0]) / math.sqrt(n)
    assert np.all(np.abs(W.mean(0) - [0.5, -1.0]) < se)
    assert np.all(np.abs(W.std(0) / [1.0, 3.0] - 1) < 0.06)
    assert np.allclose(lp, logp(W))


def test_slice_sampler_respects_bounds_and_masks():
    from paper_1803_00113_gb300 import mcmc
    rng = np.random.default_rng(1)
    n = 2000
    W = rng.uniform(0, 1, (n, 2))
    mov = np.ones((n, 2), dtype=bool)
    mov[:, 1] = False                          # the second coordinate stays put

    def logp(P):
        inside = (P[:, 0] > 0) & (P[:, 0] < 1)
        return np.where(inside, 0.0, -np.inf)  # uniform on (0, 1)

    W0 = W.copy()
    lp = logp(W)
    for _ in range(10):
        W, lp = mcmc.slice_sweep(logp, W, lp, rng, np.array([0.3, 0.3]), np.array([0.0, -np.inf]),
                                 np.array([1.0, np.inf]), mov)
    assert np.all((W[:, 0] > 0) & (W[:, 0] < 1))
    assert np.array_equal(W[:, 1], W0[:, 1])
    assert abs(W[:, 0].mean() - 0.5) < 0.03 and abs(W[:, 0].var() - 1 / 12) < 0.01


def test_ais_estimates_the_gaussian_evidence_and_posterior():
    from paper_1803_00113_gb300 import mcmc
    d, s2, x = 2, 0.25, np.array([1.0, -0.5])
    t = _Gaussian(d, x, s2, 200)
    rng = np.random.default_rng(2)
    logw, W, samples = mcmc.ais(t, 100, rng, np.ones(d), B=10)
    logz = mcmc.log_mean_exp(logw)
    ref = -0.5 * np.sum(x ** 2) / (1 + s2) - 0.5 * d * math.log(2 * math.pi * (1 + s2))
    assert abs(logz - ref) < 0.05, (logz, ref)
    post_mean, post_var = x / (1 + s2), s2 / (1 + s2)
    S = samples.reshape(-1, d)
    assert np.all(np.abs(S.mean(0) - post_mean) < 4 * math.sqrt(post_var / 200))
    assert np.all(np.abs(S.var(0) / post_var - 1) < 0.15)
