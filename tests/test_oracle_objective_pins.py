"""Pins of the oracle's assembled objective and of its trust-region iteration.

The pieces of the objective are pinned one by one elsewhere (the band
moments, the profiles, the pixel term, each KL piece).  These tests pin how
they are put together, against quantities the oracle does not compute:

* KL_s of Eq. kleq (Supplement A, Sec. 4.2.3) against a Monte Carlo estimate
  of E_q[log q(z) - log p(z)] over z ~ q (the type a, the log flux and the
  colours drawn from the variational distribution; the point masses u and e
  enter through -log p_prior(point), the cross-entropy reading).  With a
  single colour component per type the colour bound is exact, so the two
  must agree within Monte Carlo error; with the full mixture the oracle's
  value is an upper bound.  Planted mistakes in the assembly (the type
  weights swapped, the Bernoulli term dropped) fail the check.
* The whole per-source objective L_s of Eq. elbo: its pixel sum against a
  Monte Carlo estimate of E_q[log p(x | z)] with the exact log of the rate
  (the delta method of Sec. 4.2.2 may differ by at most its Taylor
  remainder), and L_s against that estimate minus the Monte Carlo KL.
* One iteration of the trust-region loop (Sec. 4.3, read as Nocedal &
  Wright's Algorithm 4.1 with the exact subproblem solution) on analytic
  objectives whose subproblem solution, ratio rho, radius update and
  acceptance are worked out by hand below.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch
from scipy import special, stats

import fields
from oracle import elbo as E
from oracle import newton as N

DT = torch.float64


# ---------------------------------------------------------------------------
# a tiny source with both types in play
# ---------------------------------------------------------------------------

def _one_colour_model(m, j=3):
    """The model with a single colour-prior component per type (J = 1)."""
    return dataclasses.replace(m, color_w=np.ones((2, 1)),
                               color_mean=m.color_mean[:, j:j + 1].copy(),
                               color_cov=m.color_cov[:, j:j + 1].copy())


def _tiny_source(model, faint=True):
    """A 9 x 9 px source in 2 bands whose per-type KL terms differ clearly,
    with q(star) = 0.65 (away from 1/2 and from the prior 0.3)."""
    p = fields.plain_source(side=9, bands=2, seed=31, model=model)
    t = p.theta[0]
    t[0] = math.log(0.65 / 0.35)
    # galaxy flux near the prior mean, star flux far above it: the two
    # types' log-normal KLs differ by about a nat
    t[1], t[3] = math.log(0.6 if faint else 6.0), math.log(1.2 if faint else 12.0)
    t[2], t[4] = math.log(0.05), math.log(0.08)
    t[13:21] = math.log(0.02)
    return p


def _theta(p):
    return E.Theta.from_vector(torch.tensor(p.theta[0], dtype=DT))


def _draw_types_fluxes_colours(th, rng, ns):
    """a ~ Bernoulli(q(star)); log r, c ~ q( . | a) (Eqs. eq0-eq1)."""
    a = rng.uniform(size=ns) < float(th.a_star)
    logr = np.empty(ns)
    c = np.empty((ns, 4))
    for i in (0, 1):
        sel = a == bool(i)
        k = int(sel.sum())
        logr[sel] = rng.normal(float(th.logr_mean[i]), math.sqrt(float(th.logr_var[i])), k)
        c[sel] = rng.normal(th.color_mean[i].numpy(), np.sqrt(th.color_var[i].numpy()), (k, 4))
    return a, logr, c


def _kl_monte_carlo(th, model, rng, ns=1_000_000):
    """E_q[log q(a, r, c) - log p(a, r, c)] by sampling, plus the point-mass
    terms -log p(e) from SciPy's densities.  Returns (estimate, std. error)."""
    a, logr, c = _draw_types_fluxes_colours(th, rng, ns)
    qs, pa = float(th.a_star), float(model.prior_a)
    d = np.where(a, math.log(qs / pa), math.log((1 - qs) / (1 - pa)))
    for i in (0, 1):
        sel = a == bool(i)
        m, v = float(th.logr_mean[i]), float(th.logr_var[i])
        pm, pv = float(model.prior_r[i, 0]), float(model.prior_r[i, 1])
        # densities of log r: the Jacobian of r -> log r cancels in the ratio
        d[sel] += (stats.norm(m, math.sqrt(v)).logpdf(logr[sel])
                   - stats.norm(pm, math.sqrt(pv)).logpdf(logr[sel]))
        cm, cv = th.color_mean[i].numpy(), th.color_var[i].numpy()
        logq = stats.multivariate_normal(cm, np.diag(cv)).logpdf(c[sel])
        logp = special.logsumexp(np.stack([
            math.log(model.color_w[i, j])
            + stats.multivariate_normal(model.color_mean[i, j], model.color_cov[i, j]).logpdf(c[sel])
            for j in range(model.color_w.shape[1])]), axis=0)
        d[sel] += logq - logp
    er_m, er_v = float(model.e_radius[0]), float(model.e_radius[1])
    point = (-stats.lognorm(s=math.sqrt(er_v), scale=math.exp(er_m)).logpdf(float(th.radius))
             - stats.beta(*model.e_axis).logpdf(float(th.axis))
             - stats.beta(*model.e_profile).logpdf(float(th.profile)))
    return float(d.mean()) + float(point), float(d.std()) / math.sqrt(ns)


def _band_log_flux(logr, c, band):
    """log l_b = log r + the colours between band b and the r band (index 2),
    with c_k = log(l_{k+1} / l_k)."""
    if band == 0:
        return logr - c[:, 0] - c[:, 1]
    if band == 1:
        return logr - c[:, 1]
    if band == 2:
        return logr
    if band == 3:
        return logr + c[:, 2]
    return logr + c[:, 2] + c[:, 3]


def _loglik_monte_carlo(p, th, rng, ns=400_000, chunk=20_000):
    """E_q[sum_m -lambda_m + x_m log lambda_m] over z ~ q with the exact log,
    where lambda_m = sky_m + l_b f_a(m) (u and e are point masses; the
    profiles f_a are the oracle's, pinned on their own by convolution and
    closed-form tests).  Returns (estimate, std. error, Taylor bound of the
    delta method: sum_m x_m E|lambda_m - E lambda_m|^3 / (3 sky_m^3))."""
    patches = E.gather_patches(p, 0)
    prof = [(E.galaxy_profile(th, pd, p.model, pd.px, pd.py).numpy(),
             E.star_profile(th, pd, pd.px, pd.py).numpy()) for pd in patches]
    totals = []
    lam_sum = [np.zeros(pd.px.shape[0]) for pd in patches]
    lam_chunks = [[] for _ in patches]
    for c0 in range(0, ns, chunk):
        k = min(chunk, ns - c0)
        a, logr, c = _draw_types_fluxes_colours(th, rng, k)
        tot = np.zeros(k)
        for n, (pd, (fg, fs)) in enumerate(zip(patches, prof)):
            l = np.exp(_band_log_flux(logr, c, pd.band))
            f = np.where(a[:, None], fs[None, :], fg[None, :])
            lam = pd.sky.numpy()[None, :] + l[:, None] * f
            tot += np.sum(-lam + pd.x.numpy()[None, :] * np.log(lam), axis=1)
            lam_sum[n] += lam.sum(0)
            lam_chunks[n].append(lam)
        totals.append(tot)
    tot = np.concatenate(totals)
    bound = 0.0
    for n, pd in enumerate(patches):
        lam = np.concatenate(lam_chunks[n])
        mean = lam_sum[n] / ns
        r3 = np.mean(np.abs(lam - mean[None, :]) ** 3, axis=0)
        bound += float(np.sum(pd.x.numpy() * r3 / (3.0 * pd.sky.numpy() ** 3)))
    return float(tot.mean()), float(tot.std()) / math.sqrt(ns), bound


# ---------------------------------------------------------------------------
# KL_s: Monte Carlo over q
# ---------------------------------------------------------------------------

def _kl_swapped_weights(th, model):
    """kl_source with the type weights (1 - a, a) exchanged (a planted mistake)."""
    a = th.a_star
    kl = E.kl_bernoulli(a, model.prior_a)
    for i, qi in ((0, a), (1, 1 - a)):
        kl = kl + qi * (E.kl_lognormal(th.logr_mean[i], th.logr_var[i],
                                       float(model.prior_r[i, 0]), float(model.prior_r[i, 1]))
                        + E.kl_color_bound(th.color_mean[i], th.color_var[i], model.color_w[i],
                                           model.color_mean[i], model.color_cov[i]))
    kl = kl + E.neglog_lognormal(th.radius, float(model.e_radius[0]), float(model.e_radius[1]))
    kl = kl + E.neglog_beta(th.axis, float(model.e_axis[0]), float(model.e_axis[1]))
    return kl + E.neglog_beta(th.profile, float(model.e_profile[0]), float(model.e_profile[1]))


def test_kl_source_equals_monte_carlo_kl_for_one_colour_component():
    model = _one_colour_model(fields.make_model())
    p = _tiny_source(model)
    th = _theta(p)
    mc, se = _kl_monte_carlo(th, model, np.random.default_rng(7))
    kl = float(E.kl_source(th, model))
    assert abs(kl - mc) <= 4 * se, (kl, mc, se)


def test_kl_source_bounds_monte_carlo_kl_for_the_colour_mixture():
    model = fields.make_model()
    p = _tiny_source(model)
    th = _theta(p)
    mc, se = _kl_monte_carlo(th, model, np.random.default_rng(8))
    kl = float(E.kl_source(th, model))
    assert kl >= mc - 4 * se, (kl, mc, se)


def test_kl_monte_carlo_check_catches_planted_assembly_mistakes(monkeypatch):
    """The check above fails when the assembly of KL_s is wrong."""
    model = _one_colour_model(fields.make_model())
    p = _tiny_source(model)
    th = _theta(p)
    mc, se = _kl_monte_carlo(th, model, np.random.default_rng(7))
    swapped = float(_kl_swapped_weights(th, model))
    assert abs(swapped - mc) > 10 * se, (swapped, mc, se)
    monkeypatch.setattr(E, "kl_bernoulli", lambda a, prior: torch.zeros((), dtype=DT))
    dropped = float(E.kl_source(th, model))
    assert abs(dropped - mc) > 10 * se, (dropped, mc, se)


# ---------------------------------------------------------------------------
# the whole objective L_s: Monte Carlo over q with the exact log-likelihood
# ---------------------------------------------------------------------------

def test_pixel_sum_and_elbo_match_monte_carlo_over_q():
    model = _one_colour_model(fields.make_model())
    p = _tiny_source(model)
    th = _theta(p)
    t = torch.tensor(p.theta[0], dtype=DT)
    L, base, kl = E.source_elbo_parts(p, 0, t)
    pixel_sum = float(L + kl)
    rng = np.random.default_rng(11)
    ll, se_ll, taylor = _loglik_monte_carlo(p, th, rng)
    # the delta method replaces E_q[log lambda] by log E - V / (2 E^2): the
    # two differ by at most the third-order Taylor remainder
    assert abs(pixel_sum - ll) <= taylor + 4 * se_ll, (pixel_sum, ll, taylor, se_ll)
    kl_mc, se_kl = _kl_monte_carlo(th, model, rng)
    elbo_mc = ll - kl_mc
    tol = taylor + 4 * math.hypot(se_ll, se_kl)
    assert abs(float(L) - elbo_mc) <= tol, (float(L), elbo_mc, tol)
    # the check is sharp enough to see the KL (a dropped or sign-flipped KL
    # would fail it) and the delta method's variance term
    assert float(kl) > 20 * tol
    E_V = [E.source_moments(th, pd, model) for pd in E.gather_patches(p, 0)]
    var_term = sum(float(torch.sum(pd.x * V / (2 * (pd.sky + Es) ** 2)))
                   for pd, (Es, V) in zip(E.gather_patches(p, 0), E_V))
    assert var_term > 5 * (taylor + 4 * se_ll), (var_term, taylor, se_ll)


# ---------------------------------------------------------------------------
# one trust-region iteration on analytic objectives, worked by hand
# ---------------------------------------------------------------------------

class _Analytic:
    """f(theta) = c1 t0 + c2 t0^2 - c4 t0^4 - sum_{k>=1} t_k^2 / 2 with its
    exact gradient and Hessian: at t_k = 0 (k >= 1) the subproblem reduces
    to one coordinate."""

    def __init__(self, c1, c2, c4):
        self.c1, self.c2, self.c4 = c1, c2, c4

    def f(self, t):
        t0 = float(t[0])
        return self.c1 * t0 + self.c2 * t0 ** 2 - self.c4 * t0 ** 4 - 0.5 * float(np.sum(t[1:] ** 2))

    def evaluation(self, t):
        t0 = float(t[0])
        g = -np.asarray(t, dtype=np.float64).copy()
        g[0] = self.c1 + 2 * self.c2 * t0 - 4 * self.c4 * t0 ** 3
        H = -np.eye(27)
        H[0, 0] = 2 * self.c2 - 12 * self.c4 * t0 ** 2
        v = self.f(t)
        return dict(elbo=v, elbo_rel=v, grad=g, hess=H)


def _iterate(monkeypatch, obj, t0, delta):
    monkeypatch.setattr(N, "source_elbo", lambda problem, s, trial: (obj.f(trial), 0.0))
    theta = np.zeros(27)
    theta[0] = t0
    return N.newton_iteration(None, 0, theta, delta, evaluation=obj.evaluation(theta))


def test_tr_iteration_grows_the_radius_after_a_good_boundary_step(monkeypatch):
    # f = 3 t - t^4 / 4 at t = 0, Delta = 1: g = 3, H = 0, so the model is
    # linear and the step is the boundary point p = 1 with predicted gain 3;
    # f(1) = 11/4, rho = 11/12 > 3/4 at the boundary: accept, Delta = 2
    obj = _Analytic(3.0, 0.0, 0.25)
    th, d, st, info = _iterate(monkeypatch, obj, 0.0, 1.0)
    assert st == N.ST_ACCEPTED
    assert info["p"][0] == pytest.approx(1.0, rel=1e-12)
    assert np.max(np.abs(info["p"][1:])) < 1e-14
    assert info["pred"] == pytest.approx(3.0, rel=1e-12)
    assert info["rho"] == pytest.approx(11.0 / 12.0, rel=1e-12)
    assert d == 2.0 and th[0] == pytest.approx(1.0, rel=1e-12)
    # next: t = 1, Delta = 2: g = 2, H = -3, the Newton step 2/3 is inside;
    # predicted 2/3, actual f(5/3) - f(1) = 26/81, rho = 13/27 in
    # [1/4, 3/4]: accept, radius unchanged
    th, d, st, info = _iterate(monkeypatch, obj, 1.0, 2.0)
    assert st == N.ST_ACCEPTED
    assert info["p"][0] == pytest.approx(2.0 / 3.0, rel=1e-12)
    assert info["pred"] == pytest.approx(2.0 / 3.0, rel=1e-12)
    assert info["rho"] == pytest.approx(13.0 / 27.0, rel=1e-12)
    assert d == 2.0 and th[0] == pytest.approx(5.0 / 3.0, rel=1e-12)


def test_tr_iteration_interior_step_never_grows_the_radius(monkeypatch):
    # f = 3 t - t^4 / 4 at t = 5/3, Delta = 2: g = 3 - 125/27 = -44/27,
    # H = -25/3; the interior step p = g / 25 * 3 = -44/225, predicted gain
    # g^2 / (2 |H|) = (44/27)^2 * 3 / 50; rho > 3/4 but |p| < Delta: accept,
    # Delta stays 2
    obj = _Analytic(3.0, 0.0, 0.25)
    th, d, st, info = _iterate(monkeypatch, obj, 5.0 / 3.0, 2.0)
    g, h = -44.0 / 27.0, -25.0 / 3.0
    p = -g / h
    pred = g * p + 0.5 * h * p * p
    rho = (obj.f(np.r_[5.0 / 3.0 + p, np.zeros(26)]) - obj.f(np.r_[5.0 / 3.0, np.zeros(26)])) / pred
    assert info["p"][0] == pytest.approx(-44.0 / 225.0, rel=1e-12)
    assert info["pred"] == pytest.approx((44.0 / 27.0) ** 2 * 3.0 / 50.0, rel=1e-12)
    assert info["rho"] == pytest.approx(rho, rel=1e-12) and rho > 0.75
    assert st == N.ST_ACCEPTED and d == 2.0


def test_tr_iteration_shrinks_but_accepts_a_poor_step(monkeypatch):
    # f = 3 t - 5/2 t^4 at 0, Delta = 1: p = 1, predicted 3, actual 1/2,
    # rho = 1/6: below 1/4 so Delta = |p| / 4 = 1/4, above 0.1 so accepted
    obj = _Analytic(3.0, 0.0, 2.5)
    th, d, st, info = _iterate(monkeypatch, obj, 0.0, 1.0)
    assert info["rho"] == pytest.approx(1.0 / 6.0, rel=1e-12)
    assert st == N.ST_ACCEPTED and d == pytest.approx(0.25, rel=1e-12)
    assert th[0] == pytest.approx(1.0, rel=1e-12)


def test_tr_iteration_rejects_a_bad_step(monkeypatch):
    # f = 3 t - 3 t^4 at 0, Delta = 1: actual gain 0, rho = 0: rejected,
    # theta unchanged, Delta = 1/4
    obj = _Analytic(3.0, 0.0, 3.0)
    th, d, st, info = _iterate(monkeypatch, obj, 0.0, 1.0)
    assert info["rho"] == pytest.approx(0.0, abs=1e-15)
    assert st == N.ST_REJECTED and d == pytest.approx(0.25, rel=1e-12)
    assert th[0] == 0.0


def test_tr_iteration_follows_positive_curvature_to_the_boundary(monkeypatch):
    # f = t + t^2 at 0, Delta = 1: g = 1, H = 2 (B = -H has eigenvalue -2),
    # so the multiplier is 3 and p = g / (l - 2) = 1 on the boundary;
    # predicted 1 + 1 = 2 equals the actual gain: rho = 1, Delta doubles
    obj = _Analytic(1.0, 1.0, 0.0)
    th, d, st, info = _iterate(monkeypatch, obj, 0.0, 1.0)
    assert info["p"][0] == pytest.approx(1.0, rel=1e-12)
    assert info["pred"] == pytest.approx(2.0, rel=1e-12)
    assert info["rho"] == pytest.approx(1.0, rel=1e-12)
    assert st == N.ST_ACCEPTED and d == 2.0


def test_tr_iteration_caps_the_radius(monkeypatch):
    # f = 300 t - 1e-9 t^4 at 0, Delta = 80: p = 80, rho = 1 - 80^3 1e-9 / 300
    # > 3/4 at the boundary: Delta = min(160, 100) = 100
    obj = _Analytic(300.0, 0.0, 1e-9)
    th, d, st, info = _iterate(monkeypatch, obj, 0.0, 80.0)
    assert info["rho"] == pytest.approx(1.0 - 80.0 ** 3 * 1e-9 / 300.0, rel=1e-9)
    assert st == N.ST_ACCEPTED and d == 100.0


def test_tr_iteration_converges_at_a_stationary_point(monkeypatch):
    # at the maximiser of f = 3 t - t^4 / 4 (t^3 = 3) the gradient is ~0, the
    # predicted gain is below 1e-9 (1 + |f|): converged, theta unchanged
    obj = _Analytic(3.0, 0.0, 0.25)
    t_star = 3.0 ** (1.0 / 3.0)
    th, d, st, info = _iterate(monkeypatch, obj, t_star, 1.0)
    assert st == N.ST_CONVERGED and th[0] == t_star and d == 1.0
