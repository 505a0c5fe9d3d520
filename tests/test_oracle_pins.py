"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign, index or band selector, a transposed covariance) fails it:
closed forms, Monte Carlo over the variational distribution, numerical
quadrature, brute-force convolution, finite differences and KKT conditions.
"""
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy import integrate, special, stats

import fields
import oracle
from oracle import elbo as E
from oracle import newton as N

DT = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _theta(p, s=0):
    return E.Theta.from_vector(torch.tensor(p.theta[s], dtype=DT))


def _patch_on_grid(p, n, xs, ys):
    """PatchData of image n over explicit pixel centres (for profile checks)."""
    px = torch.tensor(xs, dtype=DT).reshape(-1)
    py = torch.tensor(ys, dtype=DT).reshape(-1)
    return E.PatchData(image=n, band=int(p.img_band[n]), px=px, py=py,
                       x=torch.zeros_like(px), sky=torch.full_like(px, 100.0),
                       calib=float(p.img_calib[n]), A=torch.tensor(p.img_A[n], dtype=DT),
                       t=torch.tensor(p.img_t[n], dtype=DT),
                       psf=torch.tensor(p.img_psf[n], dtype=DT), rect=(0, 0, 1, 1))


# ---------------------------------------------------------------------------
# structural constants (Table 1) -- golden fixture
# ---------------------------------------------------------------------------

def test_structural_constants_golden():
    with open(os.path.join(GOLDEN, "structural_constants.json")) as f:
        g = json.load(f)
    m = fields.make_model()
    assert E.BAND_SELECT.shape[0] == g["B"]
    assert len(m.alpha_exp) == g["K"] and len(m.alpha_dev) == g["K"]
    assert m.color_w.shape[1] == g["J"]
    assert m.color_w.shape[0] == g["I"]
    # the per-source block: 27 Newton coordinates + 2 x J profiled xi weights
    # + the complementary type probability = the paper's 44 stored values
    assert E.N_THETA + g["I"] * g["J"] + 1 == g["params_per_source"]


# ---------------------------------------------------------------------------
# galaxy profile constants: unit flux, unit half-light radius
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["exp", "dev"])
def test_profile_mixture_flux_and_half_light_radius(which):
    ae, te, ad, td = fields.load_profiles()
    alpha, tau = (ae, te) if which == "exp" else (ad, td)
    assert abs(alpha.sum() - 1.0) < 1e-12
    # enclosed flux of a circular Gaussian mixture within radius 1
    enclosed = np.sum(alpha * (1.0 - np.exp(-0.5 / tau)))
    assert abs(enclosed - 0.5) < 1e-6
    # the mixture approximates the Sersic profile it stands for (the de
    # Vaucouleurs fit is truncated at 8 half-light radii, so its renormalised
    # enclosed-flux curve sits a few per cent above the untruncated profile)
    n = 1.0 if which == "exp" else 4.0
    b = special.gammaincinv(2 * n, 0.5)
    r = np.linspace(0.2, 3.0, 30)
    sersic_enc = special.gammainc(2 * n, b * r ** (1 / n))
    mix_enc = np.array([np.sum(alpha * (1 - np.exp(-0.5 * x * x / tau))) for x in r])
    assert np.max(np.abs(sersic_enc - mix_enc)) < (0.01 if which == "exp" else 0.04)


# ---------------------------------------------------------------------------
# fluxes: log-normal moments by Monte Carlo, colours by their definition
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("i", [0, 1])
def test_band_moments_monte_carlo(i):
    p = fields.plain_source()
    th = _theta(p)
    rng = np.random.default_rng(7)
    n = 1_000_000
    logr = rng.normal(float(th.logr_mean[i]), math.sqrt(float(th.logr_var[i])), n)
    c = rng.normal(th.color_mean[i].numpy(), np.sqrt(th.color_var[i].numpy()), (n, 4))
    # build every band's flux from the definition c_k = log(l_{k+1} / l_k), l_2 = r
    l = np.empty((n, 5))
    l[:, 2] = np.exp(logr)
    l[:, 3] = l[:, 2] * np.exp(c[:, 2])
    l[:, 4] = l[:, 3] * np.exp(c[:, 3])
    l[:, 1] = l[:, 2] / np.exp(c[:, 1])
    l[:, 0] = l[:, 1] / np.exp(c[:, 0])
    for b in range(5):
        e1, e2 = (float(v) for v in E.band_moments(th, i, b))
        se1 = l[:, b].std() / math.sqrt(n)
        assert abs(l[:, b].mean() - e1) < 4 * se1
        sq = l[:, b] ** 2
        assert abs(sq.mean() - e2) < 4 * sq.std() / math.sqrt(n)


# ---------------------------------------------------------------------------
# profiles: closed forms, brute-force convolution, flux conservation
# ---------------------------------------------------------------------------

def test_star_profile_single_component_is_bivariate_normal():
    p = fields.plain_source(psf_offsets=True)
    n = 0
    p.img_psf[n, :, 0] = [1.0, 0.0, 0.0]
    pd = _patch_on_grid(p, n, np.arange(10.0, 30.0), np.full(20, 21.0))
    th = _theta(p)
    f = E.star_profile(th, pd, pd.px, pd.py).numpy()
    mu = p.img_A[n] @ p.theta[0, 21:23] + p.img_t[n] + p.img_psf[n, 0, 1:3]
    w, mx, my, cxx, cxy, cyy = p.img_psf[n, 0]
    ref = stats.multivariate_normal(mu, [[cxx, cxy], [cxy, cyy]]).pdf(
        np.column_stack([pd.px.numpy(), pd.py.numpy()]))
    np.testing.assert_allclose(f, p.img_calib[n] * ref, rtol=1e-12)


def test_galaxy_profile_matches_monte_carlo_convolution():
    """f_gal(p) = E_{x ~ h_s}[PSF(p - x)]: sample the light kernel, average the PSF."""
    p = fields.plain_source(psf_offsets=True, seed=11)
    th_vec = p.theta[0].copy()
    th_vec[24] = math.log(2.5)       # radius 2.5 px
    th_vec[25] = 0.3                 # axis ratio ~0.57
    th_vec[26] = 0.4                 # mixed profile
    p.theta[0] = th_vec
    th = _theta(p)
    n = 2
    pts = np.array([[20.0, 20.0], [22.0, 19.0], [17.0, 24.0], [25.0, 25.0]])
    pd = _patch_on_grid(p, n, pts[:, 0], pts[:, 1])
    f = E.galaxy_profile(th, pd, p.model, pd.px, pd.py).numpy() / p.img_calib[n]
    rng = np.random.default_rng(3)
    ns = 2_000_000
    m = p.model
    rho = float(th.profile)
    alphas = np.concatenate([rho * m.alpha_exp, (1 - rho) * m.alpha_dev])
    taus = np.concatenate([m.tau_exp, m.tau_dev])
    comp = rng.choice(len(alphas), size=ns, p=alphas / alphas.sum())
    # Sigma_s from the shape parameters, built by rotating the principal axes
    r, ax, ang = float(th.radius), float(th.axis), float(th.angle)
    major = np.array([math.cos(ang), -math.sin(ang)])
    minor = np.array([math.sin(ang), math.cos(ang)])
    A = p.img_A[n]
    centre = A @ p.theta[0, 21:23] + p.img_t[n]
    z = rng.standard_normal((ns, 2)) * np.sqrt(taus[comp])[:, None]
    x = centre + (z[:, :1] * r * (A @ major)[None, :] + z[:, 1:] * ax * r * (A @ minor)[None, :])
    vals = np.zeros((len(pts), ns))
    for k in range(3):
        w, mx, my, cxx, cxy, cyy = p.img_psf[n, k]
        mvn = stats.multivariate_normal([0, 0], [[cxx, cxy], [cxy, cyy]])
        for q, pt in enumerate(pts):
            vals[q] += w * mvn.pdf(pt - x - np.array([mx, my]))
    mc = vals.mean(axis=1)
    se = vals.std(axis=1) / math.sqrt(ns)
    assert np.all(np.abs(mc - f) < 4 * se + 1e-12)


@pytest.mark.parametrize("star", [True, False])
def test_flux_conservation_on_wide_patch(star):
    p = fields.plain_source(seed=5)
    n = 1
    th = _theta(p)
    mu = p.img_A[n] @ p.theta[0, 21:23] + p.img_t[n]
    half = 70
    xs, ys = np.meshgrid(np.arange(round(mu[0]) - half, round(mu[0]) + half + 1, dtype=float),
                         np.arange(round(mu[1]) - half, round(mu[1]) + half + 1, dtype=float))
    pd = _patch_on_grid(p, n, xs, ys)
    if star:
        f = E.star_profile(th, pd, pd.px, pd.py)
    else:
        f = E.galaxy_profile(th, pd, p.model, pd.px, pd.py)
    # Poisson summation: the lattice sum of a density with sigma >= 1 px
    # equals its integral to ~2 exp(-2 pi^2) ~ 5e-9
    assert abs(float(f.sum()) / p.img_calib[n] - 1.0) < 1e-7


# ---------------------------------------------------------------------------
# moments of the rate: Monte Carlo over z ~ q (Eqs. conditional, vareq)
# ---------------------------------------------------------------------------

def test_rate_moments_monte_carlo():
    p = fields.plain_source(seed=9)
    p.theta[0, 0] = 0.2    # q(star) ~ 0.55: both types matter
    th = _theta(p)
    n = 3
    pts = np.array([[20.0, 20.0], [21.0, 22.0], [18.0, 17.0]])
    pd = _patch_on_grid(p, n, pts[:, 0], pts[:, 1])
    Es, Vs = E.source_moments(th, pd, p.model)
    fg = E.galaxy_profile(th, pd, p.model, pd.px, pd.py).numpy()
    fs = E.star_profile(th, pd, pd.px, pd.py).numpy()
    b = int(p.img_band[n])
    rng = np.random.default_rng(1)
    ns = 2_000_000
    a = rng.uniform(size=ns) < float(th.a_star)
    lam = np.zeros((ns, len(pts)))
    for i, f in ((0, fg), (1, fs)):
        sel = a == bool(i)
        k = int(sel.sum())
        logr = rng.normal(float(th.logr_mean[i]), math.sqrt(float(th.logr_var[i])), k)
        c = rng.normal(th.color_mean[i].numpy(), np.sqrt(th.color_var[i].numpy()), (k, 4))
        logl = logr.copy()
        if b >= 3:
            logl += c[:, 2] + (c[:, 3] if b == 4 else 0.0)
        if b <= 1:
            logl -= c[:, 1] + (c[:, 0] if b == 0 else 0.0)
        lam[sel] = np.exp(logl)[:, None] * f[None, :]
    m = lam.mean(0)
    v = lam.var(0)
    se_m = lam.std(0) / math.sqrt(ns)
    dev2 = (lam - m) ** 2
    se_v = dev2.std(0) / math.sqrt(ns)
    assert np.all(np.abs(m - Es.numpy()) < 4 * se_m)
    assert np.all(np.abs(v - Vs.numpy()) < 4 * se_v)


# ---------------------------------------------------------------------------
# the pixel term: Poisson special case and the delta-method remainder
# ---------------------------------------------------------------------------

def test_pixel_term_zero_variance_is_poisson_loglik():
    x = torch.tensor([0.0, 1.0, 57.0, 130.0, 512.0], dtype=DT)
    lam = torch.tensor([80.0, 90.5, 60.25, 140.0, 500.0], dtype=DT)
    t = E.pixel_term(x, lam, torch.zeros_like(lam)).numpy()
    ref = stats.poisson.logpmf(x.numpy(), lam.numpy()) + special.gammaln(x.numpy() + 1)
    np.testing.assert_allclose(t, ref, rtol=1e-13)


def test_delta_method_within_taylor_remainder():
    """E_q[log lambda] by Monte Carlo vs log E - V / (2 E^2)."""
    rng = np.random.default_rng(4)
    sky = 60.0
    for mu_l, v_l, f in ((3.0, 0.3, 0.05), (5.0, 0.5, 0.01), (2.0, 0.05, 0.2)):
        ns = 2_000_000
        lam = sky + f * np.exp(rng.normal(mu_l, math.sqrt(v_l), ns))
        Eq, Vq = lam.mean(), lam.var()
        delta = float(E.pixel_term(torch.tensor(1.0, dtype=DT), torch.tensor(Eq, dtype=DT),
                                   torch.tensor(Vq, dtype=DT))) + Eq
        mc = np.log(lam).mean()
        bound = np.mean(np.abs(lam - Eq) ** 3) / (3 * sky ** 3)
        se = np.log(lam).std() / math.sqrt(ns)
        assert abs(mc - delta) <= bound + 4 * se


# ---------------------------------------------------------------------------
# KL divergences: quadrature, Monte Carlo and library densities
# ---------------------------------------------------------------------------

def test_kl_bernoulli_against_scipy_entropy():
    for a, A in ((0.3, 0.5), (0.9, 0.2), (0.01, 0.7)):
        k = float(E.kl_bernoulli(torch.tensor(a, dtype=DT), A))
        assert abs(k - stats.entropy([a, 1 - a], [A, 1 - A])) < 1e-13


def test_kl_lognormal_by_quadrature():
    for m, v, M, V in ((1.0, 0.04, 1.6, 1.44), (2.5, 0.3, 1.2, 0.5)):
        q = stats.lognorm(s=math.sqrt(v), scale=math.exp(m))
        p = stats.lognorm(s=math.sqrt(V), scale=math.exp(M))
        lo, hi = q.ppf(1e-14), q.ppf(1 - 1e-14)
        val, _ = integrate.quad(lambda x: q.pdf(x) * (q.logpdf(x) - p.logpdf(x)), lo, hi,
                                limit=400, epsabs=1e-13)
        k = float(E.kl_lognormal(torch.tensor(m, dtype=DT), torch.tensor(v, dtype=DT), M, V))
        assert abs(k - val) < 1e-8


def test_color_bound_upper_bounds_true_kl_and_is_tight_for_one_component():
    m = fields.make_model()
    rng = np.random.default_rng(2)
    mean = np.array([1.0, 0.5, 0.3, 0.2])
    var = np.array([0.02, 0.05, 0.01, 0.03])
    q = stats.multivariate_normal(mean, np.diag(var))
    xs = q.rvs(size=400_000, random_state=rng)
    logq = q.logpdf(xs)
    for i in range(2):
        logp = special.logsumexp(np.stack([
            math.log(m.color_w[i, j]) + stats.multivariate_normal(m.color_mean[i, j], m.color_cov[i, j]).logpdf(xs)
            for j in range(m.color_w.shape[1])]), axis=0)
        d = logq - logp
        true_kl, se = d.mean(), d.std() / math.sqrt(len(d))
        bound = float(E.kl_color_bound(torch.tensor(mean, dtype=DT), torch.tensor(var, dtype=DT),
                                       m.color_w[i], m.color_mean[i], m.color_cov[i]))
        assert bound >= true_kl - 4 * se
        # one component: the bound is the Gaussian KL itself
        j = 3
        one = float(E.kl_color_bound(torch.tensor(mean, dtype=DT), torch.tensor(var, dtype=DT),
                                     np.array([1.0]), m.color_mean[i, j:j + 1], m.color_cov[i, j:j + 1]))
        d1 = logq - stats.multivariate_normal(m.color_mean[i, j], m.color_cov[i, j]).logpdf(xs)
        assert abs(one - d1.mean()) < 4 * d1.std() / math.sqrt(len(d1))


def test_point_mass_terms_are_negative_log_prior_densities():
    for val, mean, var in ((1.3, math.log(1.5), 0.25), (4.0, 0.2, 0.6)):
        got = float(E.neglog_lognormal(torch.tensor(val, dtype=DT), mean, var))
        ref = -stats.lognorm(s=math.sqrt(var), scale=math.exp(mean)).logpdf(val)
        assert abs(got - ref) < 1e-12
    for val, b1, b2 in ((0.3, 2.0, 1.6), (0.85, 1.5, 1.5)):
        got = float(E.neglog_beta(torch.tensor(val, dtype=DT), b1, b2))
        assert abs(got + stats.beta(b1, b2).logpdf(val)) < 1e-12


# ---------------------------------------------------------------------------
# the galaxy shape covariance and the sky interpolation
# ---------------------------------------------------------------------------

def test_galaxy_covariance_axes():
    p = fields.plain_source()
    th = _theta(p)
    S = E.galaxy_covariance(th).numpy()
    r, ax, ang = float(th.radius), float(th.axis), float(th.angle)
    major = np.array([math.cos(ang), -math.sin(ang)])   # R^T e_1
    minor = np.array([math.sin(ang), math.cos(ang)])    # R^T e_2
    np.testing.assert_allclose(S @ major, r * r * major, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(S @ minor, (ax * r) ** 2 * minor, rtol=1e-12, atol=1e-12)


def test_sky_bilinear_reproduces_plane():
    p = fields.plain_source(sky_grid=(3, 4))
    n = 0
    H, W = int(p.img_h[n]), int(p.img_w[n])
    # overwrite the knots with a plane; bilinear interpolation reproduces it
    a, bx, by = 100.0, 0.75, -0.5
    ky = np.arange(3) * (H - 1) / 2.0
    kx = np.arange(4) * (W - 1) / 3.0
    grid = a + bx * kx[None, :] + by * ky[:, None]
    off = int(p.img_sky_off[n])
    p.sky[off:off + 12] = grid.ravel().astype(np.float32)
    grid32 = p.sky[off:off + 12].astype(np.float64).reshape(3, 4)
    xs = torch.tensor([0.0, 7.0, 13.5, 40.0], dtype=DT)
    ys = torch.tensor([0.0, 33.0, 20.0, 40.0], dtype=DT)
    got = E.sky_at(p, n, xs, ys).numpy()
    ref = np.array([np.interp(y, ky, [np.interp(x, kx, grid32[i]) for i in range(3)])
                    for x, y in zip(xs.numpy(), ys.numpy())])
    np.testing.assert_allclose(got, ref, rtol=1e-12)


# ---------------------------------------------------------------------------
# derivatives: central finite differences of the oracle's scalar objective
# ---------------------------------------------------------------------------

def _fd_problem():
    """A small blend: the returned source has neighbours in its patches."""
    p = fields.batched(seed=21, n_sources=6, min_side=15, max_side=21,
                       max_images_per_band=1, max_neighbours=2)
    s = int(np.flatnonzero(np.diff(p.nbr_ptr) > 0)[0])
    return p, s


def test_gradient_and_hessian_by_finite_differences():
    p, s = _fd_problem()
    r = oracle.elbo_grad_hess(p, s)
    patches = E.gather_patches(p, s)
    bgs = [E.background_patch(p, s, pd) for pd in patches]
    t0 = torch.tensor(p.theta[s], dtype=DT)

    def L(t):
        return E.source_elbo_parts(p, s, t, patches, bgs)[0]

    def Lrel(t):
        v, base, _ = E.source_elbo_parts(p, s, t, patches, bgs)
        return float(v - base)

    h = 1e-4
    g_fd = np.zeros(27)
    for k in range(27):
        e = torch.zeros(27, dtype=DT)
        e[k] = h
        g_fd[k] = (Lrel(t0 + e) - Lrel(t0 - e)) / (2 * h)
    scale = np.maximum(np.abs(r["grad"]), 1.0)
    assert np.max(np.abs(g_fd - r["grad"]) / scale) < 1e-6

    def grad_at(t):
        t = t.clone().requires_grad_(True)
        (g,) = torch.autograd.grad(L(t), t)
        return g.numpy()
    def dgrad(k, hh):
        e = torch.zeros(27, dtype=DT)
        e[k] = hh
        return (grad_at(t0 + e) - grad_at(t0 - e)) / (2 * hh)
    H_fd = np.zeros((27, 27))
    for k in range(27):
        # Richardson extrapolation of the central difference: O(h^4) truncation
        H_fd[:, k] = (4.0 * dgrad(k, h / 2) - dgrad(k, h)) / 3.0
    hs = np.maximum(np.abs(r["hess"]), 1.0)
    assert np.max(np.abs(H_fd - r["hess"]) / hs) < 1e-6
    assert np.max(np.abs(r["hess"] - r["hess"].T)) < 1e-9 * np.max(np.abs(r["hess"]))


def test_elbo_base_is_source_absent_value():
    p, s = _fd_problem()
    L, base = oracle.source_elbo(p, s)
    # a vanishing flux makes the source's moments (and its pixel effect) vanish
    t = p.theta[s].copy()
    t[1] = t[3] = -60.0
    patches = E.gather_patches(p, s)
    bgs = [E.background_patch(p, s, pd) for pd in patches]
    v, b2, kl = E.source_elbo_parts(p, s, torch.tensor(t, dtype=DT), patches, bgs)
    assert abs(float(v + kl) - base) < 1e-9 * abs(base)
    assert abs(b2 - base) < 1e-9 * abs(base)


# ---------------------------------------------------------------------------
# trust-region subproblem: KKT conditions, concave quadratics, the hard case
# ---------------------------------------------------------------------------

def _random_sym(rng, n, shift):
    M = rng.normal(size=(n, n))
    return 0.5 * (M + M.T) + shift * np.eye(n)


@pytest.mark.parametrize("shift,delta", [(-8.0, 0.5), (-8.0, 100.0), (0.0, 0.3), (3.0, 1.0), (8.0, 0.05)])
def test_tr_subproblem_kkt(shift, delta):
    rng = np.random.default_rng(int(abs(shift) * 10 + delta * 100))
    H = _random_sym(rng, 27, shift)
    g = rng.normal(size=27)
    p, pred, l, hard = N.tr_subproblem(g, H, delta)
    B = -H
    assert np.linalg.norm((B + l * np.eye(27)) @ p - g) < 1e-9 * (1 + np.linalg.norm(g))
    assert l >= 0.0
    assert np.linalg.norm(p) <= delta * (1 + 1e-12)
    assert abs(l * (delta - np.linalg.norm(p))) < 1e-9 * max(1.0, l)
    assert np.linalg.eigvalsh(B + l * np.eye(27))[0] > -1e-9
    # the model increase is the best over the ball: compare with random feasible points
    for _ in range(200):
        q = rng.normal(size=27)
        q *= delta * rng.uniform() ** (1 / 27) / np.linalg.norm(q)
        assert g @ q + 0.5 * q @ H @ q <= pred + 1e-9 * (1 + abs(pred))


def test_tr_concave_quadratic_one_step():
    rng = np.random.default_rng(5)
    S = _random_sym(rng, 27, 0.0)
    H = -(S @ S.T + np.eye(27))
    g = rng.normal(size=27)
    p, pred, l, hard = N.tr_subproblem(g, H, 1e6)
    np.testing.assert_allclose(p, np.linalg.solve(-H, g), rtol=1e-9, atol=1e-12)
    assert l == 0.0
    # one step lands on the maximiser of the quadratic: its gradient vanishes
    assert np.linalg.norm(g + H @ p) < 1e-9 * np.linalg.norm(g)


def test_tr_hard_case():
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.normal(size=(27, 27)))
    lam = np.sort(rng.uniform(0.5, 5.0, 27))
    lam[0] = -2.0                       # B has one negative eigenvalue
    B = Q @ np.diag(lam) @ Q.T
    H = -B
    g = Q[:, 1:] @ rng.normal(size=26)  # orthogonal to the eigenvector of lam_min
    delta = 50.0
    p, pred, l, hard = N.tr_subproblem(g, H, delta)
    assert hard
    assert abs(l - 2.0) < 1e-12
    assert abs(np.linalg.norm(p) - delta) < 1e-9 * delta
    assert np.linalg.norm((B + l * np.eye(27)) @ p - g) < 1e-9 * np.linalg.norm(g)
    z = Q[:, 0] * np.sign(Q[np.flatnonzero(np.abs(Q[:, 0]) > 0)[0], 0])
    assert p @ z > 0


# ---------------------------------------------------------------------------
# the Newton subsolver on a real source
# ---------------------------------------------------------------------------

def test_newton_fit_reaches_a_local_maximum():
    p = fields.plain_source(side=19, bands=2, seed=17)
    L0, b0 = oracle.source_elbo(p, 0)
    theta, delta, status, it = oracle.newton_fit(p, 0)
    assert status == N.ST_CONVERGED
    r = oracle.elbo_grad_hess(p, 0, theta)
    assert r["elbo"] > L0
    sc = oracle.abs_sum_scales(p, 0, theta)
    # stationary: every gradient entry is negligible against its magnitude
    # scale (flat coordinates, e.g. a star's colours when q(star) ~ 0, have
    # tiny scales, hence the absolute floor)
    assert np.all(np.abs(r["grad"]) <= 1e-4 * sc["grad"] + 1e-5)
    assert np.linalg.eigvalsh(-r["hess"])[0] > -1e-8 * np.max(np.abs(r["hess"]))
