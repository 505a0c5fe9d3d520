"""Oracle: the per-source variational objective, written out step by step.

Test infrastructure only (imported by tests, the smoke check and the CPU
baseline of the benchmark; never by the library).  Plain PyTorch CPU ops in
float64; derivatives come from autograd of the scalar objective, so they are
the exact derivatives of the function below up to rounding.

Each function follows one passage of the paper (Regier et al., "Approximate
Inference for Constructing Astronomical Catalogs from Images"):

* fluxes and colours ........ Sec. 2.1.2 (Flux), colours as log flux ratios
* light kernels ............. Sec. 2.1.3, Eq. ``eq:hsi`` and the Sigma_s, R_s
                              definitions; PSF-convolved as in Sec. 2.2.2
* rate and its moments ...... Sec. 2.2.3 (lambda_nm, f_nms), Sec. 4.2,
                              Eqs. ``conditional`` and ``vareq``
* expected log-likelihood ... Eq. ``eq:log_p_last`` with the delta-method
                              expansion of E_q[log lambda] (Sec. 4.2.2)
* KL divergence ............. Eqs. ``eq:kl``, ``kleq``, the GMM colour bound
                              (Sec. 4.2.3) and Supplement A
* ELBO ...................... Eq. ``elbo``

Readings where the paper is silent or garbled (each one is listed with its
reason in the design notes):
  - colour c_b = log(l_{b+1} / l_b); reference band r (index 2 of ugriz);
  - the profile weight multiplies the exponential profile;
  - Sigma_s = R^T diag(r^2, axis^2 r^2) R with the angle in radians;
  - pixels are point-sampled at integer centres (x = column, y = row);
  - a source lights pixel m of image n iff m lies in its patch rectangle;
  - sky: bilinear interpolation of a knot grid spanning the image;
  - log-normal KL with r_hat and R_2 both variances of log r;
  - point-mass terms of u and e contribute -log p_prior(point); their
    theta-independent constants (uniform u, uniform angle) are dropped;
  - the colour KL bound is minimised over xi in closed form:
    -log sum_j w_j exp(-KL_j);
  - -log x! is excluded from the ELBO (reported separately).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List

import numpy as np
import torch

DT = torch.float64

# ---- the 27 unconstrained coordinates of one source ----------------------
# type i = 0 galaxy, 1 star; q(a = 1) is the star probability.
IDX_A = 0
IDX_LOGR_MEAN = (1, 3)
IDX_LOGR_LOGVAR = (2, 4)
IDX_COLOR_MEAN = (5, 9)
IDX_COLOR_LOGVAR = (13, 17)
IDX_U = 21
IDX_ANGLE = 23
IDX_LOGRADIUS = 24
IDX_AXIS = 25
IDX_PROFILE = 26
N_THETA = 27

# l_b = r * exp(sum_k S[b, k] c_k) with c_k = log(l_{k+1} / l_k), r = l_2
BAND_SELECT = torch.tensor([[-1., -1., 0., 0.],
                            [0., -1., 0., 0.],
                            [0., 0., 0., 0.],
                            [0., 0., 1., 0.],
                            [0., 0., 1., 1.]], dtype=DT)


@dataclass
class Theta:
    """Constrained view of one source's variational parameters (Eqs. eq0-eq1)."""
    a_star: torch.Tensor          # q(a_s = 1)
    logr_mean: torch.Tensor       # [2]  r-acute
    logr_var: torch.Tensor        # [2]  r-hat (variance of log r)
    color_mean: torch.Tensor      # [2, 4]  c-acute
    color_var: torch.Tensor       # [2, 4]  c-hat (diagonal variances)
    u: torch.Tensor               # [2] position, reference frame
    angle: torch.Tensor
    radius: torch.Tensor
    axis: torch.Tensor
    profile: torch.Tensor         # weight of the exponential profile

    @staticmethod
    def from_vector(t: torch.Tensor) -> "Theta":
        return Theta(
            a_star=torch.sigmoid(t[IDX_A]),
            logr_mean=torch.stack([t[IDX_LOGR_MEAN[0]], t[IDX_LOGR_MEAN[1]]]),
            logr_var=torch.exp(torch.stack([t[IDX_LOGR_LOGVAR[0]], t[IDX_LOGR_LOGVAR[1]]])),
            color_mean=torch.stack([t[IDX_COLOR_MEAN[0]:IDX_COLOR_MEAN[0] + 4],
                                    t[IDX_COLOR_MEAN[1]:IDX_COLOR_MEAN[1] + 4]]),
            color_var=torch.exp(torch.stack([t[IDX_COLOR_LOGVAR[0]:IDX_COLOR_LOGVAR[0] + 4],
                                             t[IDX_COLOR_LOGVAR[1]:IDX_COLOR_LOGVAR[1] + 4]])),
            u=t[IDX_U:IDX_U + 2],
            angle=t[IDX_ANGLE],
            radius=torch.exp(t[IDX_LOGRADIUS]),
            axis=torch.sigmoid(t[IDX_AXIS]),
            profile=torch.sigmoid(t[IDX_PROFILE]),
        )


# ---------------------------------------------------------------------------
# Sec. 2.1.2 and Eq. conditional / vareq: per-band flux moments under q(.|a=i)
# ---------------------------------------------------------------------------

def band_moments(th: Theta, i: int, b: int):
    """E_q[l_b | a=i] and E_q[l_b^2 | a=i].

    log l_b = log r + S_b . c is normal under q(. | a=i) with mean
    r-acute_i + S_b . c-acute_i and variance r-hat_i + sum_k S_bk^2 c-hat_ik;
    the moments of a log-normal follow.
    """
    S = BAND_SELECT[b]
    m = th.logr_mean[i] + torch.dot(S, th.color_mean[i])
    v = th.logr_var[i] + torch.dot(S * S, th.color_var[i])
    return torch.exp(m + 0.5 * v), torch.exp(2.0 * m + 2.0 * v)


# ---------------------------------------------------------------------------
# Sec. 2.1.3: galaxy shape covariance Sigma_s = R^T diag(r^2, axis^2 r^2) R
# ---------------------------------------------------------------------------

def galaxy_covariance(th: Theta) -> torch.Tensor:
    c, s = torch.cos(th.angle), torch.sin(th.angle)
    R = torch.stack([torch.stack([c, -s]), torch.stack([s, c])])
    D = torch.diag(torch.stack([th.radius ** 2, (th.axis * th.radius) ** 2]))
    return R.T @ D @ R


# ---------------------------------------------------------------------------
# image side: pixels of one patch, with the instrument parameters of its image
# ---------------------------------------------------------------------------

@dataclass
class PatchData:
    """Pixels of patch (s, n) and image n's parameters (Sec. 2.2)."""
    image: int
    band: int
    px: torch.Tensor      # pixel-centre x (column), [P]
    py: torch.Tensor      # pixel-centre y (row), [P]
    x: torch.Tensor       # photon counts, [P]
    sky: torch.Tensor     # sigma_n(m), [P]
    calib: float
    A: torch.Tensor       # [2, 2]
    t: torch.Tensor       # [2]
    psf: torch.Tensor     # [3, 6]: weight, mean x, mean y, cov xx, xy, yy
    rect: tuple           # (x0, y0, w, h)


def sky_at(problem, n, px, py):
    """Bilinear interpolation of image n's sky knot grid (knots span the image)."""
    knots = torch.tensor(problem.sky_grid(n), dtype=DT)
    ny, nx = knots.shape
    H, W = int(problem.img_h[n]), int(problem.img_w[n])
    gx = px * ((nx - 1) / max(W - 1, 1))
    gy = py * ((ny - 1) / max(H - 1, 1))
    ix = torch.clamp(torch.floor(gx), 0, max(nx - 2, 0)).long()
    iy = torch.clamp(torch.floor(gy), 0, max(ny - 2, 0)).long()
    fx = gx - ix
    fy = gy - iy
    ix1 = torch.clamp(ix + 1, max=nx - 1)
    iy1 = torch.clamp(iy + 1, max=ny - 1)
    return ((1 - fy) * ((1 - fx) * knots[iy, ix] + fx * knots[iy, ix1])
            + fy * ((1 - fx) * knots[iy1, ix] + fx * knots[iy1, ix1]))


def gather_patches(problem, s) -> List[PatchData]:
    out = []
    for p in range(int(problem.patch_ptr[s]), int(problem.patch_ptr[s + 1])):
        n = int(problem.patch_img[p])
        x0, y0 = int(problem.patch_x0[p]), int(problem.patch_y0[p])
        w, h = int(problem.patch_w[p]), int(problem.patch_h[p])
        ys, xs = torch.meshgrid(torch.arange(y0, y0 + h, dtype=DT),
                                torch.arange(x0, x0 + w, dtype=DT), indexing="ij")
        px, py = xs.reshape(-1), ys.reshape(-1)
        img = problem.image(n)
        x = torch.tensor(np.ascontiguousarray(img[y0:y0 + h, x0:x0 + w]), dtype=DT).reshape(-1)
        out.append(PatchData(
            image=n, band=int(problem.img_band[n]), px=px, py=py, x=x,
            sky=sky_at(problem, n, px, py), calib=float(problem.img_calib[n]),
            A=torch.tensor(problem.img_A[n], dtype=DT), t=torch.tensor(problem.img_t[n], dtype=DT),
            psf=torch.tensor(problem.img_psf[n], dtype=DT), rect=(x0, y0, w, h)))
    return out


# ---------------------------------------------------------------------------
# Sec. 2.2.3: f_nms, the expected photons of a one-nanomaggy source in pixel m
# ---------------------------------------------------------------------------

def _normal_density(dx, dy, cxx, cxy, cyy):
    """Bivariate normal density at offset (dx, dy) with covariance [[cxx, cxy], [cxy, cyy]]."""
    det = cxx * cyy - cxy * cxy
    q = (cyy * dx * dx - 2.0 * cxy * dx * dy + cxx * dy * dy) / det
    return torch.exp(-0.5 * q) / (2.0 * math.pi * torch.sqrt(det))


def star_profile(th: Theta, pd: PatchData, px, py):
    """f for a star: the PSF g_nm evaluated at the star's position."""
    mu = pd.A @ th.u + pd.t
    w, mx, my, cxx, cxy, cyy = pd.psf.T                      # each [K]
    dx = px[..., None] - mu[0] - mx                          # [P, K]
    dy = py[..., None] - mu[1] - my
    return pd.calib * torch.sum(w * _normal_density(dx, dy, cxx, cxy, cyy), dim=-1)


def galaxy_profile(th: Theta, pd: PatchData, model, px, py):
    """f for a galaxy: sum over PSF components k and profile components j of
    w_k alpha_j N(p; A u + t + m_k, A tau_j Sigma_s A^T + Sigma_k)  (the
    Gaussian-Gaussian convolution of Sec. 2.2.3, in pixel coordinates);
    the exponential profile has weight e^profile, de Vaucouleurs the rest."""
    mu = pd.A @ th.u + pd.t
    G = pd.A @ galaxy_covariance(th) @ pd.A.T
    w, mx, my, cxx, cxy, cyy = pd.psf.T                      # each [K]
    tau = torch.tensor(np.concatenate([model.tau_exp, model.tau_dev]), dtype=DT)      # [J]
    alpha = torch.tensor(np.concatenate([model.alpha_exp, model.alpha_dev]), dtype=DT)
    nexp = len(model.tau_exp)
    pw = torch.cat([th.profile.expand(nexp), (1.0 - th.profile).expand(len(model.tau_dev))])
    # components indexed [K, J]
    cw = w[:, None] * (pw * alpha)[None, :]
    c_xx = cxx[:, None] + tau[None, :] * G[0, 0]
    c_xy = cxy[:, None] + tau[None, :] * G[0, 1]
    c_yy = cyy[:, None] + tau[None, :] * G[1, 1]
    dx = (px[..., None] - mu[0] - mx)[..., None]             # [P, K, 1]
    dy = (py[..., None] - mu[1] - my)[..., None]
    dens = _normal_density(dx, dy, c_xx, c_xy, c_yy)          # [P, K, J]
    return pd.calib * torch.sum(cw * dens, dim=(-2, -1))


def source_moments(th: Theta, pd: PatchData, model, px=None, py=None):
    """E_q[l f] and V_q[l f] of one source in the pixels of patch pd.

    Eq. conditional conditions on a_s; Eq. vareq gives the variance as
    E[l^2 f^2] - E[l f]^2.  u and e are point masses, so E[f^2 | a] = f^2.
    """
    px = pd.px if px is None else px
    py = pd.py if py is None else py
    e1g, e2g = band_moments(th, 0, pd.band)
    e1s, e2s = band_moments(th, 1, pd.band)
    fg = galaxy_profile(th, pd, model, px, py)
    fs = star_profile(th, pd, px, py)
    a = th.a_star
    E = (1 - a) * e1g * fg + a * e1s * fs
    M = (1 - a) * e2g * fg * fg + a * e2s * fs * fs
    return E, M - E * E


# ---------------------------------------------------------------------------
# Eq. eq:log_p_last with the delta method of Sec. 4.2.2
# ---------------------------------------------------------------------------

def pixel_term(x, E, V):
    """-E[lambda] + x (log E[lambda] - V[lambda] / (2 E[lambda]^2)); -log x! excluded."""
    return -E + x * (torch.log(E) - V / (2.0 * E * E))


def _in_rect(px, py, rect):
    x0, y0, w, h = rect
    return (px >= x0) & (px < x0 + w) & (py >= y0) & (py < y0 + h)


def background_patch(problem, s, pd: PatchData, thetas=None):
    """Sky plus the moments of every neighbour that lights pixels of patch pd.

    A neighbour s' contributes to pixel m of image n iff m lies in its own
    patch rectangle in image n (the support restriction of Sec. 2.2.3).
    """
    thetas = problem.theta if thetas is None else thetas
    bgE = pd.sky.clone()
    bgV = torch.zeros_like(pd.sky)
    for t in problem.nbr_idx[problem.nbr_ptr[s]:problem.nbr_ptr[s + 1]]:
        t = int(t)
        for p in range(int(problem.patch_ptr[t]), int(problem.patch_ptr[t + 1])):
            if int(problem.patch_img[p]) != pd.image:
                continue
            rect = (int(problem.patch_x0[p]), int(problem.patch_y0[p]),
                    int(problem.patch_w[p]), int(problem.patch_h[p]))
            mask = _in_rect(pd.px, pd.py, rect)
            if not bool(mask.any()):
                continue
            tht = Theta.from_vector(torch.as_tensor(thetas[t], dtype=DT))
            E, V = source_moments(tht, pd, problem.model, pd.px[mask], pd.py[mask])
            bgE[mask] += E
            bgV[mask] += V
    return bgE, bgV


def render_source_patch(problem, s, theta_s=None):
    """Own E_q[l f] and V_q[l f] of source s over each of its patches."""
    t = torch.as_tensor(problem.theta[s] if theta_s is None else theta_s, dtype=DT)
    th = Theta.from_vector(t)
    return [source_moments(th, pd, problem.model) for pd in gather_patches(problem, s)]


# ---------------------------------------------------------------------------
# Eqs. eq:kl, kleq, Supplement A and the GMM colour bound of Sec. 4.2.3
# ---------------------------------------------------------------------------

def _kl_gauss_diag_full(mq, vq, mp, Cp):
    """KL(N(mq, diag vq) || N(mp, Cp)) for 4-vectors."""
    P = torch.linalg.inv(Cp)
    d = mq - mp
    return 0.5 * (torch.sum(torch.diagonal(P) * vq) + d @ P @ d - mq.shape[0]
                  + torch.logdet(Cp) - torch.sum(torch.log(vq)))


def kl_bernoulli(a, prior_a):
    """KL between Bernoulli(a) and Bernoulli(prior_a) (Supplement A)."""
    return a * torch.log(a / prior_a) + (1 - a) * torch.log((1 - a) / (1 - prior_a))


def kl_lognormal(mean, var, prior_mean, prior_var):
    """KL between log-normals with log-space (mean, variance) pairs (Supplement A,
    read with both second parameters as variances of log r)."""
    return 0.5 * (math.log(prior_var) - torch.log(var)
                  + (var + (mean - prior_mean) ** 2) / prior_var - 1.0)


def kl_color_bound(mean, var, w, means, covs):
    """Sec. 4.2.3: the GMM-prior bound min over xi of
    KL(xi || w) + sum_j xi_j KL(q || N_j) = -log sum_j w_j exp(-KL(q || N_j))."""
    kls = torch.stack([
        _kl_gauss_diag_full(mean, var, torch.tensor(means[j], dtype=DT),
                            torch.tensor(covs[j], dtype=DT))
        for j in range(len(w))])
    return -torch.logsumexp(torch.log(torch.tensor(w, dtype=DT)) - kls, dim=0)


def neglog_lognormal(value, mean, var):
    """-log density of a log-normal prior at a point mass."""
    lv = torch.log(value)
    return lv + 0.5 * math.log(2 * math.pi * var) + (lv - mean) ** 2 / (2 * var)


def neglog_beta(value, b1, b2):
    """-log density of a Beta(b1, b2) prior at a point mass."""
    logB = math.lgamma(b1) + math.lgamma(b2) - math.lgamma(b1 + b2)
    return -(b1 - 1) * torch.log(value) - (b2 - 1) * torch.log(1 - value) + logB


def kl_source(th: Theta, model):
    """D_KL(q(z_s), p(z_s)) of Eq. kleq under the readings listed above."""
    a = th.a_star
    kl = kl_bernoulli(a, model.prior_a)
    for i, qi in ((0, 1 - a), (1, a)):
        kl_r = kl_lognormal(th.logr_mean[i], th.logr_var[i],
                            float(model.prior_r[i, 0]), float(model.prior_r[i, 1]))
        kl_c = kl_color_bound(th.color_mean[i], th.color_var[i], model.color_w[i],
                              model.color_mean[i], model.color_cov[i])
        kl = kl + qi * (kl_r + kl_c)
    kl = kl + neglog_lognormal(th.radius, float(model.e_radius[0]), float(model.e_radius[1]))
    kl = kl + neglog_beta(th.axis, float(model.e_axis[0]), float(model.e_axis[1]))
    kl = kl + neglog_beta(th.profile, float(model.e_profile[0]), float(model.e_profile[1]))
    return kl


# ---------------------------------------------------------------------------
# Eq. elbo, restricted to the terms that depend on theta_s
# ---------------------------------------------------------------------------

def source_elbo_parts(problem, s, theta_s, patches=None, backgrounds=None):
    """(L_s, L_s^base, KL_s).

    L_s = sum over the pixels of s's patches of the pixel term, minus KL_s.
    L_s^base is the same pixel sum with source s absent (sky and neighbours
    only); it does not depend on theta_s.
    """
    th = Theta.from_vector(theta_s)
    patches = gather_patches(problem, s) if patches is None else patches
    if backgrounds is None:
        backgrounds = [background_patch(problem, s, pd) for pd in patches]
    total = 0.0
    base = 0.0
    for pd, (bgE, bgV) in zip(patches, backgrounds):
        E, V = source_moments(th, pd, problem.model)
        total = total + torch.sum(pixel_term(pd.x, bgE + E, bgV + V))
        base = base + torch.sum(pixel_term(pd.x, bgE, bgV))
    kl = kl_source(th, problem.model)
    return total - kl, base, kl


def source_elbo(problem, s, theta_s=None):
    t = torch.as_tensor(problem.theta[s] if theta_s is None else theta_s, dtype=DT)
    L, base, _ = source_elbo_parts(problem, s, t)
    return float(L), float(base)


def elbo_grad_hess(problem, s, theta_s=None, patches=None, backgrounds=None):
    """Value, gradient and Hessian of L_s over the 27 coordinates (autograd).

    Returns a dict with 'elbo' (L_s), 'elbo_rel' (L_s - L_s^base), 'grad' [27]
    and 'hess' [27, 27], all float64 numpy.
    """
    t0 = torch.as_tensor(problem.theta[s] if theta_s is None else theta_s, dtype=DT).clone()
    patches = gather_patches(problem, s) if patches is None else patches
    if backgrounds is None:
        backgrounds = [background_patch(problem, s, pd) for pd in patches]

    def f(t):
        return source_elbo_parts(problem, s, t, patches, backgrounds)[0]

    t = t0.clone().requires_grad_(True)
    L, base, kl = source_elbo_parts(problem, s, t, patches, backgrounds)
    (g,) = torch.autograd.grad(L, t)
    H = torch.autograd.functional.hessian(f, t0)
    L, kl = L.detach(), kl.detach()
    return dict(elbo=float(L), elbo_rel=float(L - base), base=float(base),
                kl=float(kl), grad=g.detach().numpy().copy(), hess=H.detach().numpy().copy())


def abs_sum_scales(problem, s, theta_s=None, patches=None, backgrounds=None, chunk=512):
    """Magnitude scales for the parity tolerances.

    value: sum over pixels of |term - term_base| plus |KL|;
    grad[k]: sum over pixels of |d term / d theta_k| plus |d KL / d theta_k|;
    hess[j, k]: the same with second derivatives.
    """
    from torch.func import grad as fgrad, hessian as fhess, vmap
    t0 = torch.as_tensor(problem.theta[s] if theta_s is None else theta_s, dtype=DT).clone()
    patches = gather_patches(problem, s) if patches is None else patches
    if backgrounds is None:
        backgrounds = [background_patch(problem, s, pd) for pd in patches]
    model = problem.model
    sv = torch.zeros((), dtype=DT)
    sg = torch.zeros(N_THETA, dtype=DT)
    sh = torch.zeros(N_THETA, N_THETA, dtype=DT)
    for pd, (bgE, bgV) in zip(patches, backgrounds):
        def one(t, px, py, x, be, bv, pd=pd):
            th = Theta.from_vector(t)
            E, V = source_moments(th, pd, model, px, py)
            return pixel_term(x, be + E, bv + V) - pixel_term(x, be, bv)
        for c0 in range(0, pd.px.shape[0], chunk):
            sl = slice(c0, c0 + chunk)
            args = (pd.px[sl], pd.py[sl], pd.x[sl], bgE[sl], bgV[sl])
            sv = sv + vmap(one, in_dims=(None, 0, 0, 0, 0, 0))(t0, *args).abs().sum()
            sg = sg + vmap(fgrad(one), in_dims=(None, 0, 0, 0, 0, 0))(t0, *args).abs().sum(0)
            sh = sh + vmap(fhess(one), in_dims=(None, 0, 0, 0, 0, 0))(t0, *args).abs().sum(0)

    def klf(t):
        return kl_source(Theta.from_vector(t), model)
    sv = sv + klf(t0).abs()
    sg = sg + fgrad(klf)(t0).abs()
    sh = sh + fhess(klf)(t0).abs()
    return dict(elbo=float(sv), grad=sg.numpy().copy(), hess=sh.numpy().copy())


def full_field_elbo(problem, thetas=None):
    """Eq. elbo over every pixel of every image (each source on its patches).

    Sum over all pixels of the pixel term with E and V summed over the
    sources whose patches contain the pixel, minus the sum of all KL_s.
    """
    thetas = problem.theta if thetas is None else thetas
    total = 0.0
    for n in range(problem.n_images):
        H, W = int(problem.img_h[n]), int(problem.img_w[n])
        ys, xs = torch.meshgrid(torch.arange(H, dtype=DT), torch.arange(W, dtype=DT), indexing="ij")
        px, py = xs.reshape(-1), ys.reshape(-1)
        E = sky_at(problem, n, px, py)
        V = torch.zeros_like(E)
        x = torch.tensor(np.ascontiguousarray(problem.image(n)), dtype=DT).reshape(-1)
        pdn = PatchData(image=n, band=int(problem.img_band[n]), px=px, py=py, x=x, sky=E,
                        calib=float(problem.img_calib[n]),
                        A=torch.tensor(problem.img_A[n], dtype=DT),
                        t=torch.tensor(problem.img_t[n], dtype=DT),
                        psf=torch.tensor(problem.img_psf[n], dtype=DT), rect=(0, 0, W, H))
        E = E.clone()
        for s in range(problem.n_sources):
            th = Theta.from_vector(torch.as_tensor(thetas[s], dtype=DT))
            for p in range(int(problem.patch_ptr[s]), int(problem.patch_ptr[s + 1])):
                if int(problem.patch_img[p]) != n:
                    continue
                x0, y0 = int(problem.patch_x0[p]), int(problem.patch_y0[p])
                w, h = int(problem.patch_w[p]), int(problem.patch_h[p])
                idx = (torch.arange(y0, y0 + h)[:, None] * W + torch.arange(x0, x0 + w)[None, :]).reshape(-1)
                Es, Vs = source_moments(th, pdn, problem.model, px[idx], py[idx])
                E[idx] += Es
                V[idx] += Vs
        total = total + float(torch.sum(pixel_term(x, E, V)))
    for s in range(problem.n_sources):
        total -= float(kl_source(Theta.from_vector(torch.as_tensor(thetas[s], dtype=DT)), problem.model))
    return total
