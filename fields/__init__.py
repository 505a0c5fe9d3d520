"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This module only *draws inputs*: images of Poisson photon counts, per-image
instrument descriptors (band, sky knots, calibration, linear WCS, Gaussian
mixture PSF), light sources with their variational parameters, patch
rectangles, neighbour lists and the model constants (galaxy profile mixtures
and prior hyperparameters).  It contains none of the inference arithmetic:
no ELBO, no derivatives, no Newton step.  To synthesise counts it renders a
deliberately simplified "truth" (each source one PSF-convolved Gaussian per
PSF component), which is data synthesis only and is not used by either side.

Shapes follow the paper's study set (Sec. 5.1: five overlapping 2048 x 1489
images holding a few hundred sources).  Units: positions and radii are in
reference-frame pixels, fluxes in nanomaggies, images in photon counts.

Variational parameter vector (27 unconstrained coordinates per source; type
0 = galaxy, 1 = star, following Eq. ``eq0``-``eq1``):

    0        logit of q(a = star)
    1, 2     galaxy: mean of log r, log of the variance of log r
    3, 4     star:   mean of log r, log of the variance of log r
    5..8     galaxy colour means        9..12   star colour means
    13..16   galaxy log colour variances 17..20  star log colour variances
    21, 22   position u (x = column, y = row) in the reference frame
    23       angle of the major axis (radians)
    24       log half-light radius (reference-frame pixels)
    25       logit of the minor/major axis ratio
    26       logit of the profile weight (weight of the exponential profile)
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

N_THETA = 27
N_BANDS = 5
REF_BAND = 2          # r band (u, g, r, i, z order)
N_PSF = 3
N_COLOR_COMP = 8      # J, colour prior mixture components per type

I_A = 0
I_LOGR_MEAN = (1, 3)
I_LOGR_LOGVAR = (2, 4)
I_COLOR_MEAN = (5, 9)
I_COLOR_LOGVAR = (13, 17)
I_U = 21
I_ANGLE = 23
I_LOGRADIUS = 24
I_AXIS = 25
I_PROFILE = 26

_HERE = os.path.dirname(os.path.abspath(__file__))


def _logit(p):
    return math.log(p / (1.0 - p))


# --------------------------------------------------------------------------
# model constants
# --------------------------------------------------------------------------

@dataclass
class Model:
    """Galaxy profile mixtures and prior hyperparameters (Table 3)."""
    alpha_exp: np.ndarray
    tau_exp: np.ndarray
    alpha_dev: np.ndarray
    tau_dev: np.ndarray
    prior_a: float                 # prior probability of a star
    prior_r: np.ndarray            # [2, 2]: (mean, variance) of log r per type
    color_w: np.ndarray            # [2, J]
    color_mean: np.ndarray         # [2, J, 4]
    color_cov: np.ndarray          # [2, J, 4, 4]
    e_radius: np.ndarray           # (mean, variance) of log radius
    e_profile: np.ndarray          # Beta parameters
    e_axis: np.ndarray             # Beta parameters


def load_profiles():
    with open(os.path.join(_HERE, "galaxy_profiles.json")) as f:
        d = json.load(f)
    return (np.array(d["exp"]["alpha"]), np.array(d["exp"]["tau"]),
            np.array(d["dev"]["alpha"]), np.array(d["dev"]["tau"]))


def make_model(seed: int = 1803_00113) -> Model:
    """Seeded synthetic hyperparameters shaped like the paper's priors."""
    rng = np.random.default_rng(seed)
    ae, te, ad, td = load_profiles()
    J = N_COLOR_COMP
    color_w = np.empty((2, J))
    color_mean = np.empty((2, J, 4))
    color_cov = np.empty((2, J, 4, 4))
    centre = np.array([[1.2, 0.6, 0.35, 0.3],     # galaxy colour centre
                       [0.9, 0.4, 0.15, 0.08]])   # star colour centre
    for i in range(2):
        color_w[i] = rng.dirichlet(np.full(J, 3.0))
        for j in range(J):
            color_mean[i, j] = centre[i] + rng.normal(0.0, 0.3, 4)
            L = np.tril(rng.normal(0.0, 0.08, (4, 4)))
            L[np.diag_indices(4)] = rng.uniform(0.08, 0.3, 4)
            color_cov[i, j] = L @ L.T
    return Model(
        alpha_exp=ae, tau_exp=te, alpha_dev=ad, tau_dev=td,
        prior_a=0.3,
        prior_r=np.array([[math.log(5.0), 1.2 ** 2], [math.log(5.0), 1.3 ** 2]]),
        color_w=color_w, color_mean=color_mean, color_cov=color_cov,
        e_radius=np.array([math.log(1.5), 0.5 ** 2]),
        e_profile=np.array([1.5, 1.5]),
        e_axis=np.array([2.0, 1.6]),
    )


# --------------------------------------------------------------------------
# the problem container
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """Images, sources and model constants, as flat host arrays.

    Images share one float32 pixel pool (row-major, ``img_stride`` elements
    per row) and one float32 pool of sky knots (``sky_ny`` x ``sky_nx`` grid
    per image, interpolated bilinearly between knots that span the image).
    A linear WCS maps a reference-frame position u to pixel coordinates
    (x = column, y = row) of image n as ``A[n] @ u + t[n]``; pixel (row i,
    col j) has its centre at (x, y) = (j, i).  ``img_psf[n, k]`` holds the
    weight, mean offset (x, y) and covariance (xx, xy, yy) of PSF component k.

    Source s owns the patches ``patch_ptr[s]:patch_ptr[s+1]``; patch p is the
    rectangle ``[x0, x0+w) x [y0, y0+h)`` of image ``patch_img[p]``.  Its
    neighbours (other sources whose patches it overlaps) are
    ``nbr_idx[nbr_ptr[s]:nbr_ptr[s+1]]``.
    """
    model: Model
    pixels: np.ndarray
    sky: np.ndarray
    img_band: np.ndarray
    img_h: np.ndarray
    img_w: np.ndarray
    img_stride: np.ndarray
    img_pix_off: np.ndarray
    img_sky_off: np.ndarray
    img_sky_ny: np.ndarray
    img_sky_nx: np.ndarray
    img_calib: np.ndarray
    img_A: np.ndarray
    img_t: np.ndarray
    img_psf: np.ndarray
    theta: np.ndarray
    patch_ptr: np.ndarray
    patch_img: np.ndarray
    patch_x0: np.ndarray
    patch_y0: np.ndarray
    patch_w: np.ndarray
    patch_h: np.ndarray
    nbr_ptr: np.ndarray
    nbr_idx: np.ndarray
    truth: Optional[dict] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_sources(self):
        return int(self.theta.shape[0])

    @property
    def n_images(self):
        return int(self.img_band.shape[0])

    @property
    def n_patches(self):
        return int(self.patch_img.shape[0])

    def visits(self, sources=None):
        """Source-pixel visits of one evaluation: sum of patch areas."""
        area = self.patch_w.astype(np.int64) * self.patch_h.astype(np.int64)
        if sources is None:
            return int(area.sum())
        return int(sum(area[self.patch_ptr[s]:self.patch_ptr[s + 1]].sum() for s in sources))

    def image(self, n):
        off = int(self.img_pix_off[n])
        h, w, st = int(self.img_h[n]), int(self.img_w[n]), int(self.img_stride[n])
        return self.pixels[off:off + h * st].reshape(h, st)[:, :w]

    def sky_grid(self, n):
        off = int(self.img_sky_off[n])
        ny, nx = int(self.img_sky_ny[n]), int(self.img_sky_nx[n])
        return self.sky[off:off + ny * nx].reshape(ny, nx)

    def subset(self, sources):
        """A problem holding the listed sources (neighbour lists restricted)."""
        sources = [int(s) for s in sources]
        remap = {s: i for i, s in enumerate(sources)}
        pp = [0]
        keep = []
        nb = [0]
        nbi = []
        for s in sources:
            keep.extend(range(self.patch_ptr[s], self.patch_ptr[s + 1]))
            pp.append(len(keep))
            for t in self.nbr_idx[self.nbr_ptr[s]:self.nbr_ptr[s + 1]]:
                if int(t) in remap:
                    nbi.append(remap[int(t)])
            nb.append(len(nbi))
        keep = np.array(keep, dtype=np.int64)
        out = Problem(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        out.theta = self.theta[sources].copy()
        out.patch_ptr = np.array(pp, dtype=np.int32)
        for k in ("patch_img", "patch_x0", "patch_y0", "patch_w", "patch_h"):
            setattr(out, k, getattr(self, k)[keep].copy())
        out.nbr_ptr = np.array(nb, dtype=np.int32)
        out.nbr_idx = np.array(nbi, dtype=np.int32)
        out.truth = None
        return out


# --------------------------------------------------------------------------
# drawing images, PSFs and sources
# --------------------------------------------------------------------------

def _draw_psf(rng, offsets=False):
    w = np.sort(rng.dirichlet([4.0, 2.0, 1.0]))[::-1]
    psf = np.zeros((N_PSF, 6))
    for k, (lo, hi) in enumerate(((1.0, 1.6), (1.6, 2.5), (2.5, 4.0))):
        sig = rng.uniform(lo, hi)
        e = rng.uniform(0.0, 0.08)
        phi = rng.uniform(0.0, math.pi)
        R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
        C = R @ np.diag([(sig * (1 + e)) ** 2, (sig * (1 - e)) ** 2]) @ R.T
        mx, my = (rng.uniform(-0.15, 0.15, 2) if offsets else (0.0, 0.0))
        psf[k] = (w[k], mx, my, C[0, 0], C[0, 1], C[1, 1])
    return psf


def _draw_wcs(rng, jitter=True):
    if not jitter:
        return np.eye(2), np.zeros(2)
    rot = rng.uniform(-0.004, 0.004)
    sc = 1.0 + rng.uniform(-0.002, 0.002, 2)
    A = np.array([[math.cos(rot), -math.sin(rot)], [math.sin(rot), math.cos(rot)]]) @ np.diag(sc)
    t = rng.uniform(-1.5, 1.5, 2)
    return A, t


def _draw_truth(rng, model: Model, star_frac, n):
    """Per-source truth: type, reference flux, colours, shape."""
    is_star = rng.uniform(size=n) < star_frac
    logr = rng.normal(math.log(5.0), 1.2, n)
    centre = np.where(is_star[:, None], np.array([0.9, 0.4, 0.15, 0.08]),
                      np.array([1.2, 0.6, 0.35, 0.3]))
    colors = centre + rng.normal(0.0, 0.25, (n, 4))
    axis = rng.uniform(0.2, 1.0, n)
    angle = rng.uniform(0.0, math.pi, n)
    radius = np.exp(rng.normal(math.log(1.5), 0.5, n))
    profile = rng.uniform(0.0, 1.0, n)
    return dict(is_star=is_star, logr=logr, colors=colors, axis=axis,
                angle=angle, radius=radius, profile=profile)


_BAND_SEL = np.array([[-1, -1, 0, 0], [0, -1, 0, 0], [0, 0, 0, 0],
                      [0, 0, 1, 0], [0, 0, 1, 1]], dtype=np.float64)


def _band_flux(truth, s, b):
    return math.exp(truth["logr"][s] + float(_BAND_SEL[b] @ truth["colors"][s]))


def _truth_cov(truth, s):
    """Covariance of the single Gaussian standing in for source s (ref frame)."""
    if truth["is_star"][s]:
        return np.zeros((2, 2))
    r, ax, ang = truth["radius"][s], truth["axis"][s], truth["angle"][s]
    # a Gaussian with half-light radius r has variance r^2 / (2 ln 2)
    v = r * r / (2.0 * math.log(2.0))
    R = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    return R.T @ np.diag([v, v * ax * ax]) @ R


def _init_theta(rng, truth, pos, n):
    """Variational parameters near (not at) the truth."""
    th = np.zeros((n, N_THETA))
    for s in range(n):
        th[s, I_A] = _logit(0.8 if truth["is_star"][s] else 0.2) + rng.normal(0, 0.3)
        for i in range(2):
            th[s, I_LOGR_MEAN[i]] = truth["logr"][s] + rng.normal(0, 0.15)
            th[s, I_LOGR_LOGVAR[i]] = math.log(0.02) + rng.normal(0, 0.3)
            th[s, I_COLOR_MEAN[i]:I_COLOR_MEAN[i] + 4] = truth["colors"][s] + rng.normal(0, 0.08, 4)
            th[s, I_COLOR_LOGVAR[i]:I_COLOR_LOGVAR[i] + 4] = math.log(0.01) + rng.normal(0, 0.3, 4)
        th[s, I_U:I_U + 2] = pos[s] + rng.uniform(-0.3, 0.3, 2)
        th[s, I_ANGLE] = truth["angle"][s] + rng.normal(0, 0.1)
        th[s, I_LOGRADIUS] = math.log(truth["radius"][s]) + rng.normal(0, 0.1)
        th[s, I_AXIS] = _logit(min(max(truth["axis"][s], 0.05), 0.95)) + rng.normal(0, 0.2)
        th[s, I_PROFILE] = _logit(min(max(truth["profile"][s], 0.05), 0.95)) + rng.normal(0, 0.2)
    return th


def _patch_side(truth, s, sky_min, calib):
    """Odd side covering where the noiseless source exceeds 0.2 sqrt(sky)."""
    flux = max(_band_flux(truth, s, b) for b in range(N_BANDS)) * calib
    C = _truth_cov(truth, s)
    sig2 = 4.0 ** 2 + max(float(np.linalg.eigvalsh(C)[-1]), 0.0)
    peak = flux / (2.0 * math.pi * sig2)
    thr = 0.2 * math.sqrt(sky_min)
    R = math.sqrt(2.0 * sig2 * math.log(peak / thr)) if peak > thr else 0.0
    return int(min(max(2 * math.ceil(R) + 1, 15), 101))


class _Builder:
    """Accumulates images and sources into the flat arrays of a Problem."""

    def __init__(self, model):
        self.model = model
        self.pix = []
        self.sky = []
        self.npix = 0
        self.nsky = 0
        self.img = []
        self.theta = []
        self.patches = []   # per source: list of (img, x0, y0, w, h)
        self.nbrs = []

    def add_image(self, band, h, w, sky_knots, calib, A, t, psf):
        stride = w
        self.img.append(dict(band=band, h=h, w=w, stride=stride, pix_off=self.npix,
                             sky_off=self.nsky, sky_ny=sky_knots.shape[0],
                             sky_nx=sky_knots.shape[1], calib=calib, A=A, t=t, psf=psf))
        self.pix.append(np.zeros(h * stride, dtype=np.float64))
        self.npix += h * stride
        self.sky.append(sky_knots.astype(np.float32).ravel())
        self.nsky += sky_knots.size
        return len(self.img) - 1

    def sky_at(self, n):
        d = self.img[n]
        if d["sky_ny"] == 1 and d["sky_nx"] == 1:
            return np.full((d["h"], d["w"]), float(self.sky[n][0]))
        knots = self.sky[n].astype(np.float64).reshape(d["sky_ny"], d["sky_nx"])
        h, w = d["h"], d["w"]
        ys = np.arange(h) * ((d["sky_ny"] - 1) / max(h - 1, 1))
        xs = np.arange(w) * ((d["sky_nx"] - 1) / max(w - 1, 1))
        # separable linear interpolation between knots (data synthesis only)
        rows = np.array([np.interp(xs, np.arange(d["sky_nx"]), knots[i]) for i in range(d["sky_ny"])])
        return np.array([np.interp(ys, np.arange(d["sky_ny"]), rows[:, j]) for j in range(w)]).T

    def finish(self, rng, truth, name, meta):
        # photon counts: Poisson draws around sky + the simplified truth render
        # (sky >= 50 counts everywhere, so a rounded normal with variance
        # lambda stands in for the Poisson draw; this keeps large batches fast)
        lam = np.concatenate(self.pix)
        off = 0
        for n, d in enumerate(self.img):
            size = d["h"] * d["stride"]
            if d["sky_ny"] == 1 and d["sky_nx"] == 1:
                lam[off:off + size] += float(self.sky[n][0])
            else:
                lam[off:off + size] += self.sky_at(n).ravel()
            off += size
        z = rng.standard_normal(lam.size, dtype=np.float32)
        z *= np.sqrt(lam.astype(np.float32))
        counts = np.maximum(np.rint(lam + z), 0.0).astype(np.float32)
        off = 0
        for n, d in enumerate(self.img):
            size = d["h"] * d["stride"]
            self.pix[n] = counts[off:off + size]
            off += size
        pp = np.zeros(len(self.patches) + 1, dtype=np.int32)
        flat = []
        for s, pl in enumerate(self.patches):
            flat.extend(pl)
            pp[s + 1] = len(flat)
        flat = np.array(flat, dtype=np.int32).reshape(-1, 5)
        nb = np.zeros(len(self.nbrs) + 1, dtype=np.int32)
        for s, l in enumerate(self.nbrs):
            nb[s + 1] = nb[s] + len(l)
        nbi = np.array([t for l in self.nbrs for t in l], dtype=np.int32)
        I = self.img
        return Problem(
            model=self.model,
            pixels=counts,
            sky=np.concatenate(self.sky).astype(np.float32),
            img_band=np.array([d["band"] for d in I], dtype=np.int32),
            img_h=np.array([d["h"] for d in I], dtype=np.int32),
            img_w=np.array([d["w"] for d in I], dtype=np.int32),
            img_stride=np.array([d["stride"] for d in I], dtype=np.int32),
            img_pix_off=np.array([d["pix_off"] for d in I], dtype=np.int64),
            img_sky_off=np.array([d["sky_off"] for d in I], dtype=np.int64),
            img_sky_ny=np.array([d["sky_ny"] for d in I], dtype=np.int32),
            img_sky_nx=np.array([d["sky_nx"] for d in I], dtype=np.int32),
            img_calib=np.array([d["calib"] for d in I], dtype=np.float64),
            img_A=np.array([d["A"] for d in I], dtype=np.float64),
            img_t=np.array([d["t"] for d in I], dtype=np.float64),
            img_psf=np.array([d["psf"] for d in I], dtype=np.float64),
            theta=np.array(self.theta, dtype=np.float64).reshape(-1, N_THETA),
            patch_ptr=pp,
            patch_img=flat[:, 0].copy(), patch_x0=flat[:, 1].copy(),
            patch_y0=flat[:, 2].copy(), patch_w=flat[:, 3].copy(),
            patch_h=flat[:, 4].copy(),
            nbr_ptr=nb, nbr_idx=nbi, truth=truth, name=name, meta=meta)


def _render_truth(b: _Builder, n, truth, s, pos, rect):
    """Add source s's simplified truth (counts) to image n over ``rect``."""
    d = b.img[n]
    x0, y0, w, h = rect
    mu = d["A"] @ pos + d["t"]
    Cs = d["A"] @ _truth_cov(truth, s) @ d["A"].T
    flux = _band_flux(truth, s, d["band"]) * d["calib"]
    xs = np.arange(x0, x0 + w, dtype=np.float64)[None, :]
    ys = np.arange(y0, y0 + h, dtype=np.float64)[:, None]
    img = b.pix[n].reshape(d["h"], d["stride"])
    acc = np.zeros((h, w))
    for k in range(N_PSF):
        wk, mx, my, cxx, cxy, cyy = d["psf"][k]
        C = Cs + np.array([[cxx, cxy], [cxy, cyy]])
        P = np.linalg.inv(C)
        dx = xs - mu[0] - mx
        dy = ys - mu[1] - my
        q = P[0, 0] * dx * dx + 2 * P[0, 1] * dx * dy + P[1, 1] * dy * dy
        acc += wk * np.exp(-0.5 * q) / (2 * math.pi * math.sqrt(np.linalg.det(C)))
    img[y0:y0 + h, x0:x0 + w] += flux * acc


def _render_truth_images(b: _Builder, imgs, truth, s, pos, rects):
    """_render_truth for one source over several same-size rectangles at once."""
    if not imgs:
        return
    d0 = b.img[imgs[0]]
    h, w = rects[0][3], rects[0][2]
    A = np.stack([b.img[n]["A"] for n in imgs])                     # [I, 2, 2]
    t = np.stack([b.img[n]["t"] for n in imgs])
    psf = np.stack([b.img[n]["psf"] for n in imgs])                 # [I, K, 6]
    calib = np.array([b.img[n]["calib"] for n in imgs])
    flux = np.array([_band_flux(truth, s, b.img[n]["band"]) for n in imgs]) * calib
    mu = A @ pos + t                                                # [I, 2]
    Cs = A @ _truth_cov(truth, s) @ np.transpose(A, (0, 2, 1))      # [I, 2, 2]
    x0 = np.array([r[0] for r in rects], dtype=np.float64)
    y0 = np.array([r[1] for r in rects], dtype=np.float64)
    xs = x0[:, None, None] + np.arange(w, dtype=np.float64)[None, None, :]
    ys = y0[:, None, None] + np.arange(h, dtype=np.float64)[None, :, None]
    acc = np.zeros((len(imgs), h, w))
    for k in range(N_PSF):
        wk = psf[:, k, 0]
        cxx = Cs[:, 0, 0] + psf[:, k, 3]
        cxy = Cs[:, 0, 1] + psf[:, k, 4]
        cyy = Cs[:, 1, 1] + psf[:, k, 5]
        det = cxx * cyy - cxy * cxy
        dx = xs - (mu[:, 0] + psf[:, k, 1])[:, None, None]
        dy = ys - (mu[:, 1] + psf[:, k, 2])[:, None, None]
        q = (cyy[:, None, None] * dx * dx - 2 * cxy[:, None, None] * dx * dy
             + cxx[:, None, None] * dy * dy) / det[:, None, None]
        acc += (wk / (2 * math.pi * np.sqrt(det)))[:, None, None] * np.exp(-0.5 * q)
    for i, n in enumerate(imgs):
        d = b.img[n]
        img = b.pix[n].reshape(d["h"], d["stride"])
        r = rects[i]
        img[r[1]:r[1] + h, r[0]:r[0] + w] += flux[i] * acc[i]


def _rect_for(b, n, pos, side):
    """Patch rectangle of odd side centred on pos in image n, kept inside it."""
    d = b.img[n]
    p = d["A"] @ pos + d["t"]
    w = min(side, d["w"])
    h = min(side, d["h"])
    x0 = int(round(p[0])) - w // 2
    y0 = int(round(p[1])) - h // 2
    x0 = min(max(x0, 0), d["w"] - w)
    y0 = min(max(y0, 0), d["h"] - h)
    return (x0, y0, w, h)


def _overlap(r1, r2):
    return (r1[0] < r2[0] + r2[2] and r2[0] < r1[0] + r1[2] and
            r1[1] < r2[1] + r2[3] and r2[1] < r1[1] + r1[3])


def _link_neighbours(b, first, last):
    """Neighbours among sources first..last-1: patches overlap in a shared image."""
    for s in range(first, last):
        b.nbrs.append([])
    by_img = {}
    for s in range(first, last):
        for (n, x0, y0, w, h) in b.patches[s]:
            by_img.setdefault(n, []).append((s, (x0, y0, w, h)))
    pairs = set()
    for n, lst in by_img.items():
        if len(lst) > 400:
            # sort-and-sweep on x for large images
            lst = sorted(lst, key=lambda e: e[1][0])
            for i, (s, r) in enumerate(lst):
                for t, q in lst[i + 1:]:
                    if q[0] >= r[0] + r[2]:
                        break
                    if _overlap(r, q):
                        pairs.add((min(s, t), max(s, t)))
        else:
            for i, (s, r) in enumerate(lst):
                for t, q in lst[i + 1:]:
                    if s != t and _overlap(r, q):
                        pairs.add((min(s, t), max(s, t)))
    for s, t in sorted(pairs):
        b.nbrs[s].append(t)
        b.nbrs[t].append(s)
    for s in range(first, last):
        b.nbrs[s].sort()


def plain_source(seed: int = 1803_00113 + 1, side: int = 41, star: Optional[bool] = None,
                 model: Optional[Model] = None, psf_offsets=False, wcs_jitter=True,
                 sky_grid=(1, 1), bands=N_BANDS):
    """One source, one image per band, ``side`` x ``side`` pixel patch."""
    rng = np.random.default_rng(seed)
    model = model or make_model()
    b = _Builder(model)
    truth = _draw_truth(rng, model, 0.3, 1)
    if star is not None:
        truth["is_star"][0] = star
    centre = np.array([(side - 1) / 2.0, (side - 1) / 2.0]) + rng.uniform(-0.5, 0.5, 2)
    imgs = []
    for band in range(bands):
        sky0 = rng.uniform(50.0, 200.0)
        knots = sky0 * (1.0 + rng.uniform(-0.05, 0.05, sky_grid)) if sky_grid != (1, 1) \
            else np.full((1, 1), sky0)
        A, t = _draw_wcs(rng, wcs_jitter)
        # keep the patch exactly the image: shift t so the source stays centred
        t = t - (A @ centre + t - centre) if wcs_jitter else t
        imgs.append(b.add_image(band, side, side, knots, 200.0 * rng.uniform(0.9, 1.1),
                                A, t, _draw_psf(rng, psf_offsets)))
    b.patches.append([(n, 0, 0, side, side) for n in imgs])
    for n in imgs:
        _render_truth(b, n, truth, 0, centre, (0, 0, side, side))
    b.theta.extend(_init_theta(rng, truth, centre[None, :], 1).ravel())
    _link_neighbours(b, 0, 1)
    truth["pos"] = centre[None, :]
    return b.finish(rng, truth, f"plain source, {bands} bands x 1 image, {side}x{side} px", {})


def single_field(seed: int = 1803_00113 + 2, n_sources=600, height=2048, width=1489,
                 star_frac=0.3, model: Optional[Model] = None, min_side=15, max_side=101):
    """A field: one image per band, sources at uniform random positions."""
    rng = np.random.default_rng(seed)
    model = model or make_model()
    b = _Builder(model)
    truth = _draw_truth(rng, model, star_frac, n_sources)
    pos = np.column_stack([rng.uniform(5, width - 6, n_sources),
                           rng.uniform(5, height - 6, n_sources)])
    imgs = []
    for band in range(N_BANDS):
        knots = rng.uniform(50.0, 200.0) * (1.0 + rng.uniform(-0.05, 0.05, (4, 3)))
        A, t = _draw_wcs(rng)
        imgs.append(b.add_image(band, height, width, knots, 200.0 * rng.uniform(0.9, 1.1),
                                A, t, _draw_psf(rng)))
    sky_min = min(float(b.sky[n].min()) for n in imgs)
    for s in range(n_sources):
        side = min(max(_patch_side(truth, s, sky_min, 220.0), min_side), max_side)
        pl = []
        for n in imgs:
            r = _rect_for(b, n, pos[s], side)
            pl.append((n,) + r)
            _render_truth(b, n, truth, s, pos[s], r)
        b.patches.append(pl)
    b.theta.extend(_init_theta(rng, truth, pos, n_sources).ravel())
    _link_neighbours(b, 0, n_sources)
    truth["pos"] = pos
    return b.finish(rng, truth, f"single field, {N_BANDS} bands of {height}x{width} px, "
                    f"{n_sources} sources", {})


def batched(seed: int = 1803_00113 + 3, n_sources=8192, min_side=15, max_side=101,
            max_images_per_band=6, max_neighbours=10, model: Optional[Model] = None,
            star_frac=0.3):
    """Blended groups: uneven patches, 1..6 images per band, 0..10 neighbours.

    Sources come in groups of 1..max_neighbours+1 placed inside each other's
    patches; every group has its own exposures (per band a uniform number of
    images in 1..max_images_per_band, each with its own PSF, sky, calibration
    and WCS jitter).  Patch sides are odd and log-uniform on [min_side, max_side].
    """
    rng = np.random.default_rng(seed)
    model = model or make_model()
    b = _Builder(model)
    truth = _draw_truth(rng, model, star_frac, n_sources)
    pos_all = np.zeros((n_sources, 2))
    s0 = 0
    while s0 < n_sources:
        g = min(int(rng.integers(1, max_neighbours + 2)), n_sources - s0)
        sides = []
        for _ in range(g):
            v = math.exp(rng.uniform(math.log(min_side), math.log(max_side)))
            sd = int(round(v))
            sides.append(sd if sd % 2 == 1 else sd + 1)
        sides = [min(max(x, min_side), max_side) for x in sides]
        smin = min(sides)
        spread = 0.35 * smin
        region = max(sides) + int(2 * spread) + 8
        centre = np.array([region / 2.0, region / 2.0])
        pos = centre + rng.uniform(-spread, spread, (g, 2))
        imgs = []
        for band in range(N_BANDS):
            for _ in range(int(rng.integers(1, max_images_per_band + 1))):
                A, t = _draw_wcs(rng)
                imgs.append(b.add_image(band, region, region, np.full((1, 1), rng.uniform(50, 200)),
                                        200.0 * rng.uniform(0.9, 1.1), A, t, _draw_psf(rng)))
        for k in range(g):
            s = s0 + k
            rects = [_rect_for(b, n, pos[k], sides[k]) for n in imgs]
            _render_truth_images(b, imgs, truth, s, pos[k], rects)
            b.patches.append([(n,) + r for n, r in zip(imgs, rects)])
            pos_all[s] = pos[k]
        _link_neighbours(b, s0, s0 + g)
        s0 += g
    b.theta.extend(_init_theta(rng, truth, pos_all, n_sources).ravel())
    truth["pos"] = pos_all
    return b.finish(rng, truth, f"batched, {n_sources} sources, patches {min_side}..{max_side} px, "
                    f"1..{max_images_per_band} images per band, 0..{max_neighbours} neighbours", {})


def region_request(seed: int, n_sources: Optional[int] = None, side: Optional[int] = None,
                   max_images_per_band=4, max_sources=64, min_region=32, max_region=512,
                   model: Optional[Model] = None, star_frac=0.3):
    """One serving request: a square sky region and the sources inside it.

    Unless given, the source count is log-uniform on [1, max_sources] and the
    region side log-uniform on [min_region, max_region] px; every band has a
    uniform number of exposures in 1..max_images_per_band, each with its own
    PSF, constant sky, calibration and WCS jitter.  Sources sit at uniform
    positions; patches follow the field's rule (odd side where the source
    exceeds 0.2 sqrt(sky), clamped to [15, 101] and to the region).
    """
    rng = np.random.default_rng(seed)
    model = model or make_model()
    if n_sources is None:
        n_sources = int(round(math.exp(rng.uniform(0.0, math.log(max_sources)))))
    if side is None:
        side = int(round(math.exp(rng.uniform(math.log(min_region), math.log(max_region)))))
    b = _Builder(model)
    truth = _draw_truth(rng, model, star_frac, n_sources)
    pos = rng.uniform(3.0, side - 4.0, (n_sources, 2))
    imgs = []
    for band in range(N_BANDS):
        for _ in range(int(rng.integers(1, max_images_per_band + 1))):
            A, t = _draw_wcs(rng)
            imgs.append(b.add_image(band, side, side, np.full((1, 1), rng.uniform(50, 200)),
                                    200.0 * rng.uniform(0.9, 1.1), A, t, _draw_psf(rng)))
    for s in range(n_sources):
        ps = _patch_side(truth, s, 50.0, 220.0)
        rects = [_rect_for(b, n, pos[s], ps) for n in imgs]
        _render_truth_images(b, imgs, truth, s, pos[s], rects)
        b.patches.append([(n,) + r for n, r in zip(imgs, rects)])
    _link_neighbours(b, 0, n_sources)
    b.theta.extend(_init_theta(rng, truth, pos, n_sources).ravel())
    truth["pos"] = pos
    return b.finish(rng, truth, f"region {side}x{side} px, {n_sources} sources, "
                    f"1..{max_images_per_band} images per band", dict(side=side))
