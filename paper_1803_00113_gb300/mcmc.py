"""Posterior sampling of one source by annealed importance sampling (AIS) and
slice sampling (Sec. 3), on the library's log-likelihood.

For a source s with its neighbours fixed, each source type a (star or
galaxy) gets N' AIS runs from the prior to the posterior through T annealed
targets pi_t(w) = p(w | a) p(x | w, a)^gamma_t, each transition one sweep of
slice sampling within Gibbs (stepping out, then shrinkage) over the
coordinates of w.  The AIS weights estimate the marginal likelihoods
p(x | a), whose ratio with the prior gives P(a | x); the final states start
B' further slice-sampling sweeps for posterior samples.

Every chain is independent, so all chains of both types advance in lock
step: each round of the sampler asks for one log-likelihood per chain, and
all of them are one call of ``celeste.loglik`` on a problem holding one copy
of the source per chain (the copies share the source's patches and
neighbours and are not each other's neighbours).  A copy's theta encodes the
point values w: log-variances of -40 and a type logit of +-40 make the
variational moments those of the point, so the call returns
log p(x | w, a) - log p(x | source absent) (the Poisson log-likelihood up
to a constant).  The sampler's own bookkeeping (slice levels, brackets,
proposals) is vectorised numpy on the host; random numbers come from a
seeded numpy generator.

Coordinates of w: star (u_x, u_y, log r, c_1..c_4); galaxy adds (angle,
log radius, axis, profile).  Priors follow the model: log r normal, colours
a Gaussian mixture, log radius normal, axis and profile Beta, angle uniform
on (0, pi), position uniform on a box of +-``box`` pixels around the
source's current position.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np
import torch

import fields
from . import celeste as cel

POINT_LOGVAR = -40.0
TYPE_LOGIT = 40.0
STAR, GALAXY = 1, 0          # type index of the model's arrays


def _betaln(a, b):
    return math.lgamma(a) + math.lgamma(b) - math.lgamma(a + b)


class Prior:
    """p(w | a) for one type: log density, draws and support."""

    def __init__(self, model, kind: int, u0, box: float = 2.0):
        self.m = model
        self.kind = kind
        self.dim = 7 if kind == STAR else 11
        lo = np.full(self.dim, -np.inf)
        hi = np.full(self.dim, np.inf)
        lo[0:2] = np.asarray(u0) - box
        hi[0:2] = np.asarray(u0) + box
        if kind == GALAXY:
            lo[7], hi[7] = 0.0, math.pi
            lo[9], hi[9] = 0.0, 1.0
            lo[10], hi[10] = 0.0, 1.0
        self.lo, self.hi = lo, hi
        self.box = box
        i = kind
        self.cw = np.asarray(model.color_w[i])
        self.cm = np.asarray(model.color_mean[i])
        self.cc = np.asarray(model.color_cov[i])
        self.cprec = np.linalg.inv(self.cc)
        self.clogdet = np.linalg.slogdet(self.cc)[1]
        self.cchol = np.linalg.cholesky(self.cc)

    def logpdf(self, W):
        W = np.atleast_2d(W)
        inside = np.all((W > self.lo) & (W < self.hi), axis=1)
        out = np.full(W.shape[0], -np.inf)
        Wi = W[inside]
        lp = np.full(Wi.shape[0], -2.0 * math.log(2.0 * self.box))       # position box
        m, v = self.m.prior_r[self.kind]
        lp += -0.5 * ((Wi[:, 2] - m) ** 2 / v + math.log(2 * math.pi * v))
        d = Wi[:, None, 3:7] - self.cm[None]                              # [n, J, 4]
        q = np.einsum("njk,jkl,njl->nj", d, self.cprec, d)
        comp = np.log(self.cw)[None] - 0.5 * (q + self.clogdet + 4 * math.log(2 * math.pi))
        mx = comp.max(axis=1)
        lp += mx + np.log(np.exp(comp - mx[:, None]).sum(axis=1))
        if self.kind == GALAXY:
            lp += -math.log(math.pi)
            mr, vr = self.m.e_radius
            lp += -0.5 * ((Wi[:, 8] - mr) ** 2 / vr + math.log(2 * math.pi * vr))
            for col, (a, b) in ((9, self.m.e_axis), (10, self.m.e_profile)):
                x = Wi[:, col]
                lp += (a - 1) * np.log(x) + (b - 1) * np.log1p(-x) - _betaln(a, b)
        out[inside] = lp
        return out

    def sample(self, rng, n):
        W = np.empty((n, self.dim))
        W[:, 0:2] = rng.uniform(self.lo[0:2], self.hi[0:2], (n, 2))
        m, v = self.m.prior_r[self.kind]
        W[:, 2] = rng.normal(m, math.sqrt(v), n)
        j = rng.choice(len(self.cw), size=n, p=self.cw)
        W[:, 3:7] = self.cm[j] + np.einsum("nkl,nl->nk", self.cchol[j], rng.standard_normal((n, 4)))
        if self.kind == GALAXY:
            W[:, 7] = rng.uniform(0.0, math.pi, n)
            mr, vr = self.m.e_radius
            W[:, 8] = rng.normal(mr, math.sqrt(vr), n)
            W[:, 9] = rng.beta(*self.m.e_axis, n)
            W[:, 10] = rng.beta(*self.m.e_profile, n)
            W[:, 9:11] = np.clip(W[:, 9:11], 1e-6, 1 - 1e-6)
        return W


def point_theta(W, kind: int, base):
    """theta rows [n, 27] whose variational moments are those of the points W."""
    W = np.atleast_2d(W)
    th = np.tile(np.asarray(base, dtype=np.float64), (W.shape[0], 1))
    th[:, fields.I_A] = TYPE_LOGIT if kind == STAR else -TYPE_LOGIT
    for i in range(2):
        th[:, fields.I_LOGR_MEAN[i]] = W[:, 2]
        th[:, fields.I_LOGR_LOGVAR[i]] = POINT_LOGVAR
        th[:, fields.I_COLOR_MEAN[i]:fields.I_COLOR_MEAN[i] + 4] = W[:, 3:7]
        th[:, fields.I_COLOR_LOGVAR[i]:fields.I_COLOR_LOGVAR[i] + 4] = POINT_LOGVAR
    th[:, fields.I_U:fields.I_U + 2] = W[:, 0:2]
    if kind == GALAXY:
        th[:, fields.I_ANGLE] = W[:, 7]
        th[:, fields.I_LOGRADIUS] = W[:, 8]
        th[:, fields.I_AXIS] = np.log(W[:, 9] / (1 - W[:, 9]))
        th[:, fields.I_PROFILE] = np.log(W[:, 10] / (1 - W[:, 10]))
    return th


def replicate(problem, s: int, n: int):
    """A problem holding source s's neighbours (fixed) and n copies of s.

    Returns (problem, slice of the copies' source ids)."""
    nbrs = [int(t) for t in problem.nbr_idx[problem.nbr_ptr[s]:problem.nbr_ptr[s + 1]]]
    order = nbrs + [s] * n
    pp, keep, nb, nbi = [0], [], [0], []
    remap = {t: k for k, t in enumerate(nbrs)}
    for k, t in enumerate(order):
        keep.extend(range(problem.patch_ptr[t], problem.patch_ptr[t + 1]))
        pp.append(len(keep))
        if k >= len(nbrs):
            nbi.extend(remap[u] for u in nbrs)              # a copy sees s's neighbours
        else:
            nbi.extend(len(nbrs) + c for c in range(n))     # a neighbour sees every copy
        nb.append(len(nbi))
    keep = np.asarray(keep, dtype=np.int64)
    out = dataclasses.replace(problem)
    out.theta = problem.theta[order].copy()
    out.patch_ptr = np.asarray(pp, dtype=np.int32)
    for k in ("patch_img", "patch_x0", "patch_y0", "patch_w", "patch_h"):
        setattr(out, k, getattr(problem, k)[keep].copy())
    out.nbr_ptr = np.asarray(nb, dtype=np.int32)
    out.nbr_idx = np.asarray(nbi, dtype=np.int32)
    out.truth = None
    return out, slice(len(nbrs), len(nbrs) + n)


class GpuLogLik:
    """log p(x | w, a) - log p(x | absent) for batches of (w, a) of one source."""

    def __init__(self, problem, s: int, n: int, device: int = 0):
        self.n = n
        self.rep, self.sl = replicate(problem, s, n)
        self.ctx = cel.Context(problem.model, device=device)
        self.dp = cel.DeviceProblem(self.rep, torch.device("cuda", device))
        self.plan = cel.Plan(self.ctx, self.dp, list(range(self.sl.start, self.sl.stop)))
        self.base = np.asarray(problem.theta[s], dtype=np.float64)
        self.out = torch.empty(n, dtype=torch.float64, device=self.ctx.device)
        self.calls = 0

    def __call__(self, thetas):
        """thetas [n, 27] (point-value encodings) -> numpy [n]."""
        self.dp.theta[self.sl] = torch.as_tensor(thetas, dtype=torch.float64,
                                                 device=self.ctx.device)
        cel.loglik(self.plan, self.out)
        self.calls += 1
        return self.out.cpu().numpy().copy()


def slice_sweep(logp: Callable, W, lp, rng, widths, lo, hi, movable=None, m: int = 8,
                max_shrink: int = 40):
    """One sweep of slice sampling within Gibbs over every coordinate, all
    chains in lock step (Neal 2003, stepping out with at most m steps split
    at random between the sides, then shrinkage).  logp maps [n, d] to [n]
    (-inf outside the support); lp holds logp(W); lo, hi ([n, d] or [d]) are
    the support bounds; movable [n, d] marks the coordinates each chain
    samples (others stay).  Returns (W, lp)."""
    n, d = W.shape
    W = W.copy()
    lp = lp.copy()
    lo = np.broadcast_to(lo, (n, d))
    hi = np.broadcast_to(hi, (n, d))
    movable = np.ones((n, d), dtype=bool) if movable is None else movable
    for k in range(d):
        mv = movable[:, k]
        if not mv.any():
            continue
        w = widths[k]
        y = lp - rng.exponential(1.0, n)                     # log slice level
        L = W[:, k] - rng.uniform(0.0, w, n)
        R = L + w
        J = np.floor(m * rng.uniform(0.0, 1.0, n)).astype(int)
        K = (m - 1) - J
        L = np.maximum(L, lo[:, k])
        R = np.minimum(R, hi[:, k])
        # stepping out: each round a chain probes its left end while it may,
        # then its right end
        left = mv & (J > 0) & (L > lo[:, k])
        right = mv & (K > 0) & (R < hi[:, k])
        for _ in range(m + 1):
            ask = left | right
            if not ask.any():
                break
            P = W.copy()
            P[:, k] = np.where(left, L, R)
            lq = np.full(n, -np.inf)
            lq[ask] = logp(P)[ask]
            above = lq > y
            gl = left & above
            L = np.where(gl, np.maximum(L - w, lo[:, k]), L)
            J = np.where(gl, J - 1, J)
            gr = ~left & right & above
            R = np.where(gr, np.minimum(R + w, hi[:, k]), R)
            K = np.where(gr, K - 1, K)
            right = np.where(~left & right, gr & (K > 0) & (R < hi[:, k]), right)
            left = gl & (J > 0) & (L > lo[:, k])
        # shrinkage
        todo = mv.copy()
        for _ in range(max_shrink):
            if not todo.any():
                break
            x = rng.uniform(L, R)
            P = W.copy()
            P[:, k] = np.where(todo, x, W[:, k])
            lq = logp(P)
            ok = todo & (lq > y)
            W[ok, k] = x[ok]
            lp[ok] = lq[ok]
            L = np.where(todo & ~ok & (x < W[:, k]), x, L)
            R = np.where(todo & ~ok & (x >= W[:, k]), x, R)
            todo &= ~ok
        # a chain out of shrink steps keeps its state for this coordinate
    return W, lp


class JointTarget:
    """Chains of several types in one state array: prior, bounds and the
    batched log-likelihood of all chains at once."""

    def __init__(self, priors, kinds, loglik_theta: Callable, base):
        self.priors = priors
        self.kinds = np.asarray(kinds)
        self.d = max(p.dim for p in priors.values())
        n = len(kinds)
        self.lo = np.zeros((n, self.d))
        self.hi = np.zeros((n, self.d))
        self.movable = np.zeros((n, self.d), dtype=bool)
        for kind, pr in priors.items():
            r = self.kinds == kind
            self.lo[r, :pr.dim] = pr.lo
            self.hi[r, :pr.dim] = pr.hi
            self.movable[r, :pr.dim] = True
        self.lo[~self.movable] = -np.inf
        self.hi[~self.movable] = np.inf
        self.loglik_theta = loglik_theta
        self.base = base

    def sample(self, rng):
        W = np.zeros((len(self.kinds), self.d))
        for kind, pr in self.priors.items():
            r = self.kinds == kind
            W[r, :pr.dim] = pr.sample(rng, int(r.sum()))
        return W

    def logprior(self, W):
        out = np.empty(W.shape[0])
        for kind, pr in self.priors.items():
            r = self.kinds == kind
            out[r] = pr.logpdf(W[r, :pr.dim])
        return out

    def loglik(self, W):
        # proposals outside the support (their prior is zero, so their value
        # is never used) are clipped into it so that every encoding is finite
        W = np.clip(W, np.nextafter(self.lo, np.inf), np.nextafter(self.hi, -np.inf))
        th = np.empty((W.shape[0], fields.N_THETA))
        for kind, pr in self.priors.items():
            r = self.kinds == kind
            th[r] = point_theta(W[r, :pr.dim], kind, self.base)
        return self.loglik_theta(th)


def ais(target: JointTarget, T: int, rng, widths, B: int = 0):
    """AIS from the prior to prior x likelihood, gamma_t = (t / T)^4, one
    slice-sampling sweep per temperature, then B sweeps at gamma = 1.
    Returns (log weights [n], final states, samples [B, n, d])."""
    W = target.sample(rng)
    ll = target.loglik(W)
    logw = np.zeros(W.shape[0])
    gam = (np.arange(T + 1) / T) ** 4

    def make(g):
        def logp(P):
            lp = target.logprior(P)
            out = np.full(P.shape[0], -np.inf)
            fin = np.isfinite(lp)
            if fin.any():
                out[fin] = lp[fin] + g * target.loglik(P)[fin]
            return out
        return logp

    for t in range(1, T + 1):
        logw += (gam[t] - gam[t - 1]) * ll
        g = gam[t]
        logp = make(g)
        W, lpt = slice_sweep(logp, W, target.logprior(W) + g * ll, rng, widths, target.lo,
                             target.hi, target.movable)
        ll = (lpt - target.logprior(W)) / g
    samples = []
    logp = make(1.0)
    lpc = target.logprior(W) + ll
    for _ in range(B):
        W, lpc = slice_sweep(logp, W, lpc, rng, widths, target.lo, target.hi, target.movable)
        samples.append(W.copy())
    return logw, W, np.asarray(samples)


def log_mean_exp(a):
    m = np.max(a)
    return m + math.log(np.mean(np.exp(a - m)))


def type_posterior(problem, s: int, n_chains: int = 25, T: int = 200, B: int = 25,
                   seed: int = 0, device: int = 0, box: float = 2.0):
    """AIS for both types of source s (N' = n_chains runs each, all chains
    in lock step and every round one library call), then B slice-sampling
    sweeps from the final states.  Returns a dict: p_star, log evidence and
    samples per type, number of log-likelihood calls."""
    rng = np.random.default_rng(seed)
    u0 = problem.theta[s, fields.I_U:fields.I_U + 2]
    priors = {STAR: Prior(problem.model, STAR, u0, box),
              GALAXY: Prior(problem.model, GALAXY, u0, box)}
    kinds = [STAR] * n_chains + [GALAXY] * n_chains
    ev = GpuLogLik(problem, s, 2 * n_chains, device)
    target = JointTarget(priors, kinds, ev, problem.theta[s])
    widths = np.full(target.d, 0.5)
    logw, W, samples = ais(target, T, rng, widths, B)
    kinds = np.asarray(kinds)
    out = {}
    for kind in (STAR, GALAXY):
        r = kinds == kind
        out[kind] = dict(log_evidence=log_mean_exp(logw[r]), logw=logw[r],
                         samples=samples[:, r, :priors[kind].dim].reshape(-1, priors[kind].dim))
    la = math.log(problem.model.prior_a) + out[STAR]["log_evidence"]
    lb = math.log(1.0 - problem.model.prior_a) + out[GALAXY]["log_evidence"]
    p_star = 1.0 / (1.0 + math.exp(min(lb - la, 700.0)))
    return dict(p_star=p_star, star=out[STAR], galaxy=out[GALAXY], calls=ev.calls)
