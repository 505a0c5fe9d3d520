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


def replicate(problem, sources, n: int):
    """A problem holding the listed sources' neighbours (fixed, at their
    theta) and n copies of each listed source.  A copy has its source's
    patches and neighbours; copies are nobody's neighbours but their own
    source's neighbours'.  Returns (problem, [slice of each source's copies])."""
    sources = [int(s) for s in sources]
    nbrs = []
    for s in sources:
        for t in problem.nbr_idx[problem.nbr_ptr[s]:problem.nbr_ptr[s + 1]]:
            if int(t) not in nbrs:
                nbrs.append(int(t))
    remap = {t: k for k, t in enumerate(nbrs)}
    order = nbrs + [s for s in sources for _ in range(n)]
    first = {t: [] for t in nbrs}                         # copies that see neighbour t
    for c, s in enumerate(order[len(nbrs):]):
        for t in problem.nbr_idx[problem.nbr_ptr[s]:problem.nbr_ptr[s + 1]]:
            first[int(t)].append(len(nbrs) + c)
    pp, keep, nb, nbi = [0], [], [0], []
    for k, t in enumerate(order):
        keep.extend(range(problem.patch_ptr[t], problem.patch_ptr[t + 1]))
        pp.append(len(keep))
        if k >= len(nbrs):
            nbi.extend(remap[int(u)] for u in problem.nbr_idx[problem.nbr_ptr[t]:problem.nbr_ptr[t + 1]])
        else:
            nbi.extend(first[t])
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
    base = len(nbrs)
    return out, [slice(base + i * n, base + (i + 1) * n) for i in range(len(sources))]


class GpuLogLik:
    """log p(x | w, a) - log p(x | absent) for batches of point values of one
    or several sources: n chains per source, one library call per batch."""

    def __init__(self, problem, sources, n: int, device: int = 0):
        sources = [int(sources)] if np.isscalar(sources) else [int(s) for s in sources]
        self.n = n * len(sources)
        self.rep, self.slices = replicate(problem, sources, n)
        self.sl = slice(self.slices[0].start, self.slices[-1].stop)
        self.ctx = cel.Context(problem.model, device=device)
        self.dp = cel.DeviceProblem(self.rep, torch.device("cuda", device))
        self.plan = cel.Plan(self.ctx, self.dp, list(range(self.sl.start, self.sl.stop)))
        self.out = torch.empty(self.n, dtype=torch.float64, device=self.ctx.device)
        self.calls = 0

    def __call__(self, thetas):
        """thetas [n_total, 27] (point-value encodings, copies in order) -> numpy."""
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
    """Chains of several (source, type) groups in one state array: prior,
    bounds and the batched log-likelihood of all chains at once.  groups:
    list of (prior, kind, base theta, number of chains), in the row order
    of the log-likelihood's copies."""

    def __init__(self, groups, loglik_theta: Callable):
        self.groups = []
        self.d = max(g[0].dim for g in groups)
        n = sum(g[3] for g in groups)
        self.lo = np.full((n, self.d), -np.inf)
        self.hi = np.full((n, self.d), np.inf)
        self.movable = np.zeros((n, self.d), dtype=bool)
        r0 = 0
        for prior, kind, base, count in groups:
            r = slice(r0, r0 + count)
            self.lo[r, :prior.dim] = prior.lo
            self.hi[r, :prior.dim] = prior.hi
            self.movable[r, :prior.dim] = True
            self.groups.append((prior, kind, np.asarray(base, dtype=np.float64), r))
            r0 += count
        self.n = n
        self.loglik_theta = loglik_theta

    def sample(self, rng):
        W = np.zeros((self.n, self.d))
        for prior, _, _, r in self.groups:
            W[r, :prior.dim] = prior.sample(rng, r.stop - r.start)
        return W

    def logprior(self, W):
        out = np.empty(W.shape[0])
        for prior, _, _, r in self.groups:
            out[r] = prior.logpdf(W[r, :prior.dim])
        return out

    def loglik(self, W):
        # proposals outside the support (their prior is zero, so their value
        # is never used) are clipped into it so that every encoding is finite
        W = np.clip(W, np.nextafter(self.lo, np.inf), np.nextafter(self.hi, -np.inf))
        th = np.empty((W.shape[0], fields.N_THETA))
        for prior, kind, base, r in self.groups:
            th[r] = point_theta(W[r, :prior.dim], kind, base)
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


def type_posteriors(problem, sources, n_chains: int = 25, T: int = 200, B: int = 25,
                    seed: int = 0, device: int = 0, box: float = 2.0):
    """AIS for both types of each listed source (N' = n_chains runs per type,
    neighbours fixed), then B slice-sampling sweeps from the final states;
    all chains of all sources advance in lock step and every sampler round
    is one library call.  Returns one dict per source: p_star, log evidence
    and samples per type; and the number of log-likelihood calls."""
    rng = np.random.default_rng(seed)
    sources = [int(s) for s in sources]
    groups = []
    for s in sources:
        u0 = problem.theta[s, fields.I_U:fields.I_U + 2]
        for kind in (STAR, GALAXY):
            groups.append((Prior(problem.model, kind, u0, box), kind, problem.theta[s], n_chains))
    ev = GpuLogLik(problem, sources, 2 * n_chains, device)
    target = JointTarget(groups, ev)
    widths = np.full(target.d, 0.5)
    logw, W, samples = ais(target, T, rng, widths, B)
    results = []
    for i, s in enumerate(sources):
        res = {}
        for prior, kind, _, r in target.groups[2 * i:2 * i + 2]:
            res[kind] = dict(log_evidence=log_mean_exp(logw[r]), logw=logw[r],
                             samples=samples[:, r, :prior.dim].reshape(-1, prior.dim))
        la = math.log(problem.model.prior_a) + res[STAR]["log_evidence"]
        lb = math.log(1.0 - problem.model.prior_a) + res[GALAXY]["log_evidence"]
        p_star = 1.0 / (1.0 + math.exp(min(lb - la, 700.0)))
        results.append(dict(source=s, p_star=p_star, star=res[STAR], galaxy=res[GALAXY]))
    return results, ev.calls


def type_posterior(problem, s: int, n_chains: int = 25, T: int = 200, B: int = 25,
                   seed: int = 0, device: int = 0, box: float = 2.0):
    """type_posteriors for one source; the dict also holds the call count."""
    (r,), calls = type_posteriors(problem, [s], n_chains, T, B, seed, device, box)
    r["calls"] = calls
    return r
