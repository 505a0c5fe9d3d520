"""Oracle: the per-source Newton trust-region subsolver (Sec. 4.3).

Test infrastructure only.  Newton's method with a Euclidean-ball trust region
(the paper cites Nocedal & Wright); the paper gives no constants, so the
reading used here is the textbook trust-region loop (Nocedal & Wright,
Algorithm 4.1) with the exact subproblem solution of their Sec. 4.3:

  maximise  m(p) = g.p + 1/2 p.H.p   subject to  |p| <= Delta.

With B = -H = Q diag(lam) Q^T (numpy's symmetric eigensolver), the solution
is p(l) = Q diag(1/(lam + l)) Q^T g for the smallest l >= max(0, -lam_min)
with |p(l)| <= Delta, and l (Delta - |p|) = 0; the "hard case" (g orthogonal
to the eigenspace of lam_min) adds a multiple of that eigenvector, signed so
that its first nonzero entry is positive.

Constants: Delta_0 = 1, Delta_max = 100, accept when rho > 0.1, shrink to
|p|/4 when rho < 1/4, double (capped) when rho > 3/4 and the step reached the
boundary.  Stop with "converged" when the predicted gain of the step is below
1e-9 (1 + |L_rel|) or the radius falls below 1e-8; stop with "max
iterations" after 50 iterations.

Around the subsolver sits block coordinate ascent over a region (Sec. 4.3,
4.4): ``overlap_classes`` colours the overlap graph of the region greedily by
ascending source id, and ``region_fit`` runs passes over the classes in
ascending colour, one fresh subsolver call per source with every other
source held at its current value.  The paper fixes neither the schedule nor
when to stop passing; the reading here is that deterministic schedule, and
a fit that stops after the first pass whose ELBO gain (the sum of the actual
gains of its accepted steps) is at most 1e-3 nats per region source, or
after 5 passes.
"""
from __future__ import annotations

import numpy as np

import dataclasses

from .elbo import elbo_grad_hess, source_elbo

DELTA0 = 1.0
DELTA_MAX = 100.0
ETA_ACCEPT = 0.1
FTOL = 1e-9
DELTA_MIN = 1e-8
MAX_ITER = 50
MAX_PASSES = 5
PASS_TOL = 1e-3

ST_ACCEPTED = 0
ST_REJECTED = 1
ST_CONVERGED = 2
ST_MAXITER = 3
ST_FAILED = -1


def tr_subproblem(g, H, delta, hard_tol=1e-12):
    """Exact solution of max g.p + 1/2 p.H.p, |p| <= delta.

    Returns (p, pred, l, hard) with pred = g.p + 1/2 p.H.p the predicted
    gain, l the multiplier and hard True in the hard case.
    """
    g = np.asarray(g, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    B = -0.5 * (H + H.T)
    lam, Q = np.linalg.eigh(B)
    gh = Q.T @ g
    gnorm = float(np.linalg.norm(g))
    lmin = float(lam[0])

    def solve(l):
        return gh / (lam + l)

    l = None
    hard = False
    y = None
    if lmin > 0.0:
        y0 = solve(0.0)
        if np.linalg.norm(y0) <= delta:
            l, y = 0.0, y0
    if l is None:
        lo = max(0.0, -lmin)
        scale = max(1.0, float(np.max(np.abs(lam))))
        deg = lam <= lmin + 1e-12 * scale
        if np.all(np.abs(gh[deg]) <= hard_tol * max(gnorm, 1e-300)):
            yh = np.zeros_like(gh)
            nd = ~deg
            yh[nd] = gh[nd] / (lam[nd] + lo)
            if np.linalg.norm(yh) <= delta:
                hard = True
                l = lo
                z = Q[:, int(np.argmax(deg))].copy()
                nz = np.flatnonzero(np.abs(z) > 0)
                if z[nz[0]] < 0:
                    z = -z
                tau = np.sqrt(max(delta * delta - float(yh @ yh), 0.0))
                p = Q @ yh + tau * z
                pred = float(g @ p + 0.5 * p @ H @ p)
                return p, pred, l, hard
        # |p(l)| decreases on (lo, inf); bracket and bisect to machine precision
        a = lo
        b = lo + gnorm / delta + 1e-300
        while np.linalg.norm(solve(b)) > delta:
            b = lo + 2.0 * (b - lo)
        for _ in range(300):
            m = 0.5 * (a + b)
            if m <= a or m >= b:
                break
            if np.linalg.norm(solve(m)) > delta:
                a = m
            else:
                b = m
        l = b
        y = solve(l)
    p = Q @ y
    pred = float(g @ p + 0.5 * p @ H @ p)
    return p, pred, l, hard


def newton_iteration(problem, s, theta, delta, evaluation=None):
    """One trust-region Newton iteration on source s (neighbours frozen).

    Returns (theta_new, delta_new, status, info).
    """
    theta = np.asarray(theta, dtype=np.float64)
    r = evaluation if evaluation is not None else elbo_grad_hess(problem, s, theta)
    if not (np.isfinite(r["elbo"]) and np.all(np.isfinite(r["grad"])) and np.all(np.isfinite(r["hess"]))):
        return theta, delta, ST_FAILED, dict(eval=r)
    p, pred, lam, hard = tr_subproblem(r["grad"], r["hess"], delta)
    if pred <= FTOL * (1.0 + abs(r["elbo_rel"])) or delta < DELTA_MIN:
        return theta, delta, ST_CONVERGED, dict(eval=r, p=p, pred=pred)
    trial = theta + p
    Lt, base_t = source_elbo(problem, s, trial)
    actual = (Lt - base_t) - r["elbo_rel"]
    rho = actual / pred
    pn = float(np.linalg.norm(p))
    new_delta = delta
    if rho < 0.25:
        new_delta = 0.25 * pn
    elif rho > 0.75 and pn >= 0.99 * delta:
        new_delta = min(2.0 * delta, DELTA_MAX)
    if rho > ETA_ACCEPT:
        return trial, new_delta, ST_ACCEPTED, dict(eval=r, p=p, pred=pred, rho=rho, hard=hard)
    return theta, new_delta, ST_REJECTED, dict(eval=r, p=p, pred=pred, rho=rho, hard=hard)


def newton_fit(problem, s, theta=None, delta=DELTA0, max_iter=MAX_ITER, trace=None):
    """Newton trust-region iterations to convergence on source s."""
    theta = np.array(problem.theta[s] if theta is None else theta, dtype=np.float64)
    status = ST_ACCEPTED
    it = 0
    for it in range(1, max_iter + 1):
        theta, delta, status, info = newton_iteration(problem, s, theta, delta)
        if trace is not None:
            trace.append(dict(theta=theta.copy(), delta=delta, status=status,
                              elbo=info["eval"]["elbo"], elbo_rel=info["eval"]["elbo_rel"]))
        if status in (ST_CONVERGED, ST_FAILED):
            break
    else:
        status = ST_MAXITER
    return theta, delta, status, it


def overlap_classes(problem, sources=None):
    """Colour classes of the region's overlap graph (Sec. 4.4).

    Two sources of the region conflict when one is in the other's neighbour
    list (their patches overlap).  Sources are coloured greedily in ascending
    id, each with the smallest colour unused by its already coloured
    neighbours; the classes are returned in ascending colour, each sorted.
    """
    region = sorted({int(s) for s in (range(problem.n_sources) if sources is None else sources)})
    color = {}
    for s in region:
        used = {color[int(t)] for t in problem.nbr_idx[problem.nbr_ptr[s]:problem.nbr_ptr[s + 1]]
                if int(t) in color}
        c = 0
        while c in used:
            c += 1
        color[s] = c
    n_colors = max(color.values()) + 1 if color else 0
    return [[s for s in region if color[s] == c] for c in range(n_colors)]


def region_fit(problem, sources=None, max_passes=MAX_PASSES, max_iter=MAX_ITER, pass_tol=PASS_TOL,
               order=None):
    """Block coordinate ascent over the region's sources (Sec. 4.3, 4.4).

    A pass visits the colour classes of ``overlap_classes`` in ascending
    colour; every source of a class gets one subsolver call (``newton_fit``
    from Delta_0, at most max_iter iterations) with all other sources at
    their current values.  The fit stops after the first pass whose gain
    (the summed actual gains of its accepted steps) is at most pass_tol
    times the number of region sources, or after max_passes passes.
    ``order`` (a function of a class returning its sources in some order)
    only serves to show that the order inside a class does not matter.

    Returns a dict: theta [n_sources, 27] (sources outside the region keep
    their values), passes, pass_gains, and per region source its last
    status, its total iterations and accepted steps over all passes; gains
    lists the actual gain of every accepted step.
    """
    work = dataclasses.replace(problem, theta=np.array(problem.theta, dtype=np.float64, copy=True))
    classes = overlap_classes(problem, sources)
    n_region = sum(len(c) for c in classes)
    status, iters, accepted, gains, pass_gains = {}, {}, {}, [], []
    passes = 0
    for passes in range(1, max_passes + 1):
        pass_gain = 0.0
        for cls in classes:
            for s in (order(cls) if order else cls):
                trace = []
                theta, _, st, it = newton_fit(work, s, work.theta[s], DELTA0, max_iter, trace)
                acc = [k for k, e in enumerate(trace) if e["status"] == ST_ACCEPTED]
                for k in acc:
                    nxt = trace[k + 1]["elbo"] if k + 1 < len(trace) else source_elbo(work, s, theta)[0]
                    gains.append(nxt - trace[k]["elbo"])
                    pass_gain += gains[-1]
                work.theta[s] = theta
                status[s] = st
                iters[s] = iters.get(s, 0) + it
                accepted[s] = accepted.get(s, 0) + len(acc)
        pass_gains.append(pass_gain)
        if not pass_gain > pass_tol * n_region:
            break
    return dict(theta=work.theta, passes=passes, pass_gains=pass_gains, status=status,
                iters=iters, accepted=accepted, gains=gains, classes=classes)
