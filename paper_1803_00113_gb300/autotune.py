"""Autotuner of the pixel kernels' tile shape, per patch-size bucket.

Two modes, both timed with the CUDA events the library records on its
stream; the result feeds ``Plan(..., ppi_bucket=...)``.

* Per bucket (``groups=None``): for every patch-area bucket of
  ``celeste.AREA_BUCKETS`` that holds sources, the derivative pixel kernel
  on a plan of that bucket's sources, for each candidate number of pixels per
  work item; keeps the most visits per millisecond.
* Composed (``groups`` = the source groups a step plans, e.g. the colour
  classes): the plans the step builds, with every kernel of an evaluation
  timed (setup, background, derivatives, epilogue, the trial value pass and,
  with a render cache, the render), summed over the groups.  Coordinate
  descent over the buckets from 256 pixels per item: launches of one group
  mix buckets, and the tail of a launch depends on all of them.
"""
from __future__ import annotations

import numpy as np

from . import celeste as cel

CANDIDATES = (128, 256, 512, 1024, 2048)


def source_bucket(problem, s):
    area = int((problem.patch_w[problem.patch_ptr[s]:problem.patch_ptr[s + 1]].astype(np.int64)
                * problem.patch_h[problem.patch_ptr[s]:problem.patch_ptr[s + 1]]).max())
    return int(np.searchsorted(cel.AREA_BUCKETS, area, side="right"))


def _composed_ms(ctx, dprob, groups, tiles, reps):
    plans = [cel.Plan(ctx, dprob, g, ppi_bucket=tiles) for g in groups]
    try:
        def once():
            for p in plans:
                if dprob.cache is not None:
                    cel.render_cache(p)
                cel.elbo_grad_hess(p)
                cel.elbo(p)
        once()                                   # warm up
        ctx.synchronize()
        ctx.profile(True, kinds="all")
        for _ in range(reps):
            once()
        ms = sum(v[0] for v in ctx.profile_kernels(reset=True).values())
        ctx.profile(False)
        return ms / reps
    finally:
        for p in plans:
            p.close()


def autotune(ctx: cel.Context, dprob: cel.DeviceProblem, sources, candidates=CANDIDATES,
             reps: int = 3, max_sources: int = 2048, groups=None):
    """Returns (ppi_bucket [4], report) for the given sources (see the module
    docstring for the two modes)."""
    problem = dprob.host
    if groups is not None:
        groups = [np.asarray(g, dtype=np.int32) for g in groups if len(g)]
        used = sorted({source_bucket(problem, int(s)) for g in groups for s in g})
        choice = [256 if b in used else 0 for b in range(4)]
        seen = {}
        for b in used:
            for ppi in candidates:
                trial = list(choice)
                trial[b] = ppi
                key = tuple(trial)
                if key not in seen:
                    seen[key] = _composed_ms(ctx, dprob, groups, trial, reps)
            choice[b] = min(candidates, key=lambda c: seen[tuple(choice[:b] + [c] + choice[b + 1:])])
        report = {"composed_ms": {str(list(k)): v for k, v in seen.items()}}
        return choice, report
    by_bucket = {}
    for s in sources:
        by_bucket.setdefault(source_bucket(problem, int(s)), []).append(int(s))
    choice = [0, 0, 0, 0]
    report = {}
    for b, srcs in sorted(by_bucket.items()):
        srcs = srcs[:max_sources]
        best = None
        for ppi in candidates:
            plan = cel.Plan(ctx, dprob, srcs, pixels_per_item=ppi)
            cel.elbo_grad_hess(plan)          # warm up
            ctx.synchronize()
            ctx.profile(True)
            for _ in range(reps):
                cel.elbo_grad_hess(plan)
            ms, n, visits = ctx.profile_read(reset=True)
            ctx.profile(False)
            rate = visits / ms if ms > 0 else 0.0
            report.setdefault(b, {})[ppi] = rate
            if best is None or rate > best[1]:
                best = (ppi, rate)
            plan.close()
        choice[b] = best[0]
    return choice, report
