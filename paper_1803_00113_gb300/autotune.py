"""Autotuner of the pixel kernels' tile shape, per patch-size bucket.

For every patch-area bucket of ``celeste.AREA_BUCKETS`` that holds sources,
times the derivative pixel kernel (CUDA events recorded by the library on its
stream) for each candidate number of pixels per work item, on a plan of that
bucket's sources, and keeps the fastest (most visits per millisecond).  The
result feeds ``Plan(..., ppi_bucket=...)``.
"""
from __future__ import annotations

import numpy as np

from . import celeste as cel

CANDIDATES = (128, 256, 512, 1024, 2048)


def source_bucket(problem, s):
    area = int((problem.patch_w[problem.patch_ptr[s]:problem.patch_ptr[s + 1]].astype(np.int64)
                * problem.patch_h[problem.patch_ptr[s]:problem.patch_ptr[s + 1]]).max())
    return int(np.searchsorted(cel.AREA_BUCKETS, area, side="right"))


def autotune(ctx: cel.Context, dprob: cel.DeviceProblem, sources, candidates=CANDIDATES,
             reps: int = 3, max_sources: int = 2048):
    """Returns (ppi_bucket [4], report) for the given sources."""
    problem = dprob.host
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
