"""Small, self-contained cases for profiler captures of single kernels.

    python -m paper_1803_00113_gb300.profile_case derivs [n_sources]

builds a seeded blended problem of ``n_sources`` sources (default 2,000,
whose pixels exceed the L2 cache), plans its first colour class and calls
``elbo_grad_hess`` twice, so that a capture can skip the first launch of the
derivative pixel kernel and take the second.
"""
from __future__ import annotations

import sys


def derivs(n_sources: int = 2000):
    import fields
    from . import build_lib
    build_lib.build()
    from . import celeste as cel
    p = fields.batched(seed=1803_00113 + 3, n_sources=n_sources)
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    plan = cel.Plan(ctx, dp, cel.color_classes(p)[0])
    for _ in range(2):
        cel.elbo_grad_hess(plan)
    ctx.synchronize()
    print("visits", plan.visits, "pixels MB", p.pixels.nbytes / 1e6)


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "derivs"
    if case != "derivs":
        raise SystemExit(f"unknown case {case!r}")
    derivs(int(sys.argv[2]) if len(sys.argv) > 2 else 2000)
