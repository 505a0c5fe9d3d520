"""FP64 CPU oracle for the per-source ELBO, its gradient and Hessian, and the
trust-region Newton step (test infrastructure only).

This package is the checker, not the product: only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it.  It shares no
code with the CUDA library; the two meet only through the seeded inputs of
``fields``.
"""
from .elbo import (  # noqa: F401
    Theta, PatchData, gather_patches, source_elbo, source_elbo_parts, elbo_grad_hess,
    abs_sum_scales, render_source_patch, background_patch, kl_source, band_moments,
    galaxy_covariance, pixel_term, full_field_elbo)
from .newton import (  # noqa: F401
    tr_subproblem, newton_iteration, newton_fit, overlap_classes, region_fit)
