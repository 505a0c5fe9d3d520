"""Oracle: the log-likelihood of point values of a source's parameters, the
quantity the AIS and slice-sampling MCMC of Sec. 3 evaluates (test
infrastructure only).

With every variance of the variational family at zero and q(a) at 0 or 1,
the delta-method pixel term of Eq. eq:log_p_last is the Poisson
log-likelihood (up to log x!), so the sum over a source's patch pixels of
the term with the source minus the term without it is
log p(x | w_s, a_s, z_-s) - log p(x | source absent); neighbours enter
through their E and V as in the ELBO.  Computed here from the oracle's own
pieces in FP64, with the per-pixel absolute sum as the magnitude scale of
the parity tolerance.
"""
from __future__ import annotations

import torch

from .elbo import DT, Theta, background_patch, gather_patches, pixel_term, source_moments


def point_loglik(problem, s, theta_point):
    """(value, scale) for source s at the point-value encoding theta_point."""
    th = Theta.from_vector(torch.as_tensor(theta_point, dtype=DT))
    value = 0.0
    scale = 0.0
    for pd in gather_patches(problem, s):
        bgE, bgV = background_patch(problem, s, pd)
        E, V = source_moments(th, pd, problem.model)
        d = pixel_term(pd.x, bgE + E, bgV + V) - pixel_term(pd.x, bgE, bgV)
        value += float(d.sum())
        scale += float(d.abs().sum())
    return value, scale
