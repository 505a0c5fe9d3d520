"""Fit the galaxy light-profile Gaussian scale mixtures (model constants).

The light kernel of a galaxy (Sec. 2.1.3, Eq. ``eq:hsi``) is a convex
combination of two extremal radial profiles, exponential and de Vaucouleurs,
each written as a scale mixture of concentric bivariate normals with
prespecified weights alpha_j and variance multipliers tau_j.  The paper does
not print these constants, so this script derives them: a least-squares fit of
K circular zero-mean Gaussians to the Sersic n=1 (exponential) and n=4
(de Vaucouleurs) surface-brightness profiles, both normalised to unit total
flux and unit half-light radius.  After the fit the weights are renormalised
to sum to one and the variances rescaled so that the mixture's own half-light
radius is exactly one (the radius parameter of a galaxy is its half-light
radius).

The output, ``galaxy_profiles.json``, is model data: both the CPU oracle and
the CUDA library receive it as an input.  Run ``python fields/fit_profiles.py``
to regenerate it (needs scipy).
"""
import json
import os

import numpy as np
from scipy import optimize, special

K = 8
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "galaxy_profiles.json")


def sersic_profile(n):
    """Surface brightness I(R) of a Sersic-n profile, unit flux, R_e = 1."""
    b = special.gammaincinv(2.0 * n, 0.5)
    # total flux of exp(-b (R^{1/n} - 1)) over the plane
    total = 2.0 * np.pi * n * np.exp(b) * special.gamma(2.0 * n) / b ** (2.0 * n)
    return lambda r: np.exp(-b * (r ** (1.0 / n) - 1.0)) / total


def mixture_profile(alpha, tau, r):
    r = np.asarray(r)[:, None]
    return np.sum(alpha / (2 * np.pi * tau) * np.exp(-0.5 * r * r / tau), axis=1)


def mixture_enclosed(alpha, tau, r):
    return np.sum(alpha * (1.0 - np.exp(-0.5 * r * r / tau)))


def fit(n, r_max):
    target = sersic_profile(n)
    r = np.geomspace(1e-3, r_max, 600)
    w = r  # residual weight: sqrt of the area element r^2 dlog r
    y = target(r)

    def resid(p):
        alpha = np.exp(p[:K])
        tau = np.exp(p[K:])
        return (mixture_profile(alpha, tau, r) - y) * w / y.max()

    tau0 = np.geomspace(1e-3 if n == 4 else 2e-2, 8.0 if n == 4 else 1.5, K)
    p0 = np.concatenate([np.full(K, np.log(1.0 / K)), np.log(tau0)])
    sol = optimize.least_squares(resid, p0, xtol=1e-14, ftol=1e-14, gtol=1e-14,
                                 max_nfev=200000)
    alpha = np.exp(sol.x[:K])
    tau = np.exp(sol.x[K:])
    order = np.argsort(tau)
    alpha, tau = alpha[order], tau[order]
    alpha = alpha / alpha.sum()
    # rescale the variances so that the mixture's half-light radius is one
    kappa = optimize.brentq(
        lambda k: mixture_enclosed(alpha, k * tau, 1.0) - 0.5, 1e-3, 1e3, xtol=1e-15)
    tau = kappa * tau
    return alpha, tau, float(np.sqrt(np.mean(sol.fun ** 2)))


def main():
    out = {"K": K, "description": (
        "Gaussian scale mixtures for the galaxy light kernel: component j has "
        "weight alpha[j] and covariance tau[j] * Sigma_s; each profile has unit "
        "flux and unit half-light radius")}
    for name, n, r_max in (("exp", 1.0, 8.0), ("dev", 4.0, 8.0)):
        alpha, tau, rms = fit(n, r_max)
        out[name] = {"sersic_n": n, "alpha": alpha.tolist(), "tau": tau.tolist(),
                     "fit_rms": rms}
        print(name, "rms", rms)
        print("  alpha", np.array2string(alpha, precision=5))
        print("  tau  ", np.array2string(tau, precision=5))
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
