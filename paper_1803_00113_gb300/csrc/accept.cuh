// Accept rule of the trust-region loop (Sec. 4.3; Nocedal & Wright,
// Algorithm 4.1): accept the trial point when rho = actual / predicted gain
// exceeds 0.1; shrink the radius to |p| / 4 when rho < 1/4, double it (up
// to 100) when rho > 3/4 and the step reached the boundary.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace celeste {

constexpr double kEta = 0.1;
constexpr double kDeltaMax = 100.0;

// Slot j with value rel_trial at theta_trial (and elbo_rel, pred and step
// of the current iteration in the plan): new radius and status, theta
// replaced on acceptance; returns whether the step was accepted, in every
// lane of the calling warp.  The warp loads everything at once (a lane per
// coordinate) and forms |p| in coordinate order from shuffles, so the
// decision costs one memory round trip rather than one per coordinate.
__device__ __forceinline__ bool accept_trial(const PlanView& v, int j, double rel_trial,
                                             double* delta, int32_t* status, int lane) {
  const int src = v.src_ids[j];
  const double pl = lane < kTheta ? v.step[(size_t)j * kTheta + lane] : 0.0;
  const double tl = lane < kTheta ? v.theta_trial[(size_t)j * kTheta + lane] : 0.0;
  const double Dl = delta[src], L0 = v.elbo_rel[j], pred = v.pred[j];
  double pn = 0.0;
#pragma unroll
  for (int i = 0; i < kTheta; ++i) {
    const double pi = __shfl_sync(0xffffffffu, pl, i);
    pn = fma(pi, pi, pn);
  }
  pn = sqrt(pn);
  const double rho = (rel_trial - L0) / pred;
  double nd = Dl;
  if (!(rho >= 0.25)) nd = 0.25 * pn;
  else if (rho > 0.75 && pn >= 0.99 * Dl) nd = fmin(2.0 * Dl, kDeltaMax);
  const bool acc = rho > kEta && isfinite(rel_trial);
  if (lane == 0) {
    delta[src] = nd;
    status[src] = acc ? CELESTE_ST_ACCEPTED : CELESTE_ST_REJECTED;
  }
  if (acc && lane < kTheta) v.theta[(size_t)src * kTheta + lane] = tl;
  return acc;
}

}  // namespace celeste
