// Per-(source, image) setup of one pair, by one warp: the PSF-convolved
// Gaussian components of the star and galaxy light kernels in the patch's
// pixel frame, and the flux moments of each source type in the image's band,
// as an FP32 record (positions relative to the patch origin so that FP32
// keeps them exact to ~1e-6 px).
//
// Follows Sec. 2.1.2 (flux: l_b = r exp(S_b . c), log-normal r and normal
// colours under q), Sec. 2.1.3 (Eq. eq:hsi and Sigma_s = R^T D R), Sec. 2.2
// (calibration, linear WCS, Gaussian-mixture PSF) and the Gaussian-Gaussian
// convolution of Sec. 2.2.3.
//
// Included by the translation units whose kernels form records: the setup
// kernel itself, the per-class preparation kernel and the per-source step.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace celeste {

// l_b = r * exp(sum_k kSel[b][k] c_k), colours c_k = log(l_{k+1} / l_k), r = l_2
static __constant__ signed char kSel[5][4] = {
    {-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

__device__ __forceinline__ float sigmoid_f(float t) {
  return t >= 0.f ? 1.f / (1.f + expf(-t)) : expf(t) / (1.f + expf(t));
}

// Record of pair p, by the calling warp (lanes over Gaussian components).
// Only the patch-local centre needs FP64 (reference-frame positions reach
// ~2000 px); everything else is FP32, which keeps the records exact to ~1e-7
// relative.  On this GPU the FP64 pipe also carries the double -> float
// conversions, at about one warp instruction per 64 cycles of an SM
// sub-partition, so the warp converts its theta row and its image's PSF,
// WCS and calibration with one instruction each (a value per lane), shared
// through thf and imf: 32 floats each of the warp's shared memory.  Own
// pairs read theta_trial when use_trial.
__device__ __forceinline__ void setup_pair(const PlanView& v, const ModelDev* __restrict__ model,
                                           int p, bool use_trial, float* thf, float* imf,
                                           int lane) {
  const PairInfo pi = v.pairs[p];
  const celeste_image& im = v.images[pi.image];
  const double* th = (use_trial && pi.slot >= 0) ? v.theta_trial + (size_t)pi.slot * kTheta
                                                 : v.theta + (size_t)pi.source * kTheta;
  float* rec = v.records + (size_t)p * kRecF;
  constexpr int kPsfV = 6 * kPsf;                // PSF values: weight, mean (2), covariance (3)
  static_assert(kTheta <= 32 && kPsfV + 5 <= 32, "one value per lane");
  __syncwarp();
  {
    thf[lane] = (float)th[lane < kTheta ? lane : 0];
    const double* src = lane < kPsfV ? &im.psf[0][0] + lane
                                     : (lane < kPsfV + 4 ? im.wcs_A + (lane - kPsfV) : &im.calib);
    imf[lane] = (float)*src;
  }
  __syncwarp();
  const float* psf = imf;                        // psf[6 k + c]
  const float* wcs = imf + kPsfV;                // A0, A1, A2, A3, calib

  // centre in the patch's local pixel frame (FP64, then FP32)
  const double ux = th[21], uy = th[22];
  const float mux = (float)(im.wcs_A[0] * ux + im.wcs_A[1] * uy + im.wcs_t[0] - (double)pi.x0);
  const float muy = (float)(im.wcs_A[2] * ux + im.wcs_A[3] * uy + im.wcs_t[1] - (double)pi.y0);
  // Sigma_s = R^T diag(d1, d2) R, R = [[c, -s], [s, c]]  (Sec. 2.1.3)
  float s, c;
  sincosf(thf[23], &s, &c);
  const float rad2 = expf(2.f * thf[24]);
  const float axis = sigmoid_f(thf[25]);
  const float d1 = rad2, d2 = axis * axis * rad2;
  const float S11 = c * c * d1 + s * s * d2;
  const float S12 = c * s * (d2 - d1);
  const float S22 = s * s * d1 + c * c * d2;
  // G = A Sigma_s A^T
  const float a11 = wcs[0], a12 = wcs[1];
  const float a21 = wcs[2], a22 = wcs[3];
  const float t11 = a11 * S11 + a12 * S12, t12 = a11 * S12 + a12 * S22;
  const float t21 = a21 * S11 + a22 * S12, t22 = a21 * S12 + a22 * S22;
  const float g11 = t11 * a11 + t12 * a12;
  const float g12 = t11 * a21 + t12 * a22;
  const float g22 = t21 * a21 + t22 * a22;

  const int ne = model->n_exp, nd = model->n_dev;
  const int ncomp = kPsf * (1 + ne + nd);
  const float log2_2pi = 2.6514961294723187f;   // log2(2 pi)
  for (int ci = lane; ci < ncomp; ci += 32) {
    int k;
    float tau, weight;
    if (ci < kPsf) {
      k = ci;
      tau = 0.f;
      weight = psf[6 * k];
    } else {
      const int r = ci - kPsf;
      k = r / (ne + nd);
      const int j = r % (ne + nd);
      // the weight product stays FP64 (one rounding), as the oracle's
      if (j < ne) {
        tau = model->f.tau_exp[j];
        weight = (float)(im.psf[k][0] * model->alpha_exp[j]);
      } else {
        tau = model->f.tau_dev[j - ne];
        weight = (float)(im.psf[k][0] * model->alpha_dev[j - ne]);
      }
    }
    const float cxx = fmaf(tau, g11, psf[6 * k + 3]);
    const float cxy = fmaf(tau, g12, psf[6 * k + 4]);
    const float cyy = fmaf(tau, g22, psf[6 * k + 5]);
    const float det = cxx * cyy - cxy * cxy;
    const float rdet = 1.f / det;
    float* e = rec + kHdr + ci * kCompF;
    e[C_MX] = mux + psf[6 * k + 1];
    e[C_MY] = muy + psf[6 * k + 2];
    e[C_P11] = cyy * rdet;
    e[C_P12] = -cxy * rdet;
    e[C_P22] = cxx * rdet;
    e[C_LW] = log2f(weight) - log2_2pi - 0.5f * log2f(det);
    e[C_TAU] = tau;
    e[7] = 0.f;
  }

  if (lane == 0) {
    // flux moments per type in this image's band (Sec. 2.1.2)
    const int b = im.band;
    float kk[2], ev[2];
    for (int i = 0; i < 2; ++i) {
      float m = thf[1 + 2 * i];
      float var = expf(thf[2 + 2 * i]);
      for (int q = 0; q < 4; ++q) {
        const float sel = (float)kSel[b][q];
        m += sel * thf[5 + 4 * i + q];
        var += sel * sel * expf(thf[13 + 4 * i + q]);
      }
      kk[i] = wcs[4] * expf(m + 0.5f * var);          // calib E[l_b | a=i]
      ev[i] = expm1f(var);                              // E[l^2] / E[l]^2 - 1
    }
    const float q1 = sigmoid_f(thf[0]);
    const float q0 = sigmoid_f(-thf[0]);
    rec[H_CE0] = q0 * kk[0];
    rec[H_CE1] = q1 * kk[1];
    rec[H_CM0] = q0 * kk[0] * kk[0] * (1.f + ev[0]);
    rec[H_CM1] = q1 * kk[1] * kk[1] * (1.f + ev[1]);
    rec[H_K0] = kk[0];
    rec[H_K1] = kk[1];
    rec[H_EV0] = ev[0];
    rec[H_EV1] = ev[1];
    rec[H_Q0] = q0;
    rec[H_Q1] = q1;
    rec[H_RHO] = sigmoid_f(thf[26]);
    rec[H_RHO1] = sigmoid_f(-thf[26]);
    rec[12] = rec[13] = rec[14] = rec[15] = 0.f;
  }
}

}  // namespace celeste
