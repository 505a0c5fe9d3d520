// Per-(source, image) setup: the PSF-convolved Gaussian components of the
// star and galaxy light kernels in the patch's pixel frame, and the flux
// moments of each source type in the image's band, as FP32 records
// (positions relative to the patch origin so that FP32 keeps them exact to
// ~1e-6 px).
//
// Follows Sec. 2.1.2 (flux: l_b = r exp(S_b . c), log-normal r and normal
// colours under q), Sec. 2.1.3 (Eq. eq:hsi and Sigma_s = R^T D R), Sec. 2.2
// (calibration, linear WCS, Gaussian-mixture PSF) and the Gaussian-Gaussian
// convolution of Sec. 2.2.3.
#include <math.h>

#include "internal.cuh"

namespace celeste {

// l_b = r * exp(sum_k kSel[b][k] c_k), colours c_k = log(l_{k+1} / l_k), r = l_2
__constant__ signed char kSel[5][4] = {
    {-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

__device__ __forceinline__ float sigmoid_f(float t) {
  return t >= 0.f ? 1.f / (1.f + expf(-t)) : expf(t) / (1.f + expf(t));
}

// One warp per pair; lanes over Gaussian components.  Only the patch-local
// centre needs FP64 (reference-frame positions reach ~2000 px); everything
// else is FP32, which keeps the records exact to ~1e-7 relative.
__global__ void setup_kernel(PlanView v, const ModelDev* __restrict__ model, int first_pair,
                             int n_pairs, int use_trial) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_pairs) return;
  const int p = first_pair + warp;
  const PairInfo pi = v.pairs[p];
  const celeste_image& im = v.images[pi.image];
  const double* th = (use_trial && pi.slot >= 0) ? v.theta_trial + (size_t)pi.slot * kTheta
                                                 : v.theta + (size_t)pi.source * kTheta;
  float* rec = v.records + (size_t)p * kRecF;

  // centre in the patch's local pixel frame (FP64, then FP32)
  const double ux = th[21], uy = th[22];
  const float mux = (float)(im.wcs_A[0] * ux + im.wcs_A[1] * uy + im.wcs_t[0] - (double)pi.x0);
  const float muy = (float)(im.wcs_A[2] * ux + im.wcs_A[3] * uy + im.wcs_t[1] - (double)pi.y0);
  // Sigma_s = R^T diag(d1, d2) R, R = [[c, -s], [s, c]]  (Sec. 2.1.3)
  float s, c;
  sincosf((float)th[23], &s, &c);
  const float rad2 = expf(2.f * (float)th[24]);
  const float axis = sigmoid_f((float)th[25]);
  const float d1 = rad2, d2 = axis * axis * rad2;
  const float S11 = c * c * d1 + s * s * d2;
  const float S12 = c * s * (d2 - d1);
  const float S22 = s * s * d1 + c * c * d2;
  // G = A Sigma_s A^T
  const float a11 = (float)im.wcs_A[0], a12 = (float)im.wcs_A[1];
  const float a21 = (float)im.wcs_A[2], a22 = (float)im.wcs_A[3];
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
      weight = (float)im.psf[k][0];
    } else {
      const int r = ci - kPsf;
      k = r / (ne + nd);
      const int j = r % (ne + nd);
      if (j < ne) {
        tau = (float)model->tau_exp[j];
        weight = (float)(im.psf[k][0] * model->alpha_exp[j]);
      } else {
        tau = (float)model->tau_dev[j - ne];
        weight = (float)(im.psf[k][0] * model->alpha_dev[j - ne]);
      }
    }
    const float cxx = fmaf(tau, g11, (float)im.psf[k][3]);
    const float cxy = fmaf(tau, g12, (float)im.psf[k][4]);
    const float cyy = fmaf(tau, g22, (float)im.psf[k][5]);
    const float det = cxx * cyy - cxy * cxy;
    const float rdet = 1.f / det;
    float* e = rec + kHdr + ci * kCompF;
    e[C_MX] = mux + (float)im.psf[k][1];
    e[C_MY] = muy + (float)im.psf[k][2];
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
      float m = (float)th[1 + 2 * i];
      float var = expf((float)th[2 + 2 * i]);
      for (int q = 0; q < 4; ++q) {
        const float sel = (float)kSel[b][q];
        m += sel * (float)th[5 + 4 * i + q];
        var += sel * sel * expf((float)th[13 + 4 * i + q]);
      }
      kk[i] = (float)im.calib * expf(m + 0.5f * var);   // calib E[l_b | a=i]
      ev[i] = expm1f(var);                              // E[l^2] / E[l]^2 - 1
    }
    const float q1 = sigmoid_f((float)th[0]);
    const float q0 = sigmoid_f(-(float)th[0]);
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
    rec[H_RHO] = sigmoid_f((float)th[26]);
    rec[H_RHO1] = sigmoid_f(-(float)th[26]);
    rec[12] = rec[13] = rec[14] = rec[15] = 0.f;
  }
}

cudaError_t launch_setup(const Launch& L, const PlanView& v, const ModelDev* model,
                         int first_pair, int n_pairs, bool use_trial) {
  if (n_pairs <= 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (n_pairs * 32 + threads - 1) / threads;
  setup_kernel<<<blocks, threads, 0, L.stream>>>(v, model, first_pair, n_pairs, use_trial ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace celeste
