// Per-(source, image) setup: the PSF-convolved Gaussian components of the
// star and galaxy light kernels in the patch's pixel frame, and the flux
// moments of each source type in the image's band.  FP64 arithmetic, FP32
// records (positions relative to the patch origin so that FP32 keeps them
// exact to ~1e-6 px).
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

__device__ __forceinline__ double sigmoid_d(double t) {
  return t >= 0.0 ? 1.0 / (1.0 + exp(-t)) : exp(t) / (1.0 + exp(t));
}

struct PairShared {
  double mux, muy;          // source centre, local pixel frame
  double g11, g12, g22;     // A Sigma_s A^T
};

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

  // per-pair quantities (every lane computes them: cheaper than a broadcast)
  const double ux = th[21], uy = th[22];
  const double mux = im.wcs_A[0] * ux + im.wcs_A[1] * uy + im.wcs_t[0] - (double)pi.x0;
  const double muy = im.wcs_A[2] * ux + im.wcs_A[3] * uy + im.wcs_t[1] - (double)pi.y0;
  const double ang = th[23];
  const double rad = exp(th[24]);
  const double axis = sigmoid_d(th[25]);
  const double rho = sigmoid_d(th[26]);
  const double c = cos(ang), s = sin(ang);
  const double d1 = rad * rad, d2 = axis * axis * rad * rad;
  // Sigma_s = R^T diag(d1, d2) R, R = [[c, -s], [s, c]]
  const double S11 = c * c * d1 + s * s * d2;
  const double S12 = c * s * (d2 - d1);
  const double S22 = s * s * d1 + c * c * d2;
  // G = A Sigma_s A^T
  const double a11 = im.wcs_A[0], a12 = im.wcs_A[1], a21 = im.wcs_A[2], a22 = im.wcs_A[3];
  const double t11 = a11 * S11 + a12 * S12, t12 = a11 * S12 + a12 * S22;
  const double t21 = a21 * S11 + a22 * S12, t22 = a21 * S12 + a22 * S22;
  const double g11 = t11 * a11 + t12 * a12;
  const double g12 = t11 * a21 + t12 * a22;
  const double g22 = t21 * a21 + t22 * a22;

  const int ne = model->n_exp, nd = model->n_dev;
  const int ncomp = kPsf * (1 + ne + nd);
  for (int ci = lane; ci < ncomp; ci += 32) {
    int k;
    double tau, weight;
    if (ci < kPsf) {
      k = ci;
      tau = 0.0;
      weight = im.psf[k][0];
    } else {
      const int r = ci - kPsf;
      k = r / (ne + nd);
      const int j = r % (ne + nd);
      if (j < ne) {
        tau = model->tau_exp[j];
        weight = im.psf[k][0] * model->alpha_exp[j];
      } else {
        tau = model->tau_dev[j - ne];
        weight = im.psf[k][0] * model->alpha_dev[j - ne];
      }
    }
    const double cxx = im.psf[k][3] + tau * g11;
    const double cxy = im.psf[k][4] + tau * g12;
    const double cyy = im.psf[k][5] + tau * g22;
    const double det = cxx * cyy - cxy * cxy;
    float* e = rec + kHdr + ci * kCompF;
    e[C_MX] = (float)(mux + im.psf[k][1]);
    e[C_MY] = (float)(muy + im.psf[k][2]);
    e[C_P11] = (float)(cyy / det);
    e[C_P12] = (float)(-cxy / det);
    e[C_P22] = (float)(cxx / det);
    e[C_LW] = (float)(log2(weight) - log2(2.0 * M_PI * sqrt(det)));
    e[C_TAU] = (float)tau;
    e[7] = 0.f;
  }

  if (lane == 0) {
    // flux moments per type in this image's band (Sec. 2.1.2)
    const int b = im.band;
    double kk[2], ev[2];
    for (int i = 0; i < 2; ++i) {
      const double mlr = th[1 + 2 * i];
      const double vlr = exp(th[2 + 2 * i]);
      double m = mlr, var = vlr;
      for (int q = 0; q < 4; ++q) {
        const double sel = (double)kSel[b][q];
        m += sel * th[5 + 4 * i + q];
        var += sel * sel * exp(th[13 + 4 * i + q]);
      }
      kk[i] = im.calib * exp(m + 0.5 * var);   // calib E[l_b | a=i]
      ev[i] = expm1(var);                       // E[l^2] / E[l]^2 - 1
    }
    const double q1 = sigmoid_d(th[0]);
    const double q0 = sigmoid_d(-th[0]);
    rec[H_CE0] = (float)(q0 * kk[0]);
    rec[H_CE1] = (float)(q1 * kk[1]);
    rec[H_CM0] = (float)(q0 * kk[0] * kk[0] * (1.0 + ev[0]));
    rec[H_CM1] = (float)(q1 * kk[1] * kk[1] * (1.0 + ev[1]));
    rec[H_K0] = (float)kk[0];
    rec[H_K1] = (float)kk[1];
    rec[H_EV0] = (float)ev[0];
    rec[H_EV1] = (float)ev[1];
    rec[H_Q0] = (float)q0;
    rec[H_Q1] = (float)q1;
    rec[H_RHO] = (float)rho;
    rec[H_RHO1] = (float)sigmoid_d(-th[26]);
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
