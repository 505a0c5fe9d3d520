// Per-source epilogue (FP64): reduce the per-tile sums of a source, map them
// from each image's natural coordinates to the source's 27 unconstrained
// coordinates, and add the KL term.
//
// Chain rule, exact because each map below is applied to reduced sums:
//   per image (affine):  cE_i = calib * kE_i[b], cM_i = calib^2 * kM_i[b],
//                        mu = A u + t, G = A Sigma_s A^T, rho = rho;
//   per source:          kE_i[b] = q_i exp(m_ib + v_ib / 2),
//                        kM_i[b] = q_i exp(2 m_ib + 2 v_ib)     (Sec. 2.1.2,
//                        Eq. conditional, vareq: E[l|a], E[l^2|a] with
//                        log l ~ N(m, v)),
//                        Sigma_s(angle, radius, axis) = R^T D R (Sec. 2.1.3),
//                        rho = sigmoid(theta_26).
//   grad_theta = J^T grad_nu,
//   hess_theta = J^T H_nu J + sum_a grad_nu[a] * hess_theta(nu_a).
// KL_s follows Eq. kleq, Supplement A and the GMM colour bound of Sec. 4.2.3
// with xi minimised in closed form: -log sum_j w_j exp(-KL(q(c|a) || N_j)).
#include <math.h>

#include "internal.cuh"

namespace celeste {

__constant__ signed char kSelE[5][4] = {
    {-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

constexpr int kNu = 26;     // 20 flux moments (5 bands x {kE0, kE1, kM0, kM1}), u (2), Sigma_s (3), rho
constexpr int kNuPad = 32;

__device__ __forceinline__ double sigm(double t) {
  return t >= 0.0 ? 1.0 / (1.0 + exp(-t)) : exp(t) / (1.0 + exp(t));
}
// log(1 + exp(t)) without overflow
__device__ __forceinline__ double softplus(double t) {
  return t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t));
}

// Stored Hessian entry (k, l) of the per-image sums (k, l in 0..9).
__device__ __forceinline__ double hw(const double* W, int k, int l) {
  if (k > l) { int t = k; k = l; l = t; }
  if ((k == 2 || k == 3) && (l == 2 || l == 3)) return 0.0;
  return W[hidx(k, l)];
}

// Shared-memory layout of one epilogue block (one warp per source).
struct EpiSmem {
  double W[kAcc];
  double gnu[kNuPad];
  double Hnu[kNu * kNu];
  double J[kNu * kTheta];
  double X[kNu * kTheta];
  double gth[kNuPad];
  double Hth[kTheta * kTheta];
  double T[10 * 10];
  double kl[kNuPad];
  double DL[20 * kTheta];    // d log kappa_a / d theta
  double D2L[20 * kTheta];   // diagonal second derivatives of log kappa_a
  double kw[kNuPad];         // grad_nu[a] * kappa_a
};

// KL_s value, gradient and Hessian over theta (added with weight `sign`).
__device__ void kl_terms(const double* th, const ModelDev* m, double* val, double* g, double* H,
                         int lane) {
  // lanes 0 and 1 handle the two source types; lane 2 the rest
  const double a = sigm(th[0]);
  const double wq = a * (1.0 - a);
  if (lane < 2) {
    const int i = lane;
    // log-normal KL of r (Supplement A; both second parameters variances)
    const double R1 = m->prior_r[i][0], R2 = m->prior_r[i][1];
    const int ir = 1 + 2 * i, iv = 2 + 2 * i;
    const double rm = th[ir], rv = exp(th[iv]);
    double K = 0.5 * (log(R2) - th[iv] + (rv + (rm - R1) * (rm - R1)) / R2 - 1.0);
    double gK[10] = {0}, hK[10][10] = {{0}};
    // local index: 0 r-mean, 1 log r-var, 2..5 colour means, 6..9 log colour vars
    gK[0] = (rm - R1) / R2;
    hK[0][0] = 1.0 / R2;
    gK[1] = 0.5 * (rv / R2 - 1.0);
    hK[1][1] = 0.5 * rv / R2;
    // colour bound: B = -log sum_j w_j exp(-K_j)
    const double* cm = th + 5 + 4 * i;
    const double* lcv = th + 13 + 4 * i;
    double cv[4];
    for (int k = 0; k < 4; ++k) cv[k] = exp(lcv[k]);
    const int J = m->n_color;
    double lg[kMaxColor], Kj[kMaxColor];
    double mx = -1e300;
    for (int j = 0; j < J; ++j) {
      const double(*P)[4] = m->color_prec[i][j];
      double d[4];
      for (int k = 0; k < 4; ++k) d[k] = cm[k] - m->color_mean[i][j][k];
      double tr = 0.0, quad = 0.0, slv = 0.0;
      for (int k = 0; k < 4; ++k) {
        tr += P[k][k] * cv[k];
        slv += lcv[k];
        double pk = 0.0;
        for (int l = 0; l < 4; ++l) pk += P[k][l] * d[l];
        quad += d[k] * pk;
      }
      Kj[j] = 0.5 * (tr + quad - 4.0 + m->color_logdet[i][j] - slv);
      lg[j] = log(m->color_w[i][j]) - Kj[j];
      mx = fmax(mx, lg[j]);
    }
    double se = 0.0;
    for (int j = 0; j < J; ++j) se += exp(lg[j] - mx);
    const double B = -(mx + log(se));
    double gB[8] = {0}, hB[8][8] = {{0}};
    for (int j = 0; j < J; ++j) {
      const double pj = exp(lg[j] - mx) / se;
      const double(*P)[4] = m->color_prec[i][j];
      double gk[8];
      for (int k = 0; k < 4; ++k) {
        double pk = 0.0;
        for (int l = 0; l < 4; ++l) pk += P[k][l] * (cm[l] - m->color_mean[i][j][l]);
        gk[k] = pk;
        gk[4 + k] = 0.5 * (P[k][k] * cv[k] - 1.0);
      }
      for (int k = 0; k < 8; ++k) {
        gB[k] += pj * gk[k];
        for (int l = 0; l < 8; ++l) hB[k][l] -= pj * gk[k] * gk[l];
      }
      for (int k = 0; k < 4; ++k) {
        for (int l = 0; l < 4; ++l) hB[k][l] += pj * P[k][l];
        hB[4 + k][4 + k] += pj * 0.5 * P[k][k] * cv[k];
      }
    }
    for (int k = 0; k < 8; ++k)
      for (int l = 0; l < 8; ++l) hB[k][l] += gB[k] * gB[l];
    K += B;
    for (int k = 0; k < 8; ++k) {
      gK[2 + k] = gB[k];
      for (int l = 0; l < 8; ++l) hK[2 + k][2 + l] = hB[k][l];
    }
    // weight q_i: q_1 = a, q_0 = 1 - a
    const double qi = i ? a : 1.0 - a;
    const double dq = i ? wq : -wq;
    const double d2q = (i ? 1.0 : -1.0) * wq * (1.0 - 2.0 * a);
    int idx[10];
    idx[0] = ir;
    idx[1] = iv;
    for (int k = 0; k < 4; ++k) {
      idx[2 + k] = 5 + 4 * i + k;
      idx[6 + k] = 13 + 4 * i + k;
    }
    // lanes 0 and 1 write disjoint index sets, except the theta_0 entries,
    // which are combined below through val[1..2] and g/H row 0 by lane 2
    val[i] = qi * K;
    val[3 + i] = dq * K;    // d/dtheta_0 part
    val[5 + i] = d2q * K;   // d2/dtheta_0^2 part
    for (int k = 0; k < 10; ++k) {
      g[idx[k]] += qi * gK[k];
      H[idx[k] * kTheta + 0] += dq * gK[k];
      H[0 * kTheta + idx[k]] += dq * gK[k];
      for (int l = 0; l < 10; ++l) H[idx[k] * kTheta + idx[l]] += qi * hK[k][l];
    }
  }
  __syncwarp();
  if (lane == 2) {
    // Bernoulli KL of a (Supplement A)
    const double pa = m->prior_a;
    const double la = log(pa) - log1p(-pa);
    const double la1 = -softplus(-th[0]), la0 = -softplus(th[0]);   // log a, log(1-a)
    double v = a * (la1 - log(pa)) + (1.0 - a) * (la0 - log1p(-pa));
    g[0] += wq * (th[0] - la) + val[3] + val[4];
    H[0] += wq * ((1.0 - 2.0 * a) * (th[0] - la) + 1.0) + val[5] + val[6];
    v += val[0] + val[1];
    // point masses: -log prior density at the point
    const double lr = th[24];
    const double E1 = m->e_radius[0], E2 = m->e_radius[1];
    v += lr + 0.5 * log(2.0 * M_PI * E2) + (lr - E1) * (lr - E1) / (2.0 * E2);
    g[24] += 1.0 + (lr - E1) / E2;
    H[24 * kTheta + 24] += 1.0 / E2;
    for (int which = 0; which < 2; ++which) {
      const int t = which ? 26 : 25;
      const double b1 = which ? m->e_profile[0] : m->e_axis[0];
      const double b2 = which ? m->e_profile[1] : m->e_axis[1];
      const double sg = sigm(th[t]);
      const double logB = lgamma(b1) + lgamma(b2) - lgamma(b1 + b2);
      v += (b1 - 1.0) * softplus(-th[t]) + (b2 - 1.0) * softplus(th[t]) + logB;
      g[t] += -(b1 - 1.0) * (1.0 - sg) + (b2 - 1.0) * sg;
      H[t * kTheta + t] += (b1 + b2 - 2.0) * sg * (1.0 - sg);
    }
    val[2] = v;
  }
  __syncwarp();
}

// First and second derivatives of Sigma_s entries (S11, S12, S22) over
// (angle, log radius, logit axis).
__device__ void sigma_derivs(const double* th, double dS[3][3], double d2S[3][3][3]) {
  const double phi = th[23], lr = th[24];
  const double ax = sigm(th[25]);
  const double e2 = exp(2.0 * lr);
  const double a2 = ax * ax;
  const double a2t = 2.0 * a2 * (1.0 - ax);                       // d(ax^2)/dt
  const double a2tt = 2.0 * a2 * (1.0 - ax) * (2.0 - 3.0 * ax);   // d2(ax^2)/dt2
  const double P = 0.5 * e2 * (1.0 + a2), Qd = 0.5 * e2 * (1.0 - a2);
  // derivatives over (l = log radius, t = logit axis)
  const double Pl = 2.0 * P, Pll = 4.0 * P, Pt = 0.5 * e2 * a2t, Ptt = 0.5 * e2 * a2tt, Plt = 2.0 * Pt;
  const double Ql = 2.0 * Qd, Qll = 4.0 * Qd, Qt = -0.5 * e2 * a2t, Qtt = -0.5 * e2 * a2tt, Qlt = 2.0 * Qt;
  const double C2 = cos(2.0 * phi), S2 = sin(2.0 * phi);
  // S11 = P + Qd C2, S22 = P - Qd C2, S12 = -Qd S2
  // index 0 = angle, 1 = log radius, 2 = logit axis
  const double sgn[3] = {1.0, 0.0, -1.0};
  for (int e = 0; e < 3; e += 2) {
    const double s = sgn[e];
    dS[e][0] = -2.0 * s * Qd * S2;
    dS[e][1] = Pl + s * Ql * C2;
    dS[e][2] = Pt + s * Qt * C2;
    d2S[e][0][0] = -4.0 * s * Qd * C2;
    d2S[e][0][1] = d2S[e][1][0] = -2.0 * s * Ql * S2;
    d2S[e][0][2] = d2S[e][2][0] = -2.0 * s * Qt * S2;
    d2S[e][1][1] = Pll + s * Qll * C2;
    d2S[e][1][2] = d2S[e][2][1] = Plt + s * Qlt * C2;
    d2S[e][2][2] = Ptt + s * Qtt * C2;
  }
  dS[1][0] = -2.0 * Qd * C2;
  dS[1][1] = -Ql * S2;
  dS[1][2] = -Qt * S2;
  d2S[1][0][0] = 4.0 * Qd * S2;
  d2S[1][0][1] = d2S[1][1][0] = -2.0 * Ql * C2;
  d2S[1][0][2] = d2S[1][2][0] = -2.0 * Qt * C2;
  d2S[1][1][1] = -Qll * S2;
  d2S[1][1][2] = d2S[1][2][1] = -Qlt * S2;
  d2S[1][2][2] = -Qtt * S2;
}

// d log kappa / d theta for flux-moment coordinate a (0..19): band b = a / 4,
// kind e = a % 4 (0: kE0, 1: kE1, 2: kM0, 3: kM1).  Returns kappa; fills the
// 27-entry gradient of log kappa and the diagonal second derivatives.
__device__ double kappa_logderivs(const double* th, int a, double* dl, double* d2l) {
  const int b = a >> 2, e = a & 3;
  const int i = e & 1;                   // type
  const bool second = e >= 2;            // E[l^2] rather than E[l]
  const double am = second ? 2.0 : 1.0, av = second ? 2.0 : 0.5;
  for (int c = 0; c < kTheta; ++c) dl[c] = d2l[c] = 0.0;
  const double q1 = sigm(th[0]), q0 = sigm(-th[0]);
  const double logq = i ? -softplus(-th[0]) : -softplus(th[0]);
  dl[0] = i ? q0 : -q1;
  d2l[0] = -q0 * q1;
  const int ir = 1 + 2 * i, iv = 2 + 2 * i;
  double m = th[ir], v = exp(th[iv]);
  dl[ir] = am;
  dl[iv] = av * exp(th[iv]);
  d2l[iv] = dl[iv];
  for (int k = 0; k < 4; ++k) {
    const double s = (double)kSelE[b][k];
    const double cvk = exp(th[13 + 4 * i + k]);
    m += s * th[5 + 4 * i + k];
    v += s * s * cvk;
    dl[5 + 4 * i + k] = am * s;
    dl[13 + 4 * i + k] = av * s * s * cvk;
    d2l[13 + 4 * i + k] = dl[13 + 4 * i + k];
  }
  return exp(logq + am * m + av * v);
}

template <bool kDerivs>
__global__ void epilogue_kernel(PlanView v, const ModelDev* __restrict__ model, double* elbo,
                                double* elbo_rel, double* grad_out, double* hess_out,
                                int use_trial) {
  extern __shared__ double smd[];
  EpiSmem& S = *reinterpret_cast<EpiSmem*>(smd);
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  if (!v.active[j]) return;
  const int src = v.src_ids[j];
  const double* th = use_trial ? v.theta_trial + (size_t)j * kTheta : v.theta + (size_t)src * kTheta;

  double vrel = 0.0, vbase = 0.0;
  if (kDerivs) {
    for (int e = lane; e < kNuPad; e += 32) S.gnu[e] = 0.0;
    for (int e = lane; e < kNu * kNu; e += 32) S.Hnu[e] = 0.0;
  }
  __syncwarp();
  for (int pp = v.slot_pair_ptr[j]; pp < v.slot_pair_ptr[j + 1]; ++pp) {
    const PairInfo pi = v.pairs[pp];
    if (!kDerivs) {
      double r = 0.0, b = 0.0;
      for (int it = pi.item_begin + lane; it < pi.item_end; it += 32) {
        r += (double)v.vpartials[2 * (size_t)it];
        b += (double)v.vpartials[2 * (size_t)it + 1];
      }
      vrel += warp_sum_d(r);
      vbase += warp_sum_d(b);
      continue;
    }
    double w0 = 0.0, w1 = 0.0;
    for (int it = pi.item_begin; it < pi.item_end; ++it) {
      w0 += (double)v.partials[(size_t)it * kAcc + lane];
      w1 += (double)v.partials[(size_t)it * kAcc + 32 + lane];
    }
    S.W[lane] = w0;
    S.W[lane + 32] = w1;
    const celeste_image& im = v.images[pi.image];
    const double cal = im.calib;
    const double* A = im.wcs_A;
    // local transform T[k][a]: w_k = sum_a T[k][a] nu_local_a
    for (int e = lane; e < 100; e += 32) S.T[e] = 0.0;
    __syncwarp();
    if (lane == 0) {
      S.T[0 * 10 + 0] = cal;
      S.T[1 * 10 + 1] = cal;
      S.T[2 * 10 + 2] = cal * cal;
      S.T[3 * 10 + 3] = cal * cal;
      S.T[4 * 10 + 4] = A[0];
      S.T[4 * 10 + 5] = A[1];
      S.T[5 * 10 + 4] = A[2];
      S.T[5 * 10 + 5] = A[3];
      // (g11, g12, g22) = M (S11, S12, S22) for G = A Sigma A^T
      S.T[6 * 10 + 6] = A[0] * A[0];
      S.T[6 * 10 + 7] = 2.0 * A[0] * A[1];
      S.T[6 * 10 + 8] = A[1] * A[1];
      S.T[7 * 10 + 6] = A[0] * A[2];
      S.T[7 * 10 + 7] = A[0] * A[3] + A[1] * A[2];
      S.T[7 * 10 + 8] = A[1] * A[3];
      S.T[8 * 10 + 6] = A[2] * A[2];
      S.T[8 * 10 + 7] = 2.0 * A[2] * A[3];
      S.T[8 * 10 + 8] = A[3] * A[3];
      S.T[9 * 10 + 9] = 1.0;
    }
    __syncwarp();
    const int b = im.band;
    auto nu_of = [b](int a) { return a < 4 ? 4 * b + a : 16 + a; };   // 4..9 -> 20..25
    auto lo = [](int a) { return a < 4 ? a : (a < 6 ? 4 : (a < 9 ? 6 : 9)); };
    auto hi = [](int a) { return a < 4 ? a + 1 : (a < 6 ? 6 : (a < 9 ? 9 : 10)); };
    if (lane < 10) {
      double gl = 0.0;
      for (int k = lo(lane); k < hi(lane); ++k) gl += S.T[k * 10 + lane] * S.W[2 + k];
      S.gnu[nu_of(lane)] += gl;
    }
    for (int e = lane; e < 55; e += 32) {
      // e -> (a, c) with a <= c in the 10 x 10 upper triangle
      int a = 0, rem = e;
      while (rem >= 10 - a) { rem -= 10 - a; ++a; }
      const int c = a + rem;
      double val = 0.0;
      for (int k = lo(a); k < hi(a); ++k)
        for (int l = lo(c); l < hi(c); ++l) val += S.T[k * 10 + a] * S.T[l * 10 + c] * hw(S.W, k, l);
      const int na = nu_of(a), nc = nu_of(c);
      S.Hnu[na * kNu + nc] += val;
      if (na != nc) S.Hnu[nc * kNu + na] += val;
    }
    vrel += S.W[0];
    vbase += S.W[1];
    __syncwarp();
  }

  // KL (value always; derivatives when needed)
  for (int e = lane; e < kNuPad; e += 32) S.kl[e] = 0.0;
  if (kDerivs) {
    for (int e = lane; e < kNuPad; e += 32) S.gth[e] = 0.0;
    for (int e = lane; e < kTheta * kTheta; e += 32) S.Hth[e] = 0.0;
  }
  __syncwarp();
  kl_terms(th, model, S.kl, S.gth, S.Hth, lane);
  const double kl = S.kl[2];
  // KL terms now sit in gth/Hth with a + sign; the objective subtracts them
  if (kDerivs) {
    for (int e = lane; e < kTheta; e += 32) S.gth[e] = -S.gth[e];
    for (int e = lane; e < kTheta * kTheta; e += 32) S.Hth[e] = -S.Hth[e];
    // Jacobian J[a][c] = d nu_a / d theta_c
    for (int e = lane; e < kNu * kTheta; e += 32) S.J[e] = 0.0;
    __syncwarp();
    if (lane < 20) {
      double* dl = S.DL + lane * kTheta;
      double* d2l = S.D2L + lane * kTheta;
      const double kap = kappa_logderivs(th, lane, dl, d2l);
      for (int c = 0; c < kTheta; ++c) S.J[lane * kTheta + c] = kap * dl[c];
      S.kw[lane] = S.gnu[lane] * kap;
    } else if (lane < 22) {
      S.J[lane * kTheta + 21 + (lane - 20)] = 1.0;
    } else if (lane == 22) {
      double dS[3][3], d2S[3][3][3];
      sigma_derivs(th, dS, d2S);
      for (int e = 0; e < 3; ++e)
        for (int c = 0; c < 3; ++c) S.J[(22 + e) * kTheta + 23 + c] = dS[e][c];
    } else if (lane == 25) {
      const double r = sigm(th[26]);
      S.J[25 * kTheta + 26] = r * (1.0 - r);
    }
    __syncwarp();
    // gradient
    if (lane < kTheta) {
      double gsum = 0.0;
      for (int a = 0; a < kNu; ++a) gsum += S.J[a * kTheta + lane] * S.gnu[a];
      S.gth[lane] += gsum;
    }
    // X = H_nu J
    for (int e = lane; e < kNu * kTheta; e += 32) {
      const int a = e / kTheta, c = e % kTheta;
      double x = 0.0;
      for (int bb = 0; bb < kNu; ++bb) x += S.Hnu[a * kNu + bb] * S.J[bb * kTheta + c];
      S.X[e] = x;
    }
    __syncwarp();
    // Hth += J^T X (upper triangle, mirrored)
    for (int e = lane; e < kTheta * kTheta; e += 32) {
      const int c = e / kTheta, d = e % kTheta;
      if (d < c) continue;
      double x = 0.0;
      for (int a = 0; a < kNu; ++a) x += S.J[a * kTheta + c] * S.X[a * kTheta + d];
      S.Hth[c * kTheta + d] += x;
      if (d != c) S.Hth[d * kTheta + c] += x;
    }
    __syncwarp();
    // second-order chain terms: flux moments (rank-one plus diagonal in
    // d log kappa), then Sigma_s and rho
    for (int e = lane; e < kTheta * kTheta; e += 32) {
      const int c = e / kTheta, d = e % kTheta;
      double x = 0.0;
      for (int a = 0; a < 20; ++a) {
        x += S.kw[a] * S.DL[a * kTheta + c] * S.DL[a * kTheta + d];
        if (c == d) x += S.kw[a] * S.D2L[a * kTheta + c];
      }
      S.Hth[e] += x;
    }
    __syncwarp();
    if (lane == 0) {
      double dS[3][3], d2S[3][3][3];
      sigma_derivs(th, dS, d2S);
      for (int e = 0; e < 3; ++e)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) S.Hth[(23 + c) * kTheta + 23 + d] += S.gnu[22 + e] * d2S[e][c][d];
      const double r = sigm(th[26]);
      S.Hth[26 * kTheta + 26] += S.gnu[25] * r * (1.0 - r) * (1.0 - 2.0 * r);
    }
    __syncwarp();
  }

  // outputs
  const double Lrel = vrel - kl;
  const double Lfull = vbase + vrel - kl;
  if (lane == 0) {
    if (elbo) elbo[j] = Lfull;
    if (elbo_rel) elbo_rel[j] = Lrel;
    if (!isfinite(Lfull)) set_error(v.err, CELESTE_DERR_NONFINITE);
  }
  if (kDerivs) {
    bool bad = false;
    for (int e = lane; e < kTheta; e += 32) {
      grad_out[(size_t)j * kTheta + e] = S.gth[e];
      bad |= !isfinite(S.gth[e]);
    }
    for (int e = lane; e < kTheta * kTheta; e += 32) {
      hess_out[(size_t)j * kTheta * kTheta + e] = S.Hth[e];
      bad |= !isfinite(S.Hth[e]);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(v.err, CELESTE_DERR_NONFINITE);
  }
}

cudaError_t launch_epilogue(const Launch& L, const PlanView& v, const ModelDev* model,
                            double* elbo, double* elbo_rel, double* grad, double* hess) {
  if (v.n == 0) return cudaSuccess;
  const size_t sm = sizeof(EpiSmem);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(epilogue_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  epilogue_kernel<true><<<v.n, 32, sm, L.stream>>>(v, model, elbo, elbo_rel, grad, hess, 0);
  return cudaGetLastError();
}

cudaError_t launch_epilogue_value(const Launch& L, const PlanView& v, const ModelDev* model,
                                  double* elbo, double* elbo_rel, bool use_trial) {
  if (v.n == 0) return cudaSuccess;
  const size_t sm = sizeof(EpiSmem);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(epilogue_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  epilogue_kernel<false><<<v.n, 32, sm, L.stream>>>(v, model, elbo, elbo_rel, nullptr, nullptr,
                                                    use_trial ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace celeste
