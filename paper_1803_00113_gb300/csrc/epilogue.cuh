// Per-source epilogue (device code shared by the epilogue kernels and the
// per-source Newton step): reduce the per-tile sums of a source, map them from
// each image's natural coordinates to the source's 27 unconstrained
// coordinates, and add the KL term.
//
// Chain rule, exact because every map is applied to reduced sums:
//   per image (affine):  cE_i = calib * kE_i[b], cM_i = calib^2 * kM_i[b],
//                        mu = A u + t, G = A Sigma_s A^T, rho = rho;
//   per source:          kE_i[b] = q_i exp(m_ib + v_ib / 2),
//                        kM_i[b] = q_i exp(2 m_ib + 2 v_ib)     (Sec. 2.1.2,
//                        Eqs. conditional and vareq: E[l|a], E[l^2|a] with
//                        log l ~ N(m, v)),
//                        Sigma_s(angle, radius, axis) = R^T D R (Sec. 2.1.3),
//                        rho = sigmoid(theta_26);
//   grad_theta = J^T grad_nu,
//   hess_theta = J^T H_nu J + sum_a grad_nu[a] * hess_theta(nu_a).
// KL_s follows Eq. kleq, Supplement A and the GMM colour bound of Sec. 4.2.3
// with xi minimised in closed form: -log sum_j w_j exp(-KL(q(c|a) || N_j)).
//
// Precision: the inputs of the chain rule are sums accumulated in FP32 by
// the pixel kernel, so the chain rule and the KL run in FP32 ("real"), which
// adds rounding of the same order as its inputs already carry; the value
// sums (which include the large sky baseline) stay in FP64.  On GB300 an
// FP64 instruction costs ~64 cycles per SM sub-partition, and this kernel
// is on the critical path of every colour class.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace celeste {

typedef float real;

static __constant__ signed char kSelE[5][4] = {
    {-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

constexpr int kNu = 26;   // 20 flux moments (band b, kind e at 4b+e), u (2), Sigma_s (3), rho
constexpr int kNuPad = 32;
constexpr int kKlVals = 8 + 10 + 4;       // per colour component: grad, precision, diag
constexpr int kKlSums = 64;                // per type: mean grad 8, centred outer 36, prec 10, diag 4

static __device__ __forceinline__ real sigm(real t) {
  return t >= 0.f ? 1.f / (1.f + expf(-t)) : expf(t) / (1.f + expf(t));
}
// log(1 + exp(t)) without overflow
static __device__ __forceinline__ real softplus(real t) {
  return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t));
}

constexpr int kEpiThreads = 128;   // four warps per source
constexpr int kPairThreads = kEpiThreads - 32;   // warps 1..3: the pixel sums
constexpr int kPairGroup = 4;                    // pairs reduced together

// Barrier among the kPairThreads threads of warps 1..3 (named barrier 1;
// warp 0 is busy with the KL terms meanwhile).
static __device__ __forceinline__ void pair_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kPairThreads) : "memory");
}

struct EpiSmem {
  double Wd[kPairGroup][2];        // per pair of a group: value sums (relative, base)
  float W[kPairGroup][kAcc];       // per pair of a group: the other sums (entries 2..63)
  real th[kNuPad];                 // theta of the source (FP32 copy)
  real gnu[kNuPad];
  real Hnu[kNu * kNu];
  real J[kNu * kTheta];
  real X[kNu * kTheta];
  real gth[kNuPad];
  real Hth[kTheta * kTheta];
  real DL[20 * kTheta];            // d log kappa_a / d theta
  real D2L[20 * kTheta];           // diagonal second derivatives of log kappa_a
  real kw[kNuPad];                 // grad_nu[a] * kappa_a
  real klc[2 * kMaxColor * kKlVals];   // colour-bound pieces per (type, component)
  real klj[2 * kMaxColor];         // log w_j - K_j
  real kls[8];                     // scalar KL pieces
  float T[kPairGroup][10 * 10];    // per pair of a group: affine map w <- nu (local)
  double red[2][kEpiThreads / 32]; // per-warp value sums
  double vsum[2];                  // the source's value sums (relative, base)
};

// Rows a of J with J[a][c] != 0 for column c: their number and the k-th one
// (the flux coordinates of a type feed every band's kE and kM rows).
static __device__ __forceinline__ int nrows(int c) {
  return c == 0 ? 20 : (c <= 20 ? 10 : (c <= 22 ? 1 : (c <= 25 ? 3 : 1)));
}
static __device__ __forceinline__ int rowof(int c, int k) {
  if (c == 0) return k;
  if (c <= 20) return 2 * k + (c <= 4 ? (c - 1) / 2 : ((c - 5) / 4) & 1);
  if (c <= 22) return c - 1;
  if (c <= 25) return 22 + k;
  return 25;
}


// d log kappa / d theta for flux-moment coordinate a (0..19): band b = a / 4,
// kind e = a % 4 (0: kE0, 1: kE1, 2: kM0, 3: kM1).  Returns kappa.
static __device__ real kappa_logderivs(const real* th, int a, real* dl, real* d2l) {
  const int b = a >> 2, e = a & 3;
  const int i = e & 1;
  const bool second = e >= 2;
  const real am = second ? 2.f : 1.f, av = second ? 2.f : 0.5f;
  for (int c = 0; c < kTheta; ++c) dl[c] = d2l[c] = 0.f;
  const real q1 = sigm(th[0]), q0 = sigm(-th[0]);
  const real logq = i ? -softplus(-th[0]) : -softplus(th[0]);
  dl[0] = i ? q0 : -q1;
  d2l[0] = -q0 * q1;
  const int ir = 1 + 2 * i, iv = 2 + 2 * i;
  real m = th[ir], v = expf(th[iv]);
  dl[ir] = am;
  dl[iv] = av * v;
  d2l[iv] = dl[iv];
  for (int k = 0; k < 4; ++k) {
    const real s = (real)kSelE[b][k];
    const real cvk = expf(th[13 + 4 * i + k]);
    m += s * th[5 + 4 * i + k];
    v += s * s * cvk;
    dl[5 + 4 * i + k] = am * s;
    dl[13 + 4 * i + k] = av * s * s * cvk;
    d2l[13 + 4 * i + k] = dl[13 + 4 * i + k];
  }
  return expf(logq + am * m + av * v);
}

// Derivatives of Sigma_s = (S11, S12, S22) over (angle, log radius, logit axis).
static __device__ void sigma_derivs(const real* th, real dS[3][3], real d2S[3][3][3]) {
  const real phi = th[23], lr = th[24];
  const real ax = sigm(th[25]);
  const real e2 = expf(2.f * lr);
  const real a2 = ax * ax;
  const real a2t = 2.f * a2 * (1.f - ax);
  const real a2tt = 2.f * a2 * (1.f - ax) * (2.f - 3.f * ax);
  const real P = 0.5f * e2 * (1.f + a2), Qd = 0.5f * e2 * (1.f - a2);
  const real Pl = 2.f * P, Pll = 4.f * P, Pt = 0.5f * e2 * a2t, Ptt = 0.5f * e2 * a2tt, Plt = 2.f * Pt;
  const real Ql = 2.f * Qd, Qll = 4.f * Qd, Qt = -0.5f * e2 * a2t, Qtt = -0.5f * e2 * a2tt, Qlt = 2.f * Qt;
  real S2, C2;
  sincosf(2.f * phi, &S2, &C2);
  // S11 = P + Qd C2, S22 = P - Qd C2, S12 = -Qd S2
  for (int e = 0; e < 3; e += 2) {
    const real s = e == 0 ? 1.f : -1.f;
    dS[e][0] = -2.f * s * Qd * S2;
    dS[e][1] = Pl + s * Ql * C2;
    dS[e][2] = Pt + s * Qt * C2;
    d2S[e][0][0] = -4.f * s * Qd * C2;
    d2S[e][0][1] = d2S[e][1][0] = -2.f * s * Ql * S2;
    d2S[e][0][2] = d2S[e][2][0] = -2.f * s * Qt * S2;
    d2S[e][1][1] = Pll + s * Qll * C2;
    d2S[e][1][2] = d2S[e][2][1] = Plt + s * Qlt * C2;
    d2S[e][2][2] = Ptt + s * Qtt * C2;
  }
  dS[1][0] = -2.f * Qd * C2;
  dS[1][1] = -Ql * S2;
  dS[1][2] = -Qt * S2;
  d2S[1][0][0] = 4.f * Qd * S2;
  d2S[1][0][1] = d2S[1][1][0] = -2.f * Ql * C2;
  d2S[1][0][2] = d2S[1][2][0] = -2.f * Qt * C2;
  d2S[1][1][1] = -Qll * S2;
  d2S[1][1][2] = d2S[1][2][1] = -Qlt * S2;
  d2S[1][2][2] = -Qtt * S2;
}

// KL_s: value into S.kls[0]; for kMode >= 1 the gradient and for kMode == 2
// also the Hessian are ADDED (with a minus sign, since L = ... - KL) into
// S.gth and S.Hth.
template <int kMode>
static __device__ void kl_terms(const real* th, const ModelDev* m, EpiSmem& S, int lane) {
  const real a = sigm(th[0]);
  const real wq = a * (1.f - a);
  const int J = m->n_color;
  // ---- colour bound, one lane per (type, component)
  if (lane < 2 * kMaxColor) {
    const int i = lane / kMaxColor, j = lane % kMaxColor;
    if (j < J) {
      const float(*P)[4] = m->f.color_prec[i][j];
      const real* cm = th + 5 + 4 * i;
      const real* lcv = th + 13 + 4 * i;
      real d[4], cv[4], pd[4];
      real tr = 0.f, quad = 0.f, slv = 0.f;
      for (int k = 0; k < 4; ++k) {
        d[k] = cm[k] - m->f.color_mean[i][j][k];
        cv[k] = expf(lcv[k]);
      }
      for (int k = 0; k < 4; ++k) {
        real s = 0.f;
        for (int l = 0; l < 4; ++l) s = fmaf(P[k][l], d[l], s);
        pd[k] = s;
        tr = fmaf(P[k][k], cv[k], tr);
        quad = fmaf(d[k], s, quad);
        slv += lcv[k];
      }
      const real K = 0.5f * (tr + quad - 4.f + m->f.color_logdet[i][j] - slv);
      S.klj[lane] = m->f.log_color_w[i][j] - K;
      if (kMode >= 1) {
        real* o = S.klc + lane * kKlVals;
        real gk[8];
        for (int k = 0; k < 4; ++k) {
          gk[k] = pd[k];
          gk[4 + k] = 0.5f * (P[k][k] * cv[k] - 1.f);
        }
        for (int k = 0; k < 8; ++k) o[k] = gk[k];
        int t = 8;
        for (int k = 0; k < 4; ++k)
          for (int l = k; l < 4; ++l) o[t++] = P[k][l];
        for (int k = 0; k < 4; ++k) o[t++] = 0.5f * P[k][k] * cv[k];
      }
    } else {
      S.klj[lane] = -INFINITY;
    }
  }
  __syncwarp();
  // ---- per type: softmax weights pi_j = w_j exp(-K_j) / sum (one exp per lane)
  if (lane < 2 * kMaxColor) {
    const int i = lane / kMaxColor;
    real mx = -INFINITY;
    for (int j = 0; j < J; ++j) mx = fmaxf(mx, S.klj[i * kMaxColor + j]);
    S.kw[lane] = (lane % kMaxColor) < J ? expf(S.klj[lane] - mx) : 0.f;   // scratch
    S.kls[4 + i] = mx;
  }
  __syncwarp();
  real Bval[2], se[2];
  for (int i = 0; i < 2; ++i) {
    se[i] = 0.f;
    for (int j = 0; j < J; ++j) se[i] += S.kw[i * kMaxColor + j];
    Bval[i] = -(S.kls[4 + i] + logf(se[i]));
  }
  if (kMode >= 1) {
    // pi-weighted sums per type (S.X as scratch, kKlSums per type): the mean
    // gradient, the precision block and the diagonal ...
    for (int e = lane; e < 2 * kKlVals; e += 32) {
      const int i = e / kKlVals, vv = e % kKlVals;
      real acc = 0.f;
      for (int j = 0; j < J; ++j)
        acc = fmaf(S.kw[i * kMaxColor + j], S.klc[(i * kMaxColor + j) * kKlVals + vv], acc);
      S.X[i * kKlSums + (vv < 8 ? vv : 36 + vv)] = acc / se[i];
    }
    __syncwarp();
    // ... then the covariance of the gradients across components in centred
    // form, sum_j pi_j (g_j - gbar)(g_j - gbar)^T, which does not cancel
    for (int e = lane; e < (kMode == 2 ? 2 * 36 : 0); e += 32) {
      const int i = e / 36;
      int u = 0, rem = e % 36;
      while (rem >= 8 - u) { rem -= 8 - u; ++u; }
      const int w = u + rem;
      const real gu = S.X[i * kKlSums + u], gw = S.X[i * kKlSums + w];
      real acc = 0.f;
      for (int j = 0; j < J; ++j) {
        const real* gj = S.klc + (i * kMaxColor + j) * kKlVals;
        acc = fmaf(S.kw[i * kMaxColor + j], (gj[u] - gu) * (gj[w] - gw), acc);
      }
      S.X[i * kKlSums + 8 + (e % 36)] = acc / se[i];
    }
  }
  __syncwarp();
  // ---- value (lane 0)
  if (lane == 0) {
    real v = a * (-softplus(-th[0]) - m->f.log_prior_a) +
             (1.f - a) * (-softplus(th[0]) - m->f.log1m_prior_a);
    for (int i = 0; i < 2; ++i) {
      const real R1 = m->f.prior_r[i][0], R2 = m->f.prior_r[i][1];
      const real rm = th[1 + 2 * i], lrv = th[2 + 2 * i], rv = expf(lrv);
      const real klr = 0.5f * (m->f.log_prior_r2[i] - lrv + (rv + (rm - R1) * (rm - R1)) / R2 - 1.f);
      S.kls[2 + i] = klr + Bval[i];
      v += (i ? a : 1.f - a) * S.kls[2 + i];
    }
    const real lr = th[24], E1 = m->f.e_radius[0], E2 = m->f.e_radius[1];
    v += lr + m->f.half_log_2pi_e2 + (lr - E1) * (lr - E1) / (2.f * E2);
    for (int which = 0; which < 2; ++which) {
      const int t = which ? 26 : 25;
      const real b1 = (which ? m->f.e_profile[0] : m->f.e_axis[0]);
      const real b2 = (which ? m->f.e_profile[1] : m->f.e_axis[1]);
      v += (b1 - 1.f) * softplus(-th[t]) + (b2 - 1.f) * softplus(th[t]) +
           (which ? m->f.log_beta_profile : m->f.log_beta_axis);
    }
    S.kls[0] = v;
  }
  __syncwarp();
  if (kMode == 0) return;
  // per type i, local coordinates 0 r-mean, 1 log r-var, 2..5 colour means,
  // 6..9 log colour vars; theta index of local k:
  auto tidx = [](int i, int k) {
    return k == 0 ? 1 + 2 * i : (k == 1 ? 2 + 2 * i : (k < 6 ? 5 + 4 * i + (k - 2) : 13 + 4 * i + (k - 6)));
  };
  // gradient-only mode visits the (i, k, l = 0) entries only
  for (int e0 = lane; e0 < (kMode == 2 ? 200 : 20); e0 += 32) {
    const int e = kMode == 2 ? e0 : (e0 / 10) * 100 + (e0 % 10) * 10;
    const int i = e / 100, k = (e % 100) / 10, l = e % 10;
    const real* pw = S.X + i * kKlSums;       // grad(8), centred outer(36), prec(10), diag(4)
    const real R2 = m->f.prior_r[i][1];
    const real rm = th[1 + 2 * i], rv = expf(th[2 + 2 * i]);
    // gradient of K_i = KL_r + B at local k
    auto gK = [&](int kk) {
      if (kk == 0) return (rm - m->f.prior_r[i][0]) / R2;
      if (kk == 1) return 0.5f * (rv / R2 - 1.f);
      return pw[kk - 2];
    };
    real h = 0.f;
    if (k < 2 || l < 2) {
      if (k == l && k == 0) h = 1.f / R2;
      if (k == l && k == 1) h = 0.5f * rv / R2;
    } else {
      const int u = k - 2, w = l - 2;        // colour block 0..7
      const int lo = u < w ? u : w, hi = u < w ? w : u;
      // sum_j pi_j H_j - sum_j pi_j (g_j - gbar)(g_j - gbar)^T
      const int oi = lo * 8 - (lo * (lo - 1)) / 2 + (hi - lo);
      h = -pw[8 + oi];
      if (u < 4 && w < 4) {
        const int po = lo * 4 - (lo * (lo - 1)) / 2 + (hi - lo);
        h += pw[44 + po];
      } else if (u == w) {
        h += pw[54 + (u - 4)];
      }
    }
    const real qi = i ? a : 1.f - a;
    if (kMode == 2) S.Hth[tidx(i, k) * kTheta + tidx(i, l)] -= qi * h;
    if (l == 0) {
      const real dq = i ? wq : -wq;
      const real g = gK(k);
      S.gth[tidx(i, k)] -= qi * g;
      if (kMode == 2) {
        S.Hth[tidx(i, k) * kTheta + 0] -= dq * g;
        S.Hth[0 * kTheta + tidx(i, k)] -= dq * g;
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    const real la = m->f.logit_prior_a;
    const real d2q = wq * (1.f - 2.f * a);
    S.gth[0] -= wq * (th[0] - la) + wq * (S.kls[3] - S.kls[2]);
    if (kMode == 2)
      S.Hth[0] -= wq * ((1.f - 2.f * a) * (th[0] - la) + 1.f) + d2q * (S.kls[3] - S.kls[2]);
    const real lr = th[24], E1 = m->f.e_radius[0], E2 = m->f.e_radius[1];
    S.gth[24] -= 1.f + (lr - E1) / E2;
    if (kMode == 2) S.Hth[24 * kTheta + 24] -= 1.f / E2;
    for (int which = 0; which < 2; ++which) {
      const int t = which ? 26 : 25;
      const real b1 = (which ? m->f.e_profile[0] : m->f.e_axis[0]);
      const real b2 = (which ? m->f.e_profile[1] : m->f.e_axis[1]);
      const real sg = sigm(th[t]);
      S.gth[t] -= -(b1 - 1.f) * (1.f - sg) + (b2 - 1.f) * sg;
      if (kMode == 2) S.Hth[t * kTheta + t] -= (b1 + b2 - 2.f) * sg * (1.f - sg);
    }
  }
  __syncwarp();
}

// Slot j of the plan, by the whole block.  kMode: 0 value, 1 value + gradient, 2 value + gradient + Hessian.  Four
// warps per source: warp 0 evaluates the KL terms while warps 1..3 reduce
// the tile sums and apply the per-image maps; then warp 0 forms the Jacobian
// rows and the two dense products (X = H_nu J, H_theta += J^T X) are spread
// over the block in register-blocked chains.
template <int kMode>
static __device__ __forceinline__ void epilogue_source(const PlanView& v,
                                                const ModelDev* __restrict__ model,
                                                EpiSmem& S, int j, double* elbo,
                                                double* elbo_rel, double* grad_out,
                                                double* hess_out, int use_trial) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (!v.active[j]) return;
  const int src = v.src_ids[j];
  // use_trial: bit 0 evaluates theta_trial; bit 1 (value mode only) asks
  // for the pixel part alone, without the KL (the log-likelihood of the
  // source's point values relative to its absence)
  const bool trial = (use_trial & 1) != 0, pixel_only = kMode == 0 && (use_trial & 2) != 0;
  const double* thd = trial ? v.theta_trial + (size_t)j * kTheta : v.theta + (size_t)src * kTheta;
  if (tid < kTheta) S.th[tid] = (real)thd[tid];
  const real* th = S.th;

  double vrel = 0.0, vbase = 0.0;
  if (kMode >= 1) {
    // the slot's tile sums (its pairs' items are contiguous, 256 B an item)
    // asked into L2 at once: the pair loop below then reads them from L2,
    // not from DRAM, pair after pair
    const int p0 = v.slot_pair_ptr[j], p1 = v.slot_pair_ptr[j + 1];
    if (p1 > p0) {
      const int64_t i0 = v.pairs[p0].item_begin, i1 = v.pairs[p1 - 1].item_end;
      const char* base = reinterpret_cast<const char*>(v.partials + i0 * kAcc);
      const int64_t lines = (i1 - i0) * (kAcc * (int64_t)sizeof(float) / 128);
      for (int64_t l = tid; l < lines; l += kEpiThreads)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + 128 * l));
    }
    for (int e = tid; e < kNuPad; e += kEpiThreads) S.gnu[e] = 0.f;
    for (int e = tid; e < kNuPad; e += kEpiThreads) S.gth[e] = 0.f;
  }
  if (kMode == 2) {
    for (int e = tid; e < kNu * kNu; e += kEpiThreads) S.Hnu[e] = 0.f;
    for (int e = tid; e < kTheta * kTheta; e += kEpiThreads) S.Hth[e] = 0.f;
  }
  __syncthreads();
  // Warp 0 evaluates the KL terms, which depend on theta alone, while warps
  // 1..3 reduce the pixel sums pair by pair (named barrier 1 among them).
  if (wid == 0) {
    if (!pixel_only) kl_terms<kMode>(th, model, S, lane);
  } else {
    const int u = tid - 32;                            // 0 .. kPairThreads - 1
    double vr = 0.0, vb = 0.0;
    if (kMode == 0) {
      // value sums of every pair's items, thread-strided, then one reduction
      for (int pp = v.slot_pair_ptr[j]; pp < v.slot_pair_ptr[j + 1]; ++pp) {
        const PairInfo pi = v.pairs[pp];
        for (int it = pi.item_begin + u; it < pi.item_end; it += kPairThreads) {
          vr += (double)v.vpartials[2 * (size_t)it];
          vb += (double)v.vpartials[2 * (size_t)it + 1];
        }
      }
      vr = warp_sum_d(vr);
      vb = warp_sum_d(vb);
      if (lane == 0) {
        S.red[0][wid - 1] = vr;
        S.red[1][wid - 1] = vb;
      }
      pair_sync();
      if (u == 0) {
        vr = S.red[0][0] + S.red[0][1] + S.red[0][2];
        vb = S.red[1][0] + S.red[1][1] + S.red[1][2];
      }
    } else {
      // kPairGroup pairs at a time: their tile sums in one loop (loads of
      // every pair in flight together) and their images' maps, then the
      // per-pair updates in pair order; each sum below is updated by one
      // thread, pair after pair, as with one pair at a time
      const int pend = v.slot_pair_ptr[j + 1];
      for (int pp = v.slot_pair_ptr[j]; pp < pend; pp += kPairGroup) {
        const int ng = min(kPairGroup, pend - pp);
        if (u < kAcc) {
          // the pairs' tile sums, accumulator u: compensated (Kahan) FP32
          // summation whose error does not grow with the number of tiles;
          // the loads are independent of the chains, so they run ahead
          float s0[kPairGroup], c0[kPairGroup];
          int ib[kPairGroup], nit[kPairGroup];
          int nmax = 0;
#pragma unroll
          for (int g = 0; g < kPairGroup; ++g) {
            s0[g] = c0[g] = 0.f;
            ib[g] = nit[g] = 0;
            if (g < ng && (kMode == 2 || u < kGradAcc)) {
              ib[g] = v.pairs[pp + g].item_begin;
              nit[g] = v.pairs[pp + g].item_end - ib[g];
              nmax = max(nmax, nit[g]);
            }
          }
#pragma unroll 4
          for (int t = 0; t < nmax; ++t) {
#pragma unroll
            for (int g = 0; g < kPairGroup; ++g) {
              if (t < nit[g]) {
                const float y0 = v.partials[(size_t)(ib[g] + t) * kAcc + u] - c0[g];
                const float t0 = s0[g] + y0;
                c0[g] = (t0 - s0[g]) - y0;
                s0[g] = t0;
              }
            }
          }
          // the value sums go on in FP64; the others are used in FP32, and
          // s0 - c0 rounded once to FP32 equals (float)((double)s0 -
          // (double)c0): that double difference is exact or off s0 by far
          // less than half an FP32 unit in the last place
#pragma unroll
          for (int g = 0; g < kPairGroup; ++g) {
            if (g < ng) {
              if (u < 2) {
                S.Wd[g][u] = (double)s0[g] - (double)c0[g];
              } else {
                S.W[g][u] = s0[g] - c0[g];
              }
            }
          }
        } else {
          // each pair's local affine map, FP32: w_k = sum_a T[k][a] nu_a
          for (int g = 0; g < ng; ++g) {
            const celeste_image& im = v.images[v.pairs[pp + g].image];
            const float cal = (float)im.calib;
            const float A0 = (float)im.wcs_A[0], A1 = (float)im.wcs_A[1];
            const float A2 = (float)im.wcs_A[2], A3 = (float)im.wcs_A[3];
            for (int e = u - kAcc; e < 100; e += kPairThreads - kAcc) {
              float t = 0.f;
              switch (e) {
                case 0: case 11: t = cal; break;
                case 22: case 33: t = cal * cal; break;
                case 44: t = A0; break;
                case 45: t = A1; break;
                case 54: t = A2; break;
                case 55: t = A3; break;
                case 66: t = A0 * A0; break;
                case 67: t = 2.f * A0 * A1; break;
                case 68: t = A1 * A1; break;
                case 76: t = A0 * A2; break;
                case 77: t = A0 * A3 + A1 * A2; break;
                case 78: t = A1 * A3; break;
                case 86: t = A2 * A2; break;
                case 87: t = 2.f * A2 * A3; break;
                case 88: t = A3 * A3; break;
                case 99: t = 1.f; break;
                default: break;
              }
              S.T[g][e] = t;
            }
          }
        }
        pair_sync();
        auto lo = [](int a) { return a < 4 ? a : (a < 6 ? 4 : (a < 9 ? 6 : 9)); };
        auto hi = [](int a) { return a < 4 ? a + 1 : (a < 6 ? 6 : (a < 9 ? 9 : 10)); };
        if (u < 10) {
          for (int g = 0; g < ng; ++g) {
            const int b = v.pairs[pp + g].band;
            const float* T = S.T[g];
            const float* W = S.W[g];
            float gl = 0.f;
            for (int k = lo(u); k < hi(u); ++k) gl += T[k * 10 + u] * W[2 + k];
            S.gnu[u < 4 ? 4 * b + u : 16 + u] += gl;    // nu of w_u (4..9 -> 20..25)
          }
        } else if (kMode == 2 && u >= 32 && u < 32 + 55) {
          const int e = u - 32;
          int a = 0, rem = e;
          while (rem >= 10 - a) { rem -= 10 - a; ++a; }
          const int c = a + rem;
          for (int g = 0; g < ng; ++g) {
            const int b = v.pairs[pp + g].band;
            const float* T = S.T[g];
            const float* W = S.W[g];
            float val = 0.f;
            for (int k = lo(a); k < hi(a); ++k)
              for (int l = lo(c); l < hi(c); ++l) {
                const int kk = k < l ? k : l, ll = k < l ? l : k;
                const bool zero = (kk == 2 || kk == 3) && (ll == 2 || ll == 3);
                const float hwv = zero ? 0.f : W[hidx(kk, ll)];
                val = fmaf(T[k * 10 + a] * T[l * 10 + c], hwv, val);
              }
            const int na = a < 4 ? 4 * b + a : 16 + a, nc = c < 4 ? 4 * b + c : 16 + c;
            S.Hnu[na * kNu + nc] += val;
            if (na != nc) S.Hnu[nc * kNu + na] += val;
          }
        }
        if (u == 0) {
          for (int g = 0; g < ng; ++g) {
            vr += S.Wd[g][0];
            vb += S.Wd[g][1];
          }
        }
        pair_sync();
      }
    }
    if (u == 0) {
      S.vsum[0] = vr;
      S.vsum[1] = vb;
    }
  }
  __syncthreads();
  vrel = S.vsum[0];
  vbase = S.vsum[1];
  const double kl = pixel_only ? 0.0 : (double)S.kls[0];
  if (kMode >= 1) {
    if (wid == 0) {
      // Jacobian rows: flux moments (lanes 0..19), u, Sigma_s, rho
      for (int e = lane; e < kNu * kTheta; e += 32) S.J[e] = 0.f;
      __syncwarp();
      if (lane < 20) {
        real* dl = S.DL + lane * kTheta;
        real* d2l = S.D2L + lane * kTheta;
        const real kap = kappa_logderivs(th, lane, dl, d2l);
        for (int c = 0; c < kTheta; ++c) S.J[lane * kTheta + c] = kap * dl[c];
        S.kw[lane] = S.gnu[lane] * kap;
      } else if (lane < 22) {
        S.J[lane * kTheta + 21 + (lane - 20)] = 1.f;
      } else if (lane == 22) {
        real dS[3][3], d2S[3][3][3];
        sigma_derivs(th, dS, d2S);
        for (int e = 0; e < 3; ++e)
          for (int c = 0; c < 3; ++c) S.J[(22 + e) * kTheta + 23 + c] = dS[e][c];
        real h[3][3] = {{0.f}};
        for (int e = 0; e < 3; ++e)
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) h[c][d] += S.gnu[22 + e] * d2S[e][c][d];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) S.X[8 * 64 + c * 3 + d] = h[c][d];   // parked below
      } else if (lane == 25) {
        const real r = sigm(th[26]);
        S.J[25 * kTheta + 26] = r * (1.f - r);
      }
      __syncwarp();
      if (kMode == 2) {
        // Sigma_s second-order chain term (parked by lane 22 in X's space)
        if (lane < 9) S.Hth[(23 + lane / 3) * kTheta + 23 + lane % 3] += S.X[8 * 64 + lane];
        if (lane == 0) {
          const real r = sigm(th[26]);
          S.Hth[26 * kTheta + 26] += S.gnu[25] * r * (1.f - r) * (1.f - 2.f * r);
        }
      }
      __syncwarp();
      // gradient: J^T grad_nu over each column's rows
      if (lane < kTheta) {
        const int nr = nrows(lane);
        real gsum = 0.f;
        for (int k = 0; k < nr; ++k) {
          const int a = rowof(lane, k);
          gsum = fmaf(S.J[a * kTheta + lane], S.gnu[a], gsum);
        }
        S.gth[lane] += gsum;
      }
    }
    __syncthreads();
    if (kMode == 2) {
      // X = H_nu J where J's column has support: thread (c, g) forms rows
      // a = g, g + 4, ... of column c, seven independent chains sharing
      // each entry of J
      if (tid < 4 * kTheta) {
        const int c = tid % kTheta, g = tid / kTheta;
        const int nr = nrows(c);
        real x[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < nr; ++k) {
          const int r = rowof(c, k);
          const real jv = S.J[r * kTheta + c];
#pragma unroll
          for (int m = 0; m < 7; ++m) {
            const int a = g + 4 * m;
            if (a < kNu) x[m] = fmaf(S.Hnu[a * kNu + r], jv, x[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < 7; ++m) {
          const int a = g + 4 * m;
          if (a < kNu) S.X[a * kTheta + c] = x[m];
        }
      }
      __syncthreads();
      // Hth += J^T X over d >= c (mirrored), plus the flux-moment
      // second-order term sum_a kw_a (dl dl^T + diag d2l): thread (c, g)
      // takes d = c + g, c + g + 4, ...
      if (tid < 4 * kTheta) {
        const int c = tid % kTheta, g = tid / kTheta;
        const int nr = nrows(c);
        real x[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < nr; ++k) {
          const int r = rowof(c, k);
          const real jv = S.J[r * kTheta + c];
#pragma unroll
          for (int m = 0; m < 7; ++m) {
            const int d = c + g + 4 * m;
            if (d < kTheta) x[m] = fmaf(jv, S.X[r * kTheta + d], x[m]);
          }
        }
        if (c <= 20) {
          for (int k = 0; k < nr; ++k) {
            const int a = rowof(c, k);
            if (a >= 20) break;
            const real kd = S.kw[a] * S.DL[a * kTheta + c];
#pragma unroll
            for (int m = 0; m < 7; ++m) {
              const int d = c + g + 4 * m;
              if (d <= 20) {
                x[m] = fmaf(kd, S.DL[a * kTheta + d], x[m]);
                if (d == c) x[m] = fmaf(S.kw[a], S.D2L[a * kTheta + c], x[m]);
              }
            }
          }
        }
#pragma unroll
        for (int m = 0; m < 7; ++m) {
          const int d = c + g + 4 * m;
          if (d < kTheta) {
            S.Hth[c * kTheta + d] += x[m];
            if (d != c) S.Hth[d * kTheta + c] += x[m];
          }
        }
      }
      __syncthreads();
    }
  }

  const double Lrel = vrel - kl;
  const double Lfull = vbase + vrel - kl;
  if (tid == 0) {
    if (elbo) elbo[j] = Lfull;
    if (elbo_rel) elbo_rel[j] = Lrel;
    // a non-finite value at a trial point is a rejected step, not an error
    if (!isfinite(Lfull) && !trial) set_error(v.err, CELESTE_DERR_NONFINITE);
  }
  if (kMode >= 1) {
    int bad = 0;
    for (int e = tid; e < kTheta; e += kEpiThreads) {
      grad_out[(size_t)j * kTheta + e] = (double)S.gth[e];
      bad |= !isfinite(S.gth[e]);
    }
    for (int e = tid; e < (kMode == 2 ? kTheta * kTheta : 0); e += kEpiThreads) {
      hess_out[(size_t)j * kTheta * kTheta + e] = (double)S.Hth[e];
      bad |= !isfinite(S.Hth[e]);
    }
    if (__syncthreads_or(bad) && tid == 0) set_error(v.err, CELESTE_DERR_NONFINITE);
  }
}

}  // namespace celeste
