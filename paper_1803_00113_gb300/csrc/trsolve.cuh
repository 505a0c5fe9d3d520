// FP64 trust-region Newton step (Sec. 4.3): maximise g.p + p.H.p / 2 over
// the ball |p| <= Delta exactly, then accept or reject the trial point.
//
// GB300 issues a warp-wide FP64 instruction about every 64 cycles per SM
// sub-partition, so the cost of this kernel is its count of dependent FP64
// warp instructions, and a source gets four warps (one per sub-partition).
// The usual path is mixed: FP32 locates lambda_min and the multiplier (a
// Householder reduction and multisections, cheap on the FP32 pipes), then
// FP64 computes the answer on the full matrix with one to three LDL^T
// factorisations (safeguarded Newton on the secular equation).  Close to the
// pole, and whenever FP64 contradicts the FP32 estimate, the all-FP64 path
// below takes over:
//   * B = -H is reduced to tridiagonal form T = Q^T B Q by Householder
//     reflections; rows are spread over the lanes and columns over the four
//     warps;
//   * lambda_min(T): multisection on Sturm counts, first in FP32 on the
//     scaled matrix, then refined in FP64 with the division-free
//     characteristic-polynomial sequence (31 probes per round);
//   * the multiplier l solving |(T + l I)^{-1} Q^T g| = Delta: FP32
//     multisection for a starting point, then the safeguarded Newton
//     iteration on 1/|y(l)| - 1/Delta (Nocedal & Wright, Algorithm 4.3),
//     each FP64 evaluation one LDL^T factorisation of T + l I;
//   * the hard case (g orthogonal to the eigenvector of lambda_min) adds
//     that eigenvector, from inverse iteration, to reach the boundary; its
//     sign makes the first nonzero entry of Q z positive;
//   * p = Q y and the predicted gain g.p + p.H.p/2 = y.Q^T g - y.T.y/2.
// Trust-region constants follow the textbook loop (Nocedal & Wright,
// Algorithm 4.1): accept when rho > 0.1, shrink to |p|/4 when rho < 1/4,
// double (up to 100) when rho > 3/4 and the step reached the boundary.
#pragma once

#include <math.h>

#include "accept.cuh"
#include "internal.cuh"

namespace celeste {

constexpr int N = kTheta;
constexpr int kTrThreads = 128;
constexpr double kFtol = 1e-9;
constexpr double kDeltaMin = 1e-8;

constexpr int kTri = N * (N + 1) / 2;                        // 378 lower entries

struct TrSmem {
  double B[N * N];
  // mixed-precision path.  The FP32 reduction (Bf), then locate32's
  // per-thread elimination factors (cps, gps: [i][thread]), then the FP64
  // factorisations (W, L) use the same memory in turn.
  union Work {
    struct Fp64 {
      double W[N * N];             // factorisation work copy of B + l I
      double L[N * N];             // unit lower factor of B + l I (strict lower part)
      float Bf[N * N];             // FP32 copy of B, reduced to tridiagonal form
    } f;
    struct Sec {
      float cps[N * kTrThreads], gps[N * kTrThreads];
    } s;
  } ws;
  double Dinv[32];                 // 1 / D
  double col[2][32];               // published pivot column, double-buffered
  double p[32];
  double lam, lo, hi;              // multiplier and its bracket (unscaled)
  double lmin_lo;                  // lower bound of lambda_min (unscaled, FP32 accuracy)
  double lam_b;                    // boundary start when an interior try fails (0: none)
  int positive;                    // FP32 finds B positive definite
  int tried0;                      // l = 0 has been evaluated
  int bisects;                     // bisection steps of the FP64 iteration
  float betaf[32], dfr[32], efr[32], gfr[32];
  float loc[4];                    // locate32: scale, |g|^2 (scaled), |p(0)|^2
  unsigned hmask[2][4];            // locate32: probe ballots of the four warps
  short2 tri[kTri];                // lower entry e -> (row, column)
  int mode;                        // 0 interior candidate, 1 boundary, 2 full FP64 path
  double beta[32];
  double gh[32];
  double d[32];
  double e[32];
  double ds[32], es[32], gs[32];   // scaled T and Q^T g (|T / scale| <= 1)
  double y[32];
  double z[32];
  double w[32];
  double part[4 * 32];
  double red[8];
  float df[32], ef[32], e2f[32], gf[32];
  float hps[32], hred[8];          // block Householder: p per row, per-warp sums
  int skip[32];                    // per Householder step: column already reduced
};

// 1 / x in FP64 from an FP32 seed and one Newton step (relative error
// ~1e-14; |x| within FP32 range: callers pass scaled values).
static __device__ __forceinline__ double rcp64(double x) {
  const double r = (double)__frcp_rn((float)x);
  return r * fma(-x, r, 2.0);
}

// Sturm count of T - sigma I in FP32 (pivot recurrence; scaled T, |T| <= 1).
// d and e2 are register arrays (fully unrolled).
static __device__ __forceinline__ int sturm32(const float (&d)[N], const float (&e2)[N], float sigma) {
  int cnt = 0;
  float q = d[0] - sigma;
  cnt += q < 0.f;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const float qp = q == 0.f ? 1e-30f : q;
    q = (d[i] - sigma) - __fdividef(e2[i - 1], qp);
    cnt += q < 0.f;
  }
  return cnt;
}

// The same count reading d and e2 from shared memory (broadcast loads).
static __device__ __forceinline__ int sturm32s(const float* d, const float* e2, float sigma) {
  int cnt = 0;
  float q = d[0] - sigma;
  cnt += q < 0.f;
  for (int i = 1; i < N; ++i) {
    const float qp = q == 0.f ? 1e-30f : q;
    q = (d[i] - sigma) - __fdividef(e2[i - 1], qp);
    cnt += q < 0.f;
  }
  return cnt;
}

// Sturm count of T - sigma I in FP64 without divisions: sign changes of the
// characteristic-polynomial sequence p_0 = 1, p_1 = d_0 - sigma,
// p_{i+1} = (d_i - sigma) p_i - e_{i-1}^2 p_{i-1} (scaled T keeps |p_i| <= 3^27).
static __device__ __forceinline__ int sturm64(const double (&d)[N], const double (&e2)[N], double sigma) {
  double pm = 1.0, p = d[0] - sigma;
  int cnt = (p < 0.0);
  bool neg = p <= 0.0;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const double pn = fma(d[i] - sigma, p, -e2[i - 1] * pm);
    const bool nn = pn < 0.0 || (pn == 0.0 && !neg);
    cnt += (nn != neg);
    neg = nn;
    pm = p;
    p = pn;
  }
  return cnt;
}

// |y|^2 for (T + lam I) y = g in FP32 (scaled problem).
static __device__ __noinline__ float norm2_32(const float* d, const float* e, const float* g, float lam) {
  float cp[N], gp[N];
  float m = d[0] + lam;
  float r = __fdividef(1.f, m);
  cp[0] = e[0] * r;
  gp[0] = g[0] * r;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    m = (d[i] + lam) - e[i - 1] * cp[i - 1];
    r = __fdividef(1.f, m);
    cp[i] = i < N - 1 ? e[i] * r : 0.f;
    gp[i] = (g[i] - e[i - 1] * gp[i - 1]) * r;
  }
  float y = gp[N - 1], s = y * y;
#pragma unroll
  for (int i = N - 2; i >= 0; --i) {
    y = gp[i] - cp[i] * y;
    s += y * y;
  }
  return s;
}

// |y|^2 for (T + lam I) y = g in FP32 with the per-thread elimination
// factors in shared memory (cps, gps: [i][thread] layout, the thread's column).
static __device__ float norm2_32s(const float* d, const float* e, const float* g, float lam, float* cps,
                           float* gps) {
  float m = d[0] + lam;
  float r = __fdividef(1.f, m);
  float c = e[0] * r, gp = g[0] * r;
  cps[0] = c;
  gps[0] = gp;
  for (int i = 1; i < N; ++i) {
    m = (d[i] + lam) - e[i - 1] * c;
    r = __fdividef(1.f, m);
    c = i < N - 1 ? e[i] * r : 0.f;
    gp = (g[i] - e[i - 1] * gp) * r;
    cps[i * kTrThreads] = c;
    gps[i * kTrThreads] = gp;
  }
  float y = gp, sum = y * y;
  for (int i = N - 2; i >= 0; --i) {
    y = gps[i * kTrThreads] - cps[i * kTrThreads] * y;
    sum += y * y;
  }
  return sum;
}

// LDL^T of T + lam I (positive definite; scaled T) and y = (T + lam I)^{-1} rhs.
// Returns |y|^2; q = y^T (T + lam I)^{-1} y when q != nullptr; y into out.
static __device__ __noinline__ double ldl_solve(const double* d, const double* e, const double* rhs,
                                         double lam, double* out, double* q) {
  double l[N], rD[N], w[N];
  rD[0] = rcp64(d[0] + lam);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    l[i - 1] = e[i - 1] * rD[i - 1];
    rD[i] = rcp64((d[i] + lam) - l[i - 1] * e[i - 1]);
  }
  double z = rhs[0];
  w[0] = z * rD[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    z = fma(-l[i - 1], z, rhs[i]);
    w[i] = z * rD[i];
  }
  double y = w[N - 1], s = y * y;
  out[N - 1] = y;
#pragma unroll
  for (int i = N - 2; i >= 0; --i) {
    y = fma(-l[i], y, w[i]);
    out[i] = y;
    s = fma(y, y, s);
  }
  if (q) {
    double u = out[0], acc = u * u * rD[0];
#pragma unroll
    for (int i = 1; i < N; ++i) {
      u = fma(-l[i - 1], u, out[i]);
      acc = fma(u * u, rD[i], acc);
    }
    *q = acc;
  }
  return s;
}

// Applies the reflections (warp 0): Q^T x (H_0 first) or Q x (H_0 last).
static __device__ void apply_q(TrSmem& S, double* x, bool transpose, int lane) {
  for (int step = 0; step < N - 2; ++step) {
    const int k = transpose ? step : N - 3 - step;
    const double bt = S.beta[k];
    if (bt == 0.0) continue;
    const int m = N - 1 - k;
    const double vi = lane < m ? S.B[(k + 1 + lane) * N + k] : 0.0;
    const double xi = lane < m ? x[k + 1 + lane] : 0.0;
    const double s = warp_sum_d(vi * xi);
    if (lane < m) x[k + 1 + lane] = fma(-bt * s, vi, xi);
    __syncwarp();
  }
}

// Exact trust-region subproblem of one source, all in FP64 (the path for
// the hard and nearly hard cases); 128 threads (4 warps) enter, warp 0
// finishes: it returns true and holds p in S.y and the predicted gain in
// S.red[0].  g (27) and H (27 x 27) are in global memory.
static __device__ bool tr_solve_full(TrSmem& S, const double* __restrict__ g,
                              const double* __restrict__ H, double Delta) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < N * N; e += kTrThreads) {
    const int i = e / N, j = e % N;
    S.B[e] = -0.5 * (H[i * N + j] + H[j * N + i]);
  }
  if (tid < N) S.gh[tid] = g[tid];
  __syncthreads();
  // ---- Householder tridiagonalisation; v_k stored below the diagonal of column k
  for (int k = 0; k < N - 2; ++k) {
    const int m = N - 1 - k;
    if (wid == 0) {
      const double xv = lane < m ? S.B[(k + 1 + lane) * N + k] : 0.0;
      const double nrm2 = warp_sum_d(xv * xv);
      const double x0 = __shfl_sync(0xffffffffu, xv, 0);
      const bool skip = nrm2 - x0 * x0 <= 1e-300 * fmax(nrm2, 1.0) || nrm2 == 0.0;
      if (skip) {
        if (lane == 0) {
          S.beta[k] = 0.0;
          S.d[k] = S.B[k * N + k];
          S.e[k] = x0;
        }
      } else {
        // alpha = -sign(x0) |x|;  v = x - alpha e_1;  beta = 2 / v.v = 1 / (|x|^2 - x0 alpha)
        double r;
        if (nrm2 > 1e-30 && nrm2 < 1e30) {
          r = (double)rsqrtf((float)nrm2);                     // FP32 seed, then
          r = r * fma(-0.5 * nrm2 * r, r, 1.5);                // one Newton step
        } else {
          r = rsqrt(nrm2);
        }
        const double alpha = -copysign(nrm2 * r, x0);
        const double bt = rcp64(fma(-x0, alpha, nrm2));
        if (lane < m) S.B[(k + 1 + lane) * N + k] = xv - (lane == 0 ? alpha : 0.0);
        if (lane == 0) {
          S.beta[k] = bt;
          S.d[k] = S.B[k * N + k];
          S.e[k] = alpha;
        }
      }
      if (lane == 0) S.skip[k] = skip ? 1 : 0;
    }
    __syncthreads();
    if (S.skip[k]) continue;
    // p = beta A22 v: rows over lanes, columns over the four warps
    const int chunk = (m + 3) >> 2;
    const int c0 = wid * chunk, c1 = min(m, c0 + chunk);
    if (lane < m) {
      const double* row = S.B + (k + 1 + lane) * N + k + 1;
      double part = 0.0;
      for (int c = c0; c < c1; ++c) part = fma(row[c], S.B[(k + 1 + c) * N + k], part);
      S.part[wid * 32 + lane] = part;
    }
    __syncthreads();
    if (wid == 0) {
      const double bt = S.beta[k];
      const double vv = lane < m ? S.B[(k + 1 + lane) * N + k] : 0.0;
      const double pi = lane < m ? bt * (S.part[lane] + S.part[32 + lane] + S.part[64 + lane] +
                                         S.part[96 + lane]) : 0.0;
      const double K = 0.5 * bt * warp_sum_d(vv * pi);
      if (lane < m) S.w[lane] = fma(-K, vv, pi);
    }
    __syncthreads();
    // A22 -= v w^T + w v^T over the same (row, column chunk) split
    if (lane < m) {
      double* row = S.B + (k + 1 + lane) * N + k + 1;
      const double vr = S.B[(k + 1 + lane) * N + k], wr = S.w[lane];
      for (int c = c0; c < c1; ++c)
        row[c] = fma(-vr, S.w[c], fma(-wr, S.B[(k + 1 + c) * N + k], row[c]));
    }
    __syncthreads();
  }
  if (wid != 0) return false;
  if (lane == 0) {
    S.d[N - 2] = S.B[(N - 2) * N + N - 2];
    S.d[N - 1] = S.B[(N - 1) * N + N - 1];
    S.e[N - 2] = S.B[(N - 1) * N + N - 2];
    S.e[N - 1] = 0.0;
  }
  __syncwarp();
  apply_q(S, S.gh, true, lane);
  // ---- scale: |T / scale| <= 1 (Gershgorin), bookkeeping in FP32
  float rowf = 0.f, g2f = 0.f;
  if (lane < N) {
    rowf = fabsf((float)S.d[lane]) + fabsf((float)S.e[lane]) + (lane ? fabsf((float)S.e[lane - 1]) : 0.f);
    const float gf = (float)S.gh[lane];
    g2f = gf * gf;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rowf = fmaxf(rowf, __shfl_xor_sync(0xffffffffu, rowf, o));
    g2f += __shfl_xor_sync(0xffffffffu, g2f, o);
  }
  const double scale = (double)fmaxf(rowf, 1e-30f);
  const double inv = 1.0 / scale;
  const float gnorm_s = sqrtf(g2f) * (float)inv;   // |g| / scale
  if (lane < N) {
    S.ds[lane] = S.d[lane] * inv;
    S.es[lane] = S.e[lane] * inv;
    S.gs[lane] = S.gh[lane] * inv;
    S.df[lane] = (float)S.ds[lane];
    S.ef[lane] = (float)S.es[lane];
    S.e2f[lane] = S.ef[lane] * S.ef[lane];
    S.gf[lane] = (float)S.gs[lane];
  }
  __syncwarp();
  const double* d = S.ds;
  const double* e = S.es;
  const double* gs = S.gs;
  // ---- lambda_min of the scaled matrix: Gershgorin bracket (FP32)
  float af = 1.f, bf = -1.f;
  if (lane < N) {
    const float r = fabsf(S.ef[lane]) + (lane ? fabsf(S.ef[lane - 1]) : 0.f);
    af = S.df[lane] - r;
    bf = S.df[lane] + r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    af = fminf(af, __shfl_xor_sync(0xffffffffu, af, o));
    bf = fmaxf(bf, __shfl_xor_sync(0xffffffffu, bf, o));
  }
  double a = (double)af, b = (double)bf;
  {
    float rd[N], re2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      rd[i] = S.df[i];
      re2[i] = S.e2f[i];
    }
    float fa = (float)a - 1e-6f, fb = (float)b + 1e-6f;
    for (int round = 0; round < 5; ++round) {
      const float sig = fa + (fb - fa) * (float)(lane + 1) * (1.f / 32.f);
      const bool hit = lane < 31 && sturm32(rd, re2, sig) >= 1;
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      const int t = mask ? __ffs(mask) - 1 : 31;
      const float na = t == 0 ? fa : fa + (fb - fa) * (float)t * (1.f / 32.f);
      const float nb = t == 31 ? fb : fa + (fb - fa) * (float)(t + 1) * (1.f / 32.f);
      fa = na;
      fb = nb;
    }
    // FP32 counts are exact away from eigenvalues to ~1e-6 of the scale
    a = fmax(a - 1e-6, (double)fa - 1e-5);
    b = fmin(b + 1e-6, (double)fb + 1e-5);
  }
  {
    double rd[N], re2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      rd[i] = d[i];
      re2[i] = e[i] * e[i];
    }
    for (int round = 0; round < 3; ++round) {
      const double sig = a + (b - a) * (double)(lane + 1) * (1.0 / 32.0);
      const bool hit = lane < 31 && sturm64(rd, re2, sig) >= 1;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    const int t = mask ? __ffs(mask) - 1 : 31;
    const double na = t == 0 ? a : a + (b - a) * (double)t * (1.0 / 32.0);
    const double nb = t == 31 ? b : a + (b - a) * (double)(t + 1) * (1.0 / 32.0);
    a = na;
    b = nb;
    }
  }
  // a lower bound of lambda_min within ~1e-9 of it (scaled): T + l I is
  // positive definite for every l > -lmin
  const double lmin = a;
  // ---- multiplier (scaled units: l / scale); |y| is scale-invariant
  const double D2 = Delta * Delta;
  bool done = false, hard = false;
  if (lmin > 0.0) {
    const double n2 = ldl_solve(d, e, gs, 0.0, S.y, nullptr);
    done = n2 <= D2;
  }
  if (!done) {
    const double lo = fmax(0.0, -lmin);
    const double eps = 1e-12;
    double la = lo + eps;
    double lb = lo + (double)gnorm_s / Delta * (1.0 + 1e-6) + eps;
    // FP32 multisection for a starting point; in the first round lane 31
    // probes la itself (the hard-case test)
    float fa = (float)la, fb = (float)lb;
    bool low_inside = false;
    for (int round = 0; round < 6; ++round) {
      const float l = lane == 31 ? fa : fa + (fb - fa) * (float)(lane + 1) * (1.f / 32.f);
      const bool inside = (lane < 31 || round == 0) && norm2_32(S.df, S.ef, S.gf, l) <= (float)D2;
      const unsigned mask = __ballot_sync(0xffffffffu, inside);
      if (round == 0) low_inside = (mask >> 31) != 0u;
      const unsigned m2 = mask & 0x7fffffffu;
      const int t = m2 ? __ffs(m2) - 1 : 31;
      const float na = t == 0 ? fa : fa + (fb - fa) * (float)t * (1.f / 32.f);
      const float nb = t == 31 ? fb : fa + (fb - fa) * (float)(t + 1) * (1.f / 32.f);
      fa = na;
      fb = nb;
    }
    if (low_inside) {
      // possibly the hard case: decide in FP64 at the lowest admissible l
      hard = ldl_solve(d, e, gs, la, S.y, nullptr) <= D2;
    }
    if (!hard) {
      double l = fmin(fmax((double)fb, la), lb);
      for (int it = 0; it < 12; ++it) {
        double q;
        const double n2 = ldl_solve(d, e, gs, l, S.y, &q);
        const double ny = sqrt(n2);
        if (n2 <= D2) lb = l; else la = l;
        // stop on the norm, or when the bracket is down to rounding (close
        // to the pole |y| is too steep in l for the norm test)
        if (fabs(ny - Delta) <= 1e-12 * Delta || lb - la <= 4e-16 * lb) break;
        double ln = l + (ny - Delta) / Delta * n2 / q;
        if (!(ln > la && ln < lb)) ln = 0.5 * (la + lb);
        if (ln == l) break;
        l = ln;
      }
    }
  }
  __syncwarp();
  if (hard) {
    // eigenvector of lambda_min by inverse iteration, shifted just below it
    const double shift = -lmin + 1e-10;
    if (lane < N) S.w[lane] = 1.0 / sqrt((double)N);
    __syncwarp();
    for (int itn = 0; itn < 4; ++itn) {
      const double nz = ldl_solve(d, e, S.w, shift, S.z, nullptr);
      __syncwarp();
      const double r = 1.0 / sqrt(nz);
      if (lane < N) S.w[lane] = S.z[lane] * r;
      __syncwarp();
    }
    double zy = 0.0;
    for (int i = 0; i < N; ++i) zy = fma(S.w[i], S.y[i], zy);
    __syncwarp();
    if (lane < N) {
      S.y[lane] = fma(-zy, S.w[lane], S.y[lane]);
      S.z[lane] = S.w[lane];
    }
    __syncwarp();
    apply_q(S, S.z, false, lane);       // Q z, to fix the sign
    double first = 0.0;
    for (int i = 0; i < N; ++i) {
      if (fabs(S.z[i]) > 1e-14) {
        first = S.z[i];
        break;
      }
    }
    double ny2 = 0.0;
    for (int i = 0; i < N; ++i) ny2 = fma(S.y[i], S.y[i], ny2);
    const double tau = copysign(sqrt(fmax(D2 - ny2, 0.0)), first);
    __syncwarp();
    if (lane < N) S.y[lane] = fma(tau, S.w[lane], S.y[lane]);
    __syncwarp();
  }
  // predicted gain: y.Q^T g - y.T.y / 2 (unscaled T), one row per lane
  {
    double term = 0.0;
    if (lane < N) {
      const double yi = S.y[lane];
      double ty = S.d[lane] * yi;
      if (lane > 0) ty = fma(S.e[lane - 1], S.y[lane - 1], ty);
      if (lane < N - 1) ty = fma(S.e[lane], S.y[lane + 1], ty);
      term = yi * fma(-0.5, ty, S.gh[lane]);
    }
    term = warp_sum_d(term);
    if (lane == 0) S.red[0] = term;
  }
  __syncwarp();
  apply_q(S, S.y, false, lane);
  return true;
}

// ---- mixed-precision path ---------------------------------------------------
//
// FP32 finds where the answer is, FP64 computes it: the FP32 Householder
// reduction of B, Sturm multisection and secular-equation multisection give
// lambda_min and the multiplier to ~1e-6 of the matrix scale; then the
// safeguarded Newton iteration of Nocedal & Wright (Algorithm 4.3, one
// LDL^T factorisation of the full B + l I per step, all in FP64) converges
// from there in one to three steps.  Near the pole (the hard case or close
// to it) and whenever FP64 contradicts FP32, the full FP64 path above runs.

// 1/x in FP64 for any positive finite x (FP32 seed on a power-of-two
// rescaled value, two Newton steps).
static __device__ __forceinline__ double rcp64_any(double x) {
  int ex;
  const double m = frexp(x, &ex);                  // x = m 2^ex, m in [0.5, 1)
  double r = (double)__frcp_rn((float)m);
  r = r * fma(-m, r, 2.0);
  r = r * fma(-m, r, 2.0);
  return ldexp(r, -ex);
}

static __device__ __forceinline__ double B_diag0(const TrSmem& S, double lam) { return S.B[0] + lam; }

// 1/d in FP64 from an FP32 seed and one Newton step (relative error
// ~1e-14) when d is inside the FP32 range; 0 when d is not a positive
// finite pivot.
static __device__ __forceinline__ double pivot_rcp(double d) {
  if (!(d > 0.0 && d < 1e300)) return 0.0;
  if (d > 1e-30 && d < 1e30) {
    const double r = (double)__fdividef(1.f, (float)d);   // ~1e-7 seed
    return fma(r, fma(-d, r, 1.0), r);                     // one Newton step: ~1e-14
  }
  return rcp64_any(d);
}

// LDL^T of B + lam I in FP64 with all 128 threads, right-looking, one
// barrier per column: the m(m+1)/2 entries of the trailing triangle are
// spread evenly over the threads, each updated with the column's inverse
// pivot applied on the fly; thread 0, which updates the next diagonal entry
// first, takes its reciprocal right away.  The columns of L are scaled at
// the end.  Returns false (the same on every thread) when a pivot is not
// positive.  On success S.ws.f.L holds the unit lower factor (strictly
// lower part) and S.Dinv the inverse pivots.  S.ws.f.W is the working copy.
static __device__ bool ldl_factor(TrSmem& S, double lam) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kTri; e += kTrThreads) {
    const short2 t = S.tri[e];
    S.ws.f.W[t.x * N + t.y] = S.B[t.x * N + t.y] + (t.x == t.y ? lam : 0.0);
  }
  if (tid == 0) S.Dinv[0] = pivot_rcp(B_diag0(S, lam));
  if (__syncthreads_or(tid == 0 && S.Dinv[0] == 0.0)) return false;
  for (int j = 0; j < N - 1; ++j) {
    const int m = N - 1 - j;
    const int cnt = m * (m + 1) / 2;
    const double dinv = S.Dinv[j];
    int bad = 0;
    for (int e = tid; e < cnt; e += kTrThreads) {
      const short2 t = S.tri[e];                  // (row, col) in the trailing block
      const int i = j + 1 + t.x, k = j + 1 + t.y;
      const double w = fma(-(S.ws.f.W[i * N + j] * dinv), S.ws.f.W[k * N + j], S.ws.f.W[i * N + k]);
      S.ws.f.W[i * N + k] = w;
      if (e == 0) {                               // the next pivot
        const double r = pivot_rcp(w);
        S.Dinv[j + 1] = r;
        bad = r == 0.0;
      }
    }
    if (__syncthreads_or(bad)) return false;
  }
  for (int e = tid; e < kTri; e += kTrThreads) {
    const short2 t = S.tri[e];
    if (t.x > t.y) S.ws.f.L[t.x * N + t.y] = S.ws.f.W[t.x * N + t.y] * S.Dinv[t.y];
  }
  __syncthreads();
  return true;
}

// Warp 0: p = (L D L^T)^{-1} rhs into out; returns |p|^2, and in *q2 (when
// non-null) p^T (L D L^T)^{-1} p.  Rows live on lanes; each elimination step
// broadcasts one solved entry.
static __device__ double ldl_solve_full(TrSmem& S, const double* rhs, double* out, int lane,
                                 double* q2) {
  double b = lane < N ? rhs[lane] : 0.0;
  for (int k = 0; k < N - 1; ++k) {
    const double wk = __shfl_sync(0xffffffffu, b, k);
    if (lane > k && lane < N) b = fma(-S.ws.f.L[lane * N + k], wk, b);
  }
  double z = lane < N ? b * S.Dinv[lane] : 0.0;
  for (int k = N - 1; k > 0; --k) {
    const double pk = __shfl_sync(0xffffffffu, z, k);
    if (lane < k) z = fma(-S.ws.f.L[k * N + lane], pk, z);
  }
  if (lane < N) out[lane] = z;
  const double n2 = warp_sum_d(z * z);
  if (q2) {
    double u = z;
    for (int k = 0; k < N - 1; ++k) {
      const double uk = __shfl_sync(0xffffffffu, u, k);
      if (lane > k && lane < N) u = fma(-S.ws.f.L[lane * N + k], uk, u);
    }
    *q2 = warp_sum_d(lane < N ? u * u * S.Dinv[lane] : 0.0);
    if (lane < N) S.z[lane] = u;        // u = L^{-1} p, for first_order()
  }
  __syncwarp();
  return n2;
}

// Warp 0: p(l + dl) = p(l) - dl (B + l I)^{-1} p(l) to first order, with
// (B + l I)^{-1} p = L^{-T} D^{-1} u and u = L^{-1} p kept by ldl_solve_full.
static __device__ void first_order(TrSmem& S, int lane, double dl) {
  double z = lane < N ? S.z[lane] * S.Dinv[lane] : 0.0;
  for (int k = N - 1; k > 0; --k) {
    const double qk = __shfl_sync(0xffffffffu, z, k);
    if (lane < k) z = fma(-S.ws.f.L[k * N + lane], qk, z);
  }
  if (lane < N) S.p[lane] = fma(-dl, z, S.p[lane]);
  __syncwarp();
}

// Warp 0: x = L^{-T} z (rows on lanes).
static __device__ __forceinline__ double back_sweep(const TrSmem& S, double z, int lane) {
  for (int k = N - 1; k > 0; --k) {
    const double xk = __shfl_sync(0xffffffffu, z, k);
    if (lane < k) z = fma(-S.ws.f.L[k * N + lane], xk, z);
  }
  return z;
}

// Warp 0: x = (L D L^T)^{-1} b.
static __device__ __forceinline__ double full_solve(const TrSmem& S, double b, int lane) {
  for (int k = 0; k < N - 1; ++k) {
    const double bk = __shfl_sync(0xffffffffu, b, k);
    if (lane > k && lane < N) b = fma(-S.ws.f.L[lane * N + k], bk, b);
  }
  return back_sweep(S, lane < N ? b * S.Dinv[lane] : 0.0, lane);
}

// Warp 0: the step at the multiplier l0 + d with |p(l0 + d)| = Delta, from
// the factorisation at l0 alone.  With A = B + l0 I and w_k = A^{-k} p(l0),
// p(l0 + d) = sum_k (-d)^k w_k (a Neumann series; four terms leave a
// relative error of about (d / gap)^4, gap the distance of l0 from the
// pole) and A(d)^{-1} p(l0 + d) = sum_n (n + 1) (-d)^n w_{n+1}; Newton's
// iteration on 1/|p| - 1/Delta (Nocedal & Wright, Algorithm 4.3) then runs
// on the scalars of the Gram matrix w_i . w_j.  On entry S.p = p(l0) and
// S.z = L^{-1} p(l0) (from ldl_solve_full); d0 is the first Newton step.
// On exit S.p is the step.
static __device__ void series_finish(TrSmem& S, int lane, double d0, double Delta) {
  constexpr int K = 3;
  double w[K + 1];
  w[0] = lane < N ? S.p[lane] : 0.0;
  w[1] = back_sweep(S, lane < N ? S.z[lane] * S.Dinv[lane] : 0.0, lane);
#pragma unroll
  for (int k = 2; k <= K; ++k) w[k] = full_solve(S, w[k - 1], lane);
  double G[K + 1][K + 1];
#pragma unroll
  for (int i = 0; i <= K; ++i)
#pragma unroll
    for (int j = i; j <= K; ++j) G[i][j] = G[j][i] = warp_sum_d(w[i] * w[j]);
  double d = d0;
  double c[K + 1];
  for (int it = 0; it < 8; ++it) {
    c[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= K; ++k) c[k] = -d * c[k - 1];
    double n2 = 0.0, q = 0.0;
#pragma unroll
    for (int i = 0; i <= K; ++i) {
#pragma unroll
      for (int j = 0; j <= K; ++j) n2 = fma(c[i] * c[j], G[i][j], n2);
#pragma unroll
      for (int n = 0; n < K; ++n) q = fma(c[i] * (double)(n + 1) * c[n], G[i][n + 1], q);
    }
    const double step = (sqrt(n2) - Delta) / Delta * n2 / q;
    d += step;
    if (!(fabs(step) > 1e-15 * fabs(d))) break;
  }
  c[0] = 1.0;
#pragma unroll
  for (int k = 1; k <= K; ++k) c[k] = -d * c[k - 1];
  double x = 0.0;
#pragma unroll
  for (int k = K; k >= 0; --k) x = fma(c[k], w[k], x);
  if (lane < N) S.p[lane] = x;
  __syncwarp();
}

// Householder reduction of B (FP32, in S.ws.f.Bf) to tridiagonal form by all
// four warps: thread t owns row t / 4 of the trailing block and, in it, the
// columns c = t (mod 4); two block barriers per reflection.  Every warp
// reduces the pivot column itself (rows on lanes, the same shuffle tree in
// each), so all threads take the same branch.  The reflections are applied
// to g as they are made.  d, e into S.dfr, S.efr; Q^T g into S.gfr.
static __device__ void householder_blk(TrSmem& S) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int i = tid >> 2, sub = tid & 3;
  float* Bf = S.ws.f.Bf;
  float gi = i < N ? S.gfr[i] : 0.f;
  for (int k = 0; k < N - 2; ++k) {
    const float xl = (lane > k && lane < N) ? Bf[lane * N + k] : 0.f;
    float nrm2 = xl * xl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
    const float x0 = Bf[(k + 1) * N + k];
    if (tid == 0) S.dfr[k] = Bf[k * N + k];
    if (!(nrm2 - x0 * x0 > 1e-30f * fmaxf(nrm2, 1e-30f))) {
      if (tid == 0) S.efr[k] = x0;
      continue;
    }
    const float alpha = -copysignf(sqrtf(nrm2), x0);
    const float bt = __fdividef(1.f, fmaf(-x0, alpha, nrm2));
    if (tid == 0) S.efr[k] = alpha;
    const bool row = i > k && i < N;
    // reflector v_c = B[c][k] - alpha [c == k + 1], c > k (column k is not
    // written during this reflection)
    auto vof = [&](int c) { return Bf[c * N + k] - (c == k + 1 ? alpha : 0.f); };
    const float vi = row ? vof(i) : 0.f;
    const int c0 = k + 1 + ((sub - (k + 1)) & 3);   // first c > k with c = sub (mod 4)
    // p = bt B v over the trailing block: this thread's columns, then the row
    float pp = 0.f;
    if (row) {
      const float* r = Bf + i * N;
      for (int c = c0; c < N; c += 4) pp = fmaf(r[c], vof(c), pp);
    }
    pp += __shfl_xor_sync(0xffffffffu, pp, 1);
    pp += __shfl_xor_sync(0xffffffffu, pp, 2);
    const float p = row ? bt * pp : 0.f;
    // K = v.p and v.g over the rows (row values on sub 0), then the warps
    float K = sub == 0 ? vi * p : 0.f, vg = sub == 0 ? vi * gi : 0.f;
#pragma unroll
    for (int o = 16; o >= 4; o >>= 1) {
      K += __shfl_xor_sync(0xffffffffu, K, o);
      vg += __shfl_xor_sync(0xffffffffu, vg, o);
    }
    if (lane == 0) {
      S.hred[wid] = K;
      S.hred[4 + wid] = vg;
    }
    if (sub == 0 && row) S.hps[i] = p;
    __syncthreads();
    K = (S.hred[0] + S.hred[1]) + (S.hred[2] + S.hred[3]);
    vg = (S.hred[4] + S.hred[5]) + (S.hred[6] + S.hred[7]);
    gi = fmaf(-bt * vg, vi, gi);                  // g -= bt v (v.g)
    // B -= v w^T + w v^T with w = p - (bt K / 2) v
    const float hk = -0.5f * bt * K;
    if (row) {
      const float wi = fmaf(hk, vi, p);
      float* r = Bf + i * N;
      for (int c = c0; c < N; c += 4) {
        const float vc = vof(c);
        const float wc = fmaf(hk, vc, S.hps[c]);
        r[c] = fmaf(-vi, wc, fmaf(-wi, vc, r[c]));
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    S.dfr[N - 2] = Bf[(N - 2) * N + N - 2];
    S.dfr[N - 1] = Bf[(N - 1) * N + N - 1];
    S.efr[N - 2] = Bf[(N - 1) * N + N - 2];
    S.efr[N - 1] = 0.f;
  }
  if (sub == 0 && i < N) S.gfr[i] = gi;
  __syncthreads();
}

// The first of the block's 127 probes (threads 0..126) that is set, or 127
// when none is; one barrier (the ballot slots alternate between rounds).
static __device__ __forceinline__ int first_hit(TrSmem& S, bool hit, int round) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, hit && tid < kTrThreads - 1);
  if (lane == 0) S.hmask[round & 1][wid] = m;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < kTrThreads / 32; ++w) {
    const unsigned mw = S.hmask[round & 1][w];
    if (mw) return w * 32 + __ffs(mw) - 1;
  }
  return kTrThreads - 1;
}

// All four warps: from the FP32 tridiagonal form, lambda_min and the
// multiplier to FP32 accuracy by multisection, 127 probes a round (7 bits);
// sets S.mode, S.lam, S.lo, S.hi (unscaled).
static __device__ void locate32(TrSmem& S, double Delta) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr float kStep = 1.f / (float)kTrThreads;
  if (wid == 0) {
    float rowf = 0.f, g2f = 0.f;
    if (lane < N) {
      rowf = fabsf(S.dfr[lane]) + fabsf(S.efr[lane]) + (lane ? fabsf(S.efr[lane - 1]) : 0.f);
      g2f = S.gfr[lane] * S.gfr[lane];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rowf = fmaxf(rowf, __shfl_xor_sync(0xffffffffu, rowf, o));
      g2f += __shfl_xor_sync(0xffffffffu, g2f, o);
    }
    const float scale = fmaxf(rowf, 1e-30f);
    const float inv = 1.f / scale;
    if (lane < N) {
      S.df[lane] = S.dfr[lane] * inv;
      S.ef[lane] = S.efr[lane] * inv;
      S.e2f[lane] = S.ef[lane] * S.ef[lane];
      S.gf[lane] = S.gfr[lane] * inv;
    }
    if (lane == 0) {
      S.loc[0] = scale;
      S.loc[1] = g2f;
    }
  }
  __syncthreads();
  const float scale = S.loc[0], g2f = S.loc[1];
  const float inv = 1.f / scale;
  float* cps = S.ws.s.cps + tid;
  float* gps = S.ws.s.gps + tid;
  const float gnorm_s = sqrtf(g2f) * inv;
  const float D2 = (float)(Delta * Delta);
  int round = 0;
  float fa = -1.f - 1e-6f, fb = 1.f + 1e-6f;
  for (int r = 0; r < 4; ++r, ++round) {
    const float sig = fa + (fb - fa) * (float)(tid + 1) * kStep;
    const int t = first_hit(S, sturm32s(S.df, S.e2f, sig) >= 1, round);
    const float na = t == 0 ? fa : fa + (fb - fa) * (float)t * kStep;
    const float nb = t == kTrThreads - 1 ? fb : fa + (fb - fa) * (float)(t + 1) * kStep;
    fa = na;
    fb = nb;
  }
  // lambda_min (scaled) lies in [fa, fb] up to FP32 rounding of the counts
  const float lmin = fa;
  if (tid == 0) S.loc[2] = lmin > 0.f ? norm2_32s(S.df, S.ef, S.gf, 0.f, cps, gps) : 3.4e38f;
  __syncthreads();
  const float n0 = S.loc[2];
  // mode 0: try l = 0 first (interior Newton step); mode 1: the boundary
  // root from the bracket [la, lb]; mode 2: the all-FP64 path
  int mode = 1;
  float la = 0.f, lb = 0.f;
  bool bracket = false;
  if (!(g2f > 0.f)) {
    mode = 2;
  } else if (lmin > 1e-4f && n0 <= D2 * 0.999f) {
    mode = 0;                       // clearly interior
  } else {
    // FP32 cannot tell an interior step of an ill-conditioned B from a
    // boundary one: try l = 0 in FP64 when it may be interior, with the
    // boundary bracket as the alternative
    if (lmin > 0.f && n0 <= D2 * 1.01f) mode = 0;
    bracket = true;
    const float lo = fmaxf(0.f, -lmin);
    la = lo;
    lb = lo + gnorm_s / (float)Delta * 1.01f + 1e-6f;
    for (int r = 0; r < 4; ++r, ++round) {
      const float l = la + (lb - la) * (float)(tid + 1) * kStep;
      const bool inside = tid < kTrThreads - 1 && norm2_32s(S.df, S.ef, S.gf, l, cps, gps) <= D2;
      const int t = first_hit(S, inside, round);
      const float na = t == 0 ? la : la + (lb - la) * (float)t * kStep;
      const float nb = t == kTrThreads - 1 ? lb : la + (lb - la) * (float)(t + 1) * kStep;
      la = na;
      lb = nb;
    }
    // near the pole (nearly hard case) the FP32 bracket is still a good
    // start; the FP64 iteration below resolves it, and a true hard case
    // (no root above the pole) ends in the all-FP64 path
  }
  if (tid == 0) {
    S.mode = mode;
    const double sc = (double)scale;
    S.lmin_lo = (double)scale * (double)fa;
    S.positive = lmin > 0.f ? 1 : 0;
    // the FP32 root estimate starts the FP64 iteration (0: no estimate)
    S.lam = bracket ? sc * 0.5 * ((double)la + (double)lb) : 0.0;
    S.lam_b = S.lam;
    S.tried0 = 0;
    S.bisects = 0;
    if (mode == 0) S.lam = 0.0;
    S.lo = -1.0;                      // FP64 bounds: none yet
    S.hi = -1.0;
  }
  __syncthreads();
}

// Exact trust-region subproblem of one source; 128 threads (4 warps) enter,
// warp 0 finishes: it returns true and holds p in S.y and the predicted
// gain in S.red[0].  g (27) and H (27 x 27) are in global memory.
static __device__ bool tr_solve(TrSmem& S, const double* __restrict__ g, const double* __restrict__ H,
                         double Delta) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < N * N; e += kTrThreads) {
    const int i = e / N, j = e % N;
    const double b = -0.5 * (H[i * N + j] + H[j * N + i]);
    S.B[e] = b;
    S.ws.f.Bf[e] = (float)b;
  }
  for (int e = tid; e < kTri; e += kTrThreads) {
    // row i of lower entry e: i (i + 1) / 2 <= e < (i + 1) (i + 2) / 2
    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if (i * (i + 1) / 2 > e) --i;
    if ((i + 1) * (i + 2) / 2 <= e) ++i;
    S.tri[e] = make_short2((short)i, (short)(e - i * (i + 1) / 2));
  }
  if (tid < N) {
    S.gh[tid] = g[tid];
    S.gfr[tid] = (float)g[tid];
  }
  __syncthreads();
  householder_blk(S);
  locate32(S, Delta);
  const double D2 = Delta * Delta;
  bool done = false;
  if (S.mode != 2) {
    // safeguarded Newton on 1/|p(l)| - 1/Delta from the FP32 estimate;
    // S.mode / S.lam / S.lo / S.hi are read after a barrier and written by
    // warp 0 lane 0 only between barriers
    for (int it = 0; it < 8 && !done; ++it) {
      const double lam = S.lam;
      const bool ok = ldl_factor(S, lam);
      if (wid == 0) {
        // Bounds known in FP64 (the FP32 estimates only pick the start):
        // lo, a multiplier too small (indefinite, or |p| > Delta), < 0 for
        // none; hi, one large enough (|p| <= Delta), < 0 for none
        double lo = S.lo, hi = S.hi, next = lam;
        int mode = S.mode, tried0 = S.tried0 | (lam == 0.0), bisects = S.bisects;
        bool fin = false;
        if (!ok) {
          lo = fmax(lo, lam);
          if (mode == 0 && S.lam_b > lo && (hi < 0.0 || S.lam_b < hi)) {
            next = S.lam_b;
          } else if (hi >= 0.0) {
            next = 0.5 * (lo + hi);
            ++bisects;
          } else {
            next = 2.0 * lam + 1e-12 * (1.0 + fabs(S.lmin_lo));
          }
          mode = 1;
        } else {
          double q2;
          const double n2 = ldl_solve_full(S, S.gh, S.p, lane, &q2);
          const double np = sqrt(n2);
          if (lam == 0.0 && n2 <= D2) {
            fin = true;                 // interior Newton step
          } else if (fabs(np - Delta) <= 1e-12 * Delta) {
            fin = true;
          } else {
            if (n2 > D2) lo = fmax(lo, lam);
            else hi = hi < 0.0 ? lam : fmin(hi, lam);
            if (mode == 0 && S.lam_b > lo && (hi < 0.0 || S.lam_b < hi)) {
              next = S.lam_b;           // l = 0 was not interior: start on the boundary
            } else {
              const double dl = (np - Delta) / Delta * n2 / q2;
              double ln = lam + dl;
              // a correction far below the distance to the pole: the
              // first-order step leaves a relative error of about
              // (dl / gap)^2 <= 1e-10 in p
              const double gap = lam + S.lmin_lo;
              const bool inside = ln > fmax(lo, 0.0) && (hi < 0.0 || ln < hi);
              if (inside && gap > 0.0 && fabs(dl) <= 1e-5 * gap) {
                first_order(S, lane, dl);
                fin = true;
              } else if (inside && gap > 0.0 && fabs(dl) <= 1e-3 * gap) {
                // still close: finish on this factorisation (a series in
                // the multiplier) instead of factorising again
                series_finish(S, lane, dl, Delta);
                fin = true;
              } else if (inside) {
                next = ln;
              } else if (n2 <= D2 && !tried0 && lo < 0.0) {
                next = 0.0;             // the root may be at 0: an interior step
              } else if (hi >= 0.0) {
                next = 0.5 * (fmax(lo, 0.0) + hi);
                ++bisects;
              } else {
                next = 2.0 * lam + 1e-12 * (1.0 + fabs(S.lmin_lo));
              }
              if (next == lam) fin = true;
            }
          }
          mode = 1;
        }
        // Bisecting again and again means the root hugs the pole (a nearly
        // hard case, the multiplier within ~1e-10 of -lambda_min): the
        // eigen-based all-FP64 path resolves it.
        if (!fin && bisects >= 3) mode = 2;
        if (lane == 0) {
          S.lo = lo;
          S.hi = hi;
          S.lam = next;
          S.tried0 = tried0;
          S.bisects = bisects;
          S.mode = fin ? 3 : mode;
        }
      }
      __syncthreads();
      if (S.mode == 3) done = true;
      if (S.mode == 2) break;
    }
  }
  if (!done) {
    __syncthreads();
    return tr_solve_full(S, g, H, Delta);
  }
  if (wid != 0) return false;
  // predicted gain g.p - p.B.p / 2 in FP64 on the full matrix, one row per lane
  double term = 0.0;
  if (lane < N) {
    double bp = 0.0;
    for (int k = 0; k < N; ++k) bp = fma(S.B[lane * N + k], S.p[k], bp);
    term = S.p[lane] * fma(-0.5, bp, S.gh[lane]);
  }
  term = warp_sum_d(term);
  if (lane < N) S.y[lane] = S.p[lane];
  if (lane == 0) S.red[0] = term;
  __syncwarp();
  return true;
}

// The step of slot j of the plan from its gradient and Hessian (v.grad,
// v.hess), by the whole block: non-finite derivatives fail the source, a
// predicted gain below kFtol (1 + |L|) or a radius below kDeltaMin
// converges it (both leave the active set); otherwise the step, its
// predicted gain and theta_trial are written.  Returns true, in every
// thread, when a trial point was formed.
static __device__ __forceinline__ bool tr_step_source(const PlanView& v, TrSmem& S, int j,
                                               const double* delta, int32_t* status) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (!v.active[j]) return false;
  const int src = v.src_ids[j];
  const double Dl = delta[src];
  const double* g = v.grad + (size_t)j * N;
  const double* H = v.hess + (size_t)j * N * N;
  bool finite = true;
  for (int e = tid; e < N * N; e += kTrThreads) finite &= isfinite(H[e]);
  if (tid < N) finite &= isfinite(g[tid]);
  finite = __syncthreads_and(finite) && isfinite(v.elbo_rel[j]);
  if (!finite) {
    if (tid == 0) {
      status[src] = CELESTE_ST_FAILED;
      v.active[j] = 0;
    }
    return false;
  }
  int formed = 0;
  if (tr_solve(S, g, H, Dl)) {
    // warp 0
    double* p = v.step + (size_t)j * N;
    if (lane < N) p[lane] = S.y[lane];
    const double pred = S.red[0];
    if (lane == 0) v.pred[j] = pred;
    if (pred <= kFtol * (1.0 + fabs(v.elbo_rel[j])) || Dl < kDeltaMin) {
      if (lane == 0) {
        status[src] = CELESTE_ST_CONVERGED;
        v.active[j] = 0;
      }
    } else {
      if (lane < N) v.theta_trial[(size_t)j * N + lane] = v.theta[(size_t)src * N + lane] + S.y[lane];
      formed = 1;
    }
  }
  return __syncthreads_or(formed) != 0;
}

}  // namespace celeste
