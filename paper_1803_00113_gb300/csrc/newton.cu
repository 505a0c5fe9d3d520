// FP64 trust-region Newton step (Sec. 4.3): maximise g.p + p.H.p / 2 over
// the ball |p| <= Delta exactly, then accept or reject the trial point.
//
// GB300 issues a warp-wide FP64 instruction about every 64 cycles per SM
// sub-partition, so the cost of this kernel is its count of FP64 warp
// instructions, and a source gets four warps (one per sub-partition) for
// the part that parallelises:
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
#include <math.h>

#include "internal.cuh"

namespace celeste {

constexpr int N = kTheta;
constexpr int kTrThreads = 128;
constexpr double kEta = 0.1;
constexpr double kDeltaMax = 100.0;
constexpr double kFtol = 1e-9;
constexpr double kDeltaMin = 1e-8;

struct TrSmem {
  double B[N * N];
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
  int skip[32];                    // per Householder step: column already reduced
};

// 1 / x in FP64 from an FP32 seed and one Newton step (relative error
// ~1e-14; |x| within FP32 range: callers pass scaled values).
__device__ __forceinline__ double rcp64(double x) {
  const double r = (double)__frcp_rn((float)x);
  return r * fma(-x, r, 2.0);
}

// Sturm count of T - sigma I in FP32 (pivot recurrence; scaled T, |T| <= 1).
// d and e2 are register arrays (fully unrolled).
__device__ __forceinline__ int sturm32(const float (&d)[N], const float (&e2)[N], float sigma) {
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

// Sturm count of T - sigma I in FP64 without divisions: sign changes of the
// characteristic-polynomial sequence p_0 = 1, p_1 = d_0 - sigma,
// p_{i+1} = (d_i - sigma) p_i - e_{i-1}^2 p_{i-1} (scaled T keeps |p_i| <= 3^27).
__device__ __forceinline__ int sturm64(const double (&d)[N], const double (&e2)[N], double sigma) {
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
__device__ __noinline__ float norm2_32(const float* d, const float* e, const float* g, float lam) {
  float cp[N], gp[N];
  float m = d[0] + lam;
  float r = __frcp_rn(m);
  cp[0] = e[0] * r;
  gp[0] = g[0] * r;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    m = (d[i] + lam) - e[i - 1] * cp[i - 1];
    r = __frcp_rn(m);
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

// LDL^T of T + lam I (positive definite; scaled T) and y = (T + lam I)^{-1} rhs.
// Returns |y|^2; q = y^T (T + lam I)^{-1} y when q != nullptr; y into out.
__device__ __noinline__ double ldl_solve(const double* d, const double* e, const double* rhs,
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
__device__ void apply_q(TrSmem& S, double* x, bool transpose, int lane) {
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

// Exact trust-region subproblem of one source; 128 threads (4 warps) enter,
// warp 0 finishes: it returns true and holds p in S.y and the predicted
// gain in S.red[0].  g (27) and H (27 x 27) are in global memory.
__device__ bool tr_solve(TrSmem& S, const double* __restrict__ g, const double* __restrict__ H,
                         double Delta) {
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

__global__ void __launch_bounds__(kTrThreads, 4) tr_subproblem_kernel(int n, const double* g,
                                                                  const double* H,
                                                                  const double* delta, double* p,
                                                                  double* pred) {
  extern __shared__ double smd[];
  TrSmem& S = *reinterpret_cast<TrSmem*>(smd);
  const int j = blockIdx.x;
  if (j >= n) return;
  if (!tr_solve(S, g + (size_t)j * N, H + (size_t)j * N * N, delta[j])) return;
  const int lane = threadIdx.x & 31;
  if (lane < N) p[(size_t)j * N + lane] = S.y[lane];
  if (lane == 0) pred[j] = S.red[0];
}

// Step of every active slot: converged sources leave the active set.
__global__ void __launch_bounds__(kTrThreads, 4) tr_step_kernel(PlanView v, const double* delta,
                                                            int32_t* status) {
  extern __shared__ double smd[];
  TrSmem& S = *reinterpret_cast<TrSmem*>(smd);
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (!v.active[j]) return;
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
    return;
  }
  if (!tr_solve(S, g, H, Dl)) return;
  double* p = v.step + (size_t)j * N;
  if (lane < N) p[lane] = S.y[lane];
  const double pred = S.red[0];
  if (lane == 0) v.pred[j] = pred;
  if (pred <= kFtol * (1.0 + fabs(v.elbo_rel[j])) || Dl < kDeltaMin) {
    if (lane == 0) {
      status[src] = CELESTE_ST_CONVERGED;
      v.active[j] = 0;
    }
    return;
  }
  if (lane < N) v.theta_trial[(size_t)j * N + lane] = v.theta[(size_t)src * N + lane] + S.y[lane];
}

// Accept or reject the trial points; update radius and status.
__global__ void tr_accept_kernel(PlanView v, const double* __restrict__ rel_trial, double* delta,
                                 int32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.n || !v.active[j]) return;
  const int src = v.src_ids[j];
  const double* p = v.step + (size_t)j * N;
  double pn = 0.0;
  for (int i = 0; i < N; ++i) pn = fma(p[i], p[i], pn);
  pn = sqrt(pn);
  const double Dl = delta[src];
  const double actual = rel_trial[j] - v.elbo_rel[j];
  const double rho = actual / v.pred[j];
  double nd = Dl;
  if (!(rho >= 0.25)) nd = 0.25 * pn;
  else if (rho > 0.75 && pn >= 0.99 * Dl) nd = fmin(2.0 * Dl, kDeltaMax);
  delta[src] = nd;
  if (rho > kEta && isfinite(rel_trial[j])) {
    for (int i = 0; i < N; ++i) v.theta[(size_t)src * N + i] = v.theta_trial[(size_t)j * N + i];
    status[src] = CELESTE_ST_ACCEPTED;
  } else {
    status[src] = CELESTE_ST_REJECTED;
  }
}

__global__ void mark_active_kernel(PlanView v, const int32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.n) return;
  const int st = status[v.src_ids[j]];
  v.active[j] =
      (st == CELESTE_ST_CONVERGED || st == CELESTE_ST_FAILED || st == CELESTE_ST_MAXITER) ? 0 : 1;
}

static bool g_attr_set = false;
static void set_attrs() {
  if (g_attr_set) return;
  cudaFuncSetAttribute(tr_subproblem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(TrSmem));
  cudaFuncSetAttribute(tr_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(TrSmem));
  g_attr_set = true;
}

cudaError_t launch_tr_subproblem(const Launch& L, int n, const double* g, const double* H,
                                 const double* delta, double* p, double* pred) {
  if (n <= 0) return cudaSuccess;
  set_attrs();
  tr_subproblem_kernel<<<n, kTrThreads, sizeof(TrSmem), L.stream>>>(n, g, H, delta, p, pred);
  return cudaGetLastError();
}

cudaError_t launch_tr_step(const Launch& L, const PlanView& v, const double* delta,
                           int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  set_attrs();
  tr_step_kernel<<<v.n, kTrThreads, sizeof(TrSmem), L.stream>>>(v, delta, status);
  return cudaGetLastError();
}

cudaError_t launch_tr_accept(const Launch& L, const PlanView& v, const double* rel_trial,
                             double* delta, int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  tr_accept_kernel<<<(v.n + 127) / 128, 128, 0, L.stream>>>(v, rel_trial, delta, status);
  return cudaGetLastError();
}

cudaError_t launch_mark_active(const Launch& L, const PlanView& v, const int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  mark_active_kernel<<<(v.n + 127) / 128, 128, 0, L.stream>>>(v, status);
  return cudaGetLastError();
}

}  // namespace celeste
