// FP64 trust-region Newton step (Sec. 4.3): maximise g.p + p.H.p / 2 over
// the ball |p| <= Delta exactly, then accept or reject the trial point.
//
// GB300 has little FP64 throughput, so the 27 x 27 subproblem avoids a full
// eigendecomposition: B = -H is reduced to tridiagonal form T = Q^T B Q by
// Householder reflections (one warp, lanes over rows), and everything after
// that is O(n) per evaluation on T:
//   * lambda_min(T) by multisection on Sturm counts (31 probes per round);
//   * the multiplier l solving |(T + l I)^{-1} Q^T g| = Delta by multisection
//     on the (monotone) step norm, each lane running one tridiagonal solve;
//   * the hard case (g orthogonal to the eigenvector of lambda_min) adds
//     that eigenvector, found by inverse iteration, to reach the boundary;
//     its sign makes the first nonzero entry of Q z positive;
//   * p = Q y and the predicted gain g.p + p.H.p/2 = y.Q^T g - y.T.y/2.
// Trust-region constants follow the textbook loop (Nocedal & Wright,
// Algorithm 4.1): accept when rho > 0.1, shrink to |p|/4 when rho < 1/4,
// double (up to 100) when rho > 3/4 and the step reached the boundary.
#include <math.h>

#include "internal.cuh"

namespace celeste {

constexpr int N = kTheta;
constexpr double kEta = 0.1;
constexpr double kDeltaMax = 100.0;
constexpr double kFtol = 1e-9;
constexpr double kDeltaMin = 1e-8;

struct TrSmem {
  double B[N * N];
  double beta[N];
  double gh[32];
  double d[32];
  double e[32];
  double y[32];
  double z[32];
  double w[32];
  double red[32];
  float df[32], ef[32], e2f[32], gf[32];   // T and Q^T g scaled by 1 / scale, FP32
};

// Sturm count of T - sigma I in FP32 (pivot recurrence; scaled T, |T| <= 1).
__device__ __forceinline__ int sturm32(const float* d, const float* e2, float sigma) {
  int cnt = 0;
  float q = d[0] - sigma;
  cnt += q < 0.f;
#pragma unroll 1
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
__device__ __forceinline__ int sturm64(const double* d, const double* e, double sigma) {
  double pm = 1.0, p = d[0] - sigma;
  int cnt = (p < 0.0);
  bool neg = p < 0.0 || (p == 0.0);
#pragma unroll 1
  for (int i = 1; i < N; ++i) {
    const double pn = (d[i] - sigma) * p - e[i - 1] * e[i - 1] * pm;
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

// LDL^T of T + lam I (positive definite) and y = (T + lam I)^{-1} rhs.
// Returns |y|^2; q = y^T (T + lam I)^{-1} y (for the Newton step on the
// secular equation); writes y when out != nullptr.  One division per row.
__device__ __noinline__ double ldl_solve(const double* d, const double* e, const double* rhs, double lam,
                            double* out, double* q) {
  double l[N], rD[N], w[N];
  double D = d[0] + lam;
  rD[0] = 1.0 / D;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    l[i - 1] = e[i - 1] * rD[i - 1];
    D = (d[i] + lam) - l[i - 1] * e[i - 1];
    rD[i] = 1.0 / D;
  }
  double z = rhs[0];
  w[0] = z * rD[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    z = rhs[i] - l[i - 1] * z;
    w[i] = z * rD[i];
  }
  double y = w[N - 1], s = y * y;
  double ys[N];
  ys[N - 1] = y;
#pragma unroll
  for (int i = N - 2; i >= 0; --i) {
    y = w[i] - l[i] * y;
    ys[i] = y;
    s += y * y;
  }
  if (out) {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = ys[i];
  }
  if (q) {
    double u = ys[0], acc = u * u * rD[0];
#pragma unroll
    for (int i = 1; i < N; ++i) {
      u = ys[i] - l[i - 1] * u;
      acc += u * u * rD[i];
    }
    *q = acc;
  }
  return s;
}

// Applies the reflections: forward (Q^T x: H_0 first) or backward (Q x).
__device__ void apply_q(TrSmem& S, double* x, bool transpose, int lane) {
  for (int step = 0; step < N - 2; ++step) {
    const int k = transpose ? step : N - 3 - step;
    const double bt = S.beta[k];
    if (bt == 0.0) continue;
    const int m = N - 1 - k;
    const double vi = lane < m ? S.B[(k + 1 + lane) * N + k] : 0.0;
    const double xi = lane < m ? x[k + 1 + lane] : 0.0;
    const double s = warp_sum_d(vi * xi);
    if (lane < m) x[k + 1 + lane] = xi - bt * s * vi;
    __syncwarp();
  }
}

// Exact trust-region subproblem for one source; warp-cooperative.
// Inputs g (27) and H (27 x 27) in global memory; writes p (smem y -> out).
__device__ void tr_solve(TrSmem& S, const double* __restrict__ g, const double* __restrict__ H,
                         double Delta, double* __restrict__ p_out, double* pred_out, int lane) {
  for (int e = lane; e < N * N; e += 32) {
    const int i = e / N, j = e % N;
    S.B[e] = -0.5 * (H[i * N + j] + H[j * N + i]);
  }
  if (lane < N) S.gh[lane] = g[lane];
  __syncwarp();
  // ---- Householder tridiagonalisation; v_k stored below the diagonal
  for (int k = 0; k < N - 2; ++k) {
    const int m = N - 1 - k;
    const double xv = lane < m ? S.B[(k + 1 + lane) * N + k] : 0.0;
    const double nrm2 = warp_sum_d(xv * xv);
    const double x0 = __shfl_sync(0xffffffffu, xv, 0);
    if (nrm2 - x0 * x0 <= 1e-300 || nrm2 == 0.0) {
      if (lane == 0) {
        S.beta[k] = 0.0;
        S.d[k] = S.B[k * N + k];
        S.e[k] = x0;
      }
      __syncwarp();
      continue;
    }
    const double alpha = -copysign(sqrt(nrm2), x0);
    const double vv = xv - (lane == 0 ? alpha : 0.0);
    const double vtv = warp_sum_d(vv * vv);
    const double bt = 2.0 / vtv;
    if (lane < m) S.B[(k + 1 + lane) * N + k] = vv;
    __syncwarp();
    double pi = 0.0;
    if (lane < m) {
      const double* row = S.B + (k + 1 + lane) * N + k + 1;
      for (int jj = 0; jj < m; ++jj) pi += row[jj] * S.B[(k + 1 + jj) * N + k];
      pi *= bt;
    }
    const double K = 0.5 * bt * warp_sum_d(vv * pi);
    const double wi = pi - K * vv;
    if (lane < m) S.w[lane] = wi;
    __syncwarp();
    if (lane < m) {
      double* row = S.B + (k + 1 + lane) * N + k + 1;
      for (int jj = 0; jj < m; ++jj) row[jj] -= vv * S.w[jj] + wi * S.B[(k + 1 + jj) * N + k];
    }
    __syncwarp();
    if (lane == 0) {
      S.beta[k] = bt;
      S.d[k] = S.B[k * N + k];
      S.e[k] = alpha;
    }
    __syncwarp();
  }
  if (lane == 0) {
    S.d[N - 2] = S.B[(N - 2) * N + N - 2];
    S.d[N - 1] = S.B[(N - 1) * N + N - 1];
    S.e[N - 2] = S.B[(N - 1) * N + N - 2];
    S.e[N - 1] = 0.0;
  }
  __syncwarp();
  apply_q(S, S.gh, true, lane);
  const double* d = S.d;
  const double* e = S.e;
  const double* gh = S.gh;
  double gn2 = 0.0, scale = 0.0;
  for (int i = 0; i < N; ++i) {
    gn2 += gh[i] * gh[i];
    scale = fmax(scale, fabs(d[i]) + fabs(e[i]) + (i ? fabs(e[i - 1]) : 0.0));
  }
  scale = fmax(scale, 1e-300);
  const double inv = 1.0 / scale;
  // scaled copies: |T / scale| <= 1
  if (lane < N) {
    S.df[lane] = (float)(d[lane] * inv);
    S.ef[lane] = (float)(e[lane] * inv);
    S.e2f[lane] = S.ef[lane] * S.ef[lane];
    S.w[lane] = e[lane] * inv;      // FP64 scaled off-diagonal
    S.z[lane] = d[lane] * inv;      // FP64 scaled diagonal
  }
  __syncwarp();
  // ---- lambda_min(T): FP32 multisection on the scaled matrix, then FP64
  // multisection with the division-free Sturm sequence
  double a = 1.0, b = -1.0;
  for (int i = 0; i < N; ++i) {
    const double r = fabs(S.w[i]) + (i ? fabs(S.w[i - 1]) : 0.0);
    a = fmin(a, S.z[i] - r);
    b = fmax(b, S.z[i] + r);
  }
  a -= 1e-6;
  b += 1e-6;
  {
    float fa = (float)a, fb = (float)b;
    for (int round = 0; round < 5; ++round) {
      const float sig = fa + (fb - fa) * (float)(lane + 1) * (1.f / 32.f);
      const bool hit = lane < 31 && sturm32(S.df, S.e2f, sig) >= 1;
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      const int t = mask ? __ffs(mask) - 1 : 31;
      const float na = t == 0 ? fa : fa + (fb - fa) * (float)t * (1.f / 32.f);
      const float nb = t == 31 ? fb : fa + (fb - fa) * (float)(t + 1) * (1.f / 32.f);
      fa = na;
      fb = nb;
    }
    // FP32 counts are exact away from eigenvalues to ~1e-6 of the scale
    a = fmax(a, (double)fa - 1e-5);
    b = fmin(b, (double)fb + 1e-5);
  }
  for (int round = 0; round < 5; ++round) {
    const double sig = a + (b - a) * (double)(lane + 1) / 32.0;
    const bool hit = lane < 31 && sturm64(S.z, S.w, sig) >= 1;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    const int t = mask ? __ffs(mask) - 1 : 31;
    const double na = t == 0 ? a : a + (b - a) * (double)t / 32.0;
    const double nb = t == 31 ? b : a + (b - a) * (double)(t + 1) / 32.0;
    a = na;
    b = nb;
  }
  const double lmin = 0.5 * (a + b) * scale;
  // ---- multiplier
  const double D2 = Delta * Delta;
  double lam = 0.0;
  bool interior = false, hard = false;
  if (lmin > 0.0) interior = ldl_solve(d, e, gh, 0.0, nullptr, nullptr) <= D2;
  if (!interior) {
    const double lo = fmax(0.0, -lmin);
    const double eps = 1e-12 * scale;
    double la = lo + eps;
    double lb = lo + sqrt(gn2) / Delta + eps;
    if (ldl_solve(d, e, gh, la, nullptr, nullptr) <= D2) {
      hard = true;
      lam = la;
    } else {
      // FP32 multisection on the scaled problem for a starting point ...
      if (lane < N) S.gf[lane] = (float)(gh[lane] * inv);
      __syncwarp();
      const float D2s = (float)(D2);          // |y| is scale-invariant
      float fa = (float)(la * inv), fb = (float)(lb * inv);
      for (int round = 0; round < 6; ++round) {
        const float l = fa + (fb - fa) * (float)(lane + 1) * (1.f / 32.f);
        const bool inside = lane < 31 && norm2_32(S.df, S.ef, S.gf, l) <= D2s;
        const unsigned mask = __ballot_sync(0xffffffffu, inside);
        const int t = mask ? __ffs(mask) - 1 : 31;
        const float na = t == 0 ? fa : fa + (fb - fa) * (float)t * (1.f / 32.f);
        const float nb = t == 31 ? fb : fa + (fb - fa) * (float)(t + 1) * (1.f / 32.f);
        fa = na;
        fb = nb;
      }
      // ... then safeguarded Newton on 1/|y(l)| - 1/Delta in FP64
      // (Nocedal & Wright, Algorithm 4.3), kept inside [la, lb]
      double l = fmin(fmax((double)fb * scale, la), lb);
      for (int it = 0; it < 12; ++it) {
        double q;
        const double n2 = ldl_solve(d, e, gh, l, nullptr, &q);
        const double ny = sqrt(n2);
        if (n2 <= D2) lb = l; else la = l;
        lam = l;
        if (fabs(ny - Delta) <= 1e-13 * Delta) break;
        double ln = l + (ny - Delta) / Delta * n2 / q;
        if (!(ln > la && ln < lb)) ln = 0.5 * (la + lb);
        if (ln == l) break;
        l = ln;
      }
    }
  }
  if (lane == 0) ldl_solve(d, e, gh, lam, S.y, nullptr);
  __syncwarp();
  if (hard) {
    // eigenvector of lambda_min by inverse iteration, shifted just below it
    if (lane == 0) {
      const double shift = -lmin + 1e-10 * scale;
      for (int i = 0; i < N; ++i) S.w[i] = 1.0 / sqrt((double)N);
      for (int itn = 0; itn < 4; ++itn) {
        const double nz = ldl_solve(d, e, S.w, shift, S.z, nullptr);
        const double r = 1.0 / sqrt(nz);
        for (int i = 0; i < N; ++i) S.w[i] = S.z[i] * r;
      }
      // project z out of y
      double zy = 0.0;
      for (int i = 0; i < N; ++i) zy += S.w[i] * S.y[i];
      for (int i = 0; i < N; ++i) {
        S.y[i] -= zy * S.w[i];
        S.z[i] = S.w[i];
      }
    }
    __syncwarp();
    apply_q(S, S.z, false, lane);       // Q z, to fix the sign
    if (lane == 0) {
      double first = 0.0;
      for (int i = 0; i < N; ++i) {
        if (fabs(S.z[i]) > 1e-14) {
          first = S.z[i];
          break;
        }
      }
      double ny2 = 0.0;
      for (int i = 0; i < N; ++i) ny2 += S.y[i] * S.y[i];
      const double tau = copysign(sqrt(fmax(D2 - ny2, 0.0)), first);
      for (int i = 0; i < N; ++i) S.y[i] += tau * S.w[i];
    }
    __syncwarp();
  }
  // predicted gain in tridiagonal coordinates: y.gh - y.T.y / 2
  if (lane == 0) {
    double gy = 0.0, yty = 0.0;
    for (int i = 0; i < N; ++i) {
      const double yi = S.y[i];
      gy += yi * gh[i];
      double ty = d[i] * yi;
      if (i > 0) ty += e[i - 1] * S.y[i - 1];
      if (i < N - 1) ty += e[i] * S.y[i + 1];
      yty += yi * ty;
    }
    S.red[0] = gy - 0.5 * yty;
  }
  __syncwarp();
  apply_q(S, S.y, false, lane);
  if (lane < N) p_out[lane] = S.y[lane];
  if (pred_out && lane == 0) *pred_out = S.red[0];
  __syncwarp();
}

__global__ void tr_subproblem_kernel(int n, const double* g, const double* H, const double* delta,
                                     double* p, double* pred) {
  extern __shared__ double smd[];
  TrSmem& S = *reinterpret_cast<TrSmem*>(smd);
  const int j = blockIdx.x;
  if (j >= n) return;
  tr_solve(S, g + (size_t)j * N, H + (size_t)j * N * N, delta[j], p + (size_t)j * N, pred + j,
           threadIdx.x);
}

// Step of every active slot: converged sources leave the active set.
__global__ void tr_step_kernel(PlanView v, const double* delta, int32_t* status) {
  extern __shared__ double smd[];
  TrSmem& S = *reinterpret_cast<TrSmem*>(smd);
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  if (!v.active[j]) return;
  const int src = v.src_ids[j];
  const double Dl = delta[src];
  const double* g = v.grad + (size_t)j * N;
  const double* H = v.hess + (size_t)j * N * N;
  bool finite = true;
  for (int e = lane; e < N * N; e += 32) finite &= isfinite(H[e]);
  if (lane < N) finite &= isfinite(g[lane]);
  finite = __all_sync(0xffffffffu, finite) && isfinite(v.elbo_rel[j]);
  if (!finite) {
    if (lane == 0) {
      status[src] = CELESTE_ST_FAILED;
      v.active[j] = 0;
    }
    return;
  }
  double* p = v.step + (size_t)j * N;
  tr_solve(S, g, H, Dl, p, v.pred + j, lane);
  __syncwarp();
  const double pred = v.pred[j];
  if (pred <= kFtol * (1.0 + fabs(v.elbo_rel[j])) || Dl < kDeltaMin) {
    if (lane == 0) {
      status[src] = CELESTE_ST_CONVERGED;
      v.active[j] = 0;
    }
    return;
  }
  if (lane < N) v.theta_trial[(size_t)j * N + lane] = v.theta[(size_t)src * N + lane] + p[lane];
}

// Accept or reject the trial points; update radius and status.
__global__ void tr_accept_kernel(PlanView v, const double* __restrict__ rel_trial, double* delta,
                                 int32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.n || !v.active[j]) return;
  const int src = v.src_ids[j];
  const double* p = v.step + (size_t)j * N;
  double pn = 0.0;
  for (int i = 0; i < N; ++i) pn += p[i] * p[i];
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
  v.active[j] = (st == CELESTE_ST_CONVERGED || st == CELESTE_ST_FAILED) ? 0 : 1;
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
  tr_subproblem_kernel<<<n, 32, sizeof(TrSmem), L.stream>>>(n, g, H, delta, p, pred);
  return cudaGetLastError();
}

cudaError_t launch_tr_step(const Launch& L, const PlanView& v, const double* delta,
                           int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  set_attrs();
  tr_step_kernel<<<v.n, 32, sizeof(TrSmem), L.stream>>>(v, delta, status);
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
