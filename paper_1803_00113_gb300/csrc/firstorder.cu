// A first-order subsolver for comparison with the Newton trust-region one
// (Sec. 4.3: Newton converges in tens of iterations, first-order methods
// and BFGS can take thousands, and a gradient alone costs a third of a
// gradient with the Hessian).  Limited-memory BFGS (Nocedal & Wright,
// Algorithm 7.4, two-loop recursion) on -L_s for every source of a plan,
// with a backtracking line search on the Armijo condition (c1 = 1e-4,
// halving from a unit step), neighbours frozen.  Per iteration it evaluates
// the value and gradient at the iterate (the gradient-only pixel pass) for
// the sources that need one, and the value at the trial point for all.
#include "host.h"

using namespace celeste;

namespace celeste {
namespace {

constexpr int N = kTheta;
constexpr int kMaxHist = 16;
constexpr double kC1 = 1e-4;
// Stop when the quasi-Newton model gain falls below 1e-12 (1 + |L|): the
// L-BFGS curvature model is too rough near the optimum for the Newton
// solver's 1e-9 (it stops 0.01-0.1 nats short on bright sources).
constexpr double kFtolFo = 1e-12;
constexpr double kNoise = 1e-7;    // relative noise of an FP32-summed value

struct LbfgsView {
  int m;               // history length
  int n;               // plan slots
  double* S;           // [m][n][27] steps
  double* Y;           // [m][n][27] gradient changes of -L
  double* rho;         // [m][n]
  int32_t* head;       // [n] next ring slot
  int32_t* count;      // [n] stored pairs
  double* theta_prev;  // [n][27]
  double* g_prev;      // [n][27]
  double* g;           // [n][27] gradient of L at the iterate
  double* d;           // [n][27] ascent direction
  double* alpha;       // [n] step length
  double* gd;          // [n] g.d
  double* f;           // [n] L_rel at the iterate
  int32_t* phase;      // [n] 0: needs a gradient, 1: trial pending
  int32_t* iters;      // [n] accepted steps (= gradient evaluations after the first)
  int32_t* fevals;     // [n] trial evaluations
  int32_t* reached;    // [n] accepted steps when the target was first reached, -1 before
};

__device__ __forceinline__ bool terminal(int st) {
  return st == CELESTE_ST_CONVERGED || st == CELESTE_ST_FAILED || st == CELESTE_ST_MAXITER;
}

__global__ void lbfgs_mark_kernel(PlanView v, LbfgsView L, const int32_t* status, int need_grad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.n) return;
  const bool live = !terminal(status[v.src_ids[j]]);
  v.active[j] = live && (!need_grad || L.phase[j] == 0) ? 1 : 0;
}

// One warp per slot that has a fresh gradient: update the history, two-loop
// recursion, unit trial step along the direction.
__global__ void lbfgs_direction_kernel(PlanView v, LbfgsView L, int32_t* status) {
  const int j = blockIdx.x, lane = threadIdx.x;
  if (!v.active[j]) return;
  const int src = v.src_ids[j];
  const size_t o = (size_t)j * N;
  const double g = lane < N ? L.g[o + lane] : 0.0;
  const double th = lane < N ? v.theta[(size_t)src * N + lane] : 0.0;
  int head = L.head[j], count = L.count[j];
  if (L.iters[j] > 0) {
    const double s = lane < N ? th - L.theta_prev[o + lane] : 0.0;
    const double y = lane < N ? L.g_prev[o + lane] - g : 0.0;   // change of grad(-L)
    const double sy = warp_sum_d(s * y), yy = warp_sum_d(y * y), ss = warp_sum_d(s * s);
    if (sy > 1e-10 * sqrt(ss * yy)) {
      const size_t h = ((size_t)head * L.n + j) * N;
      if (lane < N) {
        L.S[h + lane] = s;
        L.Y[h + lane] = y;
      }
      if (lane == 0) L.rho[(size_t)head * L.n + j] = 1.0 / sy;
      head = (head + 1) % L.m;
      count = min(count + 1, L.m);
    }
  }
  __syncwarp();
  // two-loop recursion on q = grad(-L) = -g
  double q = -g, a[kMaxHist];
  for (int t = 0; t < count; ++t) {
    const int idx = (head - 1 - t + 2 * L.m) % L.m;
    const size_t h = ((size_t)idx * L.n + j) * N;
    const double r = L.rho[(size_t)idx * L.n + j];
    a[t] = r * warp_sum_d(lane < N ? L.S[h + lane] * q : 0.0);
    if (lane < N) q = fma(-a[t], L.Y[h + lane], q);
  }
  double gamma;
  if (count > 0) {
    const int idx = (head - 1 + L.m) % L.m;
    const size_t h = ((size_t)idx * L.n + j) * N;
    const double yv = lane < N ? L.Y[h + lane] : 0.0;
    gamma = 1.0 / (L.rho[(size_t)idx * L.n + j] * warp_sum_d(yv * yv));
  } else {
    gamma = 1.0 / fmax(sqrt(warp_sum_d(g * g)), 1e-300);   // first step: unit length
  }
  double r = gamma * q;
  for (int t = count - 1; t >= 0; --t) {
    const int idx = (head - 1 - t + 2 * L.m) % L.m;
    const size_t h = ((size_t)idx * L.n + j) * N;
    const double b = L.rho[(size_t)idx * L.n + j] * warp_sum_d(lane < N ? L.Y[h + lane] * r : 0.0);
    if (lane < N) r = fma(a[t] - b, L.S[h + lane], r);
  }
  double d = -r;
  double gd = warp_sum_d(g * d);
  if (!(gd > 0.0)) {
    // not an ascent direction: restart from the scaled gradient
    const double gn = fmax(sqrt(warp_sum_d(g * g)), 1e-300);
    d = g / gn;
    gd = gn;
    count = 0;
  }
  if (lane < N) {
    L.d[o + lane] = d;
    L.theta_prev[o + lane] = th;
    L.g_prev[o + lane] = g;
    v.theta_trial[o + lane] = th + d;
  }
  if (lane == 0) {
    L.head[j] = head;
    L.count[j] = count;
    L.alpha[j] = 1.0;
    L.gd[j] = gd;
    L.phase[j] = 1;
    // converged when the model gain of the full quasi-Newton step, g.d / 2,
    // is negligible (a gradient-based test: near the optimum the value
    // changes fall below their FP32 noise)
    if (0.5 * gd <= kFtolFo * (1.0 + fabs(L.f[j]))) {
      status[src] = CELESTE_ST_CONVERGED;
      L.phase[j] = 0;
    }
  }
}

// Armijo test of every pending trial: accept (the source needs a gradient
// next) or halve the step.
__global__ void lbfgs_accept_kernel(PlanView v, LbfgsView L, const double* rel_trial,
                                    const double* target, int32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.n || !v.active[j]) return;
  const int src = v.src_ids[j];
  const size_t o = (size_t)j * N;
  const double a = L.alpha[j], f0 = L.f[j], rel = rel_trial[j];
  ++L.fevals[j];
  // Armijo; when the step's expected gain is below the value's noise, a
  // value that does not drop beyond that noise is accepted too
  const double want = kC1 * a * L.gd[j], noise = kNoise * (1.0 + fabs(f0));
  if (isfinite(rel) && (rel >= f0 + want || (want < noise && rel >= f0 - noise))) {
    for (int i = 0; i < N; ++i) v.theta[(size_t)src * N + i] = v.theta_trial[o + i];
    L.phase[j] = 0;
    const int it = ++L.iters[j];
    if (target && L.reached[j] < 0 && rel >= target[j]) L.reached[j] = it;
    status[src] = CELESTE_ST_ACCEPTED;
  } else {
    const double an = 0.5 * a;
    L.alpha[j] = an;
    if (an < 1e-20) {
      status[src] = CELESTE_ST_CONVERGED;        // no ascent left along d
    } else {
      for (int i = 0; i < N; ++i)
        v.theta_trial[o + i] = v.theta[(size_t)src * N + i] + an * L.d[o + i];
      status[src] = CELESTE_ST_REJECTED;
    }
  }
}

}  // namespace
}  // namespace celeste

struct celeste_lbfgs {
  celeste_ctx* ctx = nullptr;
  celeste_plan* plan = nullptr;
  LbfgsView L{};
  double* rel_trial = nullptr;
  std::vector<void*> allocs;
};

extern "C" {

int celeste_lbfgs_destroy(celeste_lbfgs* B) {
  if (!B) return CELESTE_EINVAL;
  for (void* a : B->allocs) cudaFree(a);
  delete B;
  return CELESTE_OK;
}

int celeste_lbfgs_create(celeste_ctx* c, const celeste_plan* pc, int32_t m, celeste_lbfgs** out) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c || !out || m < 1 || m > kMaxHist) return CELESTE_EINVAL;
  *out = nullptr;
  celeste_lbfgs* B = new celeste_lbfgs();
  B->ctx = c;
  B->plan = p;
  const size_t n = (size_t)(p->v.n > 0 ? p->v.n : 1);
  int rc = CELESTE_OK;
  auto alloc = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    if (rc != CELESTE_OK) return nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      rc = CELESTE_ENOMEM;
      return nullptr;
    }
    B->allocs.push_back(ptr);
    return ptr;
  };
  LbfgsView& L = B->L;
  L.m = m;
  L.n = p->v.n;
  L.S = static_cast<double*>(alloc(m * n * N * 8));
  L.Y = static_cast<double*>(alloc(m * n * N * 8));
  L.rho = static_cast<double*>(alloc(m * n * 8));
  L.head = static_cast<int32_t*>(alloc(n * 4));
  L.count = static_cast<int32_t*>(alloc(n * 4));
  L.theta_prev = static_cast<double*>(alloc(n * N * 8));
  L.g_prev = static_cast<double*>(alloc(n * N * 8));
  L.g = static_cast<double*>(alloc(n * N * 8));
  L.d = static_cast<double*>(alloc(n * N * 8));
  L.alpha = static_cast<double*>(alloc(n * 8));
  L.gd = static_cast<double*>(alloc(n * 8));
  L.f = static_cast<double*>(alloc(n * 8));
  L.phase = static_cast<int32_t*>(alloc(n * 4));
  L.iters = static_cast<int32_t*>(alloc(n * 4));
  L.fevals = static_cast<int32_t*>(alloc(n * 4));
  L.reached = static_cast<int32_t*>(alloc(n * 4));
  B->rel_trial = static_cast<double*>(alloc(n * 8));
  if (rc != CELESTE_OK) {
    celeste_lbfgs_destroy(B);
    return rc;
  }
  *out = B;
  return celeste_lbfgs_reset(c, B);
}

int celeste_lbfgs_reset(celeste_ctx* c, celeste_lbfgs* B) {
  if (!c || !B || B->ctx != c) return CELESTE_EINVAL;
  const size_t n = (size_t)(B->L.n > 0 ? B->L.n : 1);
  CK(cudaMemsetAsync(B->L.head, 0, n * 4, c->stream));
  CK(cudaMemsetAsync(B->L.count, 0, n * 4, c->stream));
  CK(cudaMemsetAsync(B->L.phase, 0, n * 4, c->stream));
  CK(cudaMemsetAsync(B->L.iters, 0, n * 4, c->stream));
  CK(cudaMemsetAsync(B->L.fevals, 0, n * 4, c->stream));
  CK(cudaMemsetAsync(B->L.reached, 0xff, n * 4, c->stream));   // -1
  return CELESTE_OK;
}

int celeste_lbfgs_step(celeste_ctx* c, celeste_lbfgs* B, int32_t* status, const double* target) {
  if (!c || !B || B->ctx != c || !status) return CELESTE_EINVAL;
  celeste_plan* p = B->plan;
  PlanView& v = p->v;
  if (v.n == 0) return CELESTE_OK;
  const Launch L = make_launch(c, p);
  const int nb = (v.n + 127) / 128;
  // value and gradient where a step was accepted (or at the start)
  lbfgs_mark_kernel<<<nb, 128, 0, L.stream>>>(v, B->L, status, 1);
  CK(cudaGetLastError());
  CK(launch_setup(L, v, c->d_model, 0, v.n_pairs, false));
  CK(launch_background(L, v));
  CK(launch_pixels_grad(L, v));
  CK(launch_epilogue_grad(L, v, c->d_model, nullptr, B->L.f, B->L.g));
  lbfgs_direction_kernel<<<v.n, 32, 0, L.stream>>>(v, B->L, status);
  CK(cudaGetLastError());
  // value at the trial point of every live source
  lbfgs_mark_kernel<<<nb, 128, 0, L.stream>>>(v, B->L, status, 0);
  CK(cudaGetLastError());
  CK(launch_setup(L, v, c->d_model, 0, v.n_own_pairs, true));
  CK(launch_pixels_value(L, v));
  CK(launch_epilogue_value(L, v, c->d_model, nullptr, B->rel_trial, true));
  lbfgs_accept_kernel<<<nb, 128, 0, L.stream>>>(v, B->L, B->rel_trial, target, status);
  CK(cudaGetLastError());
  c->launches += 11;
  return CELESTE_OK;
}

int celeste_lbfgs_counts(celeste_ctx* c, const celeste_lbfgs* B, int32_t* iters, int32_t* fevals,
                         int32_t* reached) {
  if (!c || !B || B->ctx != c) return CELESTE_EINVAL;
  const size_t n = (size_t)B->L.n;
  if (iters) CK(cudaMemcpyAsync(iters, B->L.iters, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (fevals) CK(cudaMemcpyAsync(fevals, B->L.fevals, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (reached) CK(cudaMemcpyAsync(reached, B->L.reached, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  return CELESTE_OK;
}

}  // extern "C"
