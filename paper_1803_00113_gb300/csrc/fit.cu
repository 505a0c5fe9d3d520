// The block-coordinate-ascent region fit (Sec. 4.3, 4.4): its device
// bookkeeping and the host code that builds and runs it.
//
// A pass is one CUDA graph: per colour class, the neighbour background is
// rendered once, then a conditional WHILE node repeats one trust-region
// Newton iteration over the class until every source of the class has
// converged, failed or used its iterations; fit_check_kernel, the last node
// of the loop body, does the per-source accounting and sets the loop
// condition.  The loop is bounded twice: by each source's iteration budget
// and by a per-class trip counter.  The host waits once per pass, reads
// which segments (independent requests sharing the fit) run another pass,
// and stops when none does.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>

#include "host.h"

namespace celeste {

namespace {

constexpr int kFitThreads = 256;

__global__ void fit_reset_kernel(FitView f) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < f.n_region; j += gridDim.x * blockDim.x) {
    const int s = f.region[j];
    if (!f.seg_active[f.seg_of[s]]) {   // finished segment: frozen at its result
      f.done[s] = 1;
      continue;
    }
    f.delta[s] = kDelta0;
    f.status[s] = CELESTE_ST_ACCEPTED;
    f.iters_pass[s] = 0;
    f.done[s] = 0;
    f.gain[s] = 0.0;
  }
  if (blockIdx.x == 0) {
    for (int c = threadIdx.x; c < f.n_classes; c += blockDim.x) f.class_iter[c] = 0;
    if (threadIdx.x == 0) f.summary[0] = 0;
  }
}

// After one Newton iteration of the class: count the iteration of every
// source that took part (not yet done this pass), add the gain of accepted
// steps, retire sources that converged, failed or ran out of iterations, and
// keep the loop going while any source of the class is still iterating.
__global__ void __launch_bounds__(kFitThreads) fit_check_kernel(PlanView v, FitView f,
                                                                const double* rel_trial, int cls,
                                                                cudaGraphConditionalHandle h) {
  int busy = 0;
  for (int j = threadIdx.x; j < v.n; j += kFitThreads) {
    const int s = v.src_ids[j];
    if (f.done[s]) continue;
    const int it = ++f.iters_pass[s];
    ++f.iters_total[s];
    const int st = f.status[s];
    if (st == CELESTE_ST_ACCEPTED) {
      ++f.accepted[s];
      f.gain[s] += rel_trial[j] - v.elbo_rel[j];
    }
    if (st == CELESTE_ST_CONVERGED || st == CELESTE_ST_FAILED) {
      f.done[s] = 1;
    } else if (it >= f.max_iter) {
      f.status[s] = CELESTE_ST_MAXITER;
      f.done[s] = 1;
    } else {
      busy = 1;
    }
  }
  busy = __syncthreads_or(busy);
  if (threadIdx.x == 0) {
    const int k = ++f.class_iter[cls];
    cudaGraphSetConditional(h, (busy && k < f.max_iter) ? 1u : 0u);
  }
}

// End of a pass, one warp per segment: the segment's gain (summed in a fixed
// order), its pass count and whether it runs another pass; summary[0]
// counts the segments still running, summary[1 + c] the loop trips of
// class c.
__global__ void fit_pass_end_kernel(FitView f) {
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k < f.n_seg && f.seg_active[k]) {
    const int b = f.seg_ptr[k], e = f.seg_ptr[k + 1];
    double g = 0.0;
    for (int j = b + lane; j < e; j += 32) g += f.gain[f.region[j]];
    g = warp_sum_d(g);
    if (lane == 0) {
      const int passes = ++f.seg_passes[k];
      f.seg_gain[k] = g;
      const bool more = g > f.pass_tol * (double)(e - b) && passes < f.max_passes;
      f.seg_active[k] = more ? 1 : 0;
      if (more) atomicAdd(&f.summary[0], 1);
    }
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < f.n_classes; c += blockDim.x) f.summary[1 + c] = f.class_iter[c];
}

}  // namespace

cudaError_t launch_fit_reset(cudaStream_t stream, const FitView& f) {
  const int blocks = (f.n_region + kFitThreads - 1) / kFitThreads;
  fit_reset_kernel<<<blocks > 0 ? blocks : 1, kFitThreads, 0, stream>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_fit_check(cudaStream_t stream, const PlanView& v, const FitView& f,
                             const double* rel_trial, int cls, cudaGraphConditionalHandle h) {
  fit_check_kernel<<<1, kFitThreads, 0, stream>>>(v, f, rel_trial, cls, h);
  return cudaGetLastError();
}

cudaError_t launch_fit_pass_end(cudaStream_t stream, const FitView& f) {
  const int warps = kFitThreads / 32;
  const int blocks = (f.n_seg + warps - 1) / warps;
  fit_pass_end_kernel<<<blocks > 0 ? blocks : 1, kFitThreads, 0, stream>>>(f);
  return cudaGetLastError();
}

// ---- host side --------------------------------------------------------------

int fit_create_segments(celeste_ctx* c, const celeste_problem* pr, const int32_t* ids, int n,
                        const int32_t* seg_ptr, int n_seg, const celeste_tuning* tuning,
                        celeste_fit** out) {
  if (!c || !pr || !out || n < 0 || (n > 0 && !ids) || n_seg < 1 || !seg_ptr ||
      seg_ptr[0] != 0 || seg_ptr[n_seg] != n || !pr->h_nbr_ptr || (pr->n_nbr > 0 && !pr->h_nbr_idx))
    return CELESTE_EINVAL;
  *out = nullptr;
  std::vector<int32_t> seg_of(pr->n_sources, -1);
  for (int k = 0; k < n_seg; ++k) {
    if (seg_ptr[k + 1] < seg_ptr[k]) return CELESTE_EINVAL;
    for (int j = seg_ptr[k]; j < seg_ptr[k + 1]; ++j) {
      if (ids[j] < 0 || ids[j] >= pr->n_sources || seg_of[ids[j]] >= 0) return CELESTE_EINVAL;
      seg_of[ids[j]] = k;
    }
  }
  // greedy colouring of the region's overlap graph by ascending id
  std::vector<int32_t> sorted(ids, ids + n);
  std::sort(sorted.begin(), sorted.end());
  std::vector<int32_t> color(pr->n_sources, -1);
  int n_colors = 0;
  std::vector<char> used;
  for (int s : sorted) {
    used.assign(n_colors + 1, 0);
    for (int k = pr->h_nbr_ptr[s]; k < pr->h_nbr_ptr[s + 1]; ++k) {
      const int t = pr->h_nbr_idx[k];
      if (t < 0 || t >= pr->n_sources) return CELESTE_EINVAL;
      if (color[t] >= 0) used[color[t]] = 1;
    }
    int col = 0;
    while (used[col]) ++col;
    color[s] = col;
    n_colors = std::max(n_colors, col + 1);
  }
  celeste_fit* F = new celeste_fit();
  F->ctx = c;
  F->ctx_serial = c->serial;
  F->region.assign(ids, ids + n);
  F->seg_ptr.assign(seg_ptr, seg_ptr + n_seg + 1);
  F->n_sources = pr->n_sources;
  int rc = CELESTE_OK;
  // one plan per colour class; the classes are planned on parallel host
  // threads (planning is host work proportional to the class's pixels)
  std::vector<std::vector<int32_t>> cls(n_colors);
  for (int s : sorted) cls[color[s]].push_back(s);
  std::vector<celeste_plan*> plans(n_colors, nullptr);
  std::vector<int> rcs(n_colors, CELESTE_OK);
  int device = 0;
  cudaGetDevice(&device);
  auto plan_class = [&](int col) {
    cudaSetDevice(device);
    rcs[col] = celeste_plan_create(c, pr, cls[col].data(), (int)cls[col].size(), tuning,
                                   &plans[col]);
  };
  const int n_threads =
      std::min<int>(n_colors, std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
  if (n_threads <= 1) {
    for (int col = 0; col < n_colors; ++col) plan_class(col);
  } else {
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t)
      pool.emplace_back([&] {
        for (int col; (col = next.fetch_add(1)) < n_colors;) plan_class(col);
      });
    for (auto& t : pool) t.join();
  }
  for (int col = 0; col < n_colors; ++col) {
    if (rcs[col] != CELESTE_OK && rc == CELESTE_OK) rc = rcs[col];
    if (plans[col]) F->plans.push_back(plans[col]);
  }
  if (rc == CELESTE_OK && pr->render_cache) {
    // sources outside the region that border it: rendered into the cache
    // once per run, since backgrounds are gathered from there
    std::vector<int32_t> outside;
    std::vector<char> seen(pr->n_sources, 0);
    for (int s : sorted)
      for (int k = pr->h_nbr_ptr[s]; k < pr->h_nbr_ptr[s + 1]; ++k) {
        const int t = pr->h_nbr_idx[k];
        if (seg_of[t] < 0 && !seen[t]) {
          seen[t] = 1;
          outside.push_back(t);
        }
      }
    if (!outside.empty())
      rc = celeste_plan_create(c, pr, outside.data(), (int)outside.size(), tuning, &F->outside);
  }
  auto alloc = [&](size_t bytes) -> void* {
    if (rc != CELESTE_OK) return nullptr;
    void* ptr = ctx_alloc(c, false, bytes);
    if (!ptr) {
      rc = CELESTE_ENOMEM;
      return nullptr;
    }
    F->allocs.push_back(ptr);
    return ptr;
  };
  auto pinned = [&](size_t bytes) -> void* {
    if (rc != CELESTE_OK) return nullptr;
    void* ptr = ctx_alloc(c, true, bytes);
    if (!ptr) {
      rc = CELESTE_ENOMEM;
      return nullptr;
    }
    F->host_allocs.push_back(ptr);
    return ptr;
  };
  const size_t S = (size_t)pr->n_sources;
  FitView& f = F->f;
  int32_t* d_region = static_cast<int32_t*>(alloc(n * sizeof(int32_t)));
  int32_t* d_seg_ptr = static_cast<int32_t*>(alloc((n_seg + 1) * sizeof(int32_t)));
  int32_t* d_seg_of = static_cast<int32_t*>(alloc(S * sizeof(int32_t)));
  f.delta = static_cast<double*>(alloc(S * sizeof(double)));
  f.status = static_cast<int32_t*>(alloc(S * sizeof(int32_t)));
  f.iters_pass = static_cast<int32_t*>(alloc(S * sizeof(int32_t)));
  f.iters_total = static_cast<int32_t*>(alloc(S * sizeof(int32_t)));
  f.accepted = static_cast<int32_t*>(alloc(S * sizeof(int32_t)));
  f.done = static_cast<uint8_t*>(alloc(S));
  f.gain = static_cast<double*>(alloc(S * sizeof(double)));
  f.class_iter = static_cast<int32_t*>(alloc(n_colors * sizeof(int32_t)));
  f.seg_active = static_cast<uint8_t*>(alloc(n_seg));
  f.seg_passes = static_cast<int32_t*>(alloc(n_seg * sizeof(int32_t)));
  f.seg_gain = static_cast<double*>(alloc(n_seg * sizeof(double)));
  f.summary = static_cast<int32_t*>(alloc((1 + n_colors) * sizeof(int32_t)));
  F->h_summary = static_cast<int32_t*>(pinned((1 + n_colors) * sizeof(int32_t)));
  F->h_seg_active = static_cast<uint8_t*>(pinned(n_seg));
  F->h_seg_gain = static_cast<double*>(pinned(n_seg * sizeof(double)));
  F->h_seg_passes = static_cast<int32_t*>(pinned(n_seg * sizeof(int32_t)));
  f.region = d_region;
  f.seg_ptr = d_seg_ptr;
  f.seg_of = d_seg_of;
  f.n_region = n;
  f.n_seg = n_seg;
  f.n_classes = n_colors;
  if (rc == CELESTE_OK &&
      (cudaMemcpy(d_region, ids, n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_seg_ptr, seg_ptr, (n_seg + 1) * sizeof(int32_t), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemcpy(d_seg_of, seg_of.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemset(f.iters_total, 0, S * sizeof(int32_t)) != cudaSuccess ||
       cudaMemset(f.accepted, 0, S * sizeof(int32_t)) != cudaSuccess ||
       cudaMemset(f.status, 0, S * sizeof(int32_t)) != cudaSuccess ||
       cudaMemset(f.seg_passes, 0, n_seg * sizeof(int32_t)) != cudaSuccess ||
       cudaStreamCreateWithFlags(&F->capture, cudaStreamNonBlocking) != cudaSuccess))
    rc = CELESTE_ECUDA;
  if (rc != CELESTE_OK) {
    celeste_fit_destroy(F);
    return rc;
  }
  *out = F;
  return CELESTE_OK;
}

namespace {

// Builds the graph of one pass for the given limits.
int fit_build(celeste_fit* F) {
  celeste_ctx* c = F->ctx;
  if (F->exec) cudaGraphExecDestroy(F->exec);
  if (F->graph) cudaGraphDestroy(F->graph);
  F->exec = nullptr;
  F->graph = nullptr;
  const FitView f = F->f;
  cudaStream_t cs = F->capture;
  CK(cudaGraphCreate(&F->graph, 0));
  std::vector<cudaGraphNode_t> deps;
  auto begin = [&]() {
    return cudaStreamBeginCaptureToGraph(cs, F->graph, deps.empty() ? nullptr : deps.data(),
                                         nullptr, deps.size(), cudaStreamCaptureModeRelaxed);
  };
  auto end = [&]() {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) deps.assign(d, d + nd);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    return e != cudaSuccess ? e : e2;
  };
  CK(begin());
  cudaError_t e = launch_fit_reset(cs, f);
  cudaError_t e2 = end();
  CK(e);
  CK(e2);
  for (int k = 0; k < f.n_classes; ++k) {
    celeste_plan* p = F->plans[k];
    Launch L = make_launch(c, p);
    L.stream = cs;
    // neighbour records and background, once per class and pass (with a
    // render cache the background needs no records: one launch)
    CK(begin());
    if (p->v.cache) {
      e = launch_prepare(L, p->v, c->d_model, f.status, 0, true);
    } else {
      e = launch_prepare(L, p->v, c->d_model, f.status, p->v.n_pairs, false);
      if (e == cudaSuccess) e = launch_background(L, p->v);
    }
    e2 = end();
    CK(e);
    CK(e2);
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, F->graph, 1, cudaGraphCondAssignDefault));
    // (the parameter union has no default constructor: zeroed storage)
    alignas(cudaGraphNodeParams) unsigned char np_bytes[sizeof(cudaGraphNodeParams)];
    memset(np_bytes, 0, sizeof(np_bytes));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_bytes);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t loop;
    CK(cudaGraphAddNode(&loop, F->graph, deps.empty() ? nullptr : deps.data(), nullptr,
                        deps.size(), &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    e = enqueue_iteration(c, p, L, f.delta, f.status);
    if (e == cudaSuccess) e = launch_fit_check(cs, p->v, f, p->rel_trial, k, h);
    cudaGraph_t g = nullptr;
    e2 = cudaStreamEndCapture(cs, &g);
    CK(e);
    CK(e2);
    deps.assign(1, loop);
    if (p->v.cache) {
      // the class's final parameters into the render cache, for the
      // backgrounds of the classes after it
      CK(begin());
      e = launch_setup(L, p->v, c->d_model, 0, p->v.n_own_pairs, false);
      if (e == cudaSuccess) e = launch_render_cache(L, p->v, nullptr);
      e2 = end();
      CK(e);
      CK(e2);
    }
  }
  CK(begin());
  e = launch_fit_pass_end(cs, f);
  e2 = end();
  CK(e);
  CK(e2);
  CK(cudaGraphInstantiate(&F->exec, F->graph, 0));
  F->built_max_iter = f.max_iter;
  F->built_max_passes = f.max_passes;
  F->built_pass_tol = f.pass_tol;
  return CELESTE_OK;
}

}  // namespace

int fit_begin(celeste_ctx* c, celeste_fit* F, int max_passes, int max_iter, double pass_tol) {
  if (!c || !F || F->ctx != c || max_passes < 0 || max_passes > 1000 || max_iter < 0 ||
      max_iter > 1000 || !(pass_tol >= 0.0))
    return CELESTE_EINVAL;
  FitView& f = F->f;
  f.max_passes = max_passes ? max_passes : 5;
  f.max_iter = max_iter ? max_iter : 50;
  f.pass_tol = pass_tol;
  if (f.n_region == 0) return CELESTE_OK;
  if (!F->exec || F->built_max_iter != f.max_iter || F->built_max_passes != f.max_passes ||
      F->built_pass_tol != f.pass_tol) {
    const int rc = fit_build(F);
    if (rc) return rc;
  }
  // a run starts from the current parameters: (re)render the cache
  for (celeste_plan* p : F->plans) {
    const int rc = celeste_render_cache(c, p);
    if (rc) return rc;
  }
  if (F->outside) {
    const int rc = celeste_render_cache(c, F->outside);
    if (rc) return rc;
  }
  const size_t S = (size_t)F->n_sources;
  CK(cudaMemsetAsync(f.iters_total, 0, S * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(f.accepted, 0, S * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(f.seg_active, 1, f.n_seg, c->stream));
  CK(cudaMemsetAsync(f.seg_passes, 0, f.n_seg * sizeof(int32_t), c->stream));
  return CELESTE_OK;
}

int fit_pass_launch(celeste_ctx* c, celeste_fit* F) {
  const FitView& f = F->f;
  if (f.n_region == 0) return CELESTE_OK;
  CK(cudaGraphLaunch(F->exec, c->stream));
  CK(cudaMemcpyAsync(F->h_summary, f.summary, (1 + f.n_classes) * sizeof(int32_t),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(F->h_seg_active, f.seg_active, f.n_seg, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(F->h_seg_gain, f.seg_gain, f.n_seg * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(F->h_seg_passes, f.seg_passes, f.n_seg * sizeof(int32_t),
                     cudaMemcpyDeviceToHost, c->stream));
  return CELESTE_OK;
}

int fit_pass(celeste_ctx* c, celeste_fit* F, int* n_active) {
  *n_active = 0;
  const int rc = fit_pass_launch(c, F);
  if (rc) return rc;
  return fit_pass_finish(c, F, n_active);
}

int fit_pass_finish(celeste_ctx* c, celeste_fit* F, int* n_active) {
  const FitView& f = F->f;
  *n_active = 0;
  if (f.n_region == 0) return CELESTE_OK;
  CK(cudaStreamSynchronize(c->stream));
  // launches of the pass: reset and summary, per class 2 (with a render
  // cache: 1, and 2 to refresh it at the end) + the loop trips
  int64_t nl = 2;
  const int per_class = F->plans.empty() || !F->plans[0]->v.cache ? 2 : 3;
  for (int k = 0; k < f.n_classes; ++k)
    nl += per_class + (int64_t)F->h_summary[1 + k] * kIterationLaunches;
  c->launches += nl;
  *n_active = F->h_summary[0];
  return CELESTE_OK;
}

}  // namespace celeste

using namespace celeste;

extern "C" {

int celeste_fit_destroy(celeste_fit* F) {
  if (!F) return CELESTE_EINVAL;
  if (F->exec) cudaGraphExecDestroy(F->exec);
  if (F->graph) cudaGraphDestroy(F->graph);
  if (F->capture) cudaStreamDestroy(F->capture);
  for (celeste_plan* p : F->plans) celeste_plan_destroy(p);
  if (F->outside) celeste_plan_destroy(F->outside);
  ctx_release(F->ctx, F->ctx_serial, true, F->host_allocs);
  ctx_release(F->ctx, F->ctx_serial, false, F->allocs);
  delete F;
  return CELESTE_OK;
}

int celeste_fit_create(celeste_ctx* c, const celeste_problem* pr, const int32_t* ids, int32_t n,
                       const celeste_tuning* tuning, celeste_fit** out) {
  if (n < 0 || (n > 0 && !ids)) return CELESTE_EINVAL;
  std::vector<int32_t> region(ids, ids + n);
  std::sort(region.begin(), region.end());
  const int32_t seg_ptr[2] = {0, n};
  return fit_create_segments(c, pr, region.data(), n, seg_ptr, 1, tuning, out);
}

int celeste_fit_classes(const celeste_fit* F) { return F ? F->f.n_classes : -1; }

int celeste_fit_run(celeste_ctx* c, celeste_fit* F, int32_t max_passes, int32_t max_iter,
                    double pass_tol, int32_t* passes_out, double* pass_gain) {
  int rc = fit_begin(c, F, max_passes, max_iter, pass_tol);
  if (rc) return rc;
  if (passes_out) *passes_out = 0;
  int pass = 0, active = 1;
  while (active > 0 && pass < F->f.max_passes && F->f.n_region > 0) {
    rc = fit_pass(c, F, &active);
    if (rc) return rc;
    if (pass_gain) pass_gain[pass] = F->h_seg_gain[0];
    ++pass;
  }
  if (passes_out) *passes_out = pass;
  return CELESTE_OK;
}

int celeste_fit_results(celeste_ctx* c, const celeste_fit* F, int32_t* status, int32_t* iters,
                        int32_t* accepted, double* delta) {
  if (!c || !F || F->ctx != c) return CELESTE_EINVAL;
  const size_t S = (size_t)F->n_sources;
  const FitView& f = F->f;
  if (status) CK(cudaMemcpyAsync(status, f.status, S * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (iters) CK(cudaMemcpyAsync(iters, f.iters_total, S * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (accepted) CK(cudaMemcpyAsync(accepted, f.accepted, S * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (delta) CK(cudaMemcpyAsync(delta, f.delta, S * 8, cudaMemcpyDeviceToDevice, c->stream));
  return CELESTE_OK;
}

}  // extern "C"
