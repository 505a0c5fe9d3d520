// Device bookkeeping of the block-coordinate-ascent region fit (Sec. 4.3,
// 4.4).  A pass is one CUDA graph: per colour class, the neighbour
// background is rendered once, then a conditional WHILE node repeats one
// trust-region Newton iteration over the class until every source of the
// class has converged, failed or used its iterations; fit_check_kernel, the
// last node of the loop body, does the per-source accounting and sets the
// loop condition.  The loop is bounded twice: by each source's iteration
// budget and by a per-class iteration counter.
#include "internal.cuh"

namespace celeste {

namespace {

constexpr int kFitThreads = 256;

__global__ void fit_reset_kernel(FitView f) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < f.n_region; j += gridDim.x * blockDim.x) {
    const int s = f.region[j];
    f.delta[s] = kDelta0;
    f.status[s] = CELESTE_ST_ACCEPTED;
    f.iters_pass[s] = 0;
    f.done[s] = 0;
    f.gain[s] = 0.0;
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < f.n_classes; c += blockDim.x) f.class_iter[c] = 0;
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

// End of a pass: out[0] = the pass's total gain (summed in a fixed order),
// out[1 + c] = Newton iterations of class c.
__global__ void __launch_bounds__(kFitThreads) fit_pass_end_kernel(FitView f) {
  __shared__ double red[kFitThreads];
  double s = 0.0;
  for (int j = threadIdx.x; j < f.n_region; j += kFitThreads) s += f.gain[f.region[j]];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kFitThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) f.out[0] = red[0];
  for (int c = threadIdx.x; c < f.n_classes; c += kFitThreads) f.out[1 + c] = f.class_iter[c];
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
  fit_pass_end_kernel<<<1, kFitThreads, 0, stream>>>(f);
  return cudaGetLastError();
}

}  // namespace celeste
