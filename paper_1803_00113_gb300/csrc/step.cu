// The per-source part of a trust-region Newton iteration (Sec. 4.3) in one
// launch, one block of four warps per plan slot:
//   1. the epilogue at theta (epilogue.cuh): the source's tile sums chained
//      to its 27 coordinates plus KL_s, giving L_rel, its gradient and its
//      Hessian;
//   2. the trust-region step (trsolve.cuh): p, its predicted gain and
//      theta_trial = theta + p, or the source leaves the active set
//      (converged or failed);
//   3. at theta_trial: KL_s on warp 0, and the records of the source's own
//      pairs on warps 1..3 (setup.cuh), which the value pass then reads.
// The stages share the block's shared memory in turn.  After the value
// pass, the finish kernel (a warp per slot) forms L_rel at theta_trial and
// applies the accept rule (accept.cuh).
#include "accept.cuh"
#include "device_once.h"
#include "epilogue.cuh"
#include "setup.cuh"
#include "trsolve.cuh"

namespace celeste {

static_assert(kEpiThreads == kTrThreads, "the stages share one block shape");

union StepSmem {
  EpiSmem e;
  TrSmem t;
};
static_assert(sizeof(EpiSmem::Hnu) >= 3 * 64 * sizeof(float), "setup scratch of warps 1..3");

// Five blocks per SM (96 registers, a few hundred bytes of spills): a colour
// class of up to 760 sources runs in one round of blocks rather than two.
__global__ void __launch_bounds__(kTrThreads, 5) source_step_kernel(PlanView v,
                                                                    const ModelDev* __restrict__ model,
                                                                    double* delta, int32_t* status) {
  extern __shared__ double smd[];
  StepSmem& S = *reinterpret_cast<StepSmem*>(smd);
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (!v.active[j]) return;
  epilogue_source<2>(v, model, S.e, j, nullptr, v.elbo_rel, v.grad, v.hess, 0);
  __syncthreads();
  if (!tr_step_source(v, S.t, j, delta, status)) return;
  if (wid == 0) {
    if (lane < kTheta) S.e.th[lane] = (real)v.theta_trial[(size_t)j * kTheta + lane];
    __syncwarp();
    kl_terms<0>(S.e.th, model, S.e, lane);
    if (lane == 0) v.kl_trial[j] = (double)S.e.kls[0];
  } else {
    // each warp's 64 floats of the Hessian scratch, which KL_s does not use
    float* scratch = S.e.Hnu + (wid - 1) * 64;
    for (int p = v.slot_pair_ptr[j] + wid - 1; p < v.slot_pair_ptr[j + 1]; p += 3)
      setup_pair(v, model, p, true, scratch, scratch + 32, lane);
  }
}

// Slot j's value at theta_trial, from the value pass's item sums (FP64, in
// item order, lane-strided) and KL_s at theta_trial, then the accept rule;
// with flip set, an accepted source's trial render (written by the value
// pass into its other half of the render cache) becomes current.  A warp
// per slot.
__global__ void slot_finish_kernel(PlanView v, int flip, double* delta, int32_t* status) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= v.n || !v.active[j]) return;
  const int i0 = v.slot_items[j], i1 = v.slot_items[j + 1];
  double vr = 0.0;
  for (int it = i0 + lane; it < i1; it += 32) vr += (double)v.vpartials[2 * (size_t)it];
  vr = warp_sum_d(vr);
  const double rel = vr - v.kl_trial[j];
  if (lane == 0) v.rel_trial[j] = rel;
  const bool acc = accept_trial(v, j, rel, delta, status, lane);
  if (acc && flip && v.cache_half && lane == 0) v.cache_half[v.src_ids[j]] ^= 1;
}

cudaError_t launch_slot_finish(const Launch& L, const PlanView& v, bool flip_cache,
                               double* delta, int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  slot_finish_kernel<<<(v.n + 3) / 4, 128, 0, L.stream>>>(v, flip_cache ? 1 : 0, delta, status);
  return cudaGetLastError();
}

static DeviceOnce g_step_attr;

cudaError_t launch_source_step(const Launch& L, const PlanView& v, const ModelDev* model,
                               double* delta, int32_t* status) {
  if (v.n <= 0) return cudaSuccess;
  cudaError_t e = g_step_attr.run([] {
    return cudaFuncSetAttribute(source_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(StepSmem));
  });
  if (e != cudaSuccess) return e;
  source_step_kernel<<<v.n, kTrThreads, sizeof(StepSmem), L.stream>>>(v, model, delta, status);
  return cudaGetLastError();
}

}  // namespace celeste
