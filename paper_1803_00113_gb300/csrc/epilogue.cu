// Per-source epilogue kernels (epilogue.cuh): reduce a source's tile sums,
// chain them to the 27 coordinates and add the KL term.
#include "device_once.h"
#include "epilogue.cuh"

namespace celeste {

template <int kMode>
__global__ void __launch_bounds__(kEpiThreads) epilogue_kernel(PlanView v,
                                                               const ModelDev* __restrict__ model,
                                                               double* elbo, double* elbo_rel,
                                                               double* grad_out, double* hess_out,
                                                               int use_trial) {
  extern __shared__ double smd[];
  epilogue_source<kMode>(v, model, *reinterpret_cast<EpiSmem*>(smd), blockIdx.x, elbo, elbo_rel,
                         grad_out, hess_out, use_trial);
}

// The dynamic shared memory limit of each epilogue kernel, once per device.
template <int kMode>
static cudaError_t set_smem_attr() {
  static DeviceOnce once;
  return once.run([] {
    return cudaFuncSetAttribute(epilogue_kernel<kMode>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EpiSmem));
  });
}

cudaError_t launch_epilogue(const Launch& L, const PlanView& v, const ModelDev* model,
                            double* elbo, double* elbo_rel, double* grad, double* hess) {
  if (v.n == 0) return cudaSuccess;
  if (cudaError_t e = set_smem_attr<2>()) return e;
  epilogue_kernel<2><<<v.n, kEpiThreads, sizeof(EpiSmem), L.stream>>>(v, model, elbo, elbo_rel, grad,
                                                              hess, 0);
  return cudaGetLastError();
}

cudaError_t launch_epilogue_grad(const Launch& L, const PlanView& v, const ModelDev* model,
                                 double* elbo, double* elbo_rel, double* grad) {
  if (v.n == 0) return cudaSuccess;
  if (cudaError_t e = set_smem_attr<1>()) return e;
  epilogue_kernel<1><<<v.n, kEpiThreads, sizeof(EpiSmem), L.stream>>>(v, model, elbo, elbo_rel, grad,
                                                              nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_epilogue_value(const Launch& L, const PlanView& v, const ModelDev* model,
                                  double* elbo, double* elbo_rel, bool use_trial) {
  if (v.n == 0) return cudaSuccess;
  if (cudaError_t e = set_smem_attr<0>()) return e;
  epilogue_kernel<0><<<v.n, kEpiThreads, sizeof(EpiSmem), L.stream>>>(v, model, elbo, elbo_rel, nullptr,
                                                              nullptr, use_trial ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_epilogue_loglik(const Launch& L, const PlanView& v, const ModelDev* model,
                                   double* out) {
  if (v.n == 0) return cudaSuccess;
  if (cudaError_t e = set_smem_attr<0>()) return e;
  epilogue_kernel<0><<<v.n, kEpiThreads, sizeof(EpiSmem), L.stream>>>(v, model, nullptr, out,
                                                                      nullptr, nullptr, 2);
  return cudaGetLastError();
}

// KL_s of every slot's source at theta, into kl_out[source id] (for the
// full-field ELBO, Eq. elbo: the pixel sum minus the sum of the KL_s).
__global__ void kl_kernel(PlanView v, const ModelDev* __restrict__ model, double* kl_out) {
  extern __shared__ double smd[];
  EpiSmem& S = *reinterpret_cast<EpiSmem*>(smd);
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  const int src = v.src_ids[j];
  if (lane < kTheta) S.th[lane] = (real)v.theta[(size_t)src * kTheta + lane];
  __syncwarp();
  kl_terms<0>(S.th, model, S, lane);
  __syncwarp();
  if (lane == 0) kl_out[src] = (double)S.kls[0];
}

cudaError_t launch_kl(const Launch& L, const PlanView& v, const ModelDev* model, double* kl_out) {
  if (v.n == 0) return cudaSuccess;
  static DeviceOnce once;
  cudaError_t e = once.run([] {
    return cudaFuncSetAttribute(kl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(EpiSmem));
  });
  if (e != cudaSuccess) return e;
  kl_kernel<<<v.n, 32, sizeof(EpiSmem), L.stream>>>(v, model, kl_out);
  return cudaGetLastError();
}

}  // namespace celeste
