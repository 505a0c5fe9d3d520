// The trust-region subproblem of independent problems (Sec. 4.3; the solver
// is in trsolve.cuh; a Newton iteration's step runs in step.cu).
#include "device_once.h"
#include "trsolve.cuh"

namespace celeste {

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

// The dynamic shared memory limit of the trust-region kernels, once per device.
static DeviceOnce g_tr_attrs;
static cudaError_t set_attrs() {
  return g_tr_attrs.run([] {
    return cudaFuncSetAttribute(tr_subproblem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(TrSmem));
  });
}

cudaError_t launch_tr_subproblem(const Launch& L, int n, const double* g, const double* H,
                                 const double* delta, double* p, double* pred) {
  if (n <= 0) return cudaSuccess;
  if (cudaError_t e = set_attrs()) return e;
  tr_subproblem_kernel<<<n, kTrThreads, sizeof(TrSmem), L.stream>>>(n, g, H, delta, p, pred);
  return cudaGetLastError();
}

}  // namespace celeste
