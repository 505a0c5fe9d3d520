// Per-(source, image) setup kernel: one warp per pair (setup.cuh), four
// pairs a block.
#include <math.h>

#include "setup.cuh"

namespace celeste {

constexpr int kSetupWarps = 4;

__global__ void __launch_bounds__(32 * kSetupWarps) setup_kernel(PlanView v,
                                                                  const ModelDev* __restrict__ model,
                                                                  int first_pair, int n_pairs,
                                                                  int use_trial) {
  __shared__ float s_th[kSetupWarps][32];    // theta, FP32
  __shared__ float s_im[kSetupWarps][32];    // PSF [k][6], then wcs_A [4], calib
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * kSetupWarps + wib;
  if (warp >= n_pairs) return;
  setup_pair(v, model, first_pair + warp, use_trial != 0, s_th[wib], s_im[wib], lane);
}

cudaError_t launch_setup(const Launch& L, const PlanView& v, const ModelDev* model,
                         int first_pair, int n_pairs, bool use_trial) {
  if (n_pairs <= 0) return cudaSuccess;
  const int blocks = (n_pairs + kSetupWarps - 1) / kSetupWarps;
  setup_kernel<<<blocks, 32 * kSetupWarps, 0, L.stream>>>(v, model, first_pair, n_pairs,
                                                          use_trial ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace celeste
