// Host-side objects behind the C ABI (contexts, plans, fits) and the helpers
// the translation units that orchestrate kernels share.  Private to the
// library.
#pragma once

#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

#define CK(call)                                \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return CELESTE_ECUDA; \
  } while (0)

namespace celeste {
// Device and pinned host memory of plans and fits, cached per context.
// Building plans and fits over and over (a server that admits requests
// between passes) would otherwise pay a cudaMalloc/cudaFree pair per buffer,
// and cudaFree waits for the device.  A freed block returns to its context
// once the context's stream has finished with it, and a later request of at
// least half its size takes it back.  Blocks go back to CUDA when the
// context is destroyed.
class MemPool {
 public:
  void* get(bool host, size_t bytes);
  void put(bool host, void* ptr);
  void release_all();

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_[2];
  std::unordered_map<void*, size_t> size_[2];
};
}  // namespace celeste

struct celeste_ctx {
  int device = 0;
  uint64_t serial = 0;               // registry key (contexts outlived by plans)
  celeste::MemPool pool;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  celeste::ModelDev* d_model = nullptr;
  unsigned int* d_err = nullptr;
  int n_exp = 0, n_dev = 0;
  int64_t launches = 0;
  // event timing of kernel launches by kind (celeste_profile_*)
  unsigned profiling = 0;            // bit k: time kernels of kind k
  std::vector<cudaEvent_t> events;   // start/stop pairs, reused
  std::vector<int> kinds;            // kind of pair k
  std::vector<int64_t> visits;       // visits of pair k (pixel kernels)
  size_t n_timed = 0;                // pairs recorded since the last reset
};

struct celeste_plan {
  celeste_ctx* ctx = nullptr;
  uint64_t ctx_serial = 0;
  celeste::PlanView v{};
  const celeste_patch* d_patches = nullptr;
  double* rel_trial = nullptr;
  std::vector<void*> allocs;
  int64_t visits = 0;
  celeste_tuning tuning{};
};

struct celeste_fit {
  celeste_ctx* ctx = nullptr;
  uint64_t ctx_serial = 0;
  std::vector<int32_t> region;              // source ids, segment by segment
  std::vector<int32_t> seg_ptr;             // [n_seg + 1] into region
  std::vector<celeste_plan*> plans;         // one per colour class
  celeste_plan* outside = nullptr;          // neighbours outside the region (render cache)
  std::vector<void*> allocs;                // device blocks (context pool)
  std::vector<void*> host_allocs;           // pinned host blocks (context pool)
  celeste::FitView f{};
  // pinned host copies read after each pass
  int32_t* h_summary = nullptr;             // [1 + n_classes]
  uint8_t* h_seg_active = nullptr;          // [n_seg]
  double* h_seg_gain = nullptr;             // [n_seg]
  int32_t* h_seg_passes = nullptr;          // [n_seg]
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int built_max_iter = 0, built_max_passes = 0;
  double built_pass_tol = -1.0;
  int n_sources = 0;
};

namespace celeste {

// Memory of a plan or fit: from its context's pool while the context lives.
void* ctx_alloc(celeste_ctx* c, bool host, size_t bytes);
// Returns blocks taken with ctx_alloc: to the pool of the context with the
// given serial if it still exists (after its stream has finished with
// them), else to CUDA.
void ctx_release(celeste_ctx* c, uint64_t serial, bool host, const std::vector<void*>& blocks);

// Launch configuration of a plan's kernels on the context's stream.
Launch make_launch(const celeste_ctx* c, const celeste_plan* p);

// One trust-region Newton iteration of the plan's active sources, once the
// neighbour records and background are in place (kIterationLaunches - 1
// kernels; the fit adds its check kernel).
cudaError_t enqueue_iteration(celeste_ctx* c, celeste_plan* p, const Launch& L, double* delta,
                              int32_t* status);
constexpr int kIterationLaunches = 6;

// A fit over region sources cut into segments (independent requests):
// ids[seg_ptr[k] .. seg_ptr[k+1]) is segment k; no source may have a
// neighbour in another segment for the segments to be independent.
int fit_create_segments(celeste_ctx* c, const celeste_problem* pr, const int32_t* ids, int n,
                        const int32_t* seg_ptr, int n_seg, const celeste_tuning* tuning,
                        celeste_fit** out);
// Prepares a run (graph for these limits, every segment active).
int fit_begin(celeste_ctx* c, celeste_fit* F, int max_passes, int max_iter, double pass_tol);
// Runs one pass of every active segment and waits for it; *n_active is the
// number of segments that run another pass.  The pinned h_* arrays of F
// then hold each segment's state.  fit_pass_launch queues the pass and the
// copies of the segment state (returning at once); fit_pass_finish waits
// for them.
int fit_pass(celeste_ctx* c, celeste_fit* F, int* n_active);
int fit_pass_launch(celeste_ctx* c, celeste_fit* F);
int fit_pass_finish(celeste_ctx* c, celeste_fit* F, int* n_active);

}  // namespace celeste
