// Library-internal declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/celeste.h"

namespace celeste {

constexpr int kTheta = CELESTE_N_THETA;
constexpr int kPsf = CELESTE_N_PSF;
constexpr int kMaxProf = CELESTE_MAX_PROFILE;
constexpr int kMaxColor = CELESTE_MAX_COLOR;

// ---- per-pair record written by the setup kernel -----------------------
// A "pair" is (source, image patch).  Its record is a header of brightness
// coefficients followed by one 8-float entry per Gaussian component:
// 3 star components, then per PSF component k: n_exp exponential-profile and
// n_dev de Vaucouleurs components.  Positions are local to the patch origin.
constexpr int kHdr = 16;
constexpr int kCompF = 8;
constexpr int kMaxComp = kPsf * (1 + 2 * kMaxProf);          // 51
constexpr int kRecF = kHdr + kMaxComp * kCompF;                // 424 floats
// header slots
enum : int {
  H_CE0 = 0, H_CE1, H_CM0, H_CM1, H_K0, H_K1, H_EV0, H_EV1, H_Q0, H_Q1, H_RHO, H_RHO1
};
// component slots: mean x, mean y (local), precision P11, P12, P22,
// log2(weight / (2 pi sqrt(det C))), tau (0 for the star), unused
enum : int { C_MX = 0, C_MY, C_P11, C_P12, C_P22, C_LW, C_TAU };

// ---- accumulators of one (pair, tile) work item ------------------------
// w = (cE0, cE1, cM0, cM1, mu_x, mu_y, g11, g12, g22, rho): the per-image
// natural coordinates.  Layout: value_rel, value_base, grad[10], then the
// upper triangle of the Hessian (row-major, j <= k) without the three
// (cM, cM) entries, which vanish identically.
constexpr int kW = 10;
constexpr int kAcc = 64;
constexpr int kGradAcc = 12;   // gradient-only items: value_rel, value_base, grad[10]
__host__ __device__ constexpr int hidx(int j, int k) {
  // packed upper triangle (row-major, j <= k) of the 10 x 10 Hessian, minus
  // the entries (2,2), (2,3) and (3,3), which are never stored
  return 12 + (j * kW - (j * (j - 1)) / 2 + (k - j)) - (j == 2 ? 2 : (j >= 3 ? 3 : 0));
}

struct PairInfo {
  int32_t source;      // source id
  int32_t slot;        // plan slot of the owning source, -1 for neighbour pairs
  int32_t patch;
  int32_t image;
  int32_t x0, y0, w, h;
  int64_t pix_base;    // index of pixel (x0, y0) in the pixel pool
  int32_t stride;
  int32_t band;
  int64_t bg_base;     // own pairs: offset in the plan's background pool
  int32_t nbr_begin, nbr_end;  // own pairs: neighbour pairs in pair_nbr[]
  int32_t item_begin, item_end;
};

struct Item {
  int32_t pair;
  int32_t start;
  int32_t count;
  int32_t pad;
};

struct ModelDev {
  int32_t n_exp, n_dev, n_color, pad;
  double alpha_exp[kMaxProf], tau_exp[kMaxProf], alpha_dev[kMaxProf], tau_dev[kMaxProf];
  double prior_a;
  double prior_r[2][2];
  double color_w[2][kMaxColor];
  double color_mean[2][kMaxColor][4];
  double color_prec[2][kMaxColor][4][4];   // inverse covariances
  double color_logdet[2][kMaxColor];
  double e_radius[2], e_profile[2], e_axis[2];
  // constants of the KL terms, precomputed on the host
  double log_color_w[2][kMaxColor];
  double log_prior_a, log1m_prior_a, logit_prior_a;
  double log_prior_r2[2];
  double half_log_2pi_e2;          // 0.5 log(2 pi E_radius,2)
  double log_beta_axis, log_beta_profile;
  // FP32 copies of what the KL terms of the epilogue read (that arithmetic
  // is FP32; the host rounds each to nearest, as a device conversion would)
  struct F32 {
    float tau_exp[kMaxProf], tau_dev[kMaxProf];
    float prior_r[2][2];
    float color_mean[2][kMaxColor][4];
    float color_prec[2][kMaxColor][4][4];
    float color_logdet[2][kMaxColor], log_color_w[2][kMaxColor];
    float e_radius[2], e_profile[2], e_axis[2];
    float log_prior_a, log1m_prior_a, logit_prior_a, log_prior_r2[2], half_log_2pi_e2;
    float log_beta_axis, log_beta_profile;
  } f;
};

// Validates *m and fills *md (colour precisions, log-determinants and the KL
// constants).  Returns false for an invalid model.
bool prepare_model(const celeste_model* m, ModelDev* md);

// Everything a kernel needs about a plan, by value.
struct PlanView {
  const float* pixels;
  const float* sky;
  const celeste_image* images;
  double* theta;              // problem theta [n_sources][27]
  const int32_t* src_ids;     // [n] plan slot -> source id
  const PairInfo* pairs;      // [n_pairs]: own pairs first
  const int32_t* pair_nbr;    // neighbour pair indices per own pair
  const int32_t* slot_pair_ptr;  // [n+1] own pairs per slot
  const Item* items;          // [n_items]
  const int32_t* slot_items;  // [n+1] items of slot j: [slot_items[j], slot_items[j+1])
  float* records;             // [n_pairs][kRecF]
  float2* bg;                 // [n_bg] background (E, V) per own patch pixel
  float* partials;            // [n_items][kAcc]
  float* vpartials;           // [n_items][2]
  double* theta_trial;        // [n][27]
  double* step;               // [n][27]
  double* pred;               // [n]
  int32_t* work_ctr;          // [2] work queue of the pixel kernels (next unit, warps done;
                              //     zero between launches), or null for grid stride
  double* kl_trial;           // [n] KL_s at theta_trial (the per-source Newton step)
  double* rel_trial;          // [n] L_rel at theta_trial
  double* elbo_rel;           // [n] value at the current iterate
  double* grad;               // [n][27] scratch for newton_step
  double* hess;               // [n][27][27]
  uint8_t* active;            // [n] 1 if the slot takes part in the evaluation
  unsigned int* err;          // device error word
  float2* cache;              // problem render cache (pool layout) or null
  uint8_t* cache_half;        // [n_sources] half of the cache holding each source's
                              //     current moments (two halves of cache_n_pool), or null
  int64_t cache_n_pool;       // float2 per half
  float2* trial_render;       // [n_bg] own moments at the trial point (with a cache)
  const celeste_patch* patches;  // problem patches (pool offsets)
  int32_t n, n_pairs, n_own_pairs, n_items;
  int64_t n_bg;
};

struct Launch {
  cudaStream_t stream;
  int sm_count;
  int warps_per_block;
  int blocks_per_sm;
  int pixels_per_item;
  int n_exp, n_dev;
};

// ---- kernel launchers (one per translation unit) ------------------------
// setup.cu: per-pair records; own pairs read theta_trial when use_trial.
cudaError_t launch_setup(const Launch& L, const PlanView& v, const ModelDev* model,
                         int first_pair, int n_pairs, bool use_trial);
// pixel.cu
// Measures the resident blocks per SM of the pixel kernels (once, before any
// stream capture; launches made earlier use 3 blocks per SM).
cudaError_t init_pixel_occupancy();
cudaError_t launch_background(const Launch& L, const PlanView& v);
cudaError_t launch_pixels_derivs(const Launch& L, const PlanView& v);
cudaError_t launch_pixels_grad(const Launch& L, const PlanView& v);
// keep_render (with a render cache): also store the own moments, in the
// source's other half of the cache when it has two (the accept rule then
// flips the half), else in v.trial_render (for the commit kernel)
cudaError_t launch_pixels_value(const Launch& L, const PlanView& v, bool keep_render = false);
cudaError_t launch_render(const Launch& L, const PlanView& v, float* E_out, float* V_out,
                          const celeste_patch* patches);
cudaError_t launch_background_out(const Launch& L, const PlanView& v, float* bgE, float* bgV,
                                  const celeste_patch* patches);
// Own moments of the plan's pairs into v.cache: every slot, or (status
// non-null) only slots whose source's status is CELESTE_ST_ACCEPTED, whose
// records then hold the accepted trial point.
cudaError_t launch_render_cache(const Launch& L, const PlanView& v, const int32_t* status);
// Full-field ELBO pieces: own moments added into per-image buffers (pixel
// pool layout; the plan's sources must not share pixels), the pixel term
// over every image pixel into per-block partials, and the final sums.
cudaError_t launch_accumulate(const Launch& L, const PlanView& v, float* Eimg, float* Vimg);
cudaError_t launch_field_terms(const Launch& L, const celeste_image* images, int n_images,
                               int blocks_per_image, const float* pixels, const float* sky,
                               const float* Eimg, const float* Vimg, unsigned int* err,
                               double* parts);
cudaError_t launch_field_sum(const Launch& L, const double* parts, int n_parts, const double* kl,
                             int n_kl, double* out);
// epilogue.cu: KL_s of each slot's source at theta into kl_out[source id].
cudaError_t launch_kl(const Launch& L, const PlanView& v, const ModelDev* model, double* kl_out);
// The start of a Newton iteration of a colour class in one launch: the
// active set from status, the records of pairs [0, n_setup) at theta and,
// with background (render cache only), the backgrounds of the active slots.
cudaError_t launch_prepare(const Launch& L, const PlanView& v, const ModelDev* model,
                           const int32_t* status, int n_setup, bool background);
// Copies v.trial_render into the render cache for slots whose source's
// status is CELESTE_ST_ACCEPTED.
cudaError_t launch_commit_render(const Launch& L, const PlanView& v, const int32_t* status);
// epilogue.cu
cudaError_t launch_epilogue(const Launch& L, const PlanView& v, const ModelDev* model,
                            double* elbo, double* elbo_rel, double* grad, double* hess);
cudaError_t launch_epilogue_grad(const Launch& L, const PlanView& v, const ModelDev* model,
                                 double* elbo, double* elbo_rel, double* grad);
// The pixel part of L_rel alone (no KL) into out[n].
cudaError_t launch_epilogue_loglik(const Launch& L, const PlanView& v, const ModelDev* model,
                                   double* out);
cudaError_t launch_epilogue_value(const Launch& L, const PlanView& v, const ModelDev* model,
                                  double* elbo, double* elbo_rel, bool use_trial);
// step.cu: the per-source part of a Newton iteration in one launch: the
// epilogue at theta, the trust-region step, KL_s at theta_trial and the own
// pairs' records at theta_trial.
cudaError_t launch_source_step(const Launch& L, const PlanView& v, const ModelDev* model,
                               double* delta, int32_t* status);
// step.cu: the end of the iteration, after the value pass at theta_trial:
// L_rel at theta_trial (into v.rel_trial), the accept rule and, with
// flip_cache and two render-cache halves, the accepted sources' halves.
cudaError_t launch_slot_finish(const Launch& L, const PlanView& v, bool flip_cache,
                               double* delta, int32_t* status);
// newton.cu
cudaError_t launch_tr_subproblem(const Launch& L, int n, const double* g, const double* H,
                                 const double* delta, double* p, double* pred);

// fit.cu: the region fit's per-source state (device arrays indexed by source
// id unless noted) and its bookkeeping kernels.  The region is cut into
// segments (independent requests), each with its own pass count and
// stopping decision; a region fit has one segment.
constexpr double kDelta0 = 1.0;   // initial trust radius of a subsolver call
struct FitView {
  const int32_t* region;   // [n_region] source ids, segment by segment
  const int32_t* seg_ptr;  // [n_seg + 1] segment k = region[seg_ptr[k] .. seg_ptr[k+1])
  const int32_t* seg_of;   // segment of each source id (region sources only)
  double* delta;
  int32_t* status;
  int32_t* iters_pass;     // Newton iterations in the current pass
  int32_t* iters_total;    // over all passes
  int32_t* accepted;       // accepted steps over all passes
  uint8_t* done;           // retired for the rest of the pass
  double* gain;            // summed actual gain of accepted steps this pass
  int32_t* class_iter;     // [n_classes] loop trips of each class this pass
  uint8_t* seg_active;     // [n_seg] segment takes part in the next pass
  int32_t* seg_passes;     // [n_seg] passes run
  double* seg_gain;        // [n_seg] gain of the segment's last pass
  int32_t* summary;        // [1 + n_classes]: active segments, class loop trips
  int32_t n_region, n_seg, n_classes, max_iter, max_passes;
  double pass_tol;         // a pass gaining <= pass_tol * (segment sources) ends it
};
cudaError_t launch_fit_reset(cudaStream_t stream, const FitView& f);
cudaError_t launch_fit_check(cudaStream_t stream, const PlanView& v, const FitView& f,
                             const double* rel_trial, int cls, cudaGraphConditionalHandle h);
cudaError_t launch_fit_pass_end(cudaStream_t stream, const FitView& f);

// ---- small device helpers ----------------------------------------------
__device__ __forceinline__ void set_error(unsigned int* err, unsigned int bit) {
  atomicOr(err, bit);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A slot takes part in a Newton iteration unless its source has stopped.
__device__ __forceinline__ uint8_t active_of(int32_t st) {
  return (st == CELESTE_ST_CONVERGED || st == CELESTE_ST_FAILED || st == CELESTE_ST_MAXITER) ? 0
                                                                                             : 1;
}

// Offset of source s's current half of the render cache.
__device__ __forceinline__ int64_t cache_base(const PlanView& v, int s) {
  return v.cache_half && v.cache_half[s] ? v.cache_n_pool : 0;
}

// Bilinear sky at pixel (x, y) of image `im` (knots span the image).
__device__ __forceinline__ float sky_value(const celeste_image& im, const float* sky, float x,
                                           float y) {
  const float* k = sky + im.sky_offset;
  const int nx = im.sky_nx, ny = im.sky_ny;
  if (nx == 1 && ny == 1) return k[0];
  float gx = nx > 1 ? x * (float)(nx - 1) / (float)max(im.width - 1, 1) : 0.f;
  float gy = ny > 1 ? y * (float)(ny - 1) / (float)max(im.height - 1, 1) : 0.f;
  int ix = min(max((int)floorf(gx), 0), max(nx - 2, 0));
  int iy = min(max((int)floorf(gy), 0), max(ny - 2, 0));
  float fx = gx - (float)ix, fy = gy - (float)iy;
  int ix1 = min(ix + 1, nx - 1), iy1 = min(iy + 1, ny - 1);
  float a = k[iy * nx + ix], b = k[iy * nx + ix1], c = k[iy1 * nx + ix], d = k[iy1 * nx + ix1];
  return (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
}

}  // namespace celeste
