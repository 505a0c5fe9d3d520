// celeste_elbo_grad_hess_noalloc: the ELBO, gradient and Hessian of a few
// sources without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc -- code running while a
// memory pool is locked or being defragmented, plugins of a host program that
// owns every device allocation, and callers that cannot pay the latency or
// synchronisation of an allocation in the middle of their work.  Such
// callers cannot create a context or a plan (both allocate), so this entry
// point takes the model and the problem directly and keeps every intermediate
// (work decomposition, component tables, background, per-tile sums) in one
// file-scope device array of fixed size, CELESTE_NOALLOC_BYTES.  Each GPU
// that loads the library holds that array until the process exits.
//
// The kernels are the ones celeste_elbo_grad_hess runs, with the work
// decomposition of a plan made with the default tiles (256 pixels per item)
// and no render cache, so the outputs agree with it.
#include <math.h>
#include <string.h>

#include "device_once.h"
#include "internal.cuh"

using namespace celeste;

namespace {

constexpr size_t kScratchBytes = CELESTE_NOALLOC_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side limits of the work decomposition, staged in static host arrays
// (no heap either).
constexpr int kMaxSlots = CELESTE_NOALLOC_MAX_SOURCES;
constexpr int kMaxPairs = 4096;
constexpr int kMaxItems = 32768;
constexpr int kMaxNbrRefs = 16384;
constexpr int kPixelsPerItem = 256;   // the default tile of celeste_plan_create

struct DeviceSetup {
  unsigned char* scratch;   // device address of g_noalloc_scratch on this device
  int sm_count;
};
static DeviceSetup g_setup[kMaxDevices];
static DeviceOnce g_setup_once;

// host staging of one call
static PairInfo h_pairs[kMaxPairs];
static Item h_items[kMaxItems];
static int32_t h_nbr[kMaxNbrRefs];
static int32_t h_slot[kMaxSlots + 1];
static int32_t h_ids[kMaxSlots];
static ModelDev h_model;

// Neighbour pairs already laid out in this call, keyed by (source, patch):
// open addressing over twice kMaxPairs slots; a slot belongs to this call
// when its stamp equals the call's.
constexpr int kPairSlots = 2 * kMaxPairs;
static uint64_t h_key[kPairSlots];
static uint32_t h_stamp[kPairSlots];
static int32_t h_index[kPairSlots];
static uint32_t g_call = 0;

int* pair_slot(int32_t source, int32_t patch, bool* found) {
  const uint64_t key = ((uint64_t)(uint32_t)source << 32) | (uint32_t)patch;
  uint64_t h = key * 0x9E3779B97F4A7C15ull;
  for (uint32_t i = (uint32_t)(h >> 40) % kPairSlots;; i = (i + 1) % kPairSlots) {
    if (h_stamp[i] != g_call) {
      h_stamp[i] = g_call;
      h_key[i] = key;
      *found = false;
      return &h_index[i];
    }
    if (h_key[i] == key) {
      *found = true;
      return &h_index[i];
    }
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Once per device, with that device current: the device address of the
// scratch array (the array's name in host code is only a stand-in), the SM
// count and the pixel kernels' occupancy.
int device_setup(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= kMaxDevices) return CELESTE_EINVAL;
  DeviceSetup& d = g_setup[dev];
  const cudaError_t e = g_setup_once.run([&] {
    void* ptr = nullptr;
    cudaError_t r = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (r == cudaSuccess && ptr == nullptr) r = cudaErrorInvalidSymbol;
    int sms = 0;
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (r == cudaSuccess) r = init_pixel_occupancy();
    if (r == cudaSuccess) {
      d.scratch = static_cast<unsigned char*>(ptr);
      d.sm_count = sms;
    }
    return r;
  });
  if (e != cudaSuccess) return CELESTE_ECUDA;
  *out = &d;
  return CELESTE_OK;
}

}  // namespace

extern "C" int celeste_elbo_grad_hess_noalloc(const celeste_model* model,
                                              const celeste_problem* pr,
                                              const int32_t* ids, int32_t n, void* cuda_stream,
                                              double* elbo, double* elbo_rel, double* grad,
                                              double* hess, uint32_t* device_error) {
  if (!model || !pr || n < 0 || (n > 0 && (!ids || !elbo || !grad || !hess))) return CELESTE_EINVAL;
  if (!pr->h_patch_ptr || !pr->h_patches || !pr->h_images || !pr->h_nbr_ptr ||
      (pr->n_nbr > 0 && !pr->h_nbr_idx) || !pr->pixels || !pr->sky || !pr->images || !pr->theta)
    return CELESTE_EINVAL;
  if (n > kMaxSlots) return CELESTE_ETOOLARGE;
  if (!prepare_model(model, &h_model)) return CELESTE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CELESTE_ECUDA;
  DeviceSetup* ds = nullptr;
  int rc = device_setup(dev, &ds);
  if (rc) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // The work decomposition is staged from host arrays that the next call
  // overwrites, so work recorded for later replay would upload whatever the
  // last call left there: refuse a stream that is being captured.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return CELESTE_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return CELESTE_EINVAL;

  // ---- work decomposition (same rules and order as celeste_plan_create)
  for (int j = 0; j < n; ++j) {
    if (ids[j] < 0 || ids[j] >= pr->n_sources) return CELESTE_EINVAL;
    for (int k = 0; k < j; ++k)
      if (ids[k] == ids[j]) return CELESTE_EINVAL;
    h_ids[j] = ids[j];
  }
  auto patch_ok = [&](const celeste_patch& q) {
    if (q.image < 0 || q.image >= pr->n_images) return false;
    const celeste_image& im = pr->h_images[q.image];
    return q.w > 0 && q.h > 0 && q.x0 >= 0 && q.y0 >= 0 && q.x0 + q.w <= im.width &&
           q.y0 + q.h <= im.height;
  };
  int np = 0, ni = 0, nn = 0;
  int64_t bg = 0;
  h_slot[0] = 0;
  for (int j = 0; j < n; ++j) {
    const int s = ids[j];
    for (int q = pr->h_patch_ptr[s]; q < pr->h_patch_ptr[s + 1]; ++q) {
      const celeste_patch& P = pr->h_patches[q];
      if (!patch_ok(P)) return CELESTE_EINVAL;
      if (np >= kMaxPairs) return CELESTE_ETOOLARGE;
      const celeste_image& im = pr->h_images[P.image];
      PairInfo pi;
      memset(&pi, 0, sizeof(pi));
      pi.source = s;
      pi.slot = j;
      pi.patch = q;
      pi.image = P.image;
      pi.x0 = P.x0;
      pi.y0 = P.y0;
      pi.w = P.w;
      pi.h = P.h;
      pi.pix_base = im.pix_offset + (int64_t)P.y0 * im.row_stride + P.x0;
      pi.stride = im.row_stride;
      pi.band = im.band;
      pi.bg_base = bg;
      const int area = P.w * P.h;
      bg += area;
      pi.item_begin = ni;
      for (int st = 0; st < area; st += kPixelsPerItem) {
        if (ni >= kMaxItems) return CELESTE_ETOOLARGE;
        h_items[ni++] = Item{np, st, area - st < kPixelsPerItem ? area - st : kPixelsPerItem, 0};
      }
      pi.item_end = ni;
      h_pairs[np++] = pi;
    }
    h_slot[j + 1] = np;
  }
  const int n_own = np;
  if (++g_call == 0) {              // stamps wrapped: forget every slot
    memset(h_stamp, 0, sizeof(h_stamp));
    g_call = 1;
  }
  for (int pp = 0; pp < n_own; ++pp) {
    const PairInfo pi = h_pairs[pp];
    h_pairs[pp].nbr_begin = nn;
    for (int k = pr->h_nbr_ptr[pi.source]; k < pr->h_nbr_ptr[pi.source + 1]; ++k) {
      const int t = pr->h_nbr_idx[k];
      if (t < 0 || t >= pr->n_sources) return CELESTE_EINVAL;
      for (int q = pr->h_patch_ptr[t]; q < pr->h_patch_ptr[t + 1]; ++q) {
        const celeste_patch& P = pr->h_patches[q];
        if (P.image != pi.image) continue;
        if (!patch_ok(P)) return CELESTE_EINVAL;
        if (P.x0 >= pi.x0 + pi.w || pi.x0 >= P.x0 + P.w || P.y0 >= pi.y0 + pi.h ||
            pi.y0 >= P.y0 + P.h)
          continue;
        bool found = false;
        int* slot = pair_slot(t, q, &found);
        int idx = found ? *slot : -1;
        if (idx < 0) {
          if (np >= kMaxPairs) return CELESTE_ETOOLARGE;
          const celeste_image& im = pr->h_images[P.image];
          PairInfo qn;
          memset(&qn, 0, sizeof(qn));
          qn.source = t;
          qn.slot = -1;
          qn.patch = q;
          qn.image = P.image;
          qn.x0 = P.x0;
          qn.y0 = P.y0;
          qn.w = P.w;
          qn.h = P.h;
          qn.pix_base = im.pix_offset + (int64_t)P.y0 * im.row_stride + P.x0;
          qn.stride = im.row_stride;
          qn.band = im.band;
          qn.bg_base = -1;
          idx = np;
          *slot = idx;
          h_pairs[np++] = qn;
        }
        if (nn >= kMaxNbrRefs) return CELESTE_ETOOLARGE;
        h_nbr[nn++] = idx;
      }
    }
    h_pairs[pp].nbr_end = nn;
  }

  // ---- carve the scratch array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + (bytes ? bytes : 1));
    return at;
  };
  const size_t o_err = take(sizeof(unsigned int));
  const size_t o_model = take(sizeof(ModelDev));
  const size_t o_ids = take(sizeof(int32_t) * (size_t)n);
  const size_t o_pairs = take(sizeof(PairInfo) * (size_t)np);
  const size_t o_nbr = take(sizeof(int32_t) * (size_t)nn);
  const size_t o_slot = take(sizeof(int32_t) * (size_t)(n + 1));
  const size_t o_items = take(sizeof(Item) * (size_t)ni);
  const size_t o_rec = take(sizeof(float) * (size_t)np * kRecF);
  const size_t o_bg = take(sizeof(float2) * (size_t)bg);
  const size_t o_part = take(sizeof(float) * (size_t)ni * kAcc);
  const size_t o_active = take((size_t)n);
  if (off > kScratchBytes) return CELESTE_ETOOLARGE;
  unsigned char* S = ds->scratch;

  // ---- stage inputs; clear what must start at zero (the error word) and
  // set the active flags (the array keeps the previous call's contents)
  if (n == 0) return CELESTE_OK;
  cudaError_t e = cudaMemsetAsync(S + o_err, 0, sizeof(unsigned int), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + o_active, 1, (size_t)n, stream);
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes)
      e = cudaMemcpyAsync(S + o, src, bytes, cudaMemcpyHostToDevice, stream);
  };
  put(o_model, &h_model, sizeof(ModelDev));
  put(o_ids, h_ids, sizeof(int32_t) * (size_t)n);
  put(o_pairs, h_pairs, sizeof(PairInfo) * (size_t)np);
  put(o_nbr, h_nbr, sizeof(int32_t) * (size_t)nn);
  put(o_slot, h_slot, sizeof(int32_t) * (size_t)(n + 1));
  put(o_items, h_items, sizeof(Item) * (size_t)ni);
  if (e != cudaSuccess) return CELESTE_ECUDA;

  PlanView v;
  memset(&v, 0, sizeof(v));
  v.pixels = pr->pixels;
  v.sky = pr->sky;
  v.images = pr->images;
  v.theta = pr->theta;
  v.src_ids = reinterpret_cast<const int32_t*>(S + o_ids);
  v.pairs = reinterpret_cast<const PairInfo*>(S + o_pairs);
  v.pair_nbr = reinterpret_cast<const int32_t*>(S + o_nbr);
  v.slot_pair_ptr = reinterpret_cast<const int32_t*>(S + o_slot);
  v.items = reinterpret_cast<const Item*>(S + o_items);
  v.records = reinterpret_cast<float*>(S + o_rec);
  v.bg = reinterpret_cast<float2*>(S + o_bg);
  v.partials = reinterpret_cast<float*>(S + o_part);
  v.active = S + o_active;
  v.err = reinterpret_cast<unsigned int*>(S + o_err);
  v.cache = nullptr;            // backgrounds are always rendered here
  v.trial_render = nullptr;
  v.patches = pr->patches;
  v.n = n;
  v.n_pairs = np;
  v.n_own_pairs = n_own;
  v.n_items = ni;
  v.n_bg = bg;
  const ModelDev* d_model = reinterpret_cast<const ModelDev*>(S + o_model);

  Launch L;
  L.stream = stream;
  L.sm_count = ds->sm_count;
  L.warps_per_block = 4;
  L.blocks_per_sm = 0;            // each kernel's measured occupancy
  L.pixels_per_item = kPixelsPerItem;
  L.n_exp = model->n_exp;
  L.n_dev = model->n_dev;
  e = launch_setup(L, v, d_model, 0, np, false);
  if (e == cudaSuccess) e = launch_background(L, v);
  if (e == cudaSuccess) e = launch_pixels_derivs(L, v);
  if (e == cudaSuccess) e = launch_epilogue(L, v, d_model, elbo, elbo_rel, grad, hess);
  if (e == cudaSuccess && device_error)
    e = cudaMemcpyAsync(device_error, S + o_err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream);
  return e == cudaSuccess ? CELESTE_OK : CELESTE_ECUDA;
}
