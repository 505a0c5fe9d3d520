// Serving: region fits submitted by independent callers, batched on the GPU.
//
// A request is a small problem of its own (a sky region: its exposures and
// the sources in it).  celeste_submit validates it, copies it and queues it;
// worker threads (each with its own context, stream and resident buffers)
// take every queued request that fits their device budget, lay the batch out
// as one problem (the requests' images, patches and sources concatenated),
// and run one segmented fit over it: each request is a segment with its own
// pass count and stopping rule, so its result does not depend on what it
// was batched with.  A request completes when its segment stops, possibly
// before the rest of its batch; celeste_poll returns its result.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "host.h"

using namespace celeste;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  std::vector<float> pixels, sky;
  std::vector<celeste_image> images;
  std::vector<double> theta;
  std::vector<int32_t> patch_ptr, nbr_ptr, nbr_idx;
  std::vector<celeste_patch> patches;
  int n_sources = 0;
  int64_t bytes = 0;                 // device footprint estimate
  // result
  std::vector<double> theta_out;
  std::vector<int32_t> status_out;
  int passes = 0;
  double last_gain = 0.0;
  int state = 0;                     // 0 queued, 1 running, 2 done
  int error = CELESTE_OK;
  uint32_t device_error = 0;
  int batch_requests = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// Grow-only device and pinned host buffers of a worker.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20) + bytes / 4;
    if (cudaMalloc(&p, want) != cudaSuccess) return false;
    cap = want;
    return true;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20) + bytes / 4;
    if (cudaMallocHost(&p, want) != cudaSuccess) return false;
    cap = want;
    return true;
  }
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
};

enum { kPix, kSky, kImg, kTheta, kPatchPtr, kPatch, kNbrPtr, kNbrIdx, kStatus, kCache, kBufs };

}  // namespace

struct celeste_server {
  celeste_model model{};
  int device = 0;
  celeste_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
  uint64_t next_ticket = 1;
  int64_t queued_bytes = 0;
  bool stop = false, paused = false;
  int worker_error = CELESTE_OK;
  int64_t launches = 0, batches = 0;
  std::vector<std::thread> workers;
};

namespace {

// Device footprint of a request: its arrays, plus the plan scratch (records
// per source-image pair, background and tile sums per patch pixel, Newton
// state per source).
int64_t footprint(const Request& r) {
  int64_t visits = 0;
  for (const celeste_patch& q : r.patches) visits += (int64_t)q.w * q.h;
  const int64_t pairs = (int64_t)r.patches.size() * (1 + (int64_t)r.nbr_idx.size() /
                                                             std::max(r.n_sources, 1));
  return 4 * ((int64_t)r.pixels.size() + (int64_t)r.sky.size()) + 256 * (int64_t)r.images.size() +
         32 * (int64_t)r.patches.size() + 12 * visits + 1792 * pairs + 16384 * (int64_t)r.n_sources;
}

// Runs one batch on a worker's context.  Returns an error code for the whole
// batch (the requests then complete with it).
int run_batch(celeste_server* S, celeste_ctx* ctx, cudaStream_t stream,
              std::vector<std::shared_ptr<Request>>& batch, DevBuf* dev, HostBuf* host) {
  const int R = (int)batch.size();
  int64_t n_pix = 0, n_sky = 0;
  int n_img = 0, n_src = 0, n_patch = 0, n_nbr = 0;
  int64_t n_pool = 0;
  for (auto& r : batch) {
    for (const celeste_patch& q : r->patches) n_pool += (int64_t)q.w * q.h;
    n_pix += (int64_t)r->pixels.size();
    n_sky += (int64_t)r->sky.size();
    n_img += (int)r->images.size();
    n_src += r->n_sources;
    n_patch += (int)r->patches.size();
    n_nbr += (int)r->nbr_idx.size();
  }
  const size_t bytes[kBufs] = {(size_t)n_pix * 4,          (size_t)n_sky * 4,
                               (size_t)n_img * sizeof(celeste_image),
                               (size_t)n_src * CELESTE_N_THETA * 8,
                               (size_t)(n_src + 1) * 4,     (size_t)n_patch * sizeof(celeste_patch),
                               (size_t)(n_src + 1) * 4,     (size_t)n_nbr * 4,
                               (size_t)n_src * 4,           (size_t)n_pool * 8};
  for (int k = 0; k < kBufs; ++k)
    if (!dev[k].reserve(bytes[k]) || (k != kCache && !host[k].reserve(bytes[k])))
      return CELESTE_ENOMEM;
  float* h_pix = static_cast<float*>(host[kPix].p);
  float* h_sky = static_cast<float*>(host[kSky].p);
  celeste_image* h_img = static_cast<celeste_image*>(host[kImg].p);
  double* h_theta = static_cast<double*>(host[kTheta].p);
  int32_t* h_pp = static_cast<int32_t*>(host[kPatchPtr].p);
  celeste_patch* h_patch = static_cast<celeste_patch*>(host[kPatch].p);
  int32_t* h_np = static_cast<int32_t*>(host[kNbrPtr].p);
  int32_t* h_ni = static_cast<int32_t*>(host[kNbrIdx].p);
  // concatenate: offsets of pixels, sky, images, sources and patches shift
  std::vector<int32_t> seg_ptr(R + 1, 0), src_first(R, 0);
  int64_t op = 0, os = 0, opool = 0;
  int oi = 0, osrc = 0, opatch = 0, onbr = 0;
  h_pp[0] = 0;
  h_np[0] = 0;
  for (int k = 0; k < R; ++k) {
    const Request& r = *batch[k];
    memcpy(h_pix + op, r.pixels.data(), r.pixels.size() * 4);
    memcpy(h_sky + os, r.sky.data(), r.sky.size() * 4);
    for (size_t i = 0; i < r.images.size(); ++i) {
      celeste_image im = r.images[i];
      im.pix_offset += op;
      im.sky_offset += os;
      h_img[oi + i] = im;
    }
    memcpy(h_theta + (size_t)osrc * CELESTE_N_THETA, r.theta.data(), r.theta.size() * 8);
    for (int s = 0; s < r.n_sources; ++s) {
      h_pp[osrc + s + 1] = opatch + r.patch_ptr[s + 1];
      h_np[osrc + s + 1] = onbr + r.nbr_ptr[s + 1];
    }
    for (size_t q = 0; q < r.patches.size(); ++q) {
      celeste_patch P = r.patches[q];
      P.image += oi;
      P.pool_offset = opool;
      opool += (int64_t)P.w * P.h;
      h_patch[opatch + q] = P;
    }
    for (size_t q = 0; q < r.nbr_idx.size(); ++q) h_ni[onbr + q] = r.nbr_idx[q] + osrc;
    src_first[k] = osrc;
    op += (int64_t)r.pixels.size();
    os += (int64_t)r.sky.size();
    oi += (int)r.images.size();
    osrc += r.n_sources;
    opatch += (int)r.patches.size();
    onbr += (int)r.nbr_idx.size();
    seg_ptr[k + 1] = osrc;
  }
  for (int k = 0; k < kStatus; ++k)
    if (bytes[k]) CK(cudaMemcpyAsync(dev[k].p, host[k].p, bytes[k], cudaMemcpyHostToDevice, stream));
  celeste_problem P{};
  P.pixels = static_cast<const float*>(dev[kPix].p);
  P.sky = static_cast<const float*>(dev[kSky].p);
  P.images = static_cast<const celeste_image*>(dev[kImg].p);
  P.theta = static_cast<double*>(dev[kTheta].p);
  P.patch_ptr = static_cast<const int32_t*>(dev[kPatchPtr].p);
  P.patches = static_cast<const celeste_patch*>(dev[kPatch].p);
  P.nbr_ptr = static_cast<const int32_t*>(dev[kNbrPtr].p);
  P.nbr_idx = static_cast<const int32_t*>(dev[kNbrIdx].p);
  P.h_patch_ptr = h_pp;
  P.h_patches = h_patch;
  P.h_images = h_img;
  P.h_nbr_ptr = h_np;
  P.h_nbr_idx = h_ni;
  P.n_pixels = n_pix;
  P.n_sky = n_sky;
  P.n_pool = n_pool;
  P.render_cache = static_cast<float*>(dev[kCache].p);
  P.n_images = n_img;
  P.n_sources = n_src;
  P.n_patches = n_patch;
  P.n_nbr = n_nbr;
  std::vector<int32_t> ids(n_src);
  for (int s = 0; s < n_src; ++s) ids[s] = s;
  celeste_fit* F = nullptr;
  celeste_tuning tuning{};
  tuning.pixels_per_item = S->cfg.pixels_per_item;
  int rc = fit_create_segments(ctx, &P, ids.data(), n_src, seg_ptr.data(), R, &tuning, &F);
  if (rc) return rc;
  rc = fit_begin(ctx, F, S->cfg.max_passes, S->cfg.max_iter, S->cfg.pass_tol);
  std::vector<char> finished(R, 0);
  double* h_th = static_cast<double*>(host[kTheta].p);
  int32_t* h_st = static_cast<int32_t*>(host[kStatus].p);
  const int64_t l0 = ctx ? celeste_launch_count(ctx) : 0;
  int active = R, guard = 0;
  while (rc == CELESTE_OK && active > 0 && guard++ < F->f.max_passes) {
    rc = fit_pass(ctx, F, &active);
    if (rc) break;
    // read back every request whose segment just stopped
    std::vector<int> now_done;
    for (int k = 0; k < R; ++k)
      if (!finished[k] && (!F->h_seg_active[k] || active == 0)) now_done.push_back(k);
    for (int k : now_done) {
      const Request& r = *batch[k];
      const size_t o = (size_t)src_first[k];
      rc = cudaMemcpyAsync(h_th + o * CELESTE_N_THETA, P.theta + o * CELESTE_N_THETA,
                           (size_t)r.n_sources * CELESTE_N_THETA * 8, cudaMemcpyDeviceToHost,
                           stream) == cudaSuccess &&
                   cudaMemcpyAsync(h_st + o, F->f.status + o, (size_t)r.n_sources * 4,
                                   cudaMemcpyDeviceToHost, stream) == cudaSuccess
               ? CELESTE_OK
               : CELESTE_ECUDA;
      if (rc) break;
    }
    if (rc == CELESTE_OK && !now_done.empty()) {
      uint32_t word = 0;
      const int sync = celeste_synchronize(ctx, &word);
      const double t = now_s();
      std::lock_guard<std::mutex> lk(S->mu);
      for (int k : now_done) {
        Request& r = *batch[k];
        const size_t o = (size_t)src_first[k];
        r.theta_out.assign(h_th + o * CELESTE_N_THETA, h_th + (o + r.n_sources) * CELESTE_N_THETA);
        r.status_out.assign(h_st + o, h_st + o + r.n_sources);
        r.passes = F->h_seg_passes[k];
        r.last_gain = F->h_seg_gain[k];
        r.batch_requests = R;
        r.error = sync;
        r.device_error = word;
        r.t_done = t;
        r.state = 2;
        finished[k] = 1;
      }
      S->cv_done.notify_all();
    }
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->launches += celeste_launch_count(ctx) - l0;
    ++S->batches;
  }
  celeste_fit_destroy(F);
  return rc;
}

void worker_main(celeste_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  celeste_ctx* ctx = nullptr;
  int rc = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess
               ? celeste_create(&ctx, &S->model, S->device, stream)
               : CELESTE_ECUDA;
  DevBuf dev[kBufs];
  HostBuf host[kBufs];
  for (;;) {
    std::vector<std::shared_ptr<Request>> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || (!S->paused && !S->queue.empty()); });
      if (S->stop) break;
      int64_t bytes = 0;
      const double t = now_s();
      while (!S->queue.empty()) {
        auto& r = S->queue.front();
        if (!batch.empty() && (bytes + r->bytes > S->cfg.device_bytes ||
                               (S->cfg.max_batch > 0 && (int)batch.size() >= S->cfg.max_batch)))
          break;
        bytes += r->bytes;
        S->queued_bytes -= r->bytes;
        r->state = 1;
        r->t_start = t;
        batch.push_back(r);
        S->queue.pop_front();
      }
    }
    int brc = rc ? rc : run_batch(S, ctx, stream, batch, dev, host);
    if (brc) {
      std::lock_guard<std::mutex> lk(S->mu);
      const double t = now_s();
      for (auto& r : batch)
        if (r->state != 2) {
          r->error = brc;
          r->t_done = t;
          r->state = 2;
        }
      if (S->worker_error == CELESTE_OK) S->worker_error = brc;
      S->cv_done.notify_all();
    }
  }
  if (ctx) celeste_destroy(ctx);
  if (stream) cudaStreamDestroy(stream);
}

bool valid_request(const celeste_region_request* q) {
  if (!q || q->n_sources < 1 || q->n_images < 1 || q->n_pixels < 1 || q->n_sky < 1 ||
      q->n_patches < 0 || q->n_nbr < 0 || !q->pixels || !q->sky || !q->images || !q->theta ||
      !q->patch_ptr || !q->patches || !q->nbr_ptr || (q->n_nbr > 0 && !q->nbr_idx))
    return false;
  for (int i = 0; i < q->n_images; ++i) {
    const celeste_image& im = q->images[i];
    if (im.band < 0 || im.band >= CELESTE_N_BANDS || im.height < 1 || im.width < 1 ||
        im.row_stride < im.width || im.sky_ny < 1 || im.sky_nx < 1 || im.pix_offset < 0 ||
        im.sky_offset < 0 ||
        im.pix_offset + (int64_t)(im.height - 1) * im.row_stride + im.width > q->n_pixels ||
        im.sky_offset + (int64_t)im.sky_ny * im.sky_nx > q->n_sky)
      return false;
  }
  if (q->patch_ptr[0] != 0 || q->patch_ptr[q->n_sources] != q->n_patches || q->nbr_ptr[0] != 0 ||
      q->nbr_ptr[q->n_sources] != q->n_nbr)
    return false;
  for (int s = 0; s < q->n_sources; ++s)
    if (q->patch_ptr[s + 1] < q->patch_ptr[s] || q->nbr_ptr[s + 1] < q->nbr_ptr[s]) return false;
  for (int p = 0; p < q->n_patches; ++p) {
    const celeste_patch& P = q->patches[p];
    if (P.image < 0 || P.image >= q->n_images) return false;
    const celeste_image& im = q->images[P.image];
    if (P.w < 1 || P.h < 1 || P.x0 < 0 || P.y0 < 0 || P.x0 + P.w > im.width || P.y0 + P.h > im.height)
      return false;
  }
  for (int k = 0; k < q->n_nbr; ++k)
    if (q->nbr_idx[k] < 0 || q->nbr_idx[k] >= q->n_sources) return false;
  return true;
}

}  // namespace

extern "C" {

int celeste_server_create(const celeste_model* model, int device, const celeste_server_config* cfg,
                          celeste_server** out) {
  if (!model || !out) return CELESTE_EINVAL;
  *out = nullptr;
  ModelDev md;
  if (!prepare_model(model, &md)) return CELESTE_EINVAL;
  celeste_server* S = new celeste_server();
  S->model = *model;
  S->device = device;
  if (cfg) S->cfg = *cfg;
  if (S->cfg.workers <= 0) S->cfg.workers = 2;
  if (S->cfg.device_bytes <= 0) S->cfg.device_bytes = (int64_t)4 << 30;
  if (S->cfg.queue_bytes <= 0) S->cfg.queue_bytes = 4 * S->cfg.device_bytes * S->cfg.workers;
  if (!(S->cfg.pass_tol >= 0.0) || S->cfg.max_passes < 0 || S->cfg.max_passes > 1000 ||
      S->cfg.max_iter < 0 || S->cfg.max_iter > 1000 || S->cfg.workers > 64 ||
      (S->cfg.pixels_per_item != 0 &&
       (S->cfg.pixels_per_item < 32 || S->cfg.pixels_per_item > 65536))) {
    delete S;
    return CELESTE_EINVAL;
  }
  S->paused = S->cfg.start_paused != 0;
  for (int w = 0; w < S->cfg.workers; ++w) S->workers.emplace_back(worker_main, S);
  *out = S;
  return CELESTE_OK;
}

int celeste_server_destroy(celeste_server* S) {
  if (!S) return CELESTE_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return CELESTE_OK;
}

int celeste_server_pause(celeste_server* S, int paused) {
  if (!S) return CELESTE_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
  }
  S->cv_work.notify_all();
  return CELESTE_OK;
}

int celeste_submit(celeste_server* S, const celeste_region_request* q, uint64_t* ticket) {
  if (!S || !ticket || !valid_request(q)) return CELESTE_EINVAL;
  auto r = std::make_shared<Request>();
  r->pixels.assign(q->pixels, q->pixels + q->n_pixels);
  r->sky.assign(q->sky, q->sky + q->n_sky);
  r->images.assign(q->images, q->images + q->n_images);
  r->theta.assign(q->theta, q->theta + (size_t)q->n_sources * CELESTE_N_THETA);
  r->patch_ptr.assign(q->patch_ptr, q->patch_ptr + q->n_sources + 1);
  r->patches.assign(q->patches, q->patches + q->n_patches);
  r->nbr_ptr.assign(q->nbr_ptr, q->nbr_ptr + q->n_sources + 1);
  r->nbr_idx.assign(q->nbr_idx, q->nbr_idx + q->n_nbr);
  r->n_sources = q->n_sources;
  r->bytes = footprint(*r);
  if (r->bytes > S->cfg.device_bytes) return CELESTE_ETOOLARGE;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return CELESTE_EINVAL;
  if (S->queued_bytes + r->bytes > S->cfg.queue_bytes) return CELESTE_EAGAIN;
  r->ticket = S->next_ticket++;
  r->t_submit = now_s();
  S->queued_bytes += r->bytes;
  S->queue.push_back(r);
  S->tickets[r->ticket] = r;
  *ticket = r->ticket;
  S->cv_work.notify_one();
  return CELESTE_OK;
}

int celeste_poll(celeste_server* S, uint64_t ticket, int32_t wait_ms, double* theta_out,
                 int32_t* status_out, celeste_request_info* info) {
  if (!S) return CELESTE_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return CELESTE_ENOTFOUND;
  std::shared_ptr<Request> r = it->second;
  if (r->state != 2 && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->state == 2; });
  if (r->state != 2) return CELESTE_EBUSY;
  if (theta_out && !r->theta_out.empty())
    memcpy(theta_out, r->theta_out.data(), r->theta_out.size() * 8);
  if (status_out && !r->status_out.empty())
    memcpy(status_out, r->status_out.data(), r->status_out.size() * 4);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->n_sources = r->n_sources;
    info->passes = r->passes;
    info->batch_requests = r->batch_requests;
    info->device_error = r->device_error;
    info->last_pass_gain = r->last_gain;
    info->queue_s = r->t_start - r->t_submit;
    info->latency_s = r->t_done - r->t_submit;
  }
  const int err = r->error;
  S->tickets.erase(it);
  return err;
}

int celeste_server_stats(celeste_server* S, int64_t* launches, int64_t* batches) {
  if (!S) return CELESTE_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (launches) *launches = S->launches;
  if (batches) *batches = S->batches;
  return S->worker_error;
}

}  // extern "C"
