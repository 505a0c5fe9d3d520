// Serving: region fits submitted by independent callers, batched on the GPU.
//
// A request is a small problem of its own (a sky region: its exposures and
// the sources in it).  celeste_submit validates it, copies it and queues it.
// Each worker thread (its own context and stream) keeps a set of running
// requests and fits them together: the running requests form one problem
// (their images, patches and sources side by side) and one segmented fit in
// which every request is a segment with its own pass count and stopping
// rule, so its result does not depend on what it runs with.  Batching is
// continuous: after every pass the worker retires the requests whose
// segments stopped (their results are ready for celeste_poll at once) and
// admits queued requests into the memory they and the still-running ones
// leave free; a request that arrives while others are on the GPU starts at
// the next pass boundary, not after the others finish.
//
// Every running request keeps fixed places in the worker's device arenas
// (pixels, sky, render cache, a range of source ids for its parameters)
// from admission to completion, so admitting others moves none of its data;
// only the small tables that tie the running requests together (images,
// patches, neighbour lists) are rebuilt, with a new fit, when the set of
// running requests grows.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
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
  // places in the worker's arenas while running
  int64_t pix_off = 0, sky_off = 0, cache_off = 0, n_pool = 0;
  int src_first = 0;
  int seg = -1;                      // segment in the worker's current fit
  int passes_run = 0;                // passes run so far
};

// First-fit allocation of ranges of [0, cap) (host bookkeeping of a device
// arena); freed ranges merge with their free neighbours.
struct Arena {
  int64_t cap = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
  void init(int64_t c) {
    cap = c;
    free_.clear();
    if (c > 0) free_[0] = c;
  }
  int64_t alloc(int64_t n) {
    if (n <= 0) return 0;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      return off;
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    if (n <= 0) return;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
};

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, (size_t)1 << 16) + bytes / 4;
    if (cudaMalloc(&p, want) != cudaSuccess) return false;
    cap = want;
    return true;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

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

// A worker: its context, its arenas and the requests it is running.
struct Worker {
  celeste_server* S = nullptr;
  celeste_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  // device arenas: pixels and sky (floats), render cache (float2 per patch
  // pixel), parameters (27 doubles per source id)
  float* d_pix = nullptr;
  float* d_sky = nullptr;
  float* d_cache = nullptr;
  double* d_theta = nullptr;
  Arena a_pix, a_sky, a_cache, a_src;
  // tables of the running set (host copies, read by plan creation, and
  // their device copies)
  std::vector<celeste_image> h_img;
  std::vector<celeste_patch> h_patch;
  std::vector<int32_t> h_pp, h_np, h_ni;
  DevBuf d_img, d_patch, d_pp, d_np, d_ni, d_status;
  std::vector<double> h_theta;
  std::vector<int32_t> h_status;
  std::vector<std::shared_ptr<Request>> run;   // running requests, segment order
  celeste_problem P{};
  celeste_fit* F = nullptr;
  int64_t run_bytes = 0;
  // destroys the fit a rebuild replaced while the next pass runs (tearing
  // down a fit's graph and plans takes milliseconds of host time)
  std::thread reaper;

  void reap(celeste_fit* old) {
    if (reaper.joinable()) reaper.join();
    if (!old) return;
    const int dev = S->device;
    reaper = std::thread([old, dev] {
      cudaSetDevice(dev);
      celeste_fit_destroy(old);
    });
  }

  ~Worker() {
    if (reaper.joinable()) reaper.join();
    if (F) celeste_fit_destroy(F);
    for (void* q : {(void*)d_pix, (void*)d_sky, (void*)d_cache, (void*)d_theta})
      if (q) cudaFree(q);
    if (ctx) celeste_destroy(ctx);
    if (stream) cudaStreamDestroy(stream);
  }

  int init() {
    CK(cudaSetDevice(S->device));
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    int rc = celeste_create(&ctx, &S->model, S->device, stream);
    if (rc) return rc;
    // capacities: a request's footprint counts 4 bytes per pixel, 8 bytes of
    // cache per patch pixel among its 12 per visit, and 16 KiB per source,
    // so arenas of the budget's size hold every admissible set
    const int64_t B = S->cfg.device_bytes;
    a_pix.init(B / 4);
    a_sky.init(std::max<int64_t>(B / 64, 1024));
    a_cache.init(B / 8);
    a_src.init(std::max<int64_t>(B / 16384, 64));
    if (cudaMalloc(&d_pix, a_pix.cap * 4) != cudaSuccess ||
        cudaMalloc(&d_sky, a_sky.cap * 4) != cudaSuccess ||
        cudaMalloc(&d_cache, a_cache.cap * 8) != cudaSuccess ||
        cudaMalloc(&d_theta, a_src.cap * CELESTE_N_THETA * 8) != cudaSuccess)
      return CELESTE_ENOMEM;
    return CELESTE_OK;
  }

  // Places r in the arenas; false (nothing held) when a range does not fit.
  bool place(Request& r) {
    int64_t pool = 0;
    for (const celeste_patch& q : r.patches) pool += (int64_t)q.w * q.h;
    const int64_t op = a_pix.alloc((int64_t)r.pixels.size());
    const int64_t os = op < 0 ? -1 : a_sky.alloc((int64_t)r.sky.size());
    const int64_t oc = os < 0 ? -1 : a_cache.alloc(pool);
    const int64_t of = oc < 0 ? -1 : a_src.alloc(r.n_sources);
    if (of < 0) {
      if (oc >= 0) a_cache.release(oc, pool);
      if (os >= 0) a_sky.release(os, (int64_t)r.sky.size());
      if (op >= 0) a_pix.release(op, (int64_t)r.pixels.size());
      return false;
    }
    r.pix_off = op;
    r.sky_off = os;
    r.cache_off = oc;
    r.n_pool = pool;
    r.src_first = (int)of;
    return true;
  }

  void unplace(const Request& r) {
    a_pix.release(r.pix_off, (int64_t)r.pixels.size());
    a_sky.release(r.sky_off, (int64_t)r.sky.size());
    a_cache.release(r.cache_off, r.n_pool);
    a_src.release(r.src_first, r.n_sources);
  }

  // Uploads a newly placed request's pixels, sky and initial parameters.
  int upload(const Request& r) {
    CK(cudaMemcpyAsync(d_pix + r.pix_off, r.pixels.data(), r.pixels.size() * 4,
                       cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_sky + r.sky_off, r.sky.data(), r.sky.size() * 4, cudaMemcpyHostToDevice,
                       stream));
    CK(cudaMemcpyAsync(d_theta + (size_t)r.src_first * CELESTE_N_THETA, r.theta.data(),
                       r.theta.size() * 8, cudaMemcpyHostToDevice, stream));
    return CELESTE_OK;
  }

  // Tables of the running set and a fit over it (segments in run order);
  // continuing requests keep their pass counts.
  int rebuild() {
    reap(F);
    F = nullptr;
    // source ids in use: [0, n_ids); ids no running request holds are empty
    int n_ids = 0;
    for (auto& r : run) n_ids = std::max(n_ids, r->src_first + r->n_sources);
    std::vector<const Request*> by_id(n_ids, nullptr);
    for (auto& r : run)
      for (int s = 0; s < r->n_sources; ++s) by_id[r->src_first + s] = r.get();
    h_img.clear();
    std::unordered_map<const Request*, int> img_base;
    for (auto& r : run) {
      img_base[r.get()] = (int)h_img.size();
      for (celeste_image im : r->images) {
        im.pix_offset += r->pix_off;
        im.sky_offset += r->sky_off;
        h_img.push_back(im);
      }
    }
    h_patch.clear();
    h_ni.clear();
    h_pp.assign(n_ids + 1, 0);
    h_np.assign(n_ids + 1, 0);
    std::unordered_map<const Request*, int64_t> pool_at;
    for (int id = 0; id < n_ids; ++id) {
      const Request* r = by_id[id];
      if (r) {
        const int s = id - r->src_first;
        int64_t& pool = pool_at[r];          // running pool offset within the request
        if (s == 0) pool = 0;
        for (int q = r->patch_ptr[s]; q < r->patch_ptr[s + 1]; ++q) {
          celeste_patch P = r->patches[q];
          P.image += img_base[r];
          P.pool_offset = r->cache_off + pool;
          pool += (int64_t)P.w * P.h;
          h_patch.push_back(P);
        }
        for (int k = r->nbr_ptr[s]; k < r->nbr_ptr[s + 1]; ++k)
          h_ni.push_back(r->nbr_idx[k] + r->src_first);
      }
      h_pp[id + 1] = (int32_t)h_patch.size();
      h_np[id + 1] = (int32_t)h_ni.size();
    }
    if (h_ni.empty()) h_ni.push_back(0);
    if (!d_img.reserve(h_img.size() * sizeof(celeste_image)) ||
        !d_patch.reserve(std::max<size_t>(h_patch.size(), 1) * sizeof(celeste_patch)) ||
        !d_pp.reserve(h_pp.size() * 4) || !d_np.reserve(h_np.size() * 4) ||
        !d_ni.reserve(h_ni.size() * 4) || !d_status.reserve((size_t)std::max(n_ids, 1) * 4))
      return CELESTE_ENOMEM;
    CK(cudaMemcpyAsync(d_img.p, h_img.data(), h_img.size() * sizeof(celeste_image),
                       cudaMemcpyHostToDevice, stream));
    if (!h_patch.empty())
      CK(cudaMemcpyAsync(d_patch.p, h_patch.data(), h_patch.size() * sizeof(celeste_patch),
                         cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_pp.p, h_pp.data(), h_pp.size() * 4, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_np.p, h_np.data(), h_np.size() * 4, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_ni.p, h_ni.data(), h_ni.size() * 4, cudaMemcpyHostToDevice, stream));
    P = celeste_problem{};
    P.pixels = d_pix;
    P.sky = d_sky;
    P.images = static_cast<const celeste_image*>(d_img.p);
    P.theta = d_theta;
    P.patch_ptr = static_cast<const int32_t*>(d_pp.p);
    P.patches = static_cast<const celeste_patch*>(d_patch.p);
    P.nbr_ptr = static_cast<const int32_t*>(d_np.p);
    P.nbr_idx = static_cast<const int32_t*>(d_ni.p);
    P.h_patch_ptr = h_pp.data();
    P.h_patches = h_patch.data();
    P.h_images = h_img.data();
    P.h_nbr_ptr = h_np.data();
    P.h_nbr_idx = h_ni.data();
    P.n_pixels = a_pix.cap;
    P.n_sky = a_sky.cap;
    P.n_pool = a_cache.cap;
    P.render_cache = d_cache;
    P.n_images = (int32_t)h_img.size();
    P.n_sources = n_ids;
    P.n_patches = (int32_t)h_patch.size();
    P.n_nbr = (int32_t)(h_ni.size() == 1 && h_np[n_ids] == 0 ? 0 : h_ni.size());
    std::vector<int32_t> ids, seg_ptr(1, 0);
    std::vector<int32_t> passes;
    for (auto& r : run) {
      r->seg = (int)passes.size();
      for (int s = 0; s < r->n_sources; ++s) ids.push_back(r->src_first + s);
      seg_ptr.push_back((int32_t)ids.size());
      passes.push_back(r->passes_run);
    }
    celeste_tuning tuning{};
    tuning.pixels_per_item = S->cfg.pixels_per_item;
    int rc = fit_create_segments(ctx, &P, ids.data(), (int)ids.size(), seg_ptr.data(),
                                 (int)run.size(), &tuning, &F);
    if (rc) return rc;
    rc = fit_begin(ctx, F, S->cfg.max_passes, S->cfg.max_iter, S->cfg.pass_tol);
    if (rc) return rc;
    CK(cudaMemcpyAsync(F->f.seg_passes, passes.data(), passes.size() * 4, cudaMemcpyHostToDevice,
                       stream));
    return CELESTE_OK;
  }

  // Completes requests (under the server lock): result or error.
  void complete(const std::vector<std::shared_ptr<Request>>& done, int err, uint32_t word) {
    const double t = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& r : done) {
      r->error = err;
      r->device_error = word;
      r->t_done = t;
      r->state = 2;
    }
    S->cv_done.notify_all();
  }

  // One pass of the running set; retires the requests whose segments
  // stopped (their results read back and published).
  int pass() {
    int n_active = 0;
    int rc = fit_pass(ctx, F, &n_active);
    if (rc) return rc;
    std::vector<std::shared_ptr<Request>> done;
    std::vector<std::shared_ptr<Request>> keep;
    for (size_t k = 0; k < run.size(); ++k) {
      Request& r = *run[k];
      r.passes_run = F->h_seg_passes[r.seg];
      r.last_gain = F->h_seg_gain[r.seg];
      if (F->h_seg_active[r.seg]) {
        keep.push_back(run[k]);
        continue;
      }
      r.theta_out.resize((size_t)r.n_sources * CELESTE_N_THETA);
      r.status_out.resize(r.n_sources);
      CK(cudaMemcpyAsync(r.theta_out.data(), d_theta + (size_t)r.src_first * CELESTE_N_THETA,
                         r.theta_out.size() * 8, cudaMemcpyDeviceToHost, stream));
      CK(cudaMemcpyAsync(r.status_out.data(), F->f.status + r.src_first, (size_t)r.n_sources * 4,
                         cudaMemcpyDeviceToHost, stream));
      r.passes = r.passes_run;
      done.push_back(run[k]);
    }
    if (done.empty()) return CELESTE_OK;
    uint32_t word = 0;
    const int sync = celeste_synchronize(ctx, &word);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& r : done) {
        unplace(*r);
        run_bytes -= r->bytes;
      }
    }
    complete(done, sync, word);
    // the fit keeps the finished segments frozen until the next rebuild
    run.swap(keep);
    return CELESTE_OK;
  }
};

void worker_main(celeste_server* S) {
  Worker W;
  W.S = S;
  const int init_rc = W.init();
  for (;;) {
    std::vector<std::shared_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        return S->stop || !W.run.empty() || (!S->paused && !S->queue.empty());
      });
      if (S->stop) break;
      // admission: queued requests in order, while their footprint fits the
      // budget beside the running ones and the arenas have room
      const double t = now_s();
      while (!S->paused && !S->queue.empty() && init_rc == CELESTE_OK) {
        auto& r = S->queue.front();
        if (S->cfg.max_batch > 0 && (int)(W.run.size() + admitted.size()) >= S->cfg.max_batch)
          break;
        if (W.run_bytes + r->bytes > S->cfg.device_bytes) break;
        if (!W.place(*r)) break;
        W.run_bytes += r->bytes;
        S->queued_bytes -= r->bytes;
        r->state = 1;
        r->t_start = t;
        admitted.push_back(r);
        S->queue.pop_front();
      }
      if (init_rc != CELESTE_OK && !S->queue.empty()) {
        // a worker that could not start fails what it takes
        admitted.push_back(S->queue.front());
        S->queue.pop_front();
      }
    }
    if (init_rc != CELESTE_OK) {
      W.complete(admitted, init_rc, 0);
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->worker_error == CELESTE_OK) S->worker_error = init_rc;
      continue;
    }
    int rc = CELESTE_OK;
    const bool fresh = W.run.empty() && !admitted.empty();
    if (!admitted.empty()) {
      for (auto& r : admitted) {
        if (rc == CELESTE_OK) rc = W.upload(*r);
        W.run.push_back(r);
      }
      const int n_run = (int)W.run.size();
      for (auto& r : admitted) r->batch_requests = n_run;
      if (rc == CELESTE_OK) rc = W.rebuild();
      if (fresh) {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->batches;
      }
    }
    const int64_t l0 = celeste_launch_count(W.ctx);
    if (rc == CELESTE_OK && !W.run.empty()) rc = W.pass();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->launches += celeste_launch_count(W.ctx) - l0;
    }
    if (rc != CELESTE_OK) {
      // the running requests fail with the error; the worker starts afresh
      std::vector<std::shared_ptr<Request>> failed;
      failed.swap(W.run);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto& r : failed) {
          W.unplace(*r);
          W.run_bytes -= r->bytes;
        }
        if (S->worker_error == CELESTE_OK) S->worker_error = rc;
      }
      W.complete(failed, rc, 0);
      if (W.F) {
        celeste_fit_destroy(W.F);
        W.F = nullptr;
      }
      continue;
    }
    if (W.run.empty() && W.F) {
      celeste_fit_destroy(W.F);
      W.F = nullptr;
    }
  }
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
    info->t_start_s = r->t_start;
    info->t_done_s = r->t_done;
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
