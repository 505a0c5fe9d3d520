// C ABI of the library: contexts, plans (work decomposition and scratch),
// and the calls of celeste.h, each a short sequence of kernel launches on the
// context's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "host.h"

using namespace celeste;

Launch celeste::make_launch(const celeste_ctx* c, const celeste_plan* p) {
  Launch L;
  L.stream = c->stream;
  L.sm_count = c->sm_count;
  L.warps_per_block = p && p->tuning.warps_per_block > 0 ? p->tuning.warps_per_block : 4;
  L.blocks_per_sm = p && p->tuning.blocks_per_sm > 0 ? p->tuning.blocks_per_sm : 0;
  L.pixels_per_item = p && p->tuning.pixels_per_item > 0 ? p->tuning.pixels_per_item : 256;
  L.n_exp = c->n_exp;
  L.n_dev = c->n_dev;
  return L;
}

namespace {

int to_status(cudaError_t e) { return e == cudaSuccess ? CELESTE_OK : CELESTE_ECUDA; }

// Inverse and log-determinant of a symmetric positive-definite 4x4 matrix
// (Cholesky).  Returns false when it is not positive definite.
bool spd_inverse4(const double C[4][4], double P[4][4], double* logdet) {
  double L[4][4] = {{0}};
  double ld = 0.0;
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = C[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i][i] = sqrt(s);
        ld += 2.0 * log(L[i][i]);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  // inverse of L, then P = L^-T L^-1
  double Li[4][4] = {{0}};
  for (int i = 0; i < 4; ++i) {
    Li[i][i] = 1.0 / L[i][i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= L[i][k] * Li[k][j];
      Li[i][j] = s / L[i][i];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = std::max(i, j); k < 4; ++k) s += Li[k][i] * Li[k][j];
      P[i][j] = s;
    }
  *logdet = ld;
  return true;
}

template <typename T>
T* dev_alloc(celeste_plan* p, size_t count, int* err) {
  if (count == 0) count = 1;
  void* ptr = ctx_alloc(p->ctx, false, count * sizeof(T));
  if (!ptr) {
    *err = CELESTE_ENOMEM;
    return nullptr;
  }
  p->allocs.push_back(ptr);
  return static_cast<T*>(ptr);
}



// Runs one launch, bracketed by a pair of events when profiling (under
// stream capture an ordinary record only expresses a dependency; the
// external flag makes it an event-record node of the graph).
template <typename F>
cudaError_t timed(celeste_ctx* c, int kind, int64_t visits, cudaStream_t stream, F&& launch) {
  if (!(c->profiling >> kind & 1u)) return launch();
  if (2 * (c->n_timed + 1) > c->events.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      c->events.push_back(e);
    }
    c->kinds.push_back(0);
    c->visits.push_back(0);
  }
  cudaEvent_t e0 = c->events[2 * c->n_timed], e1 = c->events[2 * c->n_timed + 1];
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(stream, &cap);
  const unsigned flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  if (r == cudaSuccess) r = cudaEventRecordWithFlags(e0, stream, flags);
  if (r == cudaSuccess) r = launch();
  if (r == cudaSuccess) r = cudaEventRecordWithFlags(e1, stream, flags);
  if (r == cudaSuccess) {
    c->kinds[c->n_timed] = kind;
    c->visits[c->n_timed] = visits;
    ++c->n_timed;
  }
  return r;
}

cudaError_t derivs_launch(celeste_ctx* c, celeste_plan* p, const Launch& L) {
  return timed(c, CELESTE_K_DERIVS, p->visits, L.stream, [&] { return launch_pixels_derivs(L, p->v); });
}

int run_setup(celeste_ctx* c, celeste_plan* p, int first, int n, bool trial) {
  Launch L = make_launch(c, p);
  ++c->launches;
  return to_status(timed(c, CELESTE_K_SETUP, 0, L.stream,
                         [&] { return launch_setup(L, p->v, c->d_model, first, n, trial); }));
}

}  // namespace

namespace celeste {

// ---- memory pools of contexts --------------------------------------------

void* MemPool::get(bool host, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  {
    std::lock_guard<std::mutex> lk(mu_);
    auto& fr = free_[host];
    auto it = fr.lower_bound(bytes);
    if (it != fr.end() && it->first <= 2 * bytes) {
      void* ptr = it->second;
      fr.erase(it);
      return ptr;
    }
  }
  void* ptr = nullptr;
  const cudaError_t e = host ? cudaMallocHost(&ptr, bytes) : cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu_);
  size_[host][ptr] = bytes;
  return ptr;
}

void MemPool::put(bool host, void* ptr) {
  if (!ptr) return;
  std::lock_guard<std::mutex> lk(mu_);
  auto it = size_[host].find(ptr);
  if (it != size_[host].end()) free_[host].emplace(it->second, ptr);
}

// Frees the cached blocks.  Blocks still held by plans or fits stay theirs:
// they go straight back to CUDA when those are destroyed.
void MemPool::release_all() {
  std::lock_guard<std::mutex> lk(mu_);
  for (int h = 0; h < 2; ++h) {
    for (auto& kv : free_[h]) {
      if (h) cudaFreeHost(kv.second);
      else cudaFree(kv.second);
    }
    size_[h].clear();
    free_[h].clear();
  }
}

namespace {
// Live contexts by serial: plans and fits may outlive their context.
std::mutex g_ctx_mu;
std::unordered_map<uint64_t, celeste_ctx*> g_ctx_live;
uint64_t g_ctx_serial = 0;
}  // namespace

void* ctx_alloc(celeste_ctx* c, bool host, size_t bytes) {
  return c->pool.get(host, bytes);
}

void ctx_release(celeste_ctx* c, uint64_t serial, bool host,
                          const std::vector<void*>& blocks) {
  bool live = false;
  {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    auto it = g_ctx_live.find(serial);
    live = it != g_ctx_live.end() && it->second == c;
  }
  if (live) {
    // the blocks may still be read by work queued on the context's stream
    // (destroying a context while another thread destroys its plans is a
    // caller error, as for any object in use)
    cudaStreamSynchronize(c->stream);
    for (void* b : blocks) c->pool.put(host, b);
    return;
  }
  for (void* b : blocks) {
    if (host) cudaFreeHost(b);
    else cudaFree(b);
  }
}

bool prepare_model(const celeste_model* m, ModelDev* md) {
  if (m->n_exp < 1 || m->n_exp > kMaxProf || m->n_dev < 1 || m->n_dev > kMaxProf ||
      m->n_color < 1 || m->n_color > kMaxColor || !(m->prior_a > 0.0 && m->prior_a < 1.0) ||
      !(m->e_radius[1] > 0.0))
    return false;
  memset(md, 0, sizeof(*md));
  md->n_exp = m->n_exp;
  md->n_dev = m->n_dev;
  md->n_color = m->n_color;
  for (int j = 0; j < kMaxProf; ++j) {
    md->alpha_exp[j] = m->alpha_exp[j];
    md->tau_exp[j] = m->tau_exp[j];
    md->alpha_dev[j] = m->alpha_dev[j];
    md->tau_dev[j] = m->tau_dev[j];
  }
  md->prior_a = m->prior_a;
  for (int i = 0; i < 2; ++i) {
    if (!(m->prior_r[i][1] > 0.0)) return false;
    md->prior_r[i][0] = m->prior_r[i][0];
    md->prior_r[i][1] = m->prior_r[i][1];
    md->log_prior_r2[i] = log(m->prior_r[i][1]);
    for (int j = 0; j < m->n_color; ++j) {
      if (!(m->color_w[i][j] > 0.0)) return false;
      md->color_w[i][j] = m->color_w[i][j];
      md->log_color_w[i][j] = log(m->color_w[i][j]);
      for (int k = 0; k < 4; ++k) md->color_mean[i][j][k] = m->color_mean[i][j][k];
      if (!spd_inverse4(m->color_cov[i][j], md->color_prec[i][j], &md->color_logdet[i][j]))
        return false;
    }
  }
  for (int k = 0; k < 2; ++k) {
    md->e_radius[k] = m->e_radius[k];
    md->e_profile[k] = m->e_profile[k];
    md->e_axis[k] = m->e_axis[k];
  }
  if (!(m->e_axis[0] > 0.0 && m->e_axis[1] > 0.0 && m->e_profile[0] > 0.0 && m->e_profile[1] > 0.0))
    return false;
  md->log_prior_a = log(m->prior_a);
  md->log1m_prior_a = log1p(-m->prior_a);
  md->logit_prior_a = md->log_prior_a - md->log1m_prior_a;
  md->half_log_2pi_e2 = 0.5 * log(2.0 * M_PI * m->e_radius[1]);
  md->log_beta_axis = lgamma(m->e_axis[0]) + lgamma(m->e_axis[1]) - lgamma(m->e_axis[0] + m->e_axis[1]);
  md->log_beta_profile =
      lgamma(m->e_profile[0]) + lgamma(m->e_profile[1]) - lgamma(m->e_profile[0] + m->e_profile[1]);
  ModelDev::F32& f = md->f;
  for (int j = 0; j < kMaxProf; ++j) {
    f.tau_exp[j] = (float)md->tau_exp[j];
    f.tau_dev[j] = (float)md->tau_dev[j];
  }
  for (int i = 0; i < 2; ++i) {
    f.prior_r[i][0] = (float)md->prior_r[i][0];
    f.prior_r[i][1] = (float)md->prior_r[i][1];
    f.log_prior_r2[i] = (float)md->log_prior_r2[i];
    for (int j = 0; j < kMaxColor; ++j) {
      f.color_logdet[i][j] = (float)md->color_logdet[i][j];
      f.log_color_w[i][j] = (float)md->log_color_w[i][j];
      for (int k = 0; k < 4; ++k) {
        f.color_mean[i][j][k] = (float)md->color_mean[i][j][k];
        for (int l = 0; l < 4; ++l) f.color_prec[i][j][k][l] = (float)md->color_prec[i][j][k][l];
      }
    }
  }
  for (int k = 0; k < 2; ++k) {
    f.e_radius[k] = (float)md->e_radius[k];
    f.e_profile[k] = (float)md->e_profile[k];
    f.e_axis[k] = (float)md->e_axis[k];
  }
  f.log_prior_a = (float)md->log_prior_a;
  f.log1m_prior_a = (float)md->log1m_prior_a;
  f.logit_prior_a = (float)md->logit_prior_a;
  f.half_log_2pi_e2 = (float)md->half_log_2pi_e2;
  f.log_beta_axis = (float)md->log_beta_axis;
  f.log_beta_profile = (float)md->log_beta_profile;
  return true;
}

}  // namespace celeste

// One trust-region Newton iteration of the plan's active sources once the
// neighbour records and background are in place: active set and own
// records, derivative pass, the per-source step (epilogue, trust-region
// step, trial records), the value pass at the trial points, accept rule.
cudaError_t celeste::enqueue_iteration(celeste_ctx* c, celeste_plan* p, const Launch& L,
                                     double* delta, int32_t* status) {
  PlanView& v = p->v;
  cudaError_t e = launch_prepare(L, v, c->d_model, status, v.n_own_pairs, false);
  if (e == cudaSuccess) e = launch_pixels_derivs(L, v);
  if (e == cudaSuccess) e = launch_source_step(L, v, c->d_model, delta, status);
  if (e == cudaSuccess) e = launch_pixels_value(L, v, false);
  if (e == cudaSuccess) e = launch_slot_finish(L, v, false, delta, status);
  return e;
}

extern "C" {

int celeste_create(celeste_ctx** out, const celeste_model* m, int device, void* stream) {
  if (!out || !m) return CELESTE_EINVAL;
  *out = nullptr;
  ModelDev md;
  if (!prepare_model(m, &md)) return CELESTE_EINVAL;
  CK(cudaSetDevice(device));
  celeste_ctx* c = new celeste_ctx();
  c->device = device;
  {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    c->serial = ++g_ctx_serial;
    g_ctx_live[c->serial] = c;
  }
  c->stream = static_cast<cudaStream_t>(stream);
  c->n_exp = m->n_exp;
  c->n_dev = m->n_dev;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      init_pixel_occupancy() != cudaSuccess ||
      cudaMalloc(&c->d_model, sizeof(ModelDev)) != cudaSuccess ||
      cudaMalloc(&c->d_err, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemcpy(c->d_model, &md, sizeof(md), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_err, 0, sizeof(unsigned int)) != cudaSuccess) {
    cudaFree(c->d_model);
    cudaFree(c->d_err);
    {
      std::lock_guard<std::mutex> lk(g_ctx_mu);
      g_ctx_live.erase(c->serial);
    }
    delete c;
    return CELESTE_ECUDA;
  }
  *out = c;
  return CELESTE_OK;
}

int celeste_destroy(celeste_ctx* c) {
  if (!c) return CELESTE_EINVAL;
  cudaSetDevice(c->device);
  {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    g_ctx_live.erase(c->serial);
  }
  cudaStreamSynchronize(c->stream);
  c->pool.release_all();
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  cudaFree(c->d_model);
  cudaFree(c->d_err);
  delete c;
  return CELESTE_OK;
}

int celeste_synchronize(celeste_ctx* c, uint32_t* device_error) {
  if (!c) return CELESTE_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  unsigned int w = 0;
  CK(cudaMemcpy(&w, c->d_err, sizeof(w), cudaMemcpyDeviceToHost));
  if (device_error) *device_error = w;
  if (w) {
    CK(cudaMemset(c->d_err, 0, sizeof(unsigned int)));
    return CELESTE_EDEVICE;
  }
  return CELESTE_OK;
}

int64_t celeste_launch_count(const celeste_ctx* c) { return c ? c->launches : -1; }

int celeste_profile_enable(celeste_ctx* c, int on) {
  if (!c) return CELESTE_EINVAL;
  c->profiling = static_cast<unsigned>(on) & ((1u << CELESTE_K_COUNT) - 1u);
  c->n_timed = 0;
  return CELESTE_OK;
}

int celeste_profile_kernels(celeste_ctx* c, int reset, double* ms, int64_t* launches,
                            int64_t* visits) {
  if (!c || !ms || !launches) return CELESTE_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < CELESTE_K_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    if (visits) visits[k] = 0;
  }
  for (size_t k = 0; k < c->n_timed; ++k) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->events[2 * k], c->events[2 * k + 1]));
    const int kind = c->kinds[k];
    ms[kind] += t;
    ++launches[kind];
    if (visits) visits[kind] += c->visits[k];
  }
  if (reset) c->n_timed = 0;
  return CELESTE_OK;
}

int celeste_profile_read(celeste_ctx* c, int reset, double* total_ms, int64_t* launches,
                         int64_t* visits) {
  if (!c || !total_ms || !launches || !visits) return CELESTE_EINVAL;
  double ms[CELESTE_K_COUNT];
  int64_t n[CELESTE_K_COUNT], vis[CELESTE_K_COUNT];
  const int rc = celeste_profile_kernels(c, reset, ms, n, vis);
  if (rc) return rc;
  *total_ms = ms[CELESTE_K_DERIVS];
  *launches = n[CELESTE_K_DERIVS];
  *visits = vis[CELESTE_K_DERIVS];
  return CELESTE_OK;
}

int celeste_plan_create(celeste_ctx* c, const celeste_problem* pr, const int32_t* ids, int32_t n,
                        const celeste_tuning* tuning, celeste_plan** out) {
  if (!c || !pr || !out || n < 0 || (n > 0 && !ids)) return CELESTE_EINVAL;
  *out = nullptr;
  if (!pr->h_patch_ptr || !pr->h_patches || !pr->h_images || !pr->h_nbr_ptr ||
      (pr->n_nbr > 0 && !pr->h_nbr_idx) || !pr->pixels || !pr->sky || !pr->images || !pr->theta)
    return CELESTE_EINVAL;
  const int ppi = tuning && tuning->pixels_per_item > 0 ? tuning->pixels_per_item : 256;
  if (ppi < 32 || ppi > 65536) return CELESTE_EINVAL;
  std::vector<char> seen(pr->n_sources, 0);
  for (int j = 0; j < n; ++j) {
    if (ids[j] < 0 || ids[j] >= pr->n_sources || seen[ids[j]]) return CELESTE_EINVAL;
    seen[ids[j]] = 1;
  }
  std::vector<PairInfo> pairs;
  std::vector<int32_t> slot_ptr(n + 1, 0), slot_items(n + 1, 0), pair_nbr;
  std::vector<Item> items;
  int64_t bg = 0, visits = 0;
  auto patch_ok = [&](const celeste_patch& q) {
    if (q.image < 0 || q.image >= pr->n_images) return false;
    const celeste_image& im = pr->h_images[q.image];
    return q.w > 0 && q.h > 0 && q.x0 >= 0 && q.y0 >= 0 && q.x0 + q.w <= im.width &&
           q.y0 + q.h <= im.height;
  };
  // own pairs
  for (int j = 0; j < n; ++j) {
    const int s = ids[j];
    for (int q = pr->h_patch_ptr[s]; q < pr->h_patch_ptr[s + 1]; ++q) {
      const celeste_patch& P = pr->h_patches[q];
      if (!patch_ok(P)) return CELESTE_EINVAL;
      const celeste_image& im = pr->h_images[P.image];
      PairInfo pi{};
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
      visits += area;
      pi.item_begin = (int)items.size();
      const int bucket = area < 1024 ? 0 : (area < 4096 ? 1 : (area < 16384 ? 2 : 3));
      const int bp = tuning && tuning->ppi_bucket[bucket] > 0 ? tuning->ppi_bucket[bucket] : ppi;
      if (bp < 32 || bp > 65536) return CELESTE_EINVAL;
      for (int st = 0; st < area; st += bp) items.push_back(Item{(int)pairs.size(), st, std::min(bp, area - st), 0});
      pi.item_end = (int)items.size();
      pairs.push_back(pi);
    }
    slot_ptr[j + 1] = (int)pairs.size();
    slot_items[j + 1] = (int)items.size();
  }
  const int n_own = (int)pairs.size();
  // neighbour pairs: (neighbour source, its patch in the same image) that
  // overlap an own patch.  Per own source, each patch of each neighbour is
  // matched to the own pairs in its image; every own pair lists its
  // neighbour pairs in (neighbour, patch) order.
  std::unordered_map<int64_t, int> nb_index;
  std::vector<std::vector<int32_t>> per_pair(n_own);
  std::unordered_map<int32_t, std::vector<int32_t>> own_in_image;
  for (int j = 0; j < n; ++j) {
    const int s = ids[j];
    own_in_image.clear();
    for (int pp = slot_ptr[j]; pp < slot_ptr[j + 1]; ++pp) own_in_image[pairs[pp].image].push_back(pp);
    for (int k = pr->h_nbr_ptr[s]; k < pr->h_nbr_ptr[s + 1]; ++k) {
      const int t = pr->h_nbr_idx[k];
      if (t < 0 || t >= pr->n_sources) return CELESTE_EINVAL;
      for (int q = pr->h_patch_ptr[t]; q < pr->h_patch_ptr[t + 1]; ++q) {
        const celeste_patch& P = pr->h_patches[q];
        auto own = own_in_image.find(P.image);
        if (own == own_in_image.end()) continue;
        if (!patch_ok(P)) return CELESTE_EINVAL;
        for (const int32_t pp : own->second) {
          const PairInfo pi = pairs[pp];   // a copy: pairs grows below
          if (P.x0 >= pi.x0 + pi.w || pi.x0 >= P.x0 + P.w || P.y0 >= pi.y0 + pi.h ||
              pi.y0 >= P.y0 + P.h)
            continue;
          const int64_t key = (int64_t)t * (int64_t)pr->n_patches + q;
          auto it = nb_index.find(key);
          int idx;
          if (it == nb_index.end()) {
            idx = (int)pairs.size();
            nb_index.emplace(key, idx);
            const celeste_image& im = pr->h_images[P.image];
            PairInfo qn{};
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
            qn.nbr_begin = qn.nbr_end = 0;
            qn.item_begin = qn.item_end = 0;
            pairs.push_back(qn);
          } else {
            idx = it->second;
          }
          per_pair[pp].push_back(idx);
        }
      }
    }
  }
  for (int pp = 0; pp < n_own; ++pp) {
    pairs[pp].nbr_begin = (int)pair_nbr.size();
    pair_nbr.insert(pair_nbr.end(), per_pair[pp].begin(), per_pair[pp].end());
    pairs[pp].nbr_end = (int)pair_nbr.size();
  }

  celeste_plan* p = new celeste_plan();
  p->ctx = c;
  p->ctx_serial = c->serial;
  p->visits = visits;
  if (tuning) p->tuning = *tuning;
  p->tuning.pixels_per_item = ppi;
  int err = CELESTE_OK;
  PlanView& v = p->v;
  v.pixels = pr->pixels;
  v.sky = pr->sky;
  v.images = pr->images;
  v.theta = pr->theta;
  v.n = n;
  v.n_pairs = (int)pairs.size();
  v.n_own_pairs = n_own;
  v.n_items = (int)items.size();
  v.n_bg = bg;
  v.err = c->d_err;
  v.cache = reinterpret_cast<float2*>(pr->render_cache);
  v.cache_half = pr->render_cache ? pr->render_cache_half : nullptr;
  v.cache_n_pool = pr->n_pool;
  v.patches = pr->patches;
  p->d_patches = pr->patches;
  int32_t* d_ids = dev_alloc<int32_t>(p, n, &err);
  PairInfo* d_pairs = dev_alloc<PairInfo>(p, pairs.size(), &err);
  int32_t* d_nbr = dev_alloc<int32_t>(p, pair_nbr.size(), &err);
  int32_t* d_slot = dev_alloc<int32_t>(p, n + 1, &err);
  int32_t* d_slot_items = dev_alloc<int32_t>(p, n + 1, &err);
  Item* d_items = dev_alloc<Item>(p, items.size(), &err);
  v.records = dev_alloc<float>(p, pairs.size() * (size_t)kRecF, &err);
  v.bg = dev_alloc<float2>(p, (size_t)bg, &err);
  v.trial_render = pr->render_cache ? dev_alloc<float2>(p, (size_t)bg, &err) : nullptr;
  v.partials = dev_alloc<float>(p, items.size() * (size_t)kAcc, &err);
  v.vpartials = dev_alloc<float>(p, items.size() * 2, &err);
  v.theta_trial = dev_alloc<double>(p, (size_t)n * kTheta, &err);
  v.step = dev_alloc<double>(p, (size_t)n * kTheta, &err);
  v.pred = dev_alloc<double>(p, n, &err);
  v.kl_trial = dev_alloc<double>(p, n, &err);
  v.work_ctr = dev_alloc<int32_t>(p, 2, &err);
  v.elbo_rel = dev_alloc<double>(p, n, &err);
  p->rel_trial = dev_alloc<double>(p, n, &err);
  v.rel_trial = p->rel_trial;
  v.grad = dev_alloc<double>(p, (size_t)n * kTheta, &err);
  v.hess = dev_alloc<double>(p, (size_t)n * kTheta * kTheta, &err);
  v.active = dev_alloc<uint8_t>(p, n, &err);
  if (err != CELESTE_OK) {
    celeste_plan_destroy(p);
    return err;
  }
  cudaError_t ce = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (bytes && ce == cudaSuccess) ce = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cp(d_ids, ids, n * sizeof(int32_t));
  cp(d_pairs, pairs.data(), pairs.size() * sizeof(PairInfo));
  cp(d_nbr, pair_nbr.data(), pair_nbr.size() * sizeof(int32_t));
  cp(d_slot, slot_ptr.data(), (n + 1) * sizeof(int32_t));
  cp(d_slot_items, slot_items.data(), (n + 1) * sizeof(int32_t));
  cp(d_items, items.data(), items.size() * sizeof(Item));
  if (ce == cudaSuccess) ce = cudaMemset(v.theta_trial, 0, (size_t)n * kTheta * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMemset(v.active, 1, n > 0 ? n : 1);
  if (ce == cudaSuccess) ce = cudaMemset(v.work_ctr, 0, 2 * sizeof(int32_t));
  if (ce != cudaSuccess) {
    celeste_plan_destroy(p);
    return CELESTE_ECUDA;
  }
  v.src_ids = d_ids;
  v.pairs = d_pairs;
  v.pair_nbr = d_nbr;
  v.slot_pair_ptr = d_slot;
  v.slot_items = d_slot_items;
  v.items = d_items;
  *out = p;
  return CELESTE_OK;
}

int celeste_plan_destroy(celeste_plan* p) {
  if (!p) return CELESTE_EINVAL;
  ctx_release(p->ctx, p->ctx_serial, false, p->allocs);
  delete p;
  return CELESTE_OK;
}

int64_t celeste_plan_visits(const celeste_plan* p) { return p ? p->visits : -1; }

static int eval_common(celeste_ctx* c, celeste_plan* p, bool derivs) {
  Launch L = make_launch(c, p);
  CK(cudaMemsetAsync(p->v.active, 1, p->v.n > 0 ? p->v.n : 1, c->stream));
  // with a render cache the background comes from cached moments, so only
  // the own pairs need records
  int rc = run_setup(c, p, 0, p->v.cache ? p->v.n_own_pairs : p->v.n_pairs, false);
  if (rc) return rc;
  c->launches += 2;
  CK(timed(c, CELESTE_K_BACKGROUND, p->visits, L.stream, [&] { return launch_background(L, p->v); }));
  CK(derivs ? derivs_launch(c, p, L)
            : timed(c, CELESTE_K_VALUE, p->visits, L.stream, [&] { return launch_pixels_value(L, p->v); }));
  return CELESTE_OK;
}

int celeste_elbo_grad_hess(celeste_ctx* c, const celeste_plan* pc, double* elbo, double* elbo_rel,
                           double* grad, double* hess) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c) return CELESTE_EINVAL;
  if (p->v.n == 0) return CELESTE_OK;
  if (!elbo || !grad || !hess) return CELESTE_EINVAL;
  int rc = eval_common(c, p, true);
  if (rc) return rc;
  Launch L = make_launch(c, p);
  ++c->launches;
  return to_status(timed(c, CELESTE_K_EPILOGUE, 0, L.stream, [&] {
    return launch_epilogue(L, p->v, c->d_model, elbo, elbo_rel, grad, hess);
  }));
}

int celeste_elbo_grad(celeste_ctx* c, const celeste_plan* pc, double* elbo, double* elbo_rel,
                      double* grad) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c) return CELESTE_EINVAL;
  if (p->v.n == 0) return CELESTE_OK;
  if (!grad) return CELESTE_EINVAL;
  Launch L = make_launch(c, p);
  CK(cudaMemsetAsync(p->v.active, 1, p->v.n > 0 ? p->v.n : 1, c->stream));
  int rc = run_setup(c, p, 0, p->v.n_pairs, false);
  if (rc) return rc;
  c->launches += 3;
  CK(timed(c, CELESTE_K_BACKGROUND, p->visits, L.stream, [&] { return launch_background(L, p->v); }));
  CK(timed(c, CELESTE_K_GRAD, p->visits, L.stream, [&] { return launch_pixels_grad(L, p->v); }));
  return to_status(timed(c, CELESTE_K_EPILOGUE, 0, L.stream, [&] {
    return launch_epilogue_grad(L, p->v, c->d_model, elbo, elbo_rel, grad);
  }));
}

int celeste_elbo(celeste_ctx* c, const celeste_plan* pc, double* elbo, double* elbo_rel) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c) return CELESTE_EINVAL;
  if (p->v.n == 0) return CELESTE_OK;
  int rc = eval_common(c, p, false);
  if (rc) return rc;
  Launch L = make_launch(c, p);
  ++c->launches;
  return to_status(timed(c, CELESTE_K_EPILOGUE, 0, L.stream, [&] {
    return launch_epilogue_value(L, p->v, c->d_model, elbo, elbo_rel, false);
  }));
}

int celeste_loglik(celeste_ctx* c, const celeste_plan* pc, double* out) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c || !out) return CELESTE_EINVAL;
  if (p->v.n == 0) return CELESTE_OK;
  int rc = eval_common(c, p, false);
  if (rc) return rc;
  Launch L = make_launch(c, p);
  ++c->launches;
  return to_status(timed(c, CELESTE_K_EPILOGUE, 0, L.stream,
                         [&] { return launch_epilogue_loglik(L, p->v, c->d_model, out); }));
}

int celeste_newton_step(celeste_ctx* c, const celeste_plan* pc, double* delta, int32_t* status,
                        double* elbo_rel) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c || !delta || !status) return CELESTE_EINVAL;
  if (p->v.n == 0) return CELESTE_OK;
  Launch L = make_launch(c, p);
  PlanView& v = p->v;
  const bool cached = v.cache != nullptr;
  // active set and records; with a render cache the background comes from
  // cached moments, so the own records are all it needs and it joins the
  // same launch
  c->launches += 1;
  CK(timed(c, cached ? CELESTE_K_BACKGROUND : CELESTE_K_SETUP, cached ? p->visits : 0, L.stream,
           [&] {
             return launch_prepare(L, v, c->d_model, status, cached ? v.n_own_pairs : v.n_pairs,
                                   cached);
           }));
  if (!cached) {
    c->launches += 1;
    CK(timed(c, CELESTE_K_BACKGROUND, p->visits, L.stream, [&] { return launch_background(L, v); }));
  }
  c->launches += 2;
  CK(derivs_launch(c, p, L));
  CK(timed(c, CELESTE_K_TRSTEP, 0, L.stream,
           [&] { return launch_source_step(L, v, c->d_model, delta, status); }));
  if (elbo_rel) CK(cudaMemcpyAsync(elbo_rel, v.elbo_rel, v.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  c->launches += 2;
  CK(timed(c, CELESTE_K_VALUE, p->visits, L.stream,
           [&] { return launch_pixels_value(L, v, true); }));
  CK(timed(c, CELESTE_K_OTHER, 0, L.stream,
           [&] { return launch_slot_finish(L, v, true, delta, status); }));
  if (cached && !v.cache_half) {
    // one cache: accepted sources' trial renders are copied into it
    c->launches += 1;
    CK(timed(c, CELESTE_K_RENDER, p->visits, L.stream,
             [&] { return launch_commit_render(L, v, status); }));
  }
  return CELESTE_OK;
}

int celeste_render_cache(celeste_ctx* c, const celeste_plan* pc) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c) return CELESTE_EINVAL;
  if (p->v.n == 0 || !p->v.cache) return CELESTE_OK;
  Launch L = make_launch(c, p);
  CK(cudaMemsetAsync(p->v.active, 1, p->v.n, c->stream));
  int rc = run_setup(c, p, 0, p->v.n_own_pairs, false);
  if (rc) return rc;
  ++c->launches;
  return to_status(timed(c, CELESTE_K_RENDER, p->visits, L.stream,
                         [&] { return launch_render_cache(L, p->v, nullptr); }));
}

int celeste_tr_subproblem(celeste_ctx* c, int32_t n, const double* g, const double* H,
                          const double* delta, double* p, double* pred) {
  if (!c || n < 0 || (n > 0 && (!g || !H || !delta || !p || !pred))) return CELESTE_EINVAL;
  Launch L = make_launch(c, nullptr);
  ++c->launches;
  return to_status(launch_tr_subproblem(L, n, g, H, delta, p, pred));
}

int celeste_render(celeste_ctx* c, const celeste_plan* pc, float* E_out, float* V_out) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c || (!E_out && !V_out) || !p->d_patches) return CELESTE_EINVAL;
  Launch L = make_launch(c, p);
  CK(cudaMemsetAsync(p->v.active, 1, p->v.n > 0 ? p->v.n : 1, c->stream));
  int rc = run_setup(c, p, 0, p->v.n_own_pairs, false);
  if (rc) return rc;
  ++c->launches;
  return to_status(launch_render(L, p->v, E_out, V_out, p->d_patches));
}

int celeste_background(celeste_ctx* c, const celeste_plan* pc, float* bgE, float* bgV) {
  celeste_plan* p = const_cast<celeste_plan*>(pc);
  if (!c || !p || p->ctx != c || (!bgE && !bgV) || !p->d_patches) return CELESTE_EINVAL;
  Launch L = make_launch(c, p);
  CK(cudaMemsetAsync(p->v.active, 1, p->v.n > 0 ? p->v.n : 1, c->stream));
  int rc = run_setup(c, p, 0, p->v.n_pairs, false);
  if (rc) return rc;
  c->launches += 2;
  CK(launch_background(L, p->v));
  return to_status(launch_background_out(L, p->v, bgE, bgV, p->d_patches));
}

int celeste_color_sources(int32_t n, const int32_t* nbr_ptr, const int32_t* nbr_idx,
                          int32_t* color) {
  if (n < 0 || (n > 0 && (!nbr_ptr || !color))) return CELESTE_EINVAL;
  int n_colors = 0;
  std::vector<char> used;
  for (int s = 0; s < n; ++s) {
    used.assign(n_colors + 1, 0);
    for (int k = nbr_ptr[s]; k < nbr_ptr[s + 1]; ++k) {
      const int t = nbr_idx[k];
      if (t < 0 || t >= n) return CELESTE_EINVAL;
      if (t < s && color[t] <= n_colors) used[color[t]] = 1;
    }
    int col = 0;
    while (used[col]) ++col;
    color[s] = col;
    n_colors = std::max(n_colors, col + 1);
  }
  return n_colors;
}


}  // extern "C"
