// The ELBO of a whole problem (Eq. elbo over every pixel of every image,
// Sec. 2.2.3 / 4.2.2): sum over all image pixels of the delta-method pixel
// term with E and V summed over every source whose patch holds the pixel,
// minus the sum of all KL_s.  For convergence monitoring of fits; it reuses
// the setup and value-only render of the per-source path.
//
// The sources are coloured (greedy, ascending id) so that the sources of a
// class never share a pixel; each class adds its renders into per-image E
// and V buffers with plain stores, one class after another, so the result
// is deterministic.  The pixel term is then one pass over the images.
#include <algorithm>

#include "host.h"

using namespace celeste;

struct celeste_field {
  celeste_ctx* ctx = nullptr;
  std::vector<celeste_plan*> plans;
  std::vector<void*> allocs;
  float* Eimg = nullptr;
  float* Vimg = nullptr;
  double* parts = nullptr;
  double* kl = nullptr;
  const celeste_image* images = nullptr;
  const float* pixels = nullptr;
  const float* sky = nullptr;
  int64_t n_pixels = 0;
  int n_images = 0, n_sources = 0, blocks_per_image = 1;
};

extern "C" {

int celeste_field_destroy(celeste_field* F) {
  if (!F) return CELESTE_EINVAL;
  for (celeste_plan* p : F->plans) celeste_plan_destroy(p);
  for (void* a : F->allocs) cudaFree(a);
  delete F;
  return CELESTE_OK;
}

int celeste_field_create(celeste_ctx* c, const celeste_problem* pr, const celeste_tuning* tuning,
                         celeste_field** out) {
  if (!c || !pr || !out || pr->n_sources < 0 || pr->n_images < 0 || !pr->h_nbr_ptr ||
      (pr->n_nbr > 0 && !pr->h_nbr_idx) || (pr->n_images > 0 && (!pr->images || !pr->pixels)))
    return CELESTE_EINVAL;
  *out = nullptr;
  const int S = pr->n_sources;
  std::vector<int32_t> color(std::max(S, 1));
  const int n_colors = S ? celeste_color_sources(S, pr->h_nbr_ptr, pr->h_nbr_idx, color.data()) : 0;
  if (n_colors < 0) return n_colors;
  celeste_field* F = new celeste_field();
  F->ctx = c;
  F->images = pr->images;
  F->pixels = pr->pixels;
  F->sky = pr->sky;
  F->n_pixels = pr->n_pixels;
  F->n_images = pr->n_images;
  F->n_sources = S;
  int rc = CELESTE_OK;
  for (int col = 0; col < n_colors && rc == CELESTE_OK; ++col) {
    std::vector<int32_t> cls;
    for (int s = 0; s < S; ++s)
      if (color[s] == col) cls.push_back(s);
    celeste_plan* p = nullptr;
    rc = celeste_plan_create(c, pr, cls.data(), (int)cls.size(), tuning, &p);
    if (rc == CELESTE_OK) F->plans.push_back(p);
  }
  // partial sums: about eight blocks per SM over all images
  F->blocks_per_image = F->n_images ? std::max(1, 8 * c->sm_count / F->n_images) : 1;
  auto alloc = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    if (rc != CELESTE_OK) return nullptr;
    if (cudaMalloc(&ptr, bytes ? bytes : 1) != cudaSuccess) {
      rc = CELESTE_ENOMEM;
      return nullptr;
    }
    F->allocs.push_back(ptr);
    return ptr;
  };
  F->Eimg = static_cast<float*>(alloc((size_t)F->n_pixels * sizeof(float)));
  F->Vimg = static_cast<float*>(alloc((size_t)F->n_pixels * sizeof(float)));
  F->parts = static_cast<double*>(alloc((size_t)F->blocks_per_image * F->n_images * sizeof(double)));
  F->kl = static_cast<double*>(alloc((size_t)S * sizeof(double)));
  if (rc == CELESTE_OK && cudaMemset(F->kl, 0, (size_t)std::max(S, 1) * sizeof(double)) != cudaSuccess)
    rc = CELESTE_ECUDA;
  if (rc != CELESTE_OK) {
    celeste_field_destroy(F);
    return rc;
  }
  *out = F;
  return CELESTE_OK;
}

int celeste_field_elbo(celeste_ctx* c, celeste_field* F, double* out) {
  if (!c || !F || F->ctx != c || !out) return CELESTE_EINVAL;
  CK(cudaMemsetAsync(F->Eimg, 0, (size_t)F->n_pixels * sizeof(float), c->stream));
  CK(cudaMemsetAsync(F->Vimg, 0, (size_t)F->n_pixels * sizeof(float), c->stream));
  for (celeste_plan* p : F->plans) {
    const Launch L = make_launch(c, p);
    CK(launch_setup(L, p->v, c->d_model, 0, p->v.n_own_pairs, false));
    CK(launch_accumulate(L, p->v, F->Eimg, F->Vimg));
    CK(launch_kl(L, p->v, c->d_model, F->kl));
    c->launches += 3;
  }
  const Launch L = make_launch(c, nullptr);
  CK(launch_field_terms(L, F->images, F->n_images, F->blocks_per_image, F->pixels, F->sky, F->Eimg,
                        F->Vimg, c->d_err, F->parts));
  CK(launch_field_sum(L, F->parts, F->blocks_per_image * F->n_images, F->kl, F->n_sources, out));
  c->launches += 2;
  return CELESTE_OK;
}

}  // extern "C"
