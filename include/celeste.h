/*
 * celeste.h -- C ABI of the GB300 (sm_103a) library for the per-source
 * variational objective of Regier et al., "Approximate Inference for
 * Constructing Astronomical Catalogs from Images" (arXiv:1803.00113).
 *
 * What the library computes, for each light source s of a request:
 *   L_s(theta_s) = sum over the pixels m of s's patches in every image n of
 *                  -E[lambda_nm] + x_nm (log E[lambda_nm]
 *                                        - V[lambda_nm] / (2 E[lambda_nm]^2))
 *                  - KL_s(theta_s),
 * the delta-method ELBO of Eq. eq:log_p_last (Sec. 4.2.2) restricted to the
 * terms that depend on theta_s, with E and V from Eqs. conditional and vareq
 * and KL_s from Eq. kleq (Sec. 4.2.3, Supplement A); its exact gradient and
 * dense Hessian over the 27 unconstrained coordinates of theta_s; and one
 * Newton trust-region iteration on theta_s (Sec. 4.3).  -log x! is excluded.
 *
 * Conventions shared by every call
 *  - All array pointers inside celeste_problem, and every output pointer,
 *    are DEVICE pointers owned by the caller; the library never frees them.
 *    Pointers named h_* are HOST pointers read during the call only.
 *  - Every call is asynchronous on the context's stream.  The return value
 *    reports argument validation and launch errors only (0 = OK, negative =
 *    error, see CELESTE_E*); nothing aborts.  Device-side problems (a patch
 *    outside its image, non-positive sky, a non-finite value) set bits in the
 *    context's device error word, read and cleared by celeste_synchronize.
 *  - Gradients and Hessians are of L_s itself (for maximisation).
 *  - Units: pixel coordinates (x = column, y = row, pixel centres at
 *    integers); reference-frame positions in pixels; fluxes in nanomaggies.
 */
#ifndef CELESTE_H
#define CELESTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define CELESTE_OK            0
#define CELESTE_EINVAL      (-1)   /* bad argument (null, size, range)      */
#define CELESTE_ENOMEM      (-2)   /* device allocation failed              */
#define CELESTE_ECUDA       (-3)   /* a CUDA call failed                    */
#define CELESTE_EDEVICE     (-4)   /* device error word was nonzero         */
#define CELESTE_EAGAIN      (-5)   /* serving: no capacity, retry later     */
#define CELESTE_EBUSY       (-6)   /* serving: request not finished         */
#define CELESTE_ENOTFOUND   (-7)   /* serving: unknown ticket               */
#define CELESTE_ETOOLARGE   (-8)   /* request exceeds a fixed-size limit    */

/* device error word bits (celeste_synchronize returns CELESTE_EDEVICE and
 * stores the word in *device_error when any is set) */
#define CELESTE_DERR_PATCH     0x1u  /* patch rectangle outside its image */
#define CELESTE_DERR_SKY       0x2u  /* sky <= 0 at a patch pixel          */
#define CELESTE_DERR_NONFINITE 0x4u  /* non-finite value/gradient/Hessian */
#define CELESTE_DERR_TIMEOUT   0x8u  /* a bounded device wait gave up      */

/* ---- sizes ------------------------------------------------------------ */
#define CELESTE_N_THETA      27   /* Newton block per source (see layout)  */
#define CELESTE_N_BANDS       5   /* u, g, r, i, z (Table 1: B = 5)        */
#define CELESTE_N_PSF         3   /* Gaussian components of each PSF       */
#define CELESTE_MAX_PROFILE   8   /* components per galaxy profile (K)     */
#define CELESTE_MAX_COLOR     8   /* colour prior components per type (J)  */

/* ---- layout of theta (27 unconstrained doubles per source) -------------
 * Type 0 = galaxy, 1 = star; q(a_s = 1) is the star probability (Eq. eq0).
 *   0        logit q(a = star)
 *   1, 2     galaxy: mean of log r, log variance of log r   (q(r | a=0))
 *   3, 4     star:   mean of log r, log variance of log r   (q(r | a=1))
 *   5..8     galaxy colour means     9..12  star colour means
 *   13..16   galaxy log colour variances   17..20 star log colour variances
 *   21, 22   position u (x, y) in the reference frame (point mass)
 *   23       major-axis angle, radians; 24 log half-light radius (pixels);
 *   25       logit minor/major axis ratio; 26 logit profile weight (the
 *            weight of the exponential profile; de Vaucouleurs gets 1 - it)
 * Reference band r = band index 2; colour c_k = log(l_{k+1} / l_k).
 */

/* Model constants (host struct, copied into the context at creation).
 * Galaxy profiles: Eq. eq:hsi, component j of profile p has weight
 * alpha_p[j] and covariance tau_p[j] * Sigma_s.  Priors: Sec. 2.1 and
 * Table 3 (prior_r: mean and variance of log r per type; colour prior: a
 * J-component Gaussian mixture per type; e_radius: mean and variance of log
 * radius; e_profile, e_axis: Beta parameters). */
typedef struct celeste_model {
  int32_t n_exp, n_dev, n_color, reserved;
  double alpha_exp[CELESTE_MAX_PROFILE], tau_exp[CELESTE_MAX_PROFILE];
  double alpha_dev[CELESTE_MAX_PROFILE], tau_dev[CELESTE_MAX_PROFILE];
  double prior_a;
  double prior_r[2][2];
  double color_w[2][CELESTE_MAX_COLOR];
  double color_mean[2][CELESTE_MAX_COLOR][4];
  double color_cov[2][CELESTE_MAX_COLOR][4][4];
  double e_radius[2], e_profile[2], e_axis[2];
} celeste_model;

/* One image (Sec. 2.2), 256 bytes, element of a DEVICE array.
 * pixels[pix_offset + row * row_stride + col] is the photon count x_nm.
 * Sky: sky_ny x sky_nx knots at sky[sky_offset + i * sky_nx + j], spanning
 * the image (knot (i, j) at x = j (width-1)/(sky_nx-1), y = i (height-1)/
 * (sky_ny-1)), interpolated bilinearly; must be > 0.  calib: photons per
 * nanomaggy.  WCS: pixel position = wcs_A (row-major 2x2) * u + wcs_t.
 * psf[k] = {weight, mean x, mean y, cov xx, cov xy, cov yy}. */
typedef struct celeste_image {
  int64_t pix_offset, sky_offset;
  int32_t band, height, width, row_stride;
  int32_t sky_ny, sky_nx, reserved0, reserved1;
  double calib;
  double wcs_A[4];
  double wcs_t[2];
  double psf[CELESTE_N_PSF][6];
  double reserved2;
} celeste_image;

/* One patch: the pixels [x0, x0+w) x [y0, y0+h) of an image that source s
 * lights (the support restriction of Sec. 2.2.3); 32 bytes.  A patch must
 * lie inside its image.  pool_offset: where the patch's w*h pixels (row
 * major) start in the patch-pixel pool used by celeste_render/background. */
typedef struct celeste_patch {
  int32_t image, x0, y0, w, h, reserved;
  int64_t pool_offset;
} celeste_patch;

/* A problem: images, sources, patches, neighbours.  Device arrays unless
 * named h_*.  Source s owns patches[patch_ptr[s] .. patch_ptr[s+1]) and its
 * neighbours (sources whose patches overlap s's) are nbr_idx[nbr_ptr[s] ..
 * nbr_ptr[s+1]).  The h_* copies of the index arrays are read by
 * celeste_plan_create only. */
typedef struct celeste_problem {
  const float* pixels;
  const float* sky;
  const celeste_image* images;
  double* theta;                  /* [n_sources][27]; newton_step updates it */
  const int32_t* patch_ptr;
  const celeste_patch* patches;
  const int32_t* nbr_ptr;
  const int32_t* nbr_idx;
  const int32_t* h_patch_ptr;
  const celeste_patch* h_patches;
  const celeste_image* h_images;
  const int32_t* h_nbr_ptr;
  const int32_t* h_nbr_idx;
  int64_t n_pixels, n_sky, n_pool;
  int32_t n_images, n_sources, n_patches, n_nbr;
  /* Optional (may be NULL): float2 (E, V) of each source's own moments at
   * each of its patch pixels, in the patch-pool layout ([n_pool] pairs at
   * each patch's pool_offset).  With it, neighbour backgrounds are gathered
   * from the cache instead of re-rendering every neighbour (the same values,
   * bit for bit).  celeste_newton_step keeps it current for the sources
   * whose step was accepted and celeste_fit_run keeps it current; after
   * changing theta any other way, refresh it with celeste_render_cache. */
  float* render_cache;
  /* Optional (may be NULL; read only with render_cache): [n_sources] bytes,
   * 0 or 1, on the device.  When given, render_cache holds two halves of
   * n_pool float2 each (4 n_pool floats) and render_cache_half[s] names the
   * half that holds source s's current moments (zeros: all in the first).
   * celeste_newton_step then renders each trial point into the source's
   * other half and flips the entry of the sources whose step it accepts,
   * which moves no pixel data; without it the step copies the accepted
   * renders into the single cache. */
  uint8_t* render_cache_half;
} celeste_problem;

/* Tile shape of the pixel kernels: the number of pixels one warp reduces
 * into one item, by patch area bucket ([0, 1024), [1024, 4096),
 * [4096, 16384), [16384, inf) pixels), picked by the autotuner of the Python
 * layer.  Zeros select pixels_per_item (itself 0 = 256). */
typedef struct celeste_tuning {
  int32_t pixels_per_item;    /* default pixels per item, 32..65536 */
  int32_t warps_per_block;    /* reserved (the pixel kernels use 4) */
  int32_t blocks_per_sm;      /* persistent grid = SMs * blocks_per_sm (0 = as many
                                 as fit on an SM, per kernel) */
  int32_t reserved;
  int32_t ppi_bucket[4];      /* per patch-area bucket, 0 = pixels_per_item */
} celeste_tuning;

typedef struct celeste_ctx celeste_ctx;
typedef struct celeste_plan celeste_plan;

/* Creates a context on `device` that launches on `cuda_stream` (a
 * cudaStream_t, or NULL for the legacy default stream).  Copies *model.
 * Returns CELESTE_EINVAL for out-of-range model sizes. */
int celeste_create(celeste_ctx** out, const celeste_model* model, int device, void* cuda_stream);
int celeste_destroy(celeste_ctx* ctx);
/* Waits for the context's stream; returns CELESTE_EDEVICE (and the word in
 * *device_error, may be NULL) if a device error bit was set, then clears it. */
int celeste_synchronize(celeste_ctx* ctx, uint32_t* device_error);
/* Number of kernel launches this context has issued (for accounting). */
int64_t celeste_launch_count(const celeste_ctx* ctx);
/* Event timing of kernel launches: when enabled, every launch of a timed
 * kind is bracketed by a pair of CUDA events recorded on the context's
 * stream (enabling also clears the list of pairs; events are reused).  on
 * is a mask of (1 << CELESTE_K_*) bits: 0 disables, -1 times every kind.
 * celeste_profile_read synchronises the stream and returns, for the
 * derivative pixel kernel (the dominant kernel of celeste_elbo_grad_hess
 * and celeste_newton_step), the summed kernel time (ms) over the recorded
 * pairs, their number and the source-pixel visits they processed; reset !=
 * 0 clears the list.  A CUDA graph captured with timing enabled records the
 * same pairs on every replay: read with reset = 0 after each replay.
 * Launches inside a region fit (celeste_fit_run) are never timed. */
int celeste_profile_enable(celeste_ctx* ctx, int on);
int celeste_profile_read(celeste_ctx* ctx, int reset, double* total_ms, int64_t* launches,
                         int64_t* visits);
/* The same timing for every kernel kind: ms[k], launches[k] and (for pixel
 * kernels) visits[k] for k < CELESTE_K_COUNT; visits may be NULL. */
#define CELESTE_K_SETUP       0
#define CELESTE_K_BACKGROUND  1
#define CELESTE_K_DERIVS      2   /* value + gradient + Hessian pixel pass */
#define CELESTE_K_GRAD        3   /* value + gradient pixel pass */
#define CELESTE_K_VALUE       4   /* value-only pixel pass */
#define CELESTE_K_EPILOGUE    5
#define CELESTE_K_TRSTEP      6
#define CELESTE_K_OTHER       7
#define CELESTE_K_RENDER      8   /* render-cache refresh */
#define CELESTE_K_COUNT       9
int celeste_profile_kernels(celeste_ctx* ctx, int reset, double* ms, int64_t* launches,
                            int64_t* visits);

/* A plan binds a list of sources of a problem to a work decomposition
 * (per source, image and pixel tile) and owns the device scratch of the
 * calls below (component tables, background buffers, per-tile partial
 * sums, Newton state).  h_src_ids: HOST array of n distinct source ids.
 * Sources of one plan are updated together by celeste_newton_step, so they
 * should not overlap (one colour class of the overlap graph, Sec. 4.4).
 * tuning may be NULL.  The plan keeps pointers into *problem's arrays, not
 * the struct itself; it stays valid while those arrays do. */
int celeste_plan_create(celeste_ctx* ctx, const celeste_problem* problem,
                        const int32_t* h_src_ids, int32_t n, const celeste_tuning* tuning,
                        celeste_plan** out);
int celeste_plan_destroy(celeste_plan* plan);
/* Visits (source-pixel pairs) of one evaluation of the plan. */
int64_t celeste_plan_visits(const celeste_plan* plan);

/* L_s, its gradient and Hessian for every source of the plan (Eqs. elbo,
 * eq:log_p_last, conditional, vareq, kleq).  Outputs (device, n = plan
 * size, in plan order): elbo[n] = L_s; elbo_rel[n] = L_s minus the value
 * with source s absent (sky and neighbours only), may be NULL; grad[n][27];
 * hess[n][27][27] (full, symmetric).  Neighbours are frozen at theta. */
int celeste_elbo_grad_hess(celeste_ctx* ctx, const celeste_plan* plan,
                           double* elbo, double* elbo_rel, double* grad, double* hess);

/* Value and gradient only (the gradient-only mode): the pixel pass keeps 12
 * sums per tile instead of 64, about a third of the work of
 * celeste_elbo_grad_hess (Sec. 4.3 compares the two costs).  Outputs as in
 * celeste_elbo_grad_hess; elbo and elbo_rel may be NULL. */
int celeste_elbo_grad(celeste_ctx* ctx, const celeste_plan* plan, double* elbo, double* elbo_rel,
                      double* grad);

/* Value only (no derivatives): elbo[n] and elbo_rel[n] (either may be NULL). */
int celeste_elbo(celeste_ctx* ctx, const celeste_plan* plan, double* elbo, double* elbo_rel);

/* The pixel part of L_rel alone (no KL) for every source of the plan:
 * out[n] (device, plan order) = sum over the source's patch pixels of the
 * pixel term with the source minus the same sum without it.  With theta
 * encoding point values (log-variances of -40, the type logit at +-40) this
 * is log p(x | w_s, a_s, z_-s) - log p(x | source absent) of the Poisson
 * likelihood (Eq. eq:log_p_last's V terms vanish), the quantity the AIS and
 * slice-sampling MCMC of Sec. 3 evaluates for each proposal. */
int celeste_loglik(celeste_ctx* ctx, const celeste_plan* plan, double* out);

/* One trust-region Newton iteration (Sec. 4.3) on every source of the plan
 * whose status is not CONVERGED/FAILED/MAXITER: evaluate L_s, g, H at theta; solve
 * max g.p + p.H.p/2 s.t. |p| <= delta exactly in FP64; evaluate L_s at
 * theta + p; accept when the ratio of actual to predicted gain exceeds 0.1;
 * update the radius (shrink to |p|/4 below 1/4, double up to 100 above 3/4
 * when the step reached the boundary).  delta[n_sources] and
 * status[n_sources] (device, indexed by source id) carry the state between
 * calls; initialise delta to 1 and status to 0.  Status values:
 * CELESTE_ST_*.  elbo_rel (device [n], plan order, may be NULL) receives
 * L_s - L_s(absent) at the iterate before the step.  A trial point whose
 * value is not finite (an FP32 overflow far from the iterate) is rejected
 * like any other failed step and raises no device error. */
#define CELESTE_ST_ACCEPTED   0
#define CELESTE_ST_REJECTED   1
#define CELESTE_ST_CONVERGED  2
#define CELESTE_ST_MAXITER    3
#define CELESTE_ST_FAILED    (-1)
int celeste_newton_step(celeste_ctx* ctx, const celeste_plan* plan,
                        double* delta, int32_t* status, double* elbo_rel);

/* Block coordinate ascent over a region (Sec. 4.3, 4.4): a fit object
 * colours the overlap graph of the n sources h_src_ids (HOST array,
 * distinct ids) greedily in ascending id (two region sources conflict when
 * one is in the other's neighbour list) and holds one plan per colour class
 * plus the per-source Newton state.  Sources outside the region stay fixed
 * and only enter as neighbours.  tuning may be NULL. */
typedef struct celeste_fit celeste_fit;
int celeste_fit_create(celeste_ctx* ctx, const celeste_problem* problem,
                       const int32_t* h_src_ids, int32_t n, const celeste_tuning* tuning,
                       celeste_fit** out);
int celeste_fit_destroy(celeste_fit* fit);
/* Number of colour classes of the region. */
int celeste_fit_classes(const celeste_fit* fit);
/* Runs the fit: passes over the classes in ascending colour; in a pass each
 * source gets one fresh subsolver call (radius 1, status 0) of at most
 * max_iter trust-region Newton iterations (celeste_newton_step's
 * iteration) with every other source at its current value; the neighbour
 * background of a class is rendered once per pass.  Within a class the
 * iterations run on the device (a CUDA graph loop per class, no host
 * round trip); the host waits once per pass.  The fit stops after the first
 * pass whose total ELBO gain (the sum of the actual gains of its accepted
 * steps) is at most pass_tol times the region's source count, or after
 * max_passes passes.  0 selects max_passes = 5, max_iter = 50 (both at most
 * 1000).  Updates problem->theta of the region's sources in place.  Host
 * outputs (may be NULL): *passes_out, pass_gain[max_passes]. */
int celeste_fit_run(celeste_ctx* ctx, celeste_fit* fit, int32_t max_passes, int32_t max_iter,
                    double pass_tol, int32_t* passes_out, double* pass_gain);
/* Per-source results of the last run, DEVICE arrays indexed by source id
 * ([n_sources], entries of sources outside the region are unspecified; each
 * may be NULL): status of the last subsolver call (CELESTE_ST_*), Newton
 * iterations and accepted steps over all passes, final trust radius. */
int celeste_fit_results(celeste_ctx* ctx, const celeste_fit* fit, int32_t* status,
                        int32_t* iters, int32_t* accepted, double* delta);

/* A first-order subsolver, to compare with the Newton trust-region one
 * (Sec. 4.3 reports tens of Newton iterations against thousands for
 * first-order methods and at times for BFGS): limited-memory BFGS (history
 * m <= 16) on every source of the plan with a backtracking Armijo line
 * search (c1 = 1e-4, unit step halved), neighbours frozen.  One call of
 * celeste_lbfgs_step evaluates the value and gradient (the gradient-only
 * pixel pass) of the sources whose last step was accepted, makes their new
 * direction, and evaluates the value at the trial point of every source
 * still running.  status[n_sources] (device, by source id): ACCEPTED,
 * REJECTED (backtracking), CONVERGED when the model gain of the full
 * quasi-Newton step, g.d / 2, is at most 1e-12 (1 + |L_rel|) or the step
 * shrank to nothing.  A trial whose
 * expected gain is below the value's FP32 noise (1e-7 (1 + |L_rel|)) is
 * accepted unless the value drops by more than that noise.  Sources already
 * CONVERGED/FAILED/MAXITER are skipped; initialise to 0.  target (device
 * [n], plan order, may be NULL): L_rel values whose first crossing is
 * recorded.  celeste_lbfgs_counts copies, per slot (device [n]), the
 * accepted steps, the trial evaluations and the accepted steps at which the
 * target was first reached (-1 if not).  celeste_lbfgs_reset clears the
 * history and counters (not theta). */
typedef struct celeste_lbfgs celeste_lbfgs;
int celeste_lbfgs_create(celeste_ctx* ctx, const celeste_plan* plan, int32_t m,
                         celeste_lbfgs** out);
int celeste_lbfgs_destroy(celeste_lbfgs* lbfgs);
int celeste_lbfgs_reset(celeste_ctx* ctx, celeste_lbfgs* lbfgs);
int celeste_lbfgs_step(celeste_ctx* ctx, celeste_lbfgs* lbfgs, int32_t* status,
                       const double* target);
int celeste_lbfgs_counts(celeste_ctx* ctx, const celeste_lbfgs* lbfgs, int32_t* iters,
                         int32_t* fevals, int32_t* reached);

/* The ELBO of the whole problem (Eq. elbo over every pixel of every image,
 * Sec. 2.2.3 and 4.2.2): the sum over all image pixels of
 * -E + x (log E - V / (2 E^2)), E = sky + the E_q of every source whose
 * patch holds the pixel and V the sum of their V_q, minus the sum of KL_s
 * over all sources; -log x! is excluded.  For monitoring fits.  A field
 * object colours all sources (greedy, ascending id), holds one plan per
 * colour class and per-image E and V buffers (8 bytes per image pixel).
 * celeste_field_elbo writes out[0] = ELBO, out[1] = the pixel sum,
 * out[2] = the KL sum (DEVICE array of 3 doubles) at the current theta;
 * the result is deterministic.  The neighbour lists must name every pair
 * of sources whose patches overlap (the colouring relies on it). */
typedef struct celeste_field celeste_field;
int celeste_field_create(celeste_ctx* ctx, const celeste_problem* problem,
                         const celeste_tuning* tuning, celeste_field** out);
int celeste_field_destroy(celeste_field* field);
int celeste_field_elbo(celeste_ctx* ctx, celeste_field* field, double* out);

/* ---- serving (region fits submitted by independent callers) ------------
 *
 * A server owns worker threads, each with its own context, stream and
 * resident device arenas.  celeste_submit validates a region request,
 * copies it (the caller's buffers may be reused as soon as it returns) and
 * queues it.  Batching is continuous: a worker fits its running requests
 * together, pass by pass, as one fit in which each request is a segment
 * with its own passes and stopping rule (as celeste_fit_run: max_passes,
 * max_iter, pass_tol), so a request's result is the same whether it ran
 * alone or with others; after every pass it retires the requests whose
 * segments stopped and admits queued requests, in order, while their
 * footprint (device_bytes is the budget, estimated per request from its
 * pixels, patches and sources) fits beside the running ones.  A request
 * that arrives while others run thus starts at the next pass boundary.
 * celeste_poll returns the result once the request's segment has stopped.
 *
 * Errors: celeste_submit returns CELESTE_EINVAL for a malformed request
 * (sizes, offsets, a patch outside its image, a neighbour index out of
 * range), CELESTE_ETOOLARGE when the request alone exceeds device_bytes,
 * CELESTE_EAGAIN when the queued requests already hold queue_bytes.
 * celeste_poll returns CELESTE_EBUSY until the request is done (waiting up
 * to wait_ms for it), CELESTE_ENOTFOUND for an unknown or already collected
 * ticket, and otherwise the request's outcome (CELESTE_OK, or the error of
 * its batch, e.g. CELESTE_EDEVICE when a device error bit was raised). */
typedef struct celeste_server_config {
  int32_t workers;          /* worker threads (0 = 2) */
  int32_t max_batch;        /* running requests per worker (0 = no limit) */
  int64_t device_bytes;     /* per-worker budget of resident request data (0 = 4 GiB) */
  int64_t queue_bytes;      /* admission limit of queued requests (0 = 4 x budget x workers) */
  int32_t max_passes;       /* fit limits (0 = 5, 50) */
  int32_t max_iter;
  double pass_tol;          /* nats per source */
  int32_t start_paused;     /* workers take no batch until celeste_server_pause(s, 0) */
  int32_t pixels_per_item;  /* tile size of the pixel kernels (0 = 256) */
} celeste_server_config;

/* One region: HOST arrays laid out as in celeste_problem (offsets, patch
 * and neighbour indices local to the request). */
typedef struct celeste_region_request {
  const float* pixels;
  const float* sky;
  const celeste_image* images;
  const double* theta;             /* [n_sources][27] initial values */
  const int32_t* patch_ptr;        /* [n_sources + 1] */
  const celeste_patch* patches;
  const int32_t* nbr_ptr;          /* [n_sources + 1] */
  const int32_t* nbr_idx;
  int64_t n_pixels, n_sky;
  int32_t n_images, n_sources, n_patches, n_nbr;
} celeste_region_request;

typedef struct celeste_request_info {
  int32_t n_sources;
  int32_t passes;               /* passes the request's fit ran */
  int32_t batch_requests;       /* requests running beside it when it started, itself included */
  uint32_t device_error;        /* device error word of its batch (CELESTE_DERR_*) */
  double last_pass_gain;        /* ELBO gain of its last pass */
  double queue_s;               /* submit -> taken by a worker */
  double latency_s;             /* submit -> result ready */
  double t_start_s, t_done_s;   /* taken by a worker, result ready: seconds on the
                                   server's monotonic clock (comparable between
                                   requests of one server) */
} celeste_request_info;

typedef struct celeste_server celeste_server;
int celeste_server_create(const celeste_model* model, int device,
                          const celeste_server_config* config, celeste_server** out);
/* Stops the workers after their current pass; queued and unfinished
 * requests are dropped. */
int celeste_server_destroy(celeste_server* server);
int celeste_server_pause(celeste_server* server, int paused);
int celeste_submit(celeste_server* server, const celeste_region_request* request,
                   uint64_t* ticket);
/* theta_out (HOST [n_sources][27]) and status_out (HOST [n_sources],
 * CELESTE_ST_* of each source's last subsolver call) may be NULL.  A
 * collected ticket is forgotten. */
int celeste_poll(celeste_server* server, uint64_t ticket, int32_t wait_ms, double* theta_out,
                 int32_t* status_out, celeste_request_info* info);
/* Kernel launches so far and busy periods (a worker starting from no
 * running request); returns the first worker error. */
int celeste_server_stats(celeste_server* server, int64_t* launches, int64_t* batches);

/* Only the FP64 trust-region subproblem, for n independent problems:
 * maximise g.p + p.H.p/2 subject to |p| <= delta (Sec. 4.3).  g[n][27],
 * H[n][27][27], delta[n] in; p[n][27], pred[n] (= g.p + p.H.p/2) out; all
 * device arrays. */
int celeste_tr_subproblem(celeste_ctx* ctx, int32_t n, const double* g, const double* H,
                          const double* delta, double* p, double* pred);

/* Rendering (Sec. 2.2.3, Eqs. conditional and vareq): for every patch of
 * every plan source, the source's own E_q[l f] and V_q[l f] at each patch
 * pixel, written to E_out/V_out at the patch's pool_offset (row major). */
int celeste_render(celeste_ctx* ctx, const celeste_plan* plan, float* E_out, float* V_out);
/* Renders the plan's sources at theta into problem->render_cache (no-op
 * when the problem has none). */
int celeste_render_cache(celeste_ctx* ctx, const celeste_plan* plan);
/* Sky plus the moments of the neighbours at each patch pixel of every
 * plan source (the background a source is fitted against). */
int celeste_background(celeste_ctx* ctx, const celeste_plan* plan, float* bgE_out, float* bgV_out);

/* Allocation-free evaluation, for callers that must not allocate device
 * memory: code that runs while its memory pool is locked or being
 * defragmented, plugins of a host program that owns every device
 * allocation, and callers that cannot afford the synchronisation a
 * cudaMalloc may bring mid-work.  (The paper has no counterpart: this is a
 * property of the library, not of the method.)
 *
 * Computes what celeste_elbo_grad_hess computes for the n sources
 * h_src_ids (HOST array) of *problem -- the same kernels, with the work
 * decomposition of a plan made with the default tiles (256 pixels per item)
 * and without the problem's render cache, whose backgrounds are bitwise the
 * same as rendered ones -- with no context and no plan: every intermediate
 * lives in one file-scope device array of CELESTE_NOALLOC_BYTES that each
 * GPU loading the library holds until the process exits.  It calls no
 * cudaMalloc/cudaFree and no allocating routine; model constants and the
 * work decomposition are staged from static host arrays with
 * cudaMemcpyAsync.  Runs on the current device and on cuda_stream (a
 * cudaStream_t, or NULL).  Outputs as in celeste_elbo_grad_hess;
 * device_error (device uint32, may be NULL) receives the device error word
 * of this call.  Returns CELESTE_EINVAL when cuda_stream is being captured
 * (the staging arrays are rewritten by every call).
 *
 * The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and the kernels'
 * occupancy; make that first call before any stream capture on that
 * device.  Limits: at most CELESTE_NOALLOC_MAX_SOURCES
 * sources, 4096 (source, image) patches including neighbours' patches,
 * 32768 pixel tiles of 256 pixels, and everything within the byte size;
 * larger requests return CELESTE_ETOOLARGE before any work is queued.
 * Every call shares the array and finds the previous call's contents in
 * it (what must start at zero is cleared each call): calls that overlap on
 * the GPU (on different streams, or from several host threads) race, so
 * serialise them. */
#define CELESTE_NOALLOC_BYTES        (16u << 20)
#define CELESTE_NOALLOC_MAX_SOURCES  1024
int celeste_elbo_grad_hess_noalloc(const celeste_model* model, const celeste_problem* problem,
                                   const int32_t* h_src_ids, int32_t n, void* cuda_stream,
                                   double* elbo, double* elbo_rel, double* grad, double* hess,
                                   uint32_t* device_error);

/* Greedy colouring of the overlap graph by ascending source id (host):
 * colour[s] = smallest colour unused by lower-id neighbours.  Returns the
 * number of colours, or a negative error. */
int celeste_color_sources(int32_t n_sources, const int32_t* h_nbr_ptr, const int32_t* h_nbr_idx,
                          int32_t* h_color_out);

#ifdef __cplusplus
}
#endif
#endif /* CELESTE_H */
