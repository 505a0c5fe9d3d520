"""Python binding of the CUDA library (``include/celeste.h``) via ctypes.

Argument marshalling only: every step of the objective, its derivatives and
the Newton step runs in the library's kernels.  PyTorch provides device
memory and the stream.  The binding refuses to run without the compiled
library and a CUDA device; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import build_lib

N_THETA = 27
ST_ACCEPTED, ST_REJECTED, ST_CONVERGED, ST_MAXITER, ST_FAILED = 0, 1, 2, 3, -1
# device error word bits (celeste_synchronize, device_error outputs)
DERR_PATCH, DERR_SKY, DERR_NONFINITE, DERR_TIMEOUT = 0x1, 0x2, 0x4, 0x8

IMAGE_DTYPE = np.dtype([
    ("pix_offset", "<i8"), ("sky_offset", "<i8"),
    ("band", "<i4"), ("height", "<i4"), ("width", "<i4"), ("row_stride", "<i4"),
    ("sky_ny", "<i4"), ("sky_nx", "<i4"), ("reserved0", "<i4"), ("reserved1", "<i4"),
    ("calib", "<f8"), ("wcs_A", "<f8", (4,)), ("wcs_t", "<f8", (2,)),
    ("psf", "<f8", (3, 6)), ("reserved2", "<f8")])
PATCH_DTYPE = np.dtype([("image", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("w", "<i4"),
                        ("h", "<i4"), ("reserved", "<i4"), ("pool_offset", "<i8")])
assert IMAGE_DTYPE.itemsize == 256 and PATCH_DTYPE.itemsize == 32


class _Model(ctypes.Structure):
    _fields_ = [("n_exp", ctypes.c_int32), ("n_dev", ctypes.c_int32),
                ("n_color", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("alpha_exp", ctypes.c_double * 8), ("tau_exp", ctypes.c_double * 8),
                ("alpha_dev", ctypes.c_double * 8), ("tau_dev", ctypes.c_double * 8),
                ("prior_a", ctypes.c_double), ("prior_r", ctypes.c_double * 4),
                ("color_w", ctypes.c_double * 16), ("color_mean", ctypes.c_double * 64),
                ("color_cov", ctypes.c_double * 256), ("e_radius", ctypes.c_double * 2),
                ("e_profile", ctypes.c_double * 2), ("e_axis", ctypes.c_double * 2)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("queue_bytes", ctypes.c_int64),
                ("max_passes", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("pass_tol", ctypes.c_double), ("start_paused", ctypes.c_int32),
                ("pixels_per_item", ctypes.c_int32)]


class _Request(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("pixels", "sky", "images", "theta", "patch_ptr",
                                                 "patches", "nbr_ptr", "nbr_idx")] + \
               [("n_pixels", ctypes.c_int64), ("n_sky", ctypes.c_int64),
                ("n_images", ctypes.c_int32), ("n_sources", ctypes.c_int32),
                ("n_patches", ctypes.c_int32), ("n_nbr", ctypes.c_int32)]


class _RequestInfo(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("batch_requests", ctypes.c_int32), ("device_error", ctypes.c_uint32),
                ("last_pass_gain", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("t_start_s", ctypes.c_double),
                ("t_done_s", ctypes.c_double)]


class _Problem(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "pixels", "sky", "images", "theta", "patch_ptr", "patches", "nbr_ptr", "nbr_idx",
        "h_patch_ptr", "h_patches", "h_images", "h_nbr_ptr", "h_nbr_idx")] + [
        ("n_pixels", ctypes.c_int64), ("n_sky", ctypes.c_int64), ("n_pool", ctypes.c_int64),
        ("n_images", ctypes.c_int32), ("n_sources", ctypes.c_int32),
        ("n_patches", ctypes.c_int32), ("n_nbr", ctypes.c_int32),
        ("render_cache", ctypes.c_void_p), ("render_cache_half", ctypes.c_void_p)]


class _Tuning(ctypes.Structure):
    _fields_ = [("pixels_per_item", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ppi_bucket", ctypes.c_int32 * 4)]

AREA_BUCKETS = (1024, 4096, 16384)   # patch-area bucket edges of celeste_tuning


_LIB = None


def lib():
    """The loaded library; raises if it was not built or CUDA is unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(build_lib.LIB):
        raise RuntimeError(f"{build_lib.LIB} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(build_lib.LIB)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "celeste_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(_Model), ctypes.c_int, P]),
        "celeste_destroy": (ctypes.c_int, [P]),
        "celeste_synchronize": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint32)]),
        "celeste_launch_count": (I64, [P]),
        "celeste_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "celeste_profile_read": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(D),
                                                ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "celeste_profile_kernels": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "celeste_plan_create": (ctypes.c_int, [P, ctypes.POINTER(_Problem), P, I32,
                                               ctypes.POINTER(_Tuning), ctypes.POINTER(P)]),
        "celeste_plan_destroy": (ctypes.c_int, [P]),
        "celeste_plan_visits": (I64, [P]),
        "celeste_elbo_grad_hess": (ctypes.c_int, [P, P, P, P, P, P]),
        "celeste_elbo": (ctypes.c_int, [P, P, P, P]),
        "celeste_elbo_grad": (ctypes.c_int, [P, P, P, P, P]),
        "celeste_loglik": (ctypes.c_int, [P, P, P]),
        "celeste_newton_step": (ctypes.c_int, [P, P, P, P, P]),
        "celeste_tr_subproblem": (ctypes.c_int, [P, I32, P, P, P, P, P]),
        "celeste_render": (ctypes.c_int, [P, P, P, P]),
        "celeste_background": (ctypes.c_int, [P, P, P, P]),
        "celeste_render_cache": (ctypes.c_int, [P, P]),
        "celeste_color_sources": (ctypes.c_int, [I32, P, P, P]),
        "celeste_fit_create": (ctypes.c_int, [P, ctypes.POINTER(_Problem), P, I32,
                                              ctypes.POINTER(_Tuning), ctypes.POINTER(P)]),
        "celeste_fit_destroy": (ctypes.c_int, [P]),
        "celeste_fit_classes": (ctypes.c_int, [P]),
        "celeste_fit_run": (ctypes.c_int, [P, P, I32, I32, D, ctypes.POINTER(I32), P]),
        "celeste_fit_results": (ctypes.c_int, [P, P, P, P, P, P]),
        "celeste_lbfgs_create": (ctypes.c_int, [P, P, I32, ctypes.POINTER(P)]),
        "celeste_lbfgs_destroy": (ctypes.c_int, [P]),
        "celeste_lbfgs_reset": (ctypes.c_int, [P, P]),
        "celeste_lbfgs_step": (ctypes.c_int, [P, P, P, P]),
        "celeste_lbfgs_counts": (ctypes.c_int, [P, P, P, P, P]),
        "celeste_field_create": (ctypes.c_int, [P, ctypes.POINTER(_Problem),
                                                ctypes.POINTER(_Tuning), ctypes.POINTER(P)]),
        "celeste_field_destroy": (ctypes.c_int, [P]),
        "celeste_field_elbo": (ctypes.c_int, [P, P, P]),
        "celeste_server_create": (ctypes.c_int, [ctypes.POINTER(_Model), ctypes.c_int,
                                                 ctypes.POINTER(_ServerConfig), ctypes.POINTER(P)]),
        "celeste_server_destroy": (ctypes.c_int, [P]),
        "celeste_server_pause": (ctypes.c_int, [P, ctypes.c_int]),
        "celeste_submit": (ctypes.c_int, [P, ctypes.POINTER(_Request),
                                          ctypes.POINTER(ctypes.c_uint64)]),
        "celeste_poll": (ctypes.c_int, [P, ctypes.c_uint64, I32, P, P,
                                        ctypes.POINTER(_RequestInfo)]),
        "celeste_server_stats": (ctypes.c_int, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "celeste_elbo_grad_hess_noalloc": (ctypes.c_int, [ctypes.POINTER(_Model),
                                                          ctypes.POINTER(_Problem), P, I32, P,
                                                          P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def exported_symbols():
    """Names the header declares, for the load check."""
    return ["celeste_create", "celeste_destroy", "celeste_synchronize", "celeste_launch_count",
            "celeste_profile_enable", "celeste_profile_read", "celeste_profile_kernels",
            "celeste_plan_create", "celeste_plan_destroy", "celeste_plan_visits",
            "celeste_elbo_grad_hess", "celeste_elbo", "celeste_elbo_grad", "celeste_loglik",
            "celeste_newton_step",
            "celeste_tr_subproblem", "celeste_render", "celeste_background",
            "celeste_render_cache",
            "celeste_color_sources", "celeste_fit_create", "celeste_fit_destroy",
            "celeste_fit_classes", "celeste_fit_run", "celeste_fit_results",
            "celeste_lbfgs_create", "celeste_lbfgs_destroy", "celeste_lbfgs_reset",
            "celeste_lbfgs_step", "celeste_lbfgs_counts",
            "celeste_field_create", "celeste_field_destroy", "celeste_field_elbo",
            "celeste_server_create", "celeste_server_destroy", "celeste_server_pause",
            "celeste_submit", "celeste_poll", "celeste_server_stats",
            "celeste_elbo_grad_hess_noalloc"]


KERNEL_KINDS = ("setup", "background", "derivs", "grad", "value", "epilogue", "tr_step", "other",
                "render")


class CelesteError(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        raise CelesteError(f"{what} failed with code {rc}")
    return rc


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def model_struct(model) -> _Model:
    m = _Model()
    m.n_exp, m.n_dev = len(model.alpha_exp), len(model.alpha_dev)
    m.n_color = model.color_w.shape[1]
    for name in ("alpha_exp", "tau_exp", "alpha_dev", "tau_dev"):
        arr = getattr(m, name)
        for j, x in enumerate(getattr(model, name)):
            arr[j] = float(x)
    m.prior_a = float(model.prior_a)
    for k, x in enumerate(np.asarray(model.prior_r, dtype=np.float64).ravel()):
        m.prior_r[k] = x
    J = m.n_color
    w = np.zeros((2, 8)); w[:, :J] = model.color_w
    mu = np.zeros((2, 8, 4)); mu[:, :J] = model.color_mean
    cov = np.tile(np.eye(4), (2, 8, 1, 1)); cov[:, :J] = model.color_cov
    for k, x in enumerate(w.ravel()):
        m.color_w[k] = x
    for k, x in enumerate(mu.ravel()):
        m.color_mean[k] = x
    for k, x in enumerate(cov.ravel()):
        m.color_cov[k] = x
    for name in ("e_radius", "e_profile", "e_axis"):
        arr = getattr(m, name)
        for k, x in enumerate(getattr(model, name)):
            arr[k] = float(x)
    return m


class Context:
    """A library context bound to a device and a stream (default: torch's
    current stream)."""

    def __init__(self, model, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise CelesteError("no CUDA device: the library has no CPU path")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._model = model_struct(model)
        h = ctypes.c_void_p()
        _check(lib().celeste_create(ctypes.byref(h), ctypes.byref(self._model), device,
                                    ctypes.c_void_p(self.stream.cuda_stream)), "celeste_create")
        self.handle = h

    def synchronize(self):
        w = ctypes.c_uint32(0)
        rc = lib().celeste_synchronize(self.handle, ctypes.byref(w))
        if rc < 0:
            raise CelesteError(f"device error word 0x{w.value:x} (code {rc})")

    def launches(self) -> int:
        return int(lib().celeste_launch_count(self.handle))

    def profile(self, on, kinds=None):
        """Event timing: off, the derivative kernel only (on=True), or the
        named kernel kinds (kinds="all" or an iterable of KERNEL_KINDS)."""
        if not on:
            mode = 0
        elif kinds == "all":
            mode = -1
        else:
            mode = sum(1 << KERNEL_KINDS.index(k) for k in (kinds or ("derivs",)))
        _check(lib().celeste_profile_enable(self.handle, mode), "celeste_profile_enable")

    def profile_read(self, reset: bool = True):
        """(kernel ms, timed launches, visits) of the derivative kernel."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        vis = ctypes.c_int64(0)
        _check(lib().celeste_profile_read(self.handle, 1 if reset else 0, ctypes.byref(ms),
                                          ctypes.byref(n), ctypes.byref(vis)),
               "celeste_profile_read")
        return ms.value, n.value, vis.value

    def profile_kernels(self, reset: bool = True):
        """{kind: (ms, launches, visits)} of every timed kernel kind."""
        k = len(KERNEL_KINDS)
        ms = np.zeros(k)
        n = np.zeros(k, dtype=np.int64)
        vis = np.zeros(k, dtype=np.int64)
        _check(lib().celeste_profile_kernels(self.handle, 1 if reset else 0, ms.ctypes.data,
                                             n.ctypes.data, vis.ctypes.data),
               "celeste_profile_kernels")
        return {name: (float(ms[i]), int(n[i]), int(vis[i])) for i, name in enumerate(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_structs(p):
    """Image and patch struct arrays of a fields.Problem, in the C layouts."""
    img = np.zeros(p.n_images, dtype=IMAGE_DTYPE)
    img["pix_offset"] = p.img_pix_off
    img["sky_offset"] = p.img_sky_off
    img["band"] = p.img_band
    img["height"] = p.img_h
    img["width"] = p.img_w
    img["row_stride"] = p.img_stride
    img["sky_ny"] = p.img_sky_ny
    img["sky_nx"] = p.img_sky_nx
    img["calib"] = p.img_calib
    img["wcs_A"] = p.img_A.reshape(-1, 4)
    img["wcs_t"] = p.img_t
    img["psf"] = p.img_psf
    pat = np.zeros(p.n_patches, dtype=PATCH_DTYPE)
    pat["image"] = p.patch_img
    pat["x0"] = p.patch_x0
    pat["y0"] = p.patch_y0
    pat["w"] = p.patch_w
    pat["h"] = p.patch_h
    area = p.patch_w.astype(np.int64) * p.patch_h.astype(np.int64)
    pat["pool_offset"] = np.concatenate([[0], np.cumsum(area)[:-1]]) if len(area) else []
    return img, pat, int(area.sum())


class DeviceProblem:
    """A fields.Problem uploaded to the device (plus the host index copies)."""

    def __init__(self, problem, device=None, render_cache: bool = False):
        dev = device or torch.device("cuda", 0)
        self.host = problem
        p = problem
        img, pat, n_pool = _host_structs(p)
        self.n_pool = n_pool
        self.pool_offset = pat["pool_offset"].copy()
        self.h_images = img
        self.h_patches = pat
        self.h_patch_ptr = np.ascontiguousarray(p.patch_ptr, dtype=np.int32)
        self.h_nbr_ptr = np.ascontiguousarray(p.nbr_ptr, dtype=np.int32)
        self.h_nbr_idx = np.ascontiguousarray(p.nbr_idx, dtype=np.int32)
        if self.h_nbr_idx.size == 0:
            self.h_nbr_idx = np.zeros(1, dtype=np.int32)

        def up(a, dtype=None):
            t = torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype)))
            return t.to(dev)

        self.pixels = up(p.pixels, np.float32)
        self.sky = up(p.sky, np.float32)
        self.images = up(img.view(np.uint8))
        self.theta = up(p.theta, np.float64)
        self.patch_ptr = up(self.h_patch_ptr)
        self.patches = up(pat.view(np.uint8))
        self.nbr_ptr = up(self.h_nbr_ptr)
        self.nbr_idx = up(self.h_nbr_idx)
        s = _Problem()
        s.pixels, s.sky, s.images = self.pixels.data_ptr(), self.sky.data_ptr(), self.images.data_ptr()
        s.theta = self.theta.data_ptr()
        s.patch_ptr, s.patches = self.patch_ptr.data_ptr(), self.patches.data_ptr()
        s.nbr_ptr, s.nbr_idx = self.nbr_ptr.data_ptr(), self.nbr_idx.data_ptr()
        s.h_patch_ptr = self.h_patch_ptr.ctypes.data
        s.h_patches = self.h_patches.ctypes.data
        s.h_images = self.h_images.ctypes.data
        s.h_nbr_ptr = self.h_nbr_ptr.ctypes.data
        s.h_nbr_idx = self.h_nbr_idx.ctypes.data
        s.n_pixels, s.n_sky, s.n_pool = p.pixels.size, p.sky.size, self.n_pool
        s.n_images, s.n_sources, s.n_patches = p.n_images, p.n_sources, p.n_patches
        s.n_nbr = int(p.nbr_idx.size)
        # (E, V) of every source at each of its patch pixels, pool layout, in
        # two halves; cache_half[s] names the half with source s's current
        # moments (a Newton step renders trial points into the other half)
        self.cache = (torch.zeros(4 * max(self.n_pool, 1), dtype=torch.float32, device=dev)
                      if render_cache else None)
        self.cache_half = (torch.zeros(max(p.n_sources, 1), dtype=torch.uint8, device=dev)
                           if render_cache else None)
        s.render_cache = self.cache.data_ptr() if render_cache else None
        s.render_cache_half = self.cache_half.data_ptr() if render_cache else None
        self.struct = s

    @property
    def n_sources(self):
        return self.host.n_sources

    def set_theta(self, theta):
        self.theta.copy_(torch.as_tensor(np.asarray(theta, dtype=np.float64)).to(self.theta.device))


class Plan:
    """Work decomposition and scratch for a list of sources of a problem."""

    def __init__(self, ctx: Context, dprob: DeviceProblem, sources: Sequence[int],
                 pixels_per_item: int = 0, blocks_per_sm: int = 0, ppi_bucket=None):
        self.ctx = ctx
        self.dprob = dprob
        self.sources = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        self.n = int(self.sources.size)
        t = _Tuning(pixels_per_item, 0, blocks_per_sm, 0)
        for k, v in enumerate(ppi_bucket or ()):
            t.ppi_bucket[k] = int(v)
        h = ctypes.c_void_p()
        _check(lib().celeste_plan_create(ctx.handle, ctypes.byref(dprob.struct),
                                         self.sources.ctypes.data if self.n else None, self.n,
                                         ctypes.byref(t), ctypes.byref(h)), "celeste_plan_create")
        self.handle = h
        self.visits = int(lib().celeste_plan_visits(h))

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def elbo_grad_hess(plan: Plan, out=None):
    """(elbo, elbo_rel, grad [n, 27], hess [n, 27, 27]) as float64 device tensors."""
    dev = plan.ctx.device
    n = plan.n
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=dev),
               torch.empty(n, dtype=torch.float64, device=dev),
               torch.empty(n, N_THETA, dtype=torch.float64, device=dev),
               torch.empty(n, N_THETA, N_THETA, dtype=torch.float64, device=dev))
    e, er, g, H = out
    _check(lib().celeste_elbo_grad_hess(plan.ctx.handle, plan.handle, _ptr(e), _ptr(er), _ptr(g),
                                        _ptr(H)), "celeste_elbo_grad_hess")
    return out


def elbo_grad(plan: Plan, out=None):
    """(elbo, elbo_rel, grad [n, 27]) as float64 device tensors (gradient-only mode)."""
    dev = plan.ctx.device
    n = plan.n
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=dev),
               torch.empty(n, dtype=torch.float64, device=dev),
               torch.empty(n, N_THETA, dtype=torch.float64, device=dev))
    e, er, g = out
    _check(lib().celeste_elbo_grad(plan.ctx.handle, plan.handle, _ptr(e), _ptr(er), _ptr(g)),
           "celeste_elbo_grad")
    return out


def elbo(plan: Plan):
    dev = plan.ctx.device
    e = torch.empty(plan.n, dtype=torch.float64, device=dev)
    er = torch.empty(plan.n, dtype=torch.float64, device=dev)
    _check(lib().celeste_elbo(plan.ctx.handle, plan.handle, _ptr(e), _ptr(er)), "celeste_elbo")
    return e, er


def loglik(plan: Plan, out: Optional[torch.Tensor] = None):
    """Pixel part of L_rel (no KL) per plan source, float64 device tensor."""
    if out is None:
        out = torch.empty(plan.n, dtype=torch.float64, device=plan.ctx.device)
    _check(lib().celeste_loglik(plan.ctx.handle, plan.handle, _ptr(out)), "celeste_loglik")
    return out


def newton_step(plan: Plan, delta: torch.Tensor, status: torch.Tensor,
                elbo_rel: Optional[torch.Tensor] = None):
    """One trust-region iteration; delta/status are [n_sources] device tensors."""
    _check(lib().celeste_newton_step(plan.ctx.handle, plan.handle, _ptr(delta), _ptr(status),
                                     _ptr(elbo_rel)), "celeste_newton_step")


def newton_state(dprob: DeviceProblem):
    dev = dprob.theta.device
    return (torch.ones(dprob.n_sources, dtype=torch.float64, device=dev),
            torch.zeros(dprob.n_sources, dtype=torch.int32, device=dev))


def tr_subproblem(ctx: Context, g: torch.Tensor, H: torch.Tensor, delta: torch.Tensor):
    n = g.shape[0]
    g = g.contiguous().to(torch.float64)
    H = H.contiguous().to(torch.float64)
    delta = delta.contiguous().to(torch.float64)
    p = torch.empty_like(g)
    pred = torch.empty(n, dtype=torch.float64, device=g.device)
    _check(lib().celeste_tr_subproblem(ctx.handle, n, _ptr(g), _ptr(H), _ptr(delta), _ptr(p),
                                       _ptr(pred)), "celeste_tr_subproblem")
    return p, pred


def render(plan: Plan):
    """Own E and V of every plan source, in the problem's patch-pool layout."""
    dev = plan.ctx.device
    E = torch.zeros(plan.dprob.n_pool, dtype=torch.float32, device=dev)
    V = torch.zeros(plan.dprob.n_pool, dtype=torch.float32, device=dev)
    _check(lib().celeste_render(plan.ctx.handle, plan.handle, _ptr(E), _ptr(V)), "celeste_render")
    return E, V


def render_cache(plan: Plan):
    """Refreshes the problem's render cache for the plan's sources."""
    _check(lib().celeste_render_cache(plan.ctx.handle, plan.handle), "celeste_render_cache")


def background(plan: Plan):
    dev = plan.ctx.device
    E = torch.zeros(plan.dprob.n_pool, dtype=torch.float32, device=dev)
    V = torch.zeros(plan.dprob.n_pool, dtype=torch.float32, device=dev)
    _check(lib().celeste_background(plan.ctx.handle, plan.handle, _ptr(E), _ptr(V)),
           "celeste_background")
    return E, V


def color_sources(nbr_ptr: np.ndarray, nbr_idx: np.ndarray) -> np.ndarray:
    """Greedy colouring of the overlap graph by ascending source id."""
    n = len(nbr_ptr) - 1
    ptr = np.ascontiguousarray(nbr_ptr, dtype=np.int32)
    idx = np.ascontiguousarray(nbr_idx if len(nbr_idx) else np.zeros(1), dtype=np.int32)
    col = np.zeros(max(n, 1), dtype=np.int32)
    rc = lib().celeste_color_sources(n, ptr.ctypes.data, idx.ctypes.data, col.ctypes.data)
    _check(rc, "celeste_color_sources")
    return col[:n]


def color_classes(problem) -> list:
    col = color_sources(problem.nbr_ptr, problem.nbr_idx)
    return [np.flatnonzero(col == c).astype(np.int32) for c in range(int(col.max()) + 1 if len(col) else 0)]


class Fit:
    """Block coordinate ascent over a region of sources (celeste_fit_*)."""

    def __init__(self, ctx: Context, dprob: DeviceProblem, sources: Sequence[int],
                 pixels_per_item: int = 0, ppi_bucket=None):
        self.ctx = ctx
        self.dprob = dprob
        self.sources = np.ascontiguousarray(np.asarray(sorted(sources), dtype=np.int32))
        t = _Tuning(pixels_per_item, 0, 0, 0)
        for k, v in enumerate(ppi_bucket or ()):
            t.ppi_bucket[k] = int(v)
        h = ctypes.c_void_p()
        _check(lib().celeste_fit_create(ctx.handle, ctypes.byref(dprob.struct),
                                        self.sources.ctypes.data if self.sources.size else None,
                                        int(self.sources.size), ctypes.byref(t), ctypes.byref(h)),
               "celeste_fit_create")
        self.handle = h
        self.n_classes = int(lib().celeste_fit_classes(h))

    def run(self, max_passes: int = 5, max_iter: int = 50, pass_tol: float = 1e-3):
        """Runs the fit; returns (passes, [gain of each pass])."""
        passes = ctypes.c_int32(0)
        gains = np.zeros(max(max_passes, 1), dtype=np.float64)
        _check(lib().celeste_fit_run(self.ctx.handle, self.handle, int(max_passes), int(max_iter),
                                     float(pass_tol), ctypes.byref(passes), gains.ctypes.data),
               "celeste_fit_run")
        return int(passes.value), gains[:passes.value].tolist()

    def results(self):
        """(status, iterations, accepted steps, radius): [n_sources] device tensors."""
        dev = self.ctx.device
        S = self.dprob.n_sources
        st = torch.zeros(S, dtype=torch.int32, device=dev)
        it = torch.zeros(S, dtype=torch.int32, device=dev)
        acc = torch.zeros(S, dtype=torch.int32, device=dev)
        dl = torch.zeros(S, dtype=torch.float64, device=dev)
        _check(lib().celeste_fit_results(self.ctx.handle, self.handle, _ptr(st), _ptr(it),
                                         _ptr(acc), _ptr(dl)), "celeste_fit_results")
        return st, it, acc, dl

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_fit_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lbfgs:
    """The first-order comparison subsolver (celeste_lbfgs_*) on a plan."""

    def __init__(self, plan: Plan, m: int = 10):
        self.plan = plan
        self.ctx = plan.ctx
        h = ctypes.c_void_p()
        _check(lib().celeste_lbfgs_create(self.ctx.handle, plan.handle, int(m), ctypes.byref(h)),
               "celeste_lbfgs_create")
        self.handle = h

    def reset(self):
        _check(lib().celeste_lbfgs_reset(self.ctx.handle, self.handle), "celeste_lbfgs_reset")

    def step(self, status: torch.Tensor, target: Optional[torch.Tensor] = None):
        _check(lib().celeste_lbfgs_step(self.ctx.handle, self.handle, _ptr(status), _ptr(target)),
               "celeste_lbfgs_step")

    def counts(self):
        """(accepted steps, trial evaluations, steps to the target) per plan slot."""
        n = self.plan.n
        out = [torch.zeros(max(n, 1), dtype=torch.int32, device=self.ctx.device) for _ in range(3)]
        _check(lib().celeste_lbfgs_counts(self.ctx.handle, self.handle, *[_ptr(t) for t in out]),
               "celeste_lbfgs_counts")
        return [t[:n] for t in out]

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_lbfgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FieldElbo:
    """The ELBO of the whole problem (celeste_field_*)."""

    def __init__(self, ctx: Context, dprob: DeviceProblem, pixels_per_item: int = 0):
        self.ctx = ctx
        self.dprob = dprob
        t = _Tuning(pixels_per_item, 0, 0, 0)
        h = ctypes.c_void_p()
        _check(lib().celeste_field_create(ctx.handle, ctypes.byref(dprob.struct), ctypes.byref(t),
                                          ctypes.byref(h)), "celeste_field_create")
        self.handle = h
        self.out = torch.zeros(3, dtype=torch.float64, device=ctx.device)

    def __call__(self):
        """(ELBO, pixel sum, KL sum) at the current theta, as a device tensor."""
        _check(lib().celeste_field_elbo(self.ctx.handle, self.handle, _ptr(self.out)),
               "celeste_field_elbo")
        return self.out

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_field_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


EAGAIN, EBUSY, ENOTFOUND, ETOOLARGE = -5, -6, -7, -8


class Server:
    """Region fits submitted as independent requests (celeste_server_*)."""

    def __init__(self, model, device: int = 0, workers: int = 2, max_batch: int = 0,
                 device_bytes: int = 0, queue_bytes: int = 0, max_passes: int = 5,
                 max_iter: int = 50, pass_tol: float = 1e-3, start_paused: bool = False,
                 pixels_per_item: int = 0):
        if not torch.cuda.is_available():
            raise CelesteError("no CUDA device: the library has no CPU path")
        self.model_struct = model_struct(model)
        cfg = _ServerConfig(workers, max_batch, device_bytes, queue_bytes, max_passes, max_iter,
                            pass_tol, 1 if start_paused else 0, pixels_per_item)
        h = ctypes.c_void_p()
        _check(lib().celeste_server_create(ctypes.byref(self.model_struct), device,
                                           ctypes.byref(cfg), ctypes.byref(h)),
               "celeste_server_create")
        self.handle = h
        self.sizes = {}

    def pause(self, paused: bool = True):
        _check(lib().celeste_server_pause(self.handle, 1 if paused else 0), "celeste_server_pause")

    @staticmethod
    def prepare(problem):
        """The C request of a fields.Problem (arrays kept alive with it)."""
        img, pat, _ = _host_structs(problem)
        arrs = dict(pixels=np.ascontiguousarray(problem.pixels, dtype=np.float32),
                    sky=np.ascontiguousarray(problem.sky, dtype=np.float32),
                    images=img, theta=np.ascontiguousarray(problem.theta, dtype=np.float64),
                    patch_ptr=np.ascontiguousarray(problem.patch_ptr, dtype=np.int32),
                    patches=pat,
                    nbr_ptr=np.ascontiguousarray(problem.nbr_ptr, dtype=np.int32),
                    nbr_idx=np.ascontiguousarray(problem.nbr_idx if len(problem.nbr_idx)
                                                 else np.zeros(1), dtype=np.int32))
        q = _Request(*[arrs[k].ctypes.data for k in ("pixels", "sky", "images", "theta",
                                                    "patch_ptr", "patches", "nbr_ptr", "nbr_idx")],
                     problem.pixels.size, problem.sky.size, problem.n_images, problem.n_sources,
                     problem.n_patches, int(len(problem.nbr_idx)))
        q._arrays = arrs
        q.bytes_in = sum(a.nbytes for a in arrs.values())
        return q

    def submit(self, problem) -> int:
        """Queues a fields.Problem (or a prepared request) as one region;
        returns its ticket (raises CelesteError with .code EAGAIN when the
        queue is full)."""
        q = problem if isinstance(problem, _Request) else self.prepare(problem)
        t = ctypes.c_uint64(0)
        rc = lib().celeste_submit(self.handle, ctypes.byref(q), ctypes.byref(t))
        if rc < 0:
            err = CelesteError(f"celeste_submit failed with code {rc}")
            err.code = rc
            raise err
        self.sizes[t.value] = q.n_sources
        return int(t.value)

    def poll(self, ticket: int, wait_ms: int = 0):
        """None while the request runs; else a dict with theta [n, 27],
        status [n], passes, latency_s, queue_s, batch_requests, t_start_s,
        t_done_s (the server's monotonic clock) and code."""
        if ticket not in self.sizes:
            raise CelesteError(f"unknown ticket {ticket}")
        n = self.sizes[ticket]
        theta = np.zeros((n, N_THETA), dtype=np.float64)
        status = np.zeros(n, dtype=np.int32)
        info = _RequestInfo()
        rc = lib().celeste_poll(self.handle, ticket, int(wait_ms), theta.ctypes.data,
                                status.ctypes.data, ctypes.byref(info))
        if rc == EBUSY:
            return None
        if rc == ENOTFOUND or ticket not in self.sizes:
            raise CelesteError(f"unknown ticket {ticket}")
        del self.sizes[ticket]
        return dict(theta=theta, status=status, passes=info.passes, latency_s=info.latency_s,
                    queue_s=info.queue_s, batch_requests=info.batch_requests,
                    last_pass_gain=info.last_pass_gain, device_error=info.device_error, code=rc,
                    t_start_s=info.t_start_s, t_done_s=info.t_done_s)

    def stats(self):
        nl, nb = ctypes.c_int64(0), ctypes.c_int64(0)
        rc = lib().celeste_server_stats(self.handle, ctypes.byref(nl), ctypes.byref(nb))
        return dict(launches=nl.value, batches=nb.value, worker_error=rc)

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def elbo_grad_hess_noalloc(model, dprob: DeviceProblem, sources: Sequence[int], out,
                           stream: Optional[torch.cuda.Stream] = None,
                           device_error: Optional[torch.Tensor] = None):
    """The allocation-free entry point: fills ``out`` = (elbo, elbo_rel, grad,
    hess), caller-allocated device tensors, on ``stream`` (torch's current
    stream by default).  For callers that must not allocate device memory;
    see the header for its limits and its shared scratch array."""
    ids = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    m = model_struct(model)
    st = stream if stream is not None else torch.cuda.current_stream()
    e, er, g, H = out
    return _check(lib().celeste_elbo_grad_hess_noalloc(
        ctypes.byref(m), ctypes.byref(dprob.struct), ids.ctypes.data if ids.size else None,
        int(ids.size), ctypes.c_void_p(st.cuda_stream), _ptr(e), _ptr(er), _ptr(g), _ptr(H),
        _ptr(device_error)), "celeste_elbo_grad_hess_noalloc")
