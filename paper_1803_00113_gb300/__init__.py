"""GB300 (sm_103a) library for the per-source ELBO, gradient, Hessian and
trust-region Newton step of Regier et al. (arXiv:1803.00113).

The compute path is the CUDA library ``lib/libceleste.so`` (C ABI in
``include/celeste.h``); ``celeste`` is its Python binding.
"""
from . import build_lib  # noqa: F401

__all__ = ["build_lib", "celeste"]
