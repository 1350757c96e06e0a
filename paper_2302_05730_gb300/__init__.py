"""m-Cubes (VEGAS-style Monte Carlo integration, arXiv 2302.05730 Sec. 3.2) on GB300 / sm_103a.

The integrator runs in hand-written CUDA kernels behind the C ABI of include/mcubes.h
(libmcubes.so, built by ``python -m paper_2302_05730_gb300.build``). This package is a thin
ctypes binding with the same call names. ``workloads`` draws the seeded benchmark integrand
parameters and needs no GPU.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "capi", "build_library"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def __getattr__(name):
    if name == "capi":
        from . import _capi
        return _capi
    raise AttributeError(name)
