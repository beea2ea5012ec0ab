"""DetMesh-Gadep on GB300: triangulated HPGe detector surfaces and GPU photon transport.

The compute lives in ``lib/libgadep.so`` (C ABI declared in ``include/gadep.h``);
this package is its Python binding (``api``), the build step (``build``), the
synthetic workloads (``workloads``) and the autograd wrapper (``autograd``).
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "api", "capi", "build"]
