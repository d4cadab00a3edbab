"""GB300 (sm_103a) implementation of the per-point moving least squares (MLS)
projection (Sec. 1.4, Eq. 1; Algorithm 1 of arXiv 2401.03365).

The compute path is libmls (CUDA kernels behind the C ABI in include/mls.h);
``capi`` is its ctypes binding with the same names, ``mls`` the user-facing
functions built on it, ``workloads`` the seeded synthetic clouds.
Nothing here falls back to the CPU.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "capi", "mls"]


def __getattr__(name):
    # the CUDA-facing modules import torch and load libmls on first use
    if name in ("capi", "mls"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
