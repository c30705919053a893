"""Multiword (DD/TD/QD) LU with partial pivoting, substitution and mixed
precision iterative refinement on one GB300 (Kouya, arXiv 2107.12550).

The compute path is libmwlu.so (hand-written CUDA for sm_103a, C ABI in
include/mwlu.h); ``api`` is its Python binding.  Importing this package does
not load the library; the first call does, and fails loudly if it is missing.
"""
from . import _lib  # noqa: F401

__all__ = ["api", "build", "workloads"]


def __getattr__(name):
    if name in ("ludecomp", "solve", "residual", "refine", "arith", "peak_fp64"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
