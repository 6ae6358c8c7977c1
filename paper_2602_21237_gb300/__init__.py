"""GB300-native tensor-path inner equi-join and sort (arxiv 2602.21237).

The compute path is the CUDA library ``libtj.so`` built from ``csrc/`` (see
``include/tj.h`` for the C ABI).  This package is a thin ctypes binding over it:
``join_inner``, ``sort``, ``join_batch`` marshal torch tensors' device pointers
and streams into the C calls and nothing else.  Importing the package does not
load the library; the first call does, and fails loudly if it is missing.
"""
from __future__ import annotations

__all__ = ["join_inner", "sort", "sort_multi", "join_batch", "gather_pairs", "stats", "Server",
           "TjError", "lib_path", "build"]


def __getattr__(name):
    if name in ("join_inner", "sort", "sort_multi", "join_batch", "gather_pairs", "TjError",
                "lib_path", "stats", "Server"):
        from . import api

        return getattr(api, name)
    if name == "build":
        from .build import build

        return build
    raise AttributeError(name)
