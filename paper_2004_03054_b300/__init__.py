"""LUDA-B300: SSTable compaction (LUDA, arXiv 2004.03054) as hand-written CUDA for sm_103a.

The compaction job runs in libluda.so behind a C ABI (include/luda.h); ``luda`` is its
thin ctypes binding and ``workloads`` draws seeded synthetic jobs.
"""
from . import luda, workloads  # noqa: F401

__all__ = ["luda", "workloads"]
