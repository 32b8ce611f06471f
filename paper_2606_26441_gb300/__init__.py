"""GB300-native exact batched sparse scoring (GPUSparse, Sec. 3-5).

The product is libgpusparse.so (CUDA for sm_103a, C ABI in include/gpusparse.h);
this package holds its sources (csrc/), the in-tree build (_build.py) and the
ctypes binding (gpusparse.py).
"""
from .gpusparse import (GS_MAX_K, IMPACTS, Index, Queries, alloc_workspace, gs_index_build, gs_score_dense,
                        gs_search, gs_search_flags, gs_search_host, gs_version, load, make_opts)

__all__ = ["GS_MAX_K", "IMPACTS", "Index", "Queries", "alloc_workspace", "gs_index_build", "gs_score_dense",
           "gs_search", "gs_search_flags", "gs_search_host", "gs_version", "load", "make_opts"]
