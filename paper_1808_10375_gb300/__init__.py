"""GB300 multi-mode difference-map ptychography (arXiv 1808.10375, Sec. II).

The compute path is the CUDA library ``libptycho_dm.so`` (C ABI in
include/dm.h); ``paper_1808_10375_gb300.dm`` is its ctypes binding with the
same function names.  Build the library with
``paper_1808_10375_gb300.build.build()``.
"""
from . import dm  # noqa: F401
from .dm import *  # noqa: F401,F403
