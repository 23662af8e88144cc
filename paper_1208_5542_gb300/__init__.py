"""GB300-native compressed and sieved level-synchronous BFS (arXiv 1208.5542).

The search runs in hand-written CUDA kernels for sm_103a behind the C ABI of
``include/bfs_gb300.h`` (``libbfs_gb300.so``); ``bfs.Graph`` is its Python
front end.  Build the library with ``paper_1208_5542_gb300.build.build()``.
"""
from .native import MODE_COMPRESS, MODE_COMPRESS_SIEVE, MODE_PLAIN  # noqa: F401


def __getattr__(name):
    if name in ("Graph", "wah_encode", "wah_decode", "SearchStats"):
        from . import bfs
        return getattr(bfs, name)
    raise AttributeError(name)
