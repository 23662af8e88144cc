"""Seeded synthetic graph inputs (Graph500-style Kronecker and Erdos-Renyi tuples).

This module produces inputs only.  It holds none of the BFS, directory, sieve
or codec arithmetic; the CPU oracle and the CUDA library both consume its
output.  The C source is ``graphgen.c`` next to this file; ``build()`` compiles
it into ``libgraphgen.so`` in place.

Recipe (the synthetic graphs of the paper's experiments, Sec. VII-A):

* Kronecker: ``n = 2**scale`` vertices, ``m = edgefactor * n`` directed tuples,
  initiator A=0.57, B=0.19, C=0.19, D=0.05, no noise, labels mapped through a
  seeded bijection of ``[0, n)``.
* Erdos-Renyi control: uniform endpoints, same ``n`` and ``m``.
* Seeds: tuple stream ``1000 + scale`` (Kronecker) or ``2000 + scale`` (ER),
  label bijection ``seed + 1``, roots ``7``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

KRONECKER = 0
ERDOS_RENYI = 1


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` with gcc (portable C, no host-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.graphgen_splitmix64.restype = ctypes.c_uint64
            lib.graphgen_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.graphgen_permute.restype = ctypes.c_int64
            lib.graphgen_permute.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64]
            lib.graphgen_edges.restype = ctypes.c_int
            lib.graphgen_edges.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.graphgen_pick_roots.restype = ctypes.c_int64
            lib.graphgen_pick_roots.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                                ctypes.c_void_p]
            _lib = lib
    return _lib


def splitmix64(seed: int, k: int) -> int:
    """k-th output of the SplitMix64 stream started at ``seed``."""
    return int(_load().graphgen_splitmix64(seed & (2**64 - 1), k & (2**64 - 1)))


def permute(scale: int, seed: int, x: int) -> int:
    """The seeded label bijection of ``[0, 2**scale)``."""
    return int(_load().graphgen_permute(scale, seed & (2**64 - 1), x))


def default_seed(scale: int, kind: int = KRONECKER) -> int:
    return (1000 if kind == KRONECKER else 2000) + scale


def edges(scale: int, edgefactor: int = 16, kind: int = KRONECKER, seed: int | None = None,
          threads: int = 0, m: int | None = None):
    """Return ``(n, src, dst)`` with ``src``/``dst`` int32 arrays of ``m`` directed tuples."""
    if seed is None:
        seed = default_seed(scale, kind)
    n = 1 << scale
    if m is None:
        m = edgefactor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().graphgen_edges(kind, scale, m, seed, seed + 1, src.ctypes.data, dst.ctypes.data, threads)
    if rc != 0:
        raise ValueError("graphgen_edges: bad argument")
    return n, src, dst


def pick_roots(n: int, src: np.ndarray, dst: np.ndarray, count: int, seed: int = 7) -> np.ndarray:
    """Distinct seeded roots, each with at least one non-self-loop neighbour."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    out = np.empty(count, dtype=np.int32)
    got = _load().graphgen_pick_roots(n, len(src), src.ctypes.data, dst.ctypes.data, count, seed,
                                      out.ctypes.data)
    if got < 0:
        raise MemoryError("graphgen_pick_roots")
    return out[:got].copy()


def random_edges(n: int, m: int, seed: int):
    """Small uniform random directed tuples over ``[0, n)`` for any n (tests)."""
    rng = np.random.Generator(np.random.Philox(seed))
    src = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    dst = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    return src, dst


def degrees(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Directed-entry degree of each vertex after symmetrisation (self-loops count twice)."""
    return (np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)).astype(np.int64)


def traversed_tuples(deg: np.ndarray, level: np.ndarray) -> int:
    """Graph500 TEPS numerator: input tuples inside the traversed component.

    Every tuple of the component contributes two directed entries (a self-loop
    contributes two as well), so the count is half the degree sum of the
    reached vertices.
    """
    return int(deg[level >= 0].sum() // 2)
