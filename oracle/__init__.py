"""CPU oracle for the compressed and sieved BFS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never loads it, and shares no code with it.

Each function follows a passage of the paper:

* :func:`csr` -- the adjacency the search runs on (Sec. VII-A), tuples
  symmetrised with self-loops kept twice and duplicates kept.
* :func:`bfs_levels` -- BFS hop distances (Sec. II), -1 when unreachable;
  :func:`bfs_sample` the same search stopped after a budget of scanned entries.
* :func:`parents` -- the deterministic parent: the smallest neighbour on the
  previous level (the paper's (select,max) semiring of Sec. III-A picks the
  largest; ``use_max=True`` gives that reading).
* :func:`directory` / :func:`cross_directory` -- directory vectors V_{i,j}
  (Eq. 4) and the cross directory (Eq. 5).
* :func:`wah_encode` / :func:`wah_decode` -- the WAH code of Sec. IV, Table 3.
* :func:`dist_bfs` -- Algorithms 1, 2, 3 (BIT, WAH, DIR-WAH) on a simulated
  p x p grid, with every exchanged buffer recorded: the column streams of the
  frontier exchange and, for DIR-WAH, the row buffers of the fold (the WAH
  stream of what each block reached, sieved by the visited set).
* :func:`level_exchange` -- the exchanged buffers for one given frontier.

Every function is pinned by ``tests/test_oracle_*.py`` against worked examples
printed in the paper, brute force and invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PLAIN, COMPRESS, COMPRESS_SIEVE = 0, 1, 2

_i64 = ctypes.c_int64
_int = ctypes.c_int
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C11, portable)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sig = {
                "oracle_csr_size": (_i64, [_i64, _int]),
                "oracle_csr": (_int, [_i64, _i64, _ptr, _ptr, _int, _ptr, _ptr]),
                "oracle_bfs_levels": (_i64, [_i64, _ptr, _ptr, ctypes.c_int32, _ptr]),
                "oracle_bfs_sample": (_i64, [_i64, _ptr, _ptr, ctypes.c_int32, _i64, _ptr]),
                "oracle_parents": (None, [_i64, _ptr, _ptr, _ptr, ctypes.c_int32, _int, _ptr]),
                "oracle_range_begin": (_i64, [_i64, _int, _int]),
                "oracle_range_len": (_i64, [_i64, _int, _int]),
                "oracle_directory": (None, [_i64, _int, _ptr, _ptr, _int, _int, _ptr]),
                "oracle_cross_directory": (None, [_i64, _int, _ptr, _ptr, _ptr]),
                "oracle_wah_encode": (_i64, [_ptr, _i64, _int, _int, _ptr]),
                "oracle_wah_decode": (_int, [_ptr, _i64, _i64, _int, _int, _ptr]),
                "oracle_plwah_encode": (_i64, [_ptr, _i64, _ptr]),
                "oracle_plwah_decode": (_int, [_ptr, _i64, _i64, _ptr]),
                "oracle_bbc_encode": (_i64, [_ptr, _i64, _ptr]),
                "oracle_bbc_decode": (_int, [_ptr, _i64, _i64, _ptr]),
                "oracle_adaptive_encode": (_i64, [_ptr, _i64, _int, _ptr, _ptr]),
                "oracle_adaptive_decode": (_int, [_int, _ptr, _i64, _i64, _int, _ptr]),
                "oracle_dist_bfs": (_i64, [_i64, _int, _ptr, _ptr, ctypes.c_int32, _int, _int, _int,
                                           _ptr, _ptr, _ptr, _i64, _ptr, _i64, _ptr, _i64, _ptr]),
                "oracle_dynamic_sieve_stats": (_i64, [_i64, _int, _ptr, _ptr, ctypes.c_int32, _i64, _ptr]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class CSR:
    """Plain CSR by source vertex: ``row_ptr`` (int64, n+1) and ``col`` (int32)."""

    def __init__(self, n: int, row_ptr: np.ndarray, col: np.ndarray):
        self.n, self.row_ptr, self.col = n, row_ptr, col

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def csr(n: int, src: np.ndarray, dst: np.ndarray, symmetrize: bool = True) -> CSR:
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    lib = _load()
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(1, lib.oracle_csr_size(m, int(symmetrize))), dtype=np.int32)
    rc = lib.oracle_csr(n, m, _p(src), _p(dst), int(symmetrize), _p(row_ptr), _p(col))
    if rc != 0:
        raise ValueError("oracle_csr: vertex id out of range")
    return CSR(n, row_ptr, col[: lib.oracle_csr_size(m, int(symmetrize))])


def bfs_levels(g: CSR, root: int) -> np.ndarray:
    level = np.empty(g.n, dtype=np.int32)
    rc = _load().oracle_bfs_levels(g.n, _p(g.row_ptr), _p(g.col), root, _p(level))
    if rc < 0:
        raise ValueError("oracle_bfs_levels: bad root")
    return level


def bfs_sample(g: CSR, root: int, budget: int):
    """``(level, scanned)``: the queue BFS stopped once ``budget`` adjacency
    entries were scanned; assigned levels are final, the rest -1."""
    level = np.empty(g.n, dtype=np.int32)
    k = _load().oracle_bfs_sample(g.n, _p(g.row_ptr), _p(g.col), root, int(budget), _p(level))
    if k < 0:
        raise ValueError("oracle_bfs_sample: bad root")
    return level, int(k)


def parents(g: CSR, level: np.ndarray, root: int, use_max: bool = False) -> np.ndarray:
    level = np.ascontiguousarray(level, dtype=np.int32)
    parent = np.empty(g.n, dtype=np.int32)
    _load().oracle_parents(g.n, _p(g.row_ptr), _p(g.col), _p(level), root, int(use_max), _p(parent))
    return parent


def bfs(g: CSR, root: int, use_max: bool = False):
    """``(level, parent)`` by the plain definition."""
    level = bfs_levels(g, root)
    return level, parents(g, level, root, use_max)


def range_begin(n: int, p: int, b: int) -> int:
    return int(_load().oracle_range_begin(n, p, b))


def range_len(n: int, p: int, b: int) -> int:
    return int(_load().oracle_range_len(n, p, b))


def directory(g: CSR, p: int, i: int, j: int) -> np.ndarray:
    """V_{i,j} as 0/1 bytes of length range_len(j)."""
    out = np.empty(max(1, range_len(g.n, p, j)), dtype=np.uint8)
    _load().oracle_directory(g.n, p, _p(g.row_ptr), _p(g.col), i, j, _p(out))
    return out[: range_len(g.n, p, j)]


def cross_directory(g: CSR, p: int) -> np.ndarray:
    """``D[i, u]`` = bit of u in V_{i, range(u)}; shape (p, n), 0/1 bytes."""
    out = np.empty((p, g.n), dtype=np.uint8)
    _load().oracle_cross_directory(g.n, p, _p(g.row_ptr), _p(g.col), _p(out))
    return out


def wah_encode(bits: np.ndarray, w: int = 32, fill_bit: bool = True) -> np.ndarray:
    """WAH words (as uint64 values) of a 0/1 byte array."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    nbits = len(bits)
    out = np.empty(nbits // (w - 1) + 2, dtype=np.uint64)
    nw = _load().oracle_wah_encode(_p(bits) if nbits else 0, nbits, w, int(fill_bit), _p(out))
    return out[:nw].copy()


def wah_decode(words: np.ndarray, nbits: int, w: int = 32, fill_bit: bool = True):
    """0/1 byte array, or ``None`` if the stream is malformed."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    bits = np.zeros(max(1, nbits), dtype=np.uint8)
    rc = _load().oracle_wah_decode(_p(words) if len(words) else 0, len(words), nbits, w,
                                   int(fill_bit), _p(bits))
    return None if rc != 0 else bits[:nbits]


def plwah_encode(bits: np.ndarray) -> np.ndarray:
    """PLWAH words (uint32) of a 0/1 byte array."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    nbits = len(bits)
    out = np.empty(nbits // 31 + 2, dtype=np.uint32)
    nw = _load().oracle_plwah_encode(_p(bits) if nbits else 0, nbits, _p(out))
    return out[:nw].copy()


def plwah_decode(words: np.ndarray, nbits: int):
    """0/1 byte array, or ``None`` if the stream is malformed."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    bits = np.zeros(max(1, nbits), dtype=np.uint8)
    rc = _load().oracle_plwah_decode(_p(words) if len(words) else 0, len(words), nbits, _p(bits))
    return None if rc != 0 else bits[:nbits]


def bbc_encode(bits: np.ndarray) -> np.ndarray:
    """BBC bytes (uint8) of a 0/1 byte array (oracle_bbc_encode)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    nbits = len(bits)
    nbytes = (nbits + 7) // 8
    out = np.empty(nbytes + nbytes // 15 + 16, dtype=np.uint8)
    nb = _load().oracle_bbc_encode(_p(bits) if nbits else 0, nbits, _p(out))
    if nb < 0:
        raise MemoryError("oracle_bbc_encode")
    return out[:nb].copy()


def bbc_decode(data: np.ndarray, nbits: int):
    """0/1 byte array, or ``None`` if the stream is malformed."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    bits = np.zeros(max(1, nbits), dtype=np.uint8)
    rc = _load().oracle_bbc_decode(_p(data) if len(data) else 0, len(data), nbits, _p(bits))
    return None if rc != 0 else bits[:nbits]


ADAPTIVE_WAH, ADAPTIVE_LIST, ADAPTIVE_RAW = 0, 1, 2


def adaptive_encode(bits: np.ndarray, w: int = 32):
    """``(format, elements)`` of a 0/1 byte array: the smallest of its WAH stream
    (0), sparse vector of set-bit offsets (1) and raw 32-bit bitmap words (2)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    nbits = len(bits)
    out = np.empty(max(nbits // (w - 1) + 2, nbits, (nbits + 31) // 32, 1), dtype=np.uint64)
    fmt = ctypes.c_int(-1)
    k = _load().oracle_adaptive_encode(_p(bits) if nbits else 0, nbits, w, ctypes.addressof(fmt), _p(out))
    return int(fmt.value), out[:k].copy()


def adaptive_decode(fmt: int, elems: np.ndarray, nbits: int, w: int = 32):
    """0/1 byte array, or ``None`` if the elements are malformed."""
    elems = np.ascontiguousarray(elems, dtype=np.uint64)
    bits = np.zeros(max(1, nbits), dtype=np.uint8)
    rc = _load().oracle_adaptive_decode(int(fmt), _p(elems) if len(elems) else 0, len(elems), nbits, w, _p(bits))
    return None if rc != 0 else bits[:nbits]


def adaptive_trace(tr, n: int, p: int, mode: int = COMPRESS_SIEVE, w: int = 32):
    """The level-adaptive exchange of a traced search (``dist_bfs(..., trace=True)``):
    per exchange, per slot, ``(format, elements)`` of its slice re-sent as the
    smallest of WAH stream, sparse vector and raw bitmap."""
    out = []
    for level in tr:
        row = []
        for s, words in enumerate(level):
            j = s % p if mode == COMPRESS_SIEVE else s
            bits = wah_decode(np.asarray(words, np.uint64), range_len(n, p, j), w)
            if bits is None:
                raise ValueError(f"traced stream of slot {s} does not decode")
            row.append(adaptive_encode(bits, w))
        out.append(row)
    return out


def dynamic_sieve_stats(g: CSR, p: int, root: int, max_levels: int = 256):
    """Per level of the search, by definition: (static pairs, dynamic pairs,
    entries of the static pairs, entries of the dropped pairs, entries walked by
    the directory update) -- see oracle_dynamic_sieve_stats."""
    out = np.zeros(5 * max_levels, dtype=np.int64)
    k = _load().oracle_dynamic_sieve_stats(g.n, p, _p(g.row_ptr), _p(g.col), root, max_levels, _p(out))
    if k < 0:
        raise ValueError("oracle_dynamic_sieve_stats failed")
    return out[: 5 * k].reshape(k, 5)


def dist_bfs(g: CSR, p: int, root: int, mode: int = COMPRESS_SIEVE, w: int = 32,
             use_max: bool = False, trace: bool = False, max_levels: int = 256,
             trace_cap: int | None = None, rows: bool = False, dynamic: bool = False):
    """Algorithm 1/2/3 on a simulated p x p grid.

    Returns ``(level, parent, trace)``; ``trace`` is a list (one entry per
    exchange, i.e. per BFS level that had a nonempty frontier) of lists of
    word arrays, indexed by slot: ``i*p + j`` for DIR-WAH (stream from source
    range j to block-row i), ``j`` for WAH.  ``None`` unless ``trace``.

    With ``dynamic=True`` (DIR-WAH only) the cross directory is dynamic: V_{i,j}(u)
    is cleared once every entry of u into range i leads to a visited vertex.

    With ``rows=True`` (DIR-WAH only) a fourth element is returned: the row
    buffers of every level's fold, in the same layout (slot ``i*p + j`` = the
    WAH stream of the vertices of range i that block (i, j) reached, sieved by
    the visited set of range i before the level).
    """
    lib = _load()
    level = np.empty(g.n, dtype=np.int32)
    parent = np.empty(g.n, dtype=np.int32)
    slots = p * p if mode == COMPRESS_SIEVE else (p if mode == COMPRESS else 0)
    if rows and mode != COMPRESS_SIEVE:
        raise ValueError("row buffers exist for DIR-WAH (COMPRESS_SIEVE) only")
    if (trace or rows) and trace_cap is None:
        trace_cap = max_levels * (slots * 2 + (g.n * (p if mode == COMPRESS_SIEVE else 1)) // (w - 1) + 8)
    if trace and slots:
        words = np.empty(trace_cap, dtype=np.uint64)
        counts = np.zeros(max_levels * slots, dtype=np.int64)
        wp, cp = _p(words), _p(counts)
        tcap = trace_cap
    else:
        words = counts = None
        wp = cp = 0
        tcap = 0
    if rows:
        rwords = np.empty(trace_cap, dtype=np.uint64)
        rcounts = np.zeros(max_levels * slots, dtype=np.int64)
        rwp, rcp, rcap = _p(rwords), _p(rcounts), trace_cap
    else:
        rwords = rcounts = None
        rwp = rcp = rcap = 0
    if dynamic and mode != COMPRESS_SIEVE:
        raise ValueError("the dynamic directory sieves DIR-WAH (COMPRESS_SIEVE) only")
    rc = lib.oracle_dist_bfs(g.n, p, _p(g.row_ptr), _p(g.col), root, 3 if dynamic else mode, w, int(use_max),
                             _p(level), _p(parent), wp, tcap, cp, max_levels, rwp, rcap, rcp)
    if rc < 0:
        raise ValueError(f"oracle_dist_bfs failed ({rc})")

    def unpack(ws, cs):
        out, off = [], 0
        for k in range(min(rc, max_levels)):
            lv = []
            for s in range(slots):
                c = int(cs[k * slots + s])
                lv.append(ws[off: off + c].copy())
                off += c
            out.append(lv)
        return out

    tr = unpack(words, counts) if (trace and slots) else None
    if rows:
        return level, parent, tr, unpack(rwords, rcounts)
    return level, parent, tr


def level_exchange(g: CSR, p: int, frontier: np.ndarray, mode: int = COMPRESS_SIEVE, w: int = 32,
                   D: np.ndarray | None = None):
    """The buffers exchanged for one frontier (0/1 bytes of length n).

    DIR-WAH: slot ``i*p + j`` = WAH(f_j (.) V_{i,j});  WAH: slot ``j`` = WAH(f_j).
    Returns ``(streams, sieved_counts)`` where ``sieved_counts[s]`` is the
    number of set bits in the encoded slice.
    """
    n = g.n
    frontier = np.ascontiguousarray(frontier, dtype=np.uint8)
    if mode == COMPRESS_SIEVE and D is None:
        D = cross_directory(g, p)
    streams, counts = [], []
    if mode == COMPRESS_SIEVE:
        for i in range(p):
            for j in range(p):
                b, ln = range_begin(n, p, j), range_len(n, p, j)
                sl = frontier[b: b + ln] & D[i, b: b + ln]
                streams.append(wah_encode(sl, w))
                counts.append(int(sl.sum()))
    elif mode == COMPRESS:
        for j in range(p):
            b, ln = range_begin(n, p, j), range_len(n, p, j)
            sl = frontier[b: b + ln]
            streams.append(wah_encode(sl, w))
            counts.append(int(sl.sum()))
    return streams, counts


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """0/1 bytes -> little-endian bit-packed uint32 words (bit q of word k = bits[32k+q])."""
    bits = np.asarray(bits, dtype=np.uint8)
    pad = (-len(bits)) % 32
    b = np.concatenate([bits, np.zeros(pad, dtype=np.uint8)]) if pad else bits
    return np.packbits(b, bitorder="little").view(np.uint32).copy() if len(b) else np.zeros(0, np.uint32)


def unpack_bits(words: np.ndarray, nbits: int) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:nbits].copy()
