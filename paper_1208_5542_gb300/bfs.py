"""Python front end of the C ABI (``include/bfs_gb300.h``): argument marshalling only.

PyTorch provides device memory and streams; every step of the search runs in
the CUDA kernels of ``libbfs_gb300.so``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import native
from .native import (DIRECTION_BOTTOM_UP, DIRECTION_HYBRID, DIRECTION_TOP_DOWN,  # noqa: F401
                     MODE_COMPRESS, MODE_COMPRESS_SIEVE, MODE_PLAIN, check)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(x) -> int:
    if isinstance(x, torch.Tensor):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(type(x))


def _as_i32(x):
    if isinstance(x, torch.Tensor):
        return x.contiguous().to(torch.int32)
    return np.ascontiguousarray(x, dtype=np.int32)


@dataclass
class SearchStats:
    n_levels: int = 0
    levels: list = field(default_factory=list)      # dicts, one per exchange
    trace_words: torch.Tensor | None = None         # int32 view of the packed streams
    trace_counts: torch.Tensor | None = None        # [levels, slots] int64
    trace_formats: torch.Tensor | None = None       # [levels, slots] uint8 (adaptive format: 0 WAH, 1 vector, 2 raw)
    trace_used: int = 0
    row_trace_words: torch.Tensor | None = None     # int32 view of the packed row buffers of the fold
    row_trace_counts: torch.Tensor | None = None    # [levels, p*p] int64
    row_trace_used: int = 0


class Graph:
    """A graph laid out as the p x p block grid on the current CUDA device."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        info = native.GraphInfo()
        check(native.lib().bfs_graph_info(self._h, ctypes.byref(info)))
        self.n = int(info.n_vertices)
        self.n_entries = int(info.n_entries)
        self.p = int(info.p)
        self.range_size = int(info.range_size)
        self.nonempty_columns = int(info.nonempty_columns)

    # ------------------------------------------------------------ creation --
    @staticmethod
    def _options(p, mode, wah_bits, debug, autotune=False):
        o = native.Options()
        native.lib().bfs_options_default(ctypes.byref(o))
        o.grid_r = o.grid_c = int(p)
        o.mode = int(mode)
        o.wah_word_bits = int(wah_bits)
        o.debug_checks = int(bool(debug))
        o.autotune = int(bool(autotune))
        return o

    @classmethod
    def from_edges(cls, n, src, dst, symmetrize=True, p=1, mode=MODE_COMPRESS_SIEVE, wah_bits=32,
                   debug=False, stream=None, autotune=False) -> "Graph":
        src, dst = _as_i32(src), _as_i32(dst)
        if len(src) != len(dst):
            raise ValueError("src and dst differ in length")
        o = cls._options(p, mode, wah_bits, debug, autotune)
        h = ctypes.c_void_p()
        check(native.lib().bfs_graph_create_edges(int(n), len(src), _ptr(src) if len(src) else None,
                                                  _ptr(dst) if len(dst) else None, int(bool(symmetrize)),
                                                  ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def from_csr(cls, n, row_ptr, col, p=1, mode=MODE_COMPRESS_SIEVE, wah_bits=32, debug=False,
                 stream=None) -> "Graph":
        if isinstance(row_ptr, torch.Tensor):
            row_ptr = row_ptr.contiguous().to(torch.int64)
        else:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = _as_i32(col)
        o = cls._options(p, mode, wah_bits, debug)
        h = ctypes.c_void_p()
        check(native.lib().bfs_graph_create_csr(int(n), _ptr(row_ptr), _ptr(col) if len(col) else None,
                                                ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)))
        return cls(h.value)

    def close(self):
        if self._h and self._h.value:
            check(native.lib().bfs_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---------------------------------------------------------------- info --
    def footprint(self) -> int:
        b = ctypes.c_int64()
        check(native.lib().bfs_graph_footprint(self._h, ctypes.byref(b)))
        return int(b.value)

    def set_mode(self, mode: int, wah_bits: int = 32):
        check(native.lib().bfs_graph_set_mode(self._h, int(mode), int(wah_bits)))

    def set_row_exchange(self, enabled: bool):
        check(native.lib().bfs_graph_set_row_exchange(self._h, int(bool(enabled))))

    def set_exchange_format(self, adaptive: bool):
        """Every exchanged slice as the smallest of WAH stream, sparse vector and raw
        bitmap (True), or always WAH (False, the default)."""
        check(native.lib().bfs_graph_set_exchange_format(self._h, native.FORMAT_ADAPTIVE if adaptive
                                                         else native.FORMAT_WAH))

    def set_dynamic_directory(self, enabled: bool):
        """Sieve with the search's dynamic cross directory (True) or the static
        directories of Eq. 4 (False, the default); COMPRESS_SIEVE only."""
        check(native.lib().bfs_graph_set_dynamic_directory(self._h, int(bool(enabled))))

    def set_direction(self, policy: int, alpha: int = 14, beta: int = 24):
        """Top-down (the default), hybrid top-down / bottom-up, or bottom-up levels."""
        check(native.lib().bfs_graph_set_direction(self._h, int(policy), int(alpha), int(beta)))

    def mode(self):
        info = native.GraphInfo()
        check(native.lib().bfs_graph_info(self._h, ctypes.byref(info)))
        return int(info.mode), int(info.wah_word_bits)

    def range_len(self, b: int) -> int:
        lo = min(self.n, b * self.range_size)
        hi = min(self.n, (b + 1) * self.range_size)
        return hi - lo

    def directory(self, i: int, j: int, stream=None) -> torch.Tensor:
        """V_{i,j} as int32 words (bit k of the vector = bit k%32 of word k//32)."""
        words = (self.range_len(j) + 31) // 32
        out = torch.zeros(max(1, words), dtype=torch.int32, device="cuda")
        check(native.lib().bfs_graph_directory(self._h, int(i), int(j), _ptr(out), _stream_ptr(stream)))
        return out[:words]

    # -------------------------------------------------------------- search --
    def run(self, root: int, parent=None, level=None, stats: bool = False, timing: bool = False,
            trace_capacity: int = 0, max_levels: int = 256, stream=None, row_trace_capacity: int = 0):
        """One search from ``root``; returns ``(parent, level, SearchStats | None)``.

        ``parent``/``level`` may be int32 CUDA tensors (filled in place), int32
        host tensors or numpy arrays (the library copies back), or None
        (CUDA tensors are allocated).  ``trace_capacity`` / ``row_trace_capacity``
        (uint32 elements) record the column streams / the row buffers of the fold.
        """
        if parent is None:
            parent = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if level is None:
            level = torch.empty(self.n, dtype=torch.int32, device="cuda")
        rs = None
        out_stats = None
        keep = []
        if stats or timing or trace_capacity or row_trace_capacity:
            out_stats = SearchStats()
            lv = (native.LevelStats * max_levels)()
            rs = native.RunStats()
            rs.capacity_levels = max_levels
            rs.timing = int(bool(timing))
            rs.levels = ctypes.cast(lv, ctypes.POINTER(native.LevelStats))
            keep.append(lv)
            mode, _ = self.mode()
            slots = self.p * self.p if mode == MODE_COMPRESS_SIEVE else (self.p if mode == MODE_COMPRESS else 0)
            if trace_capacity and slots:
                tw = torch.zeros(int(trace_capacity), dtype=torch.int32, device="cuda")
                tc = torch.zeros((max_levels, slots), dtype=torch.int64, device="cuda")
                rs.trace_words = _ptr(tw)
                rs.trace_capacity = int(trace_capacity)
                rs.trace_counts = _ptr(tc)
                tf = torch.zeros((max_levels, slots), dtype=torch.uint8, device="cuda")
                rs.trace_formats = _ptr(tf)
                out_stats.trace_words, out_stats.trace_counts, out_stats.trace_formats = tw, tc, tf
            if row_trace_capacity:
                rw = torch.zeros(int(row_trace_capacity), dtype=torch.int32, device="cuda")
                rcn = torch.zeros((max_levels, self.p * self.p), dtype=torch.int64, device="cuda")
                rs.row_trace_words = _ptr(rw)
                rs.row_trace_capacity = int(row_trace_capacity)
                rs.row_trace_counts = _ptr(rcn)
                out_stats.row_trace_words, out_stats.row_trace_counts = rw, rcn
        check(native.lib().bfs_run(self._h, int(root), _ptr(parent), _ptr(level),
                                   ctypes.byref(rs) if rs is not None else None, _stream_ptr(stream)))
        if out_stats is not None:
            out_stats.n_levels = int(rs.n_levels)
            out_stats.trace_used = int(rs.trace_used)
            for k in range(min(out_stats.n_levels, max_levels)):
                s = lv[k]
                out_stats.levels.append({f: getattr(s, f) for f, _ in native.LevelStats._fields_})
            out_stats.row_trace_used = int(rs.row_trace_used)
            if out_stats.trace_counts is not None:
                out_stats.trace_counts = out_stats.trace_counts[: out_stats.n_levels]
                out_stats.trace_formats = out_stats.trace_formats[: out_stats.n_levels]
            if out_stats.row_trace_counts is not None:
                out_stats.row_trace_counts = out_stats.row_trace_counts[: out_stats.n_levels]
        return parent, level, out_stats

    def check_search(self, root: int, parent, level, stream=None):
        """Raise BfsError(BFS_ERR_CORRUPT) unless (parent, level) -- int32 CUDA
        tensors -- pass the level/parent checks of ``bfs_check_search``."""
        check(native.lib().bfs_check_search(self._h, int(root), _ptr(parent), _ptr(level), _stream_ptr(stream)))

    # -------------------------------------------------------------- batch --
    def run_batch(self, roots, parents: bool = False, levels=None, stream=None):
        """Up to 64 searches at once; returns ``(levels [k, n], parents [k, n] | None, stats)``."""
        roots = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
        k = len(roots)
        if levels is None:
            levels = torch.empty((k, self.n), dtype=torch.int32, device="cuda")
        par = torch.empty((k, self.n), dtype=torch.int32, device="cuda") if parents else None
        st = native.BatchStats()
        check(native.lib().bfs_run_batch(self._h, roots.ctypes.data, k, _ptr(levels),
                                         _ptr(par) if par is not None else None, ctypes.byref(st),
                                         _stream_ptr(stream)))
        return levels, par, {"n_levels": int(st.n_levels), "edges_scanned": int(st.edges_scanned)}

    def batch_autotune(self, roots, stream=None):
        """Pick the launch shape of the batched expansion for this graph; returns (threads, ctas_per_sm)."""
        roots = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
        scratch = torch.empty((len(roots), self.n), dtype=torch.int32, device="cuda")
        t, c = ctypes.c_int32(), ctypes.c_int32()
        check(native.lib().bfs_batch_autotune(self._h, roots.ctypes.data, len(roots), _ptr(scratch),
                                              ctypes.byref(t), ctypes.byref(c), _stream_ptr(stream)))
        return int(t.value), int(c.value)


def wah_encode(bits: torch.Tensor, nbits: int, word_bits: int = 32, stream=None) -> torch.Tensor:
    """Encode the first ``nbits`` bits of ``bits`` (int32 CUDA words, bit b = bit b%32 of word b//32).

    Returns the words as an int32 tensor (32-bit words) or int64 tensor (64-bit words).
    """
    words_in = (nbits + 31) // 32
    src = torch.zeros(words_in + 2, dtype=torch.int32, device="cuda")
    if words_in:
        src[:words_in] = bits[:words_in]
    cap = nbits // (word_bits - 1) + 1
    out = torch.zeros(max(1, cap), dtype=torch.int32 if word_bits == 32 else torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    check(native.lib().bfs_wah_encode(_ptr(src), int(nbits), int(word_bits), _ptr(out), int(cap), _ptr(cnt),
                                      _stream_ptr(stream)))
    return out[: int(cnt.item())]


def wah_decode(words: torch.Tensor, nbits: int, word_bits: int = 32, stream=None) -> torch.Tensor:
    """Decode a stream (int32 / int64 CUDA tensor) into int32 bitmap words; raises on a malformed stream."""
    out = torch.zeros(max(1, (nbits + 31) // 32), dtype=torch.int32, device="cuda")
    check(native.lib().bfs_wah_decode(_ptr(words) if words.numel() else None, int(words.numel()), int(nbits),
                                      int(word_bits), _ptr(out), _stream_ptr(stream)))
    return out[: (nbits + 31) // 32]


def plwah_encode(bits: torch.Tensor, nbits: int, stream=None) -> torch.Tensor:
    """PLWAH words (int32 CUDA tensor) of the first ``nbits`` bits of ``bits`` (int32 CUDA words)."""
    words_in = (nbits + 31) // 32
    src = torch.zeros(words_in + 2, dtype=torch.int32, device="cuda")
    if words_in:
        src[:words_in] = bits[:words_in]
    cap = nbits // 31 + 1
    out = torch.zeros(max(1, cap), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    check(native.lib().bfs_plwah_encode(_ptr(src), int(nbits), _ptr(out), int(cap), _ptr(cnt), _stream_ptr(stream)))
    return out[: int(cnt.item())]


def plwah_decode(words: torch.Tensor, nbits: int, stream=None) -> torch.Tensor:
    """Decode a PLWAH stream (int32 CUDA tensor) into int32 bitmap words; raises on a malformed stream."""
    out = torch.zeros(max(1, (nbits + 31) // 32), dtype=torch.int32, device="cuda")
    check(native.lib().bfs_plwah_decode(_ptr(words) if words.numel() else None, int(words.numel()), int(nbits),
                                        _ptr(out), _stream_ptr(stream)))
    return out[: (nbits + 31) // 32]


def bbc_encode(bits: torch.Tensor, nbits: int, stream=None) -> torch.Tensor:
    """BBC bytes (uint8 CUDA tensor) of the first ``nbits`` bits of ``bits`` (int32 CUDA words)."""
    words_in = (nbits + 31) // 32
    src = torch.zeros(max(1, words_in), dtype=torch.int32, device="cuda")
    if words_in:
        src[:words_in] = bits[:words_in]
    n = (nbits + 7) // 8
    cap = n + n // 15 + 11
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    check(native.lib().bfs_bbc_encode(_ptr(src), int(nbits), _ptr(out), int(cap), _ptr(cnt), _stream_ptr(stream)))
    return out[: int(cnt.item())]


def bbc_decode(data: torch.Tensor, nbits: int, stream=None) -> torch.Tensor:
    """Decode a BBC stream (uint8 CUDA tensor) into int32 bitmap words; raises on a malformed stream."""
    out = torch.zeros(max(1, (nbits + 31) // 32), dtype=torch.int32, device="cuda")
    check(native.lib().bfs_bbc_decode(_ptr(data) if data.numel() else None, int(data.numel()), int(nbits),
                                      _ptr(out), _stream_ptr(stream)))
    return out[: (nbits + 31) // 32]


class Server:
    """Continuous-batching query server over resident graphs (``bfs_server_*``)."""

    def __init__(self, hbm_budget_bytes: int, max_lanes: int = 64):
        h = ctypes.c_void_p()
        check(native.lib().bfs_server_create(int(hbm_budget_bytes), int(max_lanes), ctypes.byref(h)))
        self._h = h
        self._n = {}

    def add_graph(self, graph: Graph) -> int:
        gid = ctypes.c_int32()
        check(native.lib().bfs_server_add_graph(self._h, graph.handle, ctypes.byref(gid)))
        self._n[int(gid.value)] = graph.n
        return int(gid.value)

    def submit(self, graph_id: int, root: int, parents: bool = False) -> int:
        t = ctypes.c_int64()
        check(native.lib().bfs_server_submit_ex(self._h, int(graph_id), int(root),
                                                native.QUERY_PARENTS if parents else 0, ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        check(native.lib().bfs_server_poll(self._h, int(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, n: int, timeout_s: float = 30.0, out=None, parents: bool = False,
             timeout_us: int | None = None):
        """Level vector (int32 CUDA tensor of length n, or ``out``) of a finished
        query; with ``parents`` the pair ``(level, parent)``."""
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device="cuda")
        par = torch.empty(n, dtype=torch.int32, device="cuda") if parents else None
        us = int(timeout_s * 1e6) if timeout_us is None else int(timeout_us)
        check(native.lib().bfs_server_wait(self._h, int(ticket), us, _ptr(out),
                                           _ptr(par) if par is not None else None))
        return (out, par) if parents else out

    def set_queue_limit(self, limit: int):
        check(native.lib().bfs_server_set_queue_limit(self._h, int(limit)))

    def stats(self) -> dict:
        st = native.ServerStats()
        check(native.lib().bfs_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in native.ServerStats._fields_}

    def close(self):
        if self._h and self._h.value:
            check(native.lib().bfs_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_fail_allocation(k: int):
    """Make the k-th device allocation of the library fail (0 disarms); tests only."""
    check(native.lib().bfs_debug_fail_allocation(int(k)))


def measure_scatter_reads(region_bytes: int = 512 << 10, iterations: int = 4096, stream=None) -> float:
    """Scattered 4-byte reads per second of this GPU (``bfs_measure_scatter_reads``)."""
    out = ctypes.c_double()
    check(native.lib().bfs_measure_scatter_reads(int(region_bytes), int(iterations), ctypes.byref(out),
                                                 _stream_ptr(stream)))
    return float(out.value)
