"""ctypes binding of libbfs_gb300.so -- argument marshalling only.

Every step of the search runs in the CUDA library; this module only loads it
and declares the C signatures of ``include/bfs_gb300.h``.  Importing it fails
loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbfs_gb300.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "bfs_gb300.h")

_lock = threading.Lock()
_lib = None

i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
vp = ctypes.c_void_p
P = ctypes.POINTER

STATUS = ["BFS_OK", "BFS_ERR_INVALID_ARG", "BFS_ERR_OUT_OF_MEMORY", "BFS_ERR_CUDA", "BFS_ERR_TIMEOUT",
          "BFS_ERR_CORRUPT", "BFS_ERR_BUSY", "BFS_ERR_NOT_FOUND"]
MODE_PLAIN, MODE_COMPRESS, MODE_COMPRESS_SIEVE = 0, 1, 2
DIRECTION_TOP_DOWN, DIRECTION_HYBRID, DIRECTION_BOTTOM_UP = 0, 1, 2
QUERY_PARENTS = 1
FORMAT_WAH, FORMAT_ADAPTIVE = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("grid_r", i32), ("grid_c", i32), ("mode", i32), ("wah_word_bits", i32),
                ("autotune", i32), ("debug_checks", i32), ("row_exchange", i32)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", i64), ("n_entries", i64), ("p", i32), ("mode", i32), ("wah_word_bits", i32),
                ("row_exchange", i32), ("range_size", i64), ("nonempty_columns", i64),
                ("exchange_format", i32), ("direction", i32), ("dynamic_directory", i32), ("reserved", i32)]


class LevelStats(ctypes.Structure):
    _fields_ = [("frontier_vertices", i64), ("exchanged_vertices", i64), ("column_hits", i64),
                ("raw_bytes", i64), ("wah_bytes", i64), ("edges_scanned", i64), ("row_wah_bytes", i64),
                ("ms_compress_sieve", ctypes.c_float), ("ms_communication", ctypes.c_float),
                ("ms_traversing", ctypes.c_float), ("ms_reducing", ctypes.c_float),
                ("bottom_up", i32), ("ms_row_compress", ctypes.c_float), ("ms_row_fold", ctypes.c_float),
                ("ms_directory_update", ctypes.c_float), ("compress_chunks", i64), ("row_compress_chunks", i64)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_levels", i32), ("reserved", i32), ("edges_scanned", i64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", i64), ("completed", i64), ("rejected", i64), ("queued", i64), ("iterations", i64),
                ("peak_lanes", i32), ("graphs", i32), ("hbm_used_bytes", i64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double)]


class RunStats(ctypes.Structure):
    _fields_ = [("capacity_levels", i32), ("n_levels", i32), ("timing", i32), ("reserved", i32),
                ("levels", P(LevelStats)), ("trace_words", vp), ("trace_capacity", i64),
                ("trace_counts", vp), ("trace_used", i64), ("trace_formats", vp),
                ("row_trace_words", vp), ("row_trace_capacity", i64),
                ("row_trace_counts", vp), ("row_trace_used", i64)]


_SIGS = {
    "bfs_options_default": (None, [P(Options)]),
    "bfs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bfs_last_error": (ctypes.c_int, [ctypes.c_char_p, i64]),
    "bfs_graph_create_edges": (ctypes.c_int, [i64, i64, vp, vp, i32, P(Options), vp, P(vp)]),
    "bfs_graph_create_csr": (ctypes.c_int, [i64, vp, vp, P(Options), vp, P(vp)]),
    "bfs_graph_destroy": (ctypes.c_int, [vp]),
    "bfs_graph_footprint": (ctypes.c_int, [vp, P(i64)]),
    "bfs_graph_info": (ctypes.c_int, [vp, P(GraphInfo)]),
    "bfs_graph_set_mode": (ctypes.c_int, [vp, i32, i32]),
    "bfs_graph_set_row_exchange": (ctypes.c_int, [vp, i32]),
    "bfs_graph_set_direction": (ctypes.c_int, [vp, i32, i32, i32]),
    "bfs_graph_set_exchange_format": (ctypes.c_int, [vp, i32]),
    "bfs_graph_set_dynamic_directory": (ctypes.c_int, [vp, i32]),
    "bfs_graph_directory": (ctypes.c_int, [vp, i32, i32, vp, vp]),
    "bfs_run": (ctypes.c_int, [vp, i32, vp, vp, P(RunStats), vp]),
    "bfs_check_search": (ctypes.c_int, [vp, i32, vp, vp, vp]),
    "bfs_debug_fail_allocation": (ctypes.c_int, [i64]),
    "bfs_server_set_queue_limit": (ctypes.c_int, [vp, i64]),
    "bfs_run_batch": (ctypes.c_int, [vp, vp, i32, vp, vp, P(BatchStats), vp]),
    "bfs_batch_autotune": (ctypes.c_int, [vp, vp, i32, vp, P(i32), P(i32), vp]),
    "bfs_server_create": (ctypes.c_int, [i64, i32, P(vp)]),
    "bfs_server_add_graph": (ctypes.c_int, [vp, vp, P(i32)]),
    "bfs_server_submit": (ctypes.c_int, [vp, i32, i32, P(i64)]),
    "bfs_server_submit_ex": (ctypes.c_int, [vp, i32, i32, i32, P(i64)]),
    "bfs_server_poll": (ctypes.c_int, [vp, i64, P(i32)]),
    "bfs_server_wait": (ctypes.c_int, [vp, i64, i64, vp, vp]),
    "bfs_server_stats": (ctypes.c_int, [vp, P(ServerStats)]),
    "bfs_server_destroy": (ctypes.c_int, [vp]),
    "bfs_wah_encode": (ctypes.c_int, [vp, i64, i32, vp, i64, vp, vp]),
    "bfs_wah_decode": (ctypes.c_int, [vp, i64, i64, i32, vp, vp]),
    "bfs_wah_decode_static": (ctypes.c_int, [vp, i64, i64, i32, vp, vp]),
    "bfs_plwah_encode": (ctypes.c_int, [vp, i64, vp, i64, vp, vp]),
    "bfs_plwah_decode": (ctypes.c_int, [vp, i64, i64, vp, vp]),
    "bfs_bbc_encode": (ctypes.c_int, [vp, i64, vp, i64, vp, vp]),
    "bfs_bbc_decode": (ctypes.c_int, [vp, i64, i64, vp, vp]),
    "bfs_measure_scatter_reads": (ctypes.c_int, [i64, i32, ctypes.POINTER(ctypes.c_double), vp]),
}


class BfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")
        self.status = status


def header_symbols() -> list[str]:
    """Names of the entry points declared in include/bfs_gb300.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^BFS_API\s+[\w\s\*]*?\b(bfs_\w+)\s*\(", text, flags=re.M)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with paper_1208_5542_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int):
    if status != 0:
        buf = ctypes.create_string_buffer(512)
        lib().bfs_last_error(buf, 512)
        raise BfsError(status, buf.value.decode(errors="replace"))
