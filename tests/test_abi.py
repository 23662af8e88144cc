"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared entry point."""
import ctypes

from paper_1208_5542_gb300 import build, native


def test_library_builds_and_exports_header_symbols():
    build.build()
    lib = ctypes.CDLL(native.LIB_PATH)
    names = native.header_symbols()
    assert "bfs_run" in names and "bfs_graph_create_edges" in names and "bfs_wah_encode" in names
    for name in names:
        assert hasattr(lib, name), name
    # every declared symbol has a binding signature, and vice versa
    assert set(names) == set(native._SIGS), set(names) ^ set(native._SIGS)


def test_status_strings_and_defaults_without_gpu():
    build.build()
    lib = native.lib()
    assert lib.bfs_status_string(0) == b"BFS_OK"
    assert lib.bfs_status_string(5) == b"BFS_ERR_CORRUPT"
    o = native.Options()
    lib.bfs_options_default(ctypes.byref(o))
    assert (o.grid_r, o.grid_c, o.mode, o.wah_word_bits) == (1, 1, 2, 32)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    that a C compiler gives the header's structures."""
    import os
    import subprocess

    structs = {"bfs_options": native.Options, "bfs_graph_info_t": native.GraphInfo,
               "bfs_level_stats": native.LevelStats, "bfs_run_stats": native.RunStats,
               "bfs_batch_stats": native.BatchStats, "bfs_server_stats_t": native.ServerStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bfs_gb300.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(native.PKG), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for line in out:
        if line:
            c, f, v = line.split()
            got[(c, f)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_failure_injection_arguments_without_gpu():
    build.build()
    lib = native.lib()
    assert native.STATUS[lib.bfs_debug_fail_allocation(-1)] == "BFS_ERR_INVALID_ARG"
    assert lib.bfs_debug_fail_allocation(0) == 0
