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
