"""bench.py's reference arm (the CPU oracle) keeps the JSON-line contract and
reports the same workload keys as the GPU arm, so that the two lines pair up."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "s12", "--steps", "2",
                          "--warmup", "3", *extra], cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_line_contract():
    d = _reference_line()
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_config_matches_the_gpu_arm():
    sys.path.insert(0, ROOT)
    import bench
    for extra, argv in [((), []), (("--roots", "4", "--direction", "hybrid"), ["--roots", "4", "--direction", "hybrid"])]:
        d = _reference_line(*extra)
        old = sys.argv
        sys.argv = ["bench.py", "--workload", "s12", *argv]
        try:
            args = bench.parse()
        finally:
            sys.argv = old
        want = bench.workload_config(args, d["config"]["vertices"], d["config"]["tuples"], d["config"]["roots"])
        assert {k: d["config"][k] for k in want} == want
        assert d["config"]["roots"] == (int(argv[1]) if argv else 16)


def test_compression_factor_is_the_mean_of_the_level_ratios():
    """Sec. VI-A: C = (1/d) sum_i 1/C_i with C_i = raw / compressed at level i of
    one search (d levels); the line reports its mean over the searches."""
    sys.path.insert(0, ROOT)
    import bench
    one = [0.001, 0.5, 1.03, None]
    two = [0.002, 0.9]
    got = bench.compression_factor([one, two], 2)
    want = ((0.001 + 0.5 + 1.03) / 3 + (0.002 + 0.9) / 2) / 2
    assert got == {"symbol": "C'", "value": round(want, 6), "searches": 2, "levels_per_search": 2.5}
    assert bench.compression_factor([one], 1)["symbol"] == "C"
    assert bench.compression_factor([one], 0) is None
    assert bench.compression_factor([], 2) is None
    assert bench.compression_factor([[None]], 2) is None


def test_kernel_hash_ignores_comments_only():
    """The committed ncu counters stay valid across comment edits of the kernel
    sources, and no longer once the code changes."""
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int x) {\n    return x + 1;   // add one\n}\n/* a block\n   comment */\n"
    same = "// header comment\nint f(int x) {\n\n    return x + 1;   // a different remark\n}\n"
    other = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench.code_digest([code]) == bench.code_digest([same])
    assert bench.code_digest([code]) != bench.code_digest([other])
    assert len(bench.kernel_hash()) == 16


def test_search_roofline_arithmetic():
    """Bytes per traversed edge from the per-level counters, the GTEPS bound at
    the copy rate, and the fraction the measured value reaches."""
    sys.path.insert(0, ROOT)
    import bench
    lv = {"edges_scanned": 1000, "column_hits": 100, "wah_bytes": 50, "compress_chunks": 2, "frontier_vertices": 10}
    chunk = bench.CHUNK_GROUPS * 31 // 8
    per = (4 * 1000 + 12 * 100 + 2 * 50 + chunk * 2 + 12 * 10) / 500
    r = bench.search_roofline_of([[lv]], [500], 32, 6000.0, 100.0, "measured")
    assert r["bytes_per_edge"] == round(per, 3)
    assert r["bound_gteps"] == round(6000.0 / per, 1)
    assert r["frac"] == round(100.0 / (6000.0 / per), 4)
    assert bench.search_roofline_of([[lv]], [0], 32, 6000.0, 100.0, "measured") is None
