"""Parity of the CUDA search with the CPU oracle (levels, parents and every exchanged buffer)."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
from tests.golden_io import bfs_example, row_buffer_example

pytestmark = pytest.mark.gpu

MODES = {"plain": 0, "compress": 1, "sieve": 2}
ORACLE_MODE = {0: oracle.PLAIN, 1: oracle.COMPRESS, 2: oracle.COMPRESS_SIEVE}


def _lib():
    from paper_1208_5542_gb300 import bfs
    from paper_1208_5542_gb300 import build
    build.build()
    return bfs


def _run(g, root, **kw):
    parent, level, st = g.run(root, **kw)
    torch.cuda.synchronize()
    return parent.cpu().numpy(), level.cpu().numpy(), st


def _unpack_trace(st, wah_bits, rows=False):
    """GPU trace (column streams, or the row buffers of the fold with ``rows``) ->
    list (per exchange) of lists (per slot) of word values."""
    if rows:
        words = st.row_trace_words[: st.row_trace_used].cpu().numpy().view(np.uint32)
        counts = st.row_trace_counts.cpu().numpy()
    else:
        words = st.trace_words[: st.trace_used].cpu().numpy().view(np.uint32)
        counts = st.trace_counts.cpu().numpy()
    per = wah_bits // 32
    out, off = [], 0
    for k in range(counts.shape[0]):
        lv = []
        for c in counts[k]:
            c = int(c)
            seg = words[off: off + c * per]
            if per == 2:
                seg = seg[0::2].astype(np.uint64) | (seg[1::2].astype(np.uint64) << np.uint64(32))
            lv.append(seg.astype(np.uint64))
            off += c * per
        out.append(lv)
    return out


def _check_trace(gpu_tr, ora_tr):
    assert len(gpu_tr) == len(ora_tr)
    for k, (a, b) in enumerate(zip(gpu_tr, ora_tr)):
        assert len(a) == len(b)
        for s, (x, y) in enumerate(zip(a, b)):
            assert len(x) == len(y) and (x == y).all(), f"exchange {k}, slot {s}: {x[:8]} vs {y[:8]}"


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("wah", [32, 64])
def test_paper_example(mode, p, wah):
    bfs = _lib()
    d = bfs_example()
    g = bfs.Graph.from_edges(d["n"], d["src"], d["dst"], p=p, mode=mode, wah_bits=wah)
    parent, level, st = _run(g, d["root"], stats=True, trace_capacity=4096, row_trace_capacity=4096)
    assert level.tolist() == d["levels"]
    assert parent.tolist() == d["parents_min"]
    if mode:
        go = oracle.csr(d["n"], d["src"], d["dst"])
        _, _, tr = oracle.dist_bfs(go, p, d["root"], mode=ORACLE_MODE[mode], w=wah, trace=True)
        _check_trace(_unpack_trace(st, wah), tr)
    if mode == 2:
        # the row buffers of the fold: the hand-derived words of the fixture (p = 1, 2)
        # and the oracle's (every p)
        _, _, _, rows = oracle.dist_bfs(go, p, d["root"], mode=oracle.COMPRESS_SIEVE, w=wah, rows=True)
        got = _unpack_trace(st, wah, rows=True)
        _check_trace(got, rows)
        want = row_buffer_example().get(p)
        if want is not None:
            assert [[[int(x) for x in sl] for sl in lvl] for lvl in got] == [[[x] for x in lvl] for lvl in want]


def test_directories_match_eq4():
    bfs = _lib()
    n, src, dst = graphgen.edges(11, 16)
    go = oracle.csr(n, src, dst)
    for p in (1, 3, 8):
        g = bfs.Graph.from_edges(n, src, dst, p=p)
        assert g.nonempty_columns == int(oracle.cross_directory(go, p).sum())
        for i in range(p):
            for j in range(p):
                want = oracle.pack_bits(oracle.directory(go, p, i, j))
                got = g.directory(i, j).cpu().numpy().view(np.uint32)
                assert (got == want).all(), (p, i, j)


def test_scale12_plain_2x2_sixteen_roots():
    """The scale-12 Kronecker graph, 2x2 grid, no compression or sieve, 16 seeded roots."""
    bfs = _lib()
    n, src, dst = graphgen.edges(12, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=2, mode=0)
    roots = graphgen.pick_roots(n, src, dst, 16)
    assert len(roots) == 16
    for r in roots:
        lv, pa = oracle.bfs(go, int(r))
        parent, level, _ = _run(g, int(r))
        assert (level == lv).all() and (parent == pa).all()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("p,wah", [(2, 32), (4, 64), (8, 32), (5, 32)])
def test_kronecker_traces_bit_exact(mode, p, wah):
    bfs = _lib()
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode, wah_bits=wah)
    for r in graphgen.pick_roots(n, src, dst, 3):
        if mode == 2:
            lv, pa, tr, rows = oracle.dist_bfs(go, p, int(r), mode=oracle.COMPRESS_SIEVE, w=wah, trace=True,
                                               rows=True)
        else:
            lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=ORACLE_MODE[mode], w=wah, trace=True)
        parent, level, st = _run(g, int(r), stats=True, trace_capacity=1 << 22, row_trace_capacity=1 << 22)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, wah), tr)
        if mode == 2:
            _check_trace(_unpack_trace(st, wah, rows=True), rows)
        # per-level statistics agree with the oracle's streams
        for k, ls in enumerate(st.levels):
            assert ls["frontier_vertices"] == int((lv == k).sum())
            assert ls["wah_bytes"] == sum(len(x) for x in tr[k]) * wah // 8
            assert ls["row_wah_bytes"] == (sum(len(x) for x in rows[k]) * wah // 8 if mode == 2 else 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ragged_ranges_directed_and_multi_tile(mode):
    """n not a multiple of p (ragged last range, unaligned slices), no symmetrisation,
    ranges long enough for several encoder tiles and expansion chunks."""
    bfs = _lib()
    n = 100_003
    src, dst = graphgen.random_edges(n, 400_000, 11)
    go = oracle.csr(n, src, dst, symmetrize=False)
    for p in (3, 7):
        g = bfs.Graph.from_edges(n, src, dst, symmetrize=False, p=p, mode=mode)
        for r in (0, 77_777, n - 1):
            lv, pa = oracle.bfs(go, r)
            parent, level, _ = _run(g, r)
            assert (level == lv).all() and (parent == pa).all()


def test_dense_frontier_one_fills():
    """Root 0 reaches 1..3999 (a contiguous dense frontier), each of which reaches
    one vertex of 4000..7999: the level-1 streams hold all-one groups (1-fills)."""
    bfs = _lib()
    mid = np.arange(1, 4000)
    src = np.concatenate([np.zeros(len(mid), np.int64), mid]).astype(np.int32)
    dst = np.concatenate([mid, 4000 + (mid * 7) % 4000]).astype(np.int32)
    n = 8000
    go = oracle.csr(n, src, dst)
    for mode in (1, 2):
        for p in (1, 2):
            g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
            lv, pa, tr = oracle.dist_bfs(go, p, 0, mode=ORACLE_MODE[mode], trace=True)
            parent, level, st = _run(g, 0, stats=True, trace_capacity=1 << 20)
            assert (level == lv).all() and (parent == pa).all()
            got = _unpack_trace(st, 32)
            _check_trace(got, tr)
            one_fills = sum(int(((w >> np.uint64(30)) == 3).sum()) for lvl in got for w in lvl if len(w))
            assert one_fills > 0


def test_isolated_root_single_vertex_and_empty_graph():
    bfs = _lib()
    g = bfs.Graph.from_edges(1, np.zeros(0, np.int32), np.zeros(0, np.int32), p=1)
    parent, level, _ = _run(g, 0)
    assert parent.tolist() == [0] and level.tolist() == [0]
    src = np.array([0, 1, 5], np.int32)
    dst = np.array([1, 2, 5], np.int32)
    for mode in (0, 1, 2):
        g = bfs.Graph.from_edges(6, src, dst, p=3, mode=mode)
        parent, level, _ = _run(g, 5)
        assert level.tolist() == [-1, -1, -1, -1, -1, 0]
        assert parent.tolist() == [-1, -1, -1, -1, -1, 5]
        parent, level, _ = _run(g, 3)
        assert level.tolist() == [-1, -1, -1, 0, -1, -1]


def test_from_csr_and_host_outputs():
    bfs = _lib()
    n, src, dst = graphgen.edges(12, 8)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_csr(n, go.row_ptr, go.col, p=4)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    lv, pa = oracle.bfs(go, r)
    par = np.empty(n, np.int32)
    lev = np.empty(n, np.int32)
    g.run(r, parent=par, level=lev)
    assert (lev == lv).all() and (par == pa).all()


def test_bad_arguments_are_reported():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    with pytest.raises(BfsError, match="INVALID_ARG"):
        bfs.Graph.from_edges(10, np.array([0, 11], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(BfsError, match="INVALID_ARG"):
        bfs.Graph.from_edges(10, np.array([0], np.int32), np.array([1], np.int32), p=11)
    g = bfs.Graph.from_edges(10, np.array([0], np.int32), np.array([1], np.int32), p=2)
    with pytest.raises(BfsError, match="INVALID_ARG"):
        g.run(10)
    with pytest.raises(BfsError, match="INVALID_ARG"):
        g.set_mode(3)


@pytest.mark.parametrize("mode", [0, 2])
def test_scale20_grid8(mode):
    bfs = _lib()
    n, src, dst = graphgen.edges(20, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=8, mode=mode)
    for r in graphgen.pick_roots(n, src, dst, 2):
        lv, pa = oracle.bfs(go, int(r))
        parent, level, _ = _run(g, int(r))
        assert (level == lv).all() and (parent == pa).all()


@pytest.mark.parametrize("mode", [0, 2])
def test_ranges_too_long_for_the_shared_window(mode):
    """Scale 21 on a 2x2 grid: 1M-vertex ranges do not fit the on-chip row
    window, so the expansion takes its global-memory visiting path."""
    bfs = _lib()
    n, src, dst = graphgen.edges(21, 8)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=2, mode=mode)
    for r in graphgen.pick_roots(n, src, dst, 2):
        lv, pa = oracle.bfs(go, int(r))
        parent, level, _ = _run(g, int(r))
        assert (level == lv).all() and (parent == pa).all()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_many_rows(mode):
    """A 64 x 64 grid on a small graph: many rows for the row-affine work hand-out."""
    bfs = _lib()
    n, src, dst = graphgen.edges(13, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=64, mode=mode)
    for r in graphgen.pick_roots(n, src, dst, 3):
        lv, pa = oracle.bfs(go, int(r))
        parent, level, _ = _run(g, int(r))
        assert (level == lv).all() and (parent == pa).all()


@pytest.mark.parametrize("gap_tiles", [1, 2, 33, 40])
def test_zero_tiles_skipped_then_set_bit_at_tile_start(gap_tiles):
    """The encoder skips all-zero tiles of 1024 groups using the frontier summary.
    Put the only frontier vertex of level 1 at the first bit of a tile that
    follows gap_tiles all-zero tiles, and a second one further on, so the zero
    fill must close exactly at a tile boundary after a skip (and after a run
    of skips longer than one look-ahead of 32 tiles)."""
    bfs = _lib()
    tile_bits = 1024 * 31
    first = gap_tiles * tile_bits
    second = first + 3 * tile_bits + 5
    n = second + tile_bits + 100
    src = np.array([0, 0, first, second], np.int32)
    dst = np.array([first, second, n - 1, n - 2], np.int32)
    go = oracle.csr(n, src, dst)
    for mode in (1, 2):
        g = bfs.Graph.from_edges(n, src, dst, p=1, mode=mode)
        lv, pa, tr = oracle.dist_bfs(go, 1, 0, mode=ORACLE_MODE[mode], trace=True)
        parent, level, st = _run(g, 0, stats=True, trace_capacity=1 << 16)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, 32), tr)


def test_sieved_away_chunk_inside_a_zero_run():
    """A chunk of 1024 groups that holds frontier vertices (so the encoder reads
    it) but whose vertices all have empty columns in block (0,0), so the sieve
    clears it: it opens no word, continues the zero run carried in from the
    previous chunk, and that run ends at its last group because the next chunk
    starts with a sieved-in vertex.  The exchanged streams must equal Alg. 3's."""
    bfs = _lib()
    tile = 1024 * 31
    n = 200_000                                   # p = 2: ranges of 100,000 vertices, 4 chunks each
    root = 150_000
    mid = np.arange(tile + 100, tile + 200)       # chunk 1 of range 0: edges into range 1 only
    src = np.concatenate([[root, root, 5], np.full(len(mid), root), mid, [root, 2 * tile]]).astype(np.int32)
    dst = np.concatenate([[5, 6, 6], mid, np.full(len(mid), root + 1), [2 * tile, 7]]).astype(np.int32)
    go = oracle.csr(n, src, dst, symmetrize=False)
    for mode in (1, 2):
        g = bfs.Graph.from_edges(n, src, dst, symmetrize=False, p=2, mode=mode)
        lv, pa, tr = oracle.dist_bfs(go, 2, root, mode=ORACLE_MODE[mode], trace=True)
        parent, level, st = _run(g, root, stats=True, trace_capacity=1 << 18)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, 32), tr)
        parent, level, _ = _run(g, root)          # the graph-launched loop
        assert (level == lv).all() and (parent == pa).all()


@pytest.mark.parametrize("scale,p,wah", [(14, 4, 32), (13, 7, 64), (16, 2, 32), (21, 2, 32)])
def test_row_buffers_bit_exact(scale, p, wah):
    """COMPRESS_SIEVE with the row exchange of the fold (the default): every row
    buffer -- the WAH stream of what block (i,j) reached, sieved by not(pi_i) --
    word for word the oracle's, on ragged ranges (p = 7), 64-bit words, the
    shared-memory row window (scale 16) and the global visiting path (scale 21:
    ranges of 1M vertices); with the row exchange off the search is the same
    and carries no row buffers."""
    bfs = _lib()
    n, src, dst = graphgen.edges(scale, 16 if scale < 20 else 8)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2, wah_bits=wah)
    cap = 1 << 24
    for r in graphgen.pick_roots(n, src, dst, 2):
        lv, pa, tr, rows = oracle.dist_bfs(go, p, int(r), mode=oracle.COMPRESS_SIEVE, w=wah, trace=True,
                                           rows=True, max_levels=64, trace_cap=cap)
        parent, level, st = _run(g, int(r), stats=True, trace_capacity=2 * cap, row_trace_capacity=2 * cap)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, wah), tr)
        _check_trace(_unpack_trace(st, wah, rows=True), rows)
        parent, level, _ = _run(g, int(r))             # the graph-launched level loop
        assert (level == lv).all() and (parent == pa).all()
    g.set_row_exchange(False)
    parent, level, st = _run(g, int(r), stats=True)
    assert (level == lv).all() and (parent == pa).all()
    assert sum(ls["row_wah_bytes"] for ls in st.levels) == 0


def test_row_buffers_bench_launch_configuration_scale24():
    """Kronecker scale 24 on the 16 x 16 grid: the parent array exceeds half of
    L2 and the ranges (1M vertices) exceed the row window, so the expansion
    sweeps the block-rows in turn on its global visiting path -- the bench's
    launch configuration at scale 26.  Every row buffer of one search
    bit-exact with the oracle's."""
    bfs = _lib()
    n, src, dst = graphgen.edges(24, 16)
    p = 16
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    cap = 1 << 26
    parent, level, st = _run(g, r, stats=True, row_trace_capacity=cap)
    rows_gpu = _unpack_trace(st, 32, rows=True)
    del g
    torch.cuda.empty_cache()
    go = oracle.csr(n, src, dst)
    del src, dst
    lv, pa, _, rows = oracle.dist_bfs(go, p, r, mode=oracle.COMPRESS_SIEVE, rows=True, max_levels=64,
                                      trace_cap=cap)
    assert (level == lv).all() and (parent == pa).all()
    _check_trace(rows_gpu, rows)


def test_scale22_grid8_64bit_words_streams_bit_exact():
    """The scale-22 configuration: Kronecker scale 22, 8x8 grid, COMPRESS_SIEVE
    with 64-bit WAH words.  Levels and parents of two roots, and every exchanged
    stream and row buffer of the first, bit-exact with the oracle's Alg. 3."""
    bfs = _lib()
    n, src, dst = graphgen.edges(22, 16)
    go = oracle.csr(n, src, dst)
    p, wah = 8, 64
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2, wah_bits=wah)
    roots = graphgen.pick_roots(n, src, dst, 2)
    cap = 32 * (2 * p * p + n * p // (wah - 1) + 8)
    lv, pa, tr, rows = oracle.dist_bfs(go, p, int(roots[0]), mode=oracle.COMPRESS_SIEVE, w=wah, trace=True,
                                       max_levels=32, trace_cap=cap, rows=True)
    parent, level, st = _run(g, int(roots[0]), stats=True, trace_capacity=cap * 2, row_trace_capacity=cap * 2)
    assert (level == lv).all() and (parent == pa).all()
    _check_trace(_unpack_trace(st, wah), tr)
    _check_trace(_unpack_trace(st, wah, rows=True), rows)
    lv, pa = oracle.bfs(go, int(roots[1]))
    parent, level, _ = _run(g, int(roots[1]))
    assert (level == lv).all() and (parent == pa).all()


def test_scale26_grid16_bench_configuration_one_root():
    """The bench's workload and launch configuration: Kronecker scale 26 (67M
    vertices, 2.1G entries), 16x16 grid, COMPRESS_SIEVE, 32-bit words, the
    global-memory visiting path with rows in turn.  One seeded root: all levels
    and parents bit-exact with the oracle; the PLAIN search agrees."""
    bfs = _lib()
    n, src, dst = graphgen.edges(26, 16)
    g = bfs.Graph.from_edges(n, src, dst, p=16, mode=2)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    parent, level, _ = _run(g, r)
    g.set_mode(0)
    parent0, level0, _ = _run(g, r)
    del g
    torch.cuda.empty_cache()
    go = oracle.csr(n, src, dst)
    del src, dst
    lv, pa = oracle.bfs(go, r)
    assert (level == lv).all() and (parent == pa).all()
    assert (level0 == lv).all() and (parent0 == pa).all()


def test_erdos_renyi_scale26_grid16_control_one_root():
    """The bench's control workload: Erdos-Renyi scale 26 (uniform endpoints,
    the Kronecker graph's n and m), 16x16 grid, COMPRESS_SIEVE and PLAIN, the
    global-memory visiting path.  One seeded root: all levels and parents
    bit-exact with the oracle."""
    bfs = _lib()
    n, src, dst = graphgen.edges(26, 16, kind=graphgen.ERDOS_RENYI)
    g = bfs.Graph.from_edges(n, src, dst, p=16, mode=2)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    parent, level, _ = _run(g, r)
    g.set_mode(0)
    parent0, level0, _ = _run(g, r)
    del g
    torch.cuda.empty_cache()
    go = oracle.csr(n, src, dst)
    del src, dst
    lv, pa = oracle.bfs(go, r)
    assert (level == lv).all() and (parent == pa).all()
    assert (level0 == lv).all() and (parent0 == pa).all()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_long_columns_cut_into_pieces(mode):
    """Columns around and far above the piece length (2048 entries): stars whose
    centres have 2047, 2048, 2049, 4097 and 20000 leaves, joined by a path, on
    1 x 1 and 2 x 2 grids, from a centre and from a leaf; levels, parents and
    streams equal the oracle's, on the global visiting path too (a range too
    long for the row window)."""
    bfs = _lib()
    src, dst, base = [], [], 0
    centres = []
    for leaves in (2047, 2048, 2049, 4097, 20000):
        centres.append(base)
        src += [base] * leaves
        dst += list(range(base + 1, base + 1 + leaves))
        base += leaves + 1
    for a, b in zip(centres[:-1], centres[1:]):
        src.append(a + 1)
        dst.append(b)
    n = max(base, 2_000_000)                         # isolated tail: ranges beyond the row window
    src = np.array(src, np.int32)
    dst = np.array(dst, np.int32)
    go = oracle.csr(n, src, dst)
    for p in (1, 2):
        g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
        for r in (centres[0], centres[-1] + 7, centres[2]):
            lv, pa, tr = oracle.dist_bfs(go, p, r, mode=ORACLE_MODE[mode], trace=True)
            parent, level, st = _run(g, r, stats=True, trace_capacity=1 << 22 if mode else 0)
            assert (level == lv).all() and (parent == pa).all()
            if mode:
                _check_trace(_unpack_trace(st, 32), tr)
            parent, level, _ = _run(g, r)
            assert (level == lv).all() and (parent == pa).all()
