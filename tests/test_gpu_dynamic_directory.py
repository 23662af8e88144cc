"""The dynamic cross directory on the GPU (Sec. V-B: the directories kept up to
date on both sides as the search goes on).  Every exchanged stream (and every
row buffer of the fold) must equal the oracle's search with the dynamic
directory word for word, level by level; levels and parents stay those of the
plain search; the sieve then carries fewer vertices than with the static
directory of Alg. 3, never more."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.test_gpu_bfs import _check_trace, _lib, _run, _unpack_trace

pytestmark = pytest.mark.gpu

TOP_DOWN, HYBRID, BOTTOM_UP = 0, 1, 2


def _exchanged(st):
    return [int(ls["exchanged_vertices"]) for ls in st.levels]


@pytest.mark.parametrize("scale,p,wah", [(12, 1, 32), (14, 2, 64), (14, 4, 32), (14, 5, 32), (13, 8, 32)])
def test_dynamic_streams_equal_the_oracle(scale, p, wah):
    bfs = _lib()
    n, src, dst = graphgen.edges(scale, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2, wah_bits=wah)
    g.set_row_exchange(False)
    fewer = False
    for r in graphgen.pick_roots(n, src, dst, 3):
        lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=oracle.COMPRESS_SIEVE, w=wah, trace=True, dynamic=True)
        g.set_dynamic_directory(True)
        parent, level, st = _run(g, int(r), stats=True, trace_capacity=1 << 22)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, wah), tr)
        dyn = _exchanged(st)
        parent, level, _ = _run(g, int(r))                  # the graph-launched level loop
        assert (level == lv).all() and (parent == pa).all()
        g.set_dynamic_directory(False)
        _, _, st0 = _run(g, int(r), stats=True)
        static = _exchanged(st0)
        assert len(dyn) == len(static) and all(a <= b for a, b in zip(dyn, static))
        fewer |= sum(dyn) < sum(static)
    if p > 1:
        assert fewer


def test_dynamic_row_buffers_hybrid_and_bottom_up():
    """With the row exchange the row buffers follow the dynamically sieved
    streams (the oracle's row trace of the same search); bottom-up and hybrid
    levels exchange the same streams, since the bits depend only on the
    visited sets; repeated searches start from fresh directories."""
    bfs = _lib()
    n, src, dst = graphgen.edges(15, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
    g.set_dynamic_directory(True)
    cap = 1 << 23
    for r in graphgen.pick_roots(n, src, dst, 2):
        lv, pa, tr, rows = oracle.dist_bfs(go, p, int(r), mode=oracle.COMPRESS_SIEVE, trace=True, rows=True,
                                           dynamic=True, max_levels=64, trace_cap=cap)
        for policy in (TOP_DOWN, HYBRID, BOTTOM_UP):
            g.set_direction(policy, 4, 24)
            g.set_row_exchange(policy == TOP_DOWN)
            for _ in range(2):
                parent, level, st = _run(g, int(r), stats=True, timing=True, trace_capacity=2 * cap,
                                         row_trace_capacity=2 * cap if policy == TOP_DOWN else 0)
                assert (level == lv).all() and (parent == pa).all()
                _check_trace(_unpack_trace(st, 32), tr)
                if policy == TOP_DOWN:
                    _check_trace(_unpack_trace(st, 32, rows=True), rows)
                assert all(ls["ms_directory_update"] >= 0.0 for ls in st.levels)
                parent, level, _ = _run(g, int(r))
                assert (level == lv).all() and (parent == pa).all()


def test_dynamic_adaptive_format():
    """The level-adaptive format re-sends the dynamically sieved slices: every
    slot's format and elements equal the oracle's choice for them."""
    from tests.test_gpu_adaptive import _check, _unpack
    bfs = _lib()
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
    g.set_exchange_format(True)
    g.set_dynamic_directory(True)
    for r in graphgen.pick_roots(n, src, dst, 2):
        lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=oracle.COMPRESS_SIEVE, trace=True, dynamic=True)
        parent, level, st = g.run(int(r), stats=True, trace_capacity=1 << 22)
        assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
        _check(_unpack(st), oracle.adaptive_trace(tr, n, p))


def test_dynamic_long_columns_and_directed_graphs():
    """A star whose centre has a long column in every block (the warp-wide scan)
    plus a path, undirected and directed (a CSR graph, not symmetrised): streams
    equal the oracle's on a ragged 3 x 3 grid, from the centre, a leaf and the
    path's end."""
    bfs = _lib()
    leaves = np.arange(1, 5001)
    path = np.arange(5001, 5400)
    src = np.concatenate([np.zeros(len(leaves), np.int64), path[:-1], [4999]]).astype(np.int32)
    dst = np.concatenate([leaves, path[1:], [5001]]).astype(np.int32)
    n = 5400
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=3, mode=2)
    g.set_dynamic_directory(True)
    for r in (0, 17, 5399):
        lv, pa, tr = oracle.dist_bfs(go, 3, r, mode=oracle.COMPRESS_SIEVE, trace=True, dynamic=True)
        parent, level, st = _run(g, r, stats=True, trace_capacity=1 << 20)
        assert (level == lv).all() and (parent == pa).all()
        _check_trace(_unpack_trace(st, 32), tr)
    # directed: Kronecker edges one way only
    n2, s2, d2 = graphgen.edges(13, 16)
    gd = oracle.csr(n2, s2, d2, symmetrize=False)
    for p, wah in ((2, 32), (5, 64)):
        g2 = bfs.Graph.from_csr(n2, gd.row_ptr, gd.col, p=p, mode=2, wah_bits=wah)
        g2.set_dynamic_directory(True)
        for r in graphgen.pick_roots(n2, s2, d2, 3):
            lv, pa, tr = oracle.dist_bfs(gd, p, int(r), mode=oracle.COMPRESS_SIEVE, w=wah, trace=True, dynamic=True)
            parent, level, st = _run(g2, int(r), stats=True, trace_capacity=1 << 22)
            assert (level == lv).all() and (parent == pa).all()
            _check_trace(_unpack_trace(st, wah), tr)


def test_dynamic_scale22_grid8_one_root():
    """Kronecker scale 22 on the 8 x 8 grid: every stream of one search."""
    bfs = _lib()
    n, src, dst = graphgen.edges(22, 16)
    go = oracle.csr(n, src, dst)
    p = 8
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
    g.set_dynamic_directory(True)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    cap = 32 * (2 * p * p + n * p // 31 + 8)
    lv, pa, tr = oracle.dist_bfs(go, p, r, mode=oracle.COMPRESS_SIEVE, trace=True, dynamic=True, max_levels=32,
                                 trace_cap=cap)
    parent, level, st = _run(g, r, stats=True, trace_capacity=2 * cap)
    assert (level == lv).all() and (parent == pa).all()
    _check_trace(_unpack_trace(st, 32), tr)


def test_other_modes_ignore_the_dynamic_directory():
    bfs = _lib()
    n, src, dst = graphgen.edges(10, 16)
    go = oracle.csr(n, src, dst)
    g2 = bfs.Graph.from_edges(n, src, dst, p=2, mode=0)
    g2.set_dynamic_directory(True)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    lv, pa = oracle.bfs(go, r)
    for mode in (0, 1):
        g2.set_mode(mode)
        parent, level, st = _run(g2, r, stats=True, timing=True)
        assert (level == lv).all() and (parent == pa).all()
        assert all(ls["ms_directory_update"] == 0.0 for ls in st.levels)
