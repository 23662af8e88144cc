"""Bottom-up and hybrid levels (the top-down / bottom-up traversal the paper names
in Sec. VIII and IX as the next method to combine with compression and sieve).

Levels and parents must equal the oracle's closed form (smallest neighbour on
the previous level), every exchanged stream must equal the oracle's (the
exchange does not depend on the direction), and the per-level directions must
follow the switching rule, recomputed here from the oracle's levels and
degrees.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle
from tests.golden_io import bfs_example
from tests.test_gpu_bfs import ORACLE_MODE, _check_trace, _lib, _run, _unpack_trace

pytestmark = pytest.mark.gpu

TOP_DOWN, HYBRID, BOTTOM_UP = 0, 1, 2


def _expected_directions(go, level, root, policy, alpha=14, beta=24):
    """Direction of every exchange under the switching rule, from the oracle's
    levels: bottom-up once the growing frontier's degree sum exceeds 1/alpha of
    the unvisited vertices' degree sum, top-down again once the shrinking
    frontier has fewer than n/beta vertices."""
    deg = np.diff(go.row_ptr).astype(np.int64)
    n = go.n
    depth = int(level.max())
    sizes = [int((level == k).sum()) for k in range(depth + 2)]
    degs = [int(deg[level == k].sum()) for k in range(depth + 2)]
    bu = policy == BOTTOM_UP
    m_u = int(deg.sum()) - int(deg[root])
    out = [int(bu)]
    for k in range(depth):
        f, prev, mf = sizes[k + 1], sizes[k], degs[k + 1]
        m_u -= mf
        if policy == BOTTOM_UP:
            bu = True
        elif policy == HYBRID:
            bu = (f > prev and mf * alpha > m_u) if not bu else not (f < prev and f * beta < n)
        else:
            bu = False
        out.append(int(bu))
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("p,wah", [(1, 32), (2, 64), (4, 32), (5, 32)])
def test_bottom_up_every_level_bit_exact(mode, p, wah):
    bfs = _lib()
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode, wah_bits=wah)
    g.set_direction(BOTTOM_UP)
    for r in graphgen.pick_roots(n, src, dst, 3):
        lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=ORACLE_MODE[mode], w=wah, trace=True)
        parent, level, st = _run(g, int(r), stats=True, trace_capacity=1 << 22 if mode else 0)
        assert (level == lv).all() and (parent == pa).all()
        assert [ls["bottom_up"] for ls in st.levels] == [1] * st.n_levels
        if mode:
            _check_trace(_unpack_trace(st, wah), tr)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_hybrid_follows_the_switching_rule(mode):
    """Kronecker scale 16 on a 4 x 4 grid: the hybrid switches to bottom-up on
    the dense levels and back; results and streams equal the oracle's, and the
    CUDA-graph loop (no statistics) gives the same levels and parents."""
    bfs = _lib()
    n, src, dst = graphgen.edges(16, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
    g.set_direction(HYBRID)
    saw_switch = False
    for r in graphgen.pick_roots(n, src, dst, 4):
        lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=ORACLE_MODE[mode], trace=True)
        parent, level, st = _run(g, int(r), stats=True, trace_capacity=1 << 23 if mode else 0)
        assert (level == lv).all() and (parent == pa).all()
        if mode:
            _check_trace(_unpack_trace(st, 32), tr)
        got = [ls["bottom_up"] for ls in st.levels]
        assert got == _expected_directions(go, lv, int(r), HYBRID)
        saw_switch |= 0 < sum(got) < len(got)
        parent, level, _ = _run(g, int(r))
        assert (level == lv).all() and (parent == pa).all()
    assert saw_switch


def test_hybrid_thresholds_and_switching_back_to_top_down():
    """alpha and beta change the levels that run bottom-up; the graph's loop is
    rebuilt when the policy changes and results never change."""
    bfs = _lib()
    n, src, dst = graphgen.edges(15, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=2, mode=2)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    lv, pa = oracle.bfs(go, r)
    for policy, alpha, beta in [(HYBRID, 1, 1), (HYBRID, 1000, 2), (HYBRID, 14, 1000000), (TOP_DOWN, 14, 24),
                                (BOTTOM_UP, 14, 24), (HYBRID, 14, 24)]:
        g.set_direction(policy, alpha, beta)
        parent, level, st = _run(g, r, stats=True)
        assert (level == lv).all() and (parent == pa).all()
        got = [ls["bottom_up"] for ls in st.levels]
        assert got == _expected_directions(go, lv, r, policy, alpha, beta), (policy, alpha, beta)
        parent, level, _ = _run(g, r)
        assert (level == lv).all() and (parent == pa).all()


def test_bottom_up_ragged_ranges_er_and_one_fills():
    """n not a multiple of p (ranges that end inside a visited word), an
    Erdos-Renyi graph, and a dense contiguous frontier (1-fill runs decoded)."""
    bfs = _lib()
    n = 100_003
    src, dst = graphgen.random_edges(n, 400_000, 11)
    go = oracle.csr(n, src, dst)
    for p, mode in [(3, 2), (7, 1), (7, 0)]:
        g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
        g.set_direction(BOTTOM_UP)
        for r in (0, 77_777, n - 1):
            lv, pa = oracle.bfs(go, r)
            parent, level, _ = _run(g, r)
            assert (level == lv).all() and (parent == pa).all()
    mid = np.arange(1, 4000)
    src = np.concatenate([np.zeros(len(mid), np.int64), mid]).astype(np.int32)
    dst = np.concatenate([mid, 4000 + (mid * 7) % 4000]).astype(np.int32)
    go = oracle.csr(8000, src, dst)
    for mode in (1, 2):
        for wah in (32, 64):
            g = bfs.Graph.from_edges(8000, src, dst, p=2, mode=mode, wah_bits=wah)
            g.set_direction(BOTTOM_UP)
            lv, pa = oracle.bfs(go, 0)
            parent, level, _ = _run(g, 0)
            assert (level == lv).all() and (parent == pa).all()


def test_paper_example_and_isolated_roots_bottom_up():
    bfs = _lib()
    d = bfs_example()
    for p in (1, 2, 4):
        for mode in (0, 1, 2):
            g = bfs.Graph.from_edges(d["n"], d["src"], d["dst"], p=p, mode=mode)
            g.set_direction(BOTTOM_UP)
            parent, level, _ = _run(g, d["root"])
            assert level.tolist() == d["levels"]
            assert parent.tolist() == d["parents_min"]
    src = np.array([0, 1, 5], np.int32)
    dst = np.array([1, 2, 5], np.int32)
    g = bfs.Graph.from_edges(6, src, dst, p=3, mode=2)
    g.set_direction(HYBRID, 1, 1)
    parent, level, _ = _run(g, 5)
    assert level.tolist() == [-1, -1, -1, -1, -1, 0] and parent.tolist() == [-1, -1, -1, -1, -1, 5]
    parent, level, _ = _run(g, 0)
    assert level.tolist() == [0, 1, 2, -1, -1, -1] and parent.tolist() == [0, 0, 1, -1, -1, -1]


def test_direction_needs_an_undirected_graph():
    from paper_1208_5542_gb300 import native
    bfs = _lib()
    n, src, dst = graphgen.edges(10, 8)
    g = bfs.Graph.from_edges(n, src, dst, symmetrize=False, p=2)
    for policy in (HYBRID, BOTTOM_UP):
        with pytest.raises(native.BfsError, match="INVALID_ARG"):
            g.set_direction(policy)
    g.set_direction(TOP_DOWN)
    go = oracle.csr(n, src, dst)
    gc = bfs.Graph.from_csr(n, go.row_ptr, go.col, p=2)
    with pytest.raises(native.BfsError, match="INVALID_ARG"):
        gc.set_direction(HYBRID)
    gs = bfs.Graph.from_edges(n, src, dst, p=2)
    for bad in [(3, 14, 24), (-1, 14, 24), (HYBRID, 0, 24), (HYBRID, 14, 0), (HYBRID, 2_000_000, 24)]:
        with pytest.raises(native.BfsError, match="INVALID_ARG"):
            gs.set_direction(*bad)
    before = gs.footprint()
    gs.set_direction(HYBRID)
    assert gs.footprint() >= before + 4 * n


def test_scale22_grid8_hybrid_sampled_roots():
    """Kronecker scale 22 on the 8 x 8 grid (the scale-22 benchmark layout), hybrid
    levels in COMPRESS_SIEVE and PLAIN mode: two roots bit-exact with the oracle."""
    bfs = _lib()
    n, src, dst = graphgen.edges(22, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=8, mode=2)
    g.set_direction(HYBRID)
    roots = graphgen.pick_roots(n, src, dst, 2)
    for mode in (2, 0):
        g.set_mode(mode)
        for r in roots:
            lv, pa = oracle.bfs(go, int(r))
            parent, level, st = _run(g, int(r), stats=True)
            assert (level == lv).all() and (parent == pa).all()
            assert 0 < sum(ls["bottom_up"] for ls in st.levels) < st.n_levels
    torch.cuda.synchronize()
