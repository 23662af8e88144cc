"""The reading behind bottom-up levels, checked on the CPU against the oracle.

A bottom-up level lets every unvisited vertex v (range i) scan its neighbours
range by range (j = 0, 1, ...), in any order inside a range, and stop after the
first range holding a frontier neighbour, taking the smallest one there.  Two
facts make that exact:

* the parent it finds is the closed-form parent (the smallest neighbour on the
  previous level), because the ranges are ordered intervals of ids;
* every bit it tests is carried by the block's own sieved stream: v in range i
  adjacent to u in range j means the directory V_{i,j} (Eq. 4) has u's bit, so
  f_j sieved by V_{i,j} holds f_j(u), and an OR over the block-rows of the
  decoded streams holds exactly that bit.
"""
import numpy as np
import pytest

import graphgen
import oracle


def _bottom_up_parent(go, level, v, k, p, rng):
    """Scan v's neighbours range by range, shuffled inside each range; stop after
    the first range with a neighbour on level k; return its smallest one or -1."""
    nbrs = go.col[go.row_ptr[v]:go.row_ptr[v + 1]]
    by_range = {}
    for u in nbrs:
        j = next(b for b in range(p) if oracle.range_begin(go.n, p, b) <= u < oracle.range_begin(go.n, p, b + 1))
        by_range.setdefault(j, []).append(int(u))
    for j in sorted(by_range):
        us = by_range[j]
        rng.shuffle(us)
        hits = [u for u in us if level[u] == k]
        if hits:
            return min(hits)
    return -1


@pytest.mark.parametrize("seed,p", [(1, 1), (2, 3), (3, 4), (4, 7)])
def test_range_ordered_scan_reaches_the_smallest_parent(seed, p):
    n, src, dst = graphgen.edges(9, 8, seed=seed)
    go = oracle.csr(n, src, dst)
    rng = np.random.default_rng(seed)
    root = int(graphgen.pick_roots(n, src, dst, 1, seed=seed)[0])
    level, parent = oracle.bfs(go, root)
    for k in range(int(level.max())):
        # every vertex unvisited before level k+1 is expanded bottom-up
        for v in np.flatnonzero((level < 0) | (level > k)):
            got = _bottom_up_parent(go, level, int(v), k, p, rng)
            if level[v] == k + 1:
                assert got == parent[v], (k, v, got, parent[v])
            else:
                assert got == -1


@pytest.mark.parametrize("p", [2, 5])
def test_every_tested_bit_is_in_the_blocks_own_stream(p):
    """For every entry v -> u with v in range i and u in range j, V_{i,j} holds u:
    the stream of slot (i, j) carries f_j(u), whatever the frontier."""
    n, src, dst = graphgen.edges(9, 8)
    go = oracle.csr(n, src, dst)
    begin = [oracle.range_begin(n, p, b) for b in range(p + 1)]
    dirs = {(i, j): oracle.directory(go, p, i, j) for i in range(p) for j in range(p)}
    for v in range(n):
        i = int(np.searchsorted(begin, v, side="right") - 1)
        for u in go.col[go.row_ptr[v]:go.row_ptr[v + 1]]:
            j = int(np.searchsorted(begin, u, side="right") - 1)
            assert dirs[(i, j)][u - begin[j]] == 1, (v, int(u), i, j)
    # and the OR over the block-rows of the sieved slices is f on every vertex with an edge
    rng = np.random.default_rng(3)
    f = rng.random(n) < 0.3
    has_edge = np.diff(go.row_ptr) > 0
    folded = np.zeros(n, bool)
    for (i, j), d in dirs.items():
        folded[begin[j]:begin[j + 1]] |= f[begin[j]:begin[j + 1]] & (d == 1)
    assert (folded[has_edge] == f[has_edge]).all()
    assert not folded[~has_edge].any()
