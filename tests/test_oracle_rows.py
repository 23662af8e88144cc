"""Pins of the oracle's row buffers: the compressed fold of a block-row (DIR-WAH
with the 2D partitioning of Sec. VIII).  Row buffer (i, j) at level k = the WAH
stream of the vertices of range i reached by block (i, j) from the frontier it
received, sieved by the visited set of range i before the level."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.golden_io import bfs_example, row_buffer_example


def _ranges(n, p):
    nb = -(-n // p)
    return [(min(n, b * nb), min(n, (b + 1) * nb)) for b in range(p)]


def _dense_rows(n, src, dst, root, p, symmetrize=True):
    """Row buffers by dense boolean algebra, level by level: f_0 = {root};
    block (i, j) reaches (A_{i,j} f_j > 0); sieve by not(visited); the next
    frontier is the reached set minus the visited one.  Returns per level the
    list of p*p 0/1 vectors and the next frontier."""
    A = np.zeros((n, n), dtype=np.int64)      # A[v, u] = 1 for an entry u -> v
    A[dst, src] = 1
    if symmetrize:
        A[src, dst] = 1
    f = np.zeros(n, dtype=bool)
    f[root] = True
    vis = f.copy()
    out = []
    rg = _ranges(n, p)
    while f.any():
        reach = (A @ f.astype(np.int64)) > 0
        nxt = reach & ~vis
        blocks = []
        for (ib, ie) in rg:
            for (jb, je) in rg:
                t = (A[ib:ie, jb:je] @ f[jb:je].astype(np.int64)) > 0
                blocks.append((t & ~vis[ib:ie]).astype(np.uint8))
        out.append((blocks, nxt))
        vis |= nxt
        f = nxt
    return out


def test_paper_example_row_words():
    """The hand-derived row buffers of the Sec. III-A graph for p = 1 and 2, both word widths."""
    d = bfs_example()
    g = oracle.csr(d["n"], d["src"], d["dst"])
    want = row_buffer_example()
    for p, levels in want.items():
        for w in (32, 64):
            lv, pa, _, rows = oracle.dist_bfs(g, p, d["root"], mode=oracle.COMPRESS_SIEVE, w=w, rows=True)
            assert lv.tolist() == d["levels"] and pa.tolist() == d["parents_min"]
            got = [[[int(x) for x in s] for s in level] for level in rows]
            assert got == [[[x] for x in level] for level in levels], (p, w)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("p", [2, 3])
def test_row_buffers_vs_dense_products(seed, p):
    """Every row buffer decodes to the block's dense product sieved by not(visited);
    their OR over j is the next frontier of range i (Lemma 2 for the fold)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(p, 41))
    m = int(rng.integers(n, 4 * n))
    sym = seed % 3 != 0
    src, dst = graphgen.random_edges(n, m, seed)
    g = oracle.csr(n, src, dst, symmetrize=sym)
    root = int(rng.integers(0, n))
    for w in (32, 64):
        _, _, _, rows = oracle.dist_bfs(g, p, root, mode=oracle.COMPRESS_SIEVE, w=w, rows=True)
        dense = _dense_rows(n, src, dst, root, p, symmetrize=sym)
        assert len(rows) == len(dense)
        rg = _ranges(n, p)
        for k, (level_rows, (blocks, nxt)) in enumerate(zip(rows, dense)):
            for i, (ib, ie) in enumerate(rg):
                acc = np.zeros(ie - ib, dtype=np.uint8)
                for j in range(p):
                    s = i * p + j
                    bits = oracle.wah_decode(level_rows[s], ie - ib, w)
                    assert bits is not None and (bits == blocks[s]).all(), (k, i, j)
                    acc |= bits
                assert (acc.astype(bool) == nxt[ib:ie]).all(), (k, i)


def test_row_buffers_kronecker_runs_and_literals():
    """A Kronecker graph of scale 10 on a 3 x 3 grid (ragged ranges of 342 bits:
    literals, zero fills and active words): the decoded row buffers equal the
    dense products, and the sieve by the visited set clears something."""
    n, src, dst = graphgen.edges(10, 16)
    g = oracle.csr(n, src, dst)
    p = 3
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    _, _, _, rows = oracle.dist_bfs(g, p, root, mode=oracle.COMPRESS_SIEVE, rows=True)
    dense = _dense_rows(n, src, dst, root, p)
    rg = _ranges(n, p)
    cleared = 0
    kinds = set()
    for level_rows, (blocks, _) in zip(rows, dense):
        for s, words in enumerate(level_rows):
            ib, ie = rg[s // p]
            assert (oracle.wah_decode(words, ie - ib) == blocks[s]).all()
            for x in words:
                kinds.add("fill" if int(x) >> 31 else "literal")
    # the unsieved products hold visited vertices that the buffers drop
    A = np.zeros((n, n), dtype=np.int64)
    A[dst, src] = 1
    A[src, dst] = 1
    lv = oracle.bfs_levels(g, root)
    for k in range(len(rows)):
        f = lv == k
        vis = (lv >= 0) & (lv <= k)
        cleared += int((((A @ f.astype(np.int64)) > 0) & vis).sum())
    assert cleared > 0 and kinds == {"fill", "literal"}


def test_modes_without_a_sieve_have_no_row_buffers():
    d = bfs_example()
    g = oracle.csr(d["n"], d["src"], d["dst"])
    with pytest.raises(ValueError):
        oracle.dist_bfs(g, 2, d["root"], mode=oracle.COMPRESS, rows=True)
