"""Pins of the CPU oracle against the worked examples printed in the paper.

Sources: the 8-vertex BFS example of Sec. III-A, the partition / directory /
sieve example of Sec. V-A (Eq. 3-4), and the WAH examples of Table 3.
"""
import numpy as np

import oracle
from tests.golden_io import bfs_example, directory_example, wah_examples


def _paper_graph():
    d = bfs_example()
    g = oracle.csr(d["n"], d["src"], d["dst"], symmetrize=True)
    return d, g


def test_paper_graph_adjacency_matches_printed_matrix():
    d, g = _paper_graph()
    A = np.zeros((d["n"], d["n"]), dtype=np.uint8)
    for u in range(d["n"]):
        for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            A[u, v] = 1
    assert (A == d["A"]).all()
    assert len(g.col) == 20          # 10 undirected edges, both directions


def test_paper_levels_and_frontiers():
    d, g = _paper_graph()
    level = oracle.bfs_levels(g, d["root"])
    assert level.tolist() == d["levels"]
    for k, members in d["frontiers"].items():
        assert sorted(np.nonzero(level == k)[0].tolist()) == members


def test_paper_parents_min_and_max():
    d, g = _paper_graph()
    level, parent = oracle.bfs(g, d["root"])
    assert parent.tolist() == d["parents_min"]
    assert oracle.parents(g, level, d["root"], use_max=True).tolist() == d["parents_max"]


def test_paper_first_spmv_step():
    """A^T (x) f_L0 (.) not(pi_0) = f_L1 as printed in Sec. III-A."""
    d, _ = _paper_graph()
    A = d["A"].astype(np.int64)
    f0 = np.zeros(8, dtype=np.int64)
    f0[0] = 1
    pi0 = f0.copy()
    f1 = ((A.T @ f0) > 0).astype(np.int64) * (1 - pi0)
    assert np.nonzero(f1)[0].tolist() == d["frontiers"][1]


def test_paper_directory_and_sieve_example():
    d, g = _paper_graph()
    ex = directory_example()
    p = ex["p"]
    i, j = ex["block"]
    assert [oracle.range_len(8, p, b) for b in range(p)] == [2, 2, 2, 2]
    # the printed block A_{4,2}: rows = range i (destinations), cols = range j (sources)
    ib, jb = oracle.range_begin(8, p, i), oracle.range_begin(8, p, j)
    blk = d["A"][jb:jb + 2, ib:ib + 2].T          # A[u, v] = entry u -> v
    assert blk.flatten().tolist() == ex["A_block"]
    V = oracle.directory(g, p, i, j)
    assert V.tolist() == ex["V"]
    sieved = np.array(ex["f_j"], dtype=np.uint8) & V
    assert sieved.tolist() == ex["sieved"]
    D = oracle.cross_directory(g, p)
    assert D[i, jb:jb + 2].tolist() == ex["V"]


def test_paper_wah_examples():
    for name, ex in wah_examples().items():
        words = oracle.wah_encode(ex["bits"], w=ex["w"], fill_bit=bool(ex["fill_bit"]))
        assert [int(x) for x in words] == ex["words"], name
        back = oracle.wah_decode(words, len(ex["bits"]), w=ex["w"], fill_bit=bool(ex["fill_bit"]))
        assert back is not None and (back == ex["bits"]).all(), name


def test_paper_dirwah_exchange_on_example():
    """Alg. 3 on the example: the stream P2 sends to P4 for f_L1 carries only v3.

    f_L1 = {2,3,5}; range 1 = {2,3}; V for block-row 3 = (0,1) -> sieved (0,1);
    two bits, no full 31-bit group, so the stream is one active word 0b01.
    """
    d, g = _paper_graph()
    level, parent, tr = oracle.dist_bfs(g, 4, d["root"], mode=oracle.COMPRESS_SIEVE, trace=True)
    assert level.tolist() == d["levels"]
    assert parent.tolist() == d["parents_min"]
    assert len(tr) == 4                      # exchanges feeding levels 0..3
    assert [int(x) for x in tr[1][3 * 4 + 1]] == [0b01]
    # the root's exchange: only vertex 0 set; block-row 0 has no entry from v0
    # (v0's neighbours 2,3,5 live in ranges 1 and 2), so that stream is zero
    assert [int(x) for x in tr[0][0 * 4 + 0]] == [0b00]
    assert [int(x) for x in tr[0][1 * 4 + 0]] == [0b10]
    assert [int(x) for x in tr[0][2 * 4 + 0]] == [0b10]
    assert [int(x) for x in tr[0][3 * 4 + 0]] == [0b00]
