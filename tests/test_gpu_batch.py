"""Batched multi-source search (64 bit-parallel lanes, one CUDA-graph launch) vs the oracle."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1208_5542_gb300 import bfs, build
    build.build()
    return bfs


def _check(go, roots, levels, parents=None):
    lv = levels.cpu().numpy()
    pa = parents.cpu().numpy() if parents is not None else None
    for r, root in enumerate(roots):
        want_l, want_p = oracle.bfs(go, int(root))
        assert (lv[r] == want_l).all(), f"lane {r} (root {root}) levels differ"
        if pa is not None:
            assert (pa[r] == want_p).all(), f"lane {r} (root {root}) parents differ"


@pytest.mark.parametrize("p", [1, 3, 4])
@pytest.mark.parametrize("k", [1, 17, 64])
def test_batch_levels_and_parents_scale14(p, k):
    bfs = _lib()
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p)
    roots = graphgen.pick_roots(n, src, dst, k, seed=3)
    levels, parents, st = g.run_batch(roots, parents=True)
    torch.cuda.synchronize()
    _check(go, roots, levels, parents)
    assert st["n_levels"] == int(levels.max().item()) + 1
    levels2, _, _ = g.run_batch(roots)            # the graph is reused: same answer without parents
    assert torch.equal(levels, levels2)


def test_batch_duplicate_roots_isolated_and_directed():
    bfs = _lib()
    src = np.array([0, 1, 2, 5, 7], np.int32)
    dst = np.array([1, 2, 3, 5, 6], np.int32)
    go = oracle.csr(8, src, dst, symmetrize=False)
    g = bfs.Graph.from_edges(8, src, dst, symmetrize=False, p=2)
    roots = [0, 0, 5, 3, 4, 7, 2, 0]
    levels, parents, _ = g.run_batch(roots, parents=True)
    _check(go, roots, levels, parents)


def test_batch_scale20_grid8_sixty_four_roots():
    """The batched configuration: scale-20 Kronecker graph, 64 roots in one launch."""
    bfs = _lib()
    n, src, dst = graphgen.edges(20, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=8)
    roots = graphgen.pick_roots(n, src, dst, 64)
    levels, _, st = g.run_batch(roots)
    _check(go, roots, levels)
    assert st["edges_scanned"] > 0


def test_batch_autotune_keeps_results():
    bfs = _lib()
    n, src, dst = graphgen.edges(16, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=4)
    roots = graphgen.pick_roots(n, src, dst, 64)
    t, c = g.batch_autotune(roots)
    assert t in (128, 256, 512, 1024) and c in (1, 2, 4, 8, 16) and t * c <= 2048
    levels, parents, _ = g.run_batch(roots[:8], parents=True)
    _check(go, roots[:8], levels, parents)


def test_batch_bad_arguments():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    g = bfs.Graph.from_edges(10, np.array([0], np.int32), np.array([1], np.int32))
    with pytest.raises(BfsError, match="INVALID_ARG"):
        g.run_batch(list(range(10)) * 7)            # 70 roots
    with pytest.raises(BfsError, match="INVALID_ARG"):
        g.run_batch([10])
