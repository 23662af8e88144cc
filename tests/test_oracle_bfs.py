"""Pins of the oracle's BFS, parents and Algorithms 1-3 against brute force and invariants."""
import numpy as np
import pytest

import graphgen
import oracle


def _dense(n, src, dst, symmetrize=True):
    A = np.zeros((n, n), dtype=bool)          # A[u, v]: entry u -> v
    A[src, dst] = True
    if symmetrize:
        A[dst, src] = True
    return A


def _floyd_levels(A, root):
    """All-pairs hop distances by Floyd-Warshall on the dense matrix."""
    n = A.shape[0]
    INF = 10 ** 9
    dist = np.full((n, n), INF, dtype=np.int64)
    dist[A] = 1
    np.fill_diagonal(dist, 0)
    for k in range(n):
        dist = np.minimum(dist, dist[:, k:k + 1] + dist[k:k + 1, :])
    d = dist[root]
    return np.where(d >= INF, -1, d).astype(np.int32)


def _brute_parents(A, level, root, use_max=False):
    n = A.shape[0]
    par = np.full(n, -1, dtype=np.int32)
    for v in range(n):
        if v == root:
            par[v] = root
            continue
        if level[v] < 0:
            continue
        cands = [u for u in range(n) if A[u, v] and level[u] == level[v] - 1]
        par[v] = max(cands) if use_max else min(cands)
    return par


@pytest.mark.parametrize("seed", range(12))
def test_levels_and_parents_vs_floyd_warshall(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 49))
    m = int(rng.integers(0, 3 * n))
    sym = bool(seed % 3)
    src, dst = graphgen.random_edges(n, m, seed)
    g = oracle.csr(n, src, dst, symmetrize=sym)
    A = _dense(n, src, dst, sym)
    for root in rng.choice(n, size=min(n, 4), replace=False):
        level, parent = oracle.bfs(g, int(root))
        assert (level == _floyd_levels(A, int(root))).all()
        assert (parent == _brute_parents(A, level, int(root))).all()
        pmax = oracle.parents(g, level, int(root), use_max=True)
        assert (pmax == _brute_parents(A, level, int(root), use_max=True)).all()


def _check_tree(g, root, level, parent):
    n = g.n
    assert level[root] == 0 and parent[root] == root
    u = np.repeat(np.arange(n), np.diff(g.row_ptr))
    v = g.col
    # every vertex in the root's component is reached (no edge leaves the reached set)
    assert not ((level[u] >= 0) & (level[v] < 0)).any()
    # levels differ by at most one across every edge
    both = (level[u] >= 0) & (level[v] >= 0)
    assert (np.abs(level[u][both] - level[v][both]) <= 1).all()
    reached = np.nonzero((level >= 0) & (np.arange(n) != root))[0]
    p = parent[reached]
    assert (p >= 0).all()
    # levels differ by exactly one along tree edges
    assert (level[p] == level[reached] - 1).all()
    # every tree edge exists
    have = set(zip(u.tolist(), v.tolist()))
    assert all((int(a), int(b)) in have for a, b in zip(p, reached))
    assert (parent[level < 0] == -1).all()


def test_kronecker_tree_invariants():
    n, src, dst = graphgen.edges(10, 16)
    g = oracle.csr(n, src, dst)
    for r in graphgen.pick_roots(n, src, dst, 4):
        level, parent = oracle.bfs(g, int(r))
        _check_tree(g, int(r), level, parent)
        # parents are the smallest previous-level neighbour
        u = np.repeat(np.arange(n), np.diff(g.row_ptr))
        v = g.col
        on = (level[u] >= 0) & (level[v] == level[u] + 1) & (v != r)
        best = np.full(n, np.iinfo(np.int32).max, dtype=np.int64)
        np.minimum.at(best, v[on], u[on])
        reached = (level > 0)
        assert (parent[reached] == best[reached]).all()


@pytest.mark.parametrize("mode", [oracle.PLAIN, oracle.COMPRESS, oracle.COMPRESS_SIEVE])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 7])
def test_algorithms_1_2_3_equal_plain_bfs(mode, p):
    """Lemma 2: sieving and compressing never change t_i, so Alg. 1-3 give the plain BFS."""
    n = 97                                   # not a multiple of p: ragged last range
    src, dst = graphgen.random_edges(n, 160, 5 + p)
    g = oracle.csr(n, src, dst)
    for root in (0, 13, 96):
        lv, pa = oracle.bfs(g, root)
        l2, p2, _ = oracle.dist_bfs(g, p, root, mode=mode)
        assert (lv == l2).all() and (pa == p2).all()
        _, pmax, _ = oracle.dist_bfs(g, p, root, mode=mode, use_max=True)
        assert (pmax == oracle.parents(g, lv, root, use_max=True)).all()


def test_dist_bfs_kronecker_grid_invariance():
    n, src, dst = graphgen.edges(9, 16)
    g = oracle.csr(n, src, dst)
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    lv, pa = oracle.bfs(g, root)
    for p in (2, 4, 8):
        for mode in (oracle.COMPRESS, oracle.COMPRESS_SIEVE):
            for w in (32, 64):
                l2, p2, tr = oracle.dist_bfs(g, p, root, mode=mode, w=w, trace=True)
                assert (lv == l2).all() and (pa == p2).all()
                assert len(tr) == int(lv.max()) + 1


def test_isolated_root_and_directed_input():
    # vertex 5 has only a self-loop: its BFS reaches only itself
    src = np.array([0, 1, 5, 2], dtype=np.int32)
    dst = np.array([1, 2, 5, 3], dtype=np.int32)
    g = oracle.csr(6, src, dst)
    lv, pa = oracle.bfs(g, 5)
    assert lv.tolist() == [-1, -1, -1, -1, -1, 0]
    assert pa.tolist() == [-1, -1, -1, -1, -1, 5]
    # directed (no symmetrisation): from 3 nothing is reachable
    gd = oracle.csr(6, src, dst, symmetrize=False)
    lv, _ = oracle.bfs(gd, 3)
    assert lv.tolist() == [-1, -1, -1, 0, -1, -1]
    lv, pa = oracle.bfs(gd, 0)
    assert lv.tolist() == [0, 1, 2, 3, -1, -1]
    assert pa.tolist() == [0, 0, 1, 2, -1, -1]


def test_self_loops_and_duplicates_counted_twice():
    src = np.array([0, 0, 1, 1], dtype=np.int32)
    dst = np.array([1, 1, 1, 2], dtype=np.int32)
    g = oracle.csr(3, src, dst)
    assert g.degree().tolist() == [2, 5, 1]     # 0-1 twice, 1-1 self-loop twice, 1-2
    assert sorted(g.col[g.row_ptr[1]:g.row_ptr[2]].tolist()) == [0, 0, 1, 1, 2]


def test_bounded_sample_is_a_prefix_of_the_search():
    """oracle_bfs_sample: with an unlimited budget it is oracle_bfs_levels; with a
    small one every level it assigns is the full search's, the assigned levels
    form a prefix (all of levels < L, some of level L), and it scanned at least
    the budget unless the component ended."""
    n, src, dst = graphgen.edges(12, 16)
    g = oracle.csr(n, src, dst)
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    full = oracle.bfs_levels(g, root)
    lv, k = oracle.bfs_sample(g, root, 1 << 62)
    assert (lv == full).all() and k == int(g.degree()[full >= 0].sum())
    for budget in (1, 50, 5000, 40000):
        lv, k = oracle.bfs_sample(g, root, budget)
        got = lv >= 0
        assert (lv[got] == full[got]).all()
        top = lv.max()
        assert ((full < top) & (full >= 0) <= got).all()
        assert k >= min(budget, int(g.degree()[full >= 0].sum()))
