"""Pins of the dynamic cross directory (the reading of Sec. V-B, "update them
synchronously on each side"): V_{i,j}(u) is cleared once every entry of u
into range i leads to a visited vertex.  It must never change the search; it
sends exactly the pairs its definition keeps; it drops work only."""
import numpy as np
import pytest

import graphgen
import oracle


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("p", [2, 3, 5])
def test_dynamic_directory_never_changes_the_search(seed, p):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(p, 60))
    m = int(rng.integers(n, 5 * n))
    sym = seed % 2 == 0
    src, dst = graphgen.random_edges(n, m, seed)
    g = oracle.csr(n, src, dst, symmetrize=sym)
    root = int(rng.integers(0, n))
    lv, pa = oracle.bfs(g, root)
    for use_max in (False, True):
        l2, p2, _ = oracle.dist_bfs(g, p, root, dynamic=True, use_max=use_max)
        assert (l2 == lv).all()
        assert (p2 == oracle.parents(g, lv, root, use_max=use_max)).all()


def _sent_per_level(tr, n, p):
    """Set bits of every traced slice, per level (the (u, i) pairs sent)."""
    out = []
    for level in tr:
        tot = 0
        for s, words in enumerate(level):
            bits = oracle.wah_decode(words, oracle.range_len(n, p, s % p))
            tot += int(bits.sum())
        out.append(tot)
    return out


def test_traced_pairs_equal_the_definition():
    """The pairs the dynamic sieve of the traced search sends (its streams'
    set bits) equal the dynamic pairs counted by definition, level by level;
    the static search's equal the static pairs; dropped pairs drop entries."""
    n, src, dst = graphgen.edges(12, 16)
    g = oracle.csr(n, src, dst)
    p = 4
    for root in graphgen.pick_roots(n, src, dst, 2):
        st = oracle.dynamic_sieve_stats(g, p, int(root))
        _, _, tr_dyn = oracle.dist_bfs(g, p, int(root), trace=True, dynamic=True)
        _, _, tr_sta = oracle.dist_bfs(g, p, int(root), trace=True)
        assert _sent_per_level(tr_dyn, n, p) == [int(x) for x in st[:, 1]]
        assert _sent_per_level(tr_sta, n, p) == [int(x) for x in st[:, 0]]
        assert (st[:, 1] <= st[:, 0]).all() and (st[:, 3] <= st[:, 2]).all()
        assert ((st[:, 0] - st[:, 1] > 0) == (st[:, 3] > 0)).all()
        # the update walks every entry into a reached vertex exactly once
        lv = oracle.bfs_levels(g, int(root))
        assert int(st[:, 4].sum()) == int(np.bincount(g.col, minlength=n)[lv >= 0].sum())


def test_dense_brute_force_on_a_tiny_graph():
    """Dense boolean algebra on a 40-vertex graph: the dynamic pairs of level k
    are the (u, i) with u in F_k and A[range i, u] & not(pi_k) nonzero."""
    rng = np.random.default_rng(7)
    n, p = 40, 3
    src, dst = graphgen.random_edges(n, 90, 3)
    g = oracle.csr(n, src, dst)
    A = np.zeros((n, n), dtype=bool)            # A[v, u]: entry u -> v
    A[dst, src] = True
    A[src, dst] = True
    root = int(rng.integers(0, n))
    lv = oracle.bfs_levels(g, root)
    st = oracle.dynamic_sieve_stats(g, p, root)
    nb = -(-n // p)
    for k in range(st.shape[0]):
        F = lv == k
        pik = (lv >= 0) & (lv <= k)
        sta = dyn = 0
        for i in range(p):
            rows = slice(i * nb, min(n, (i + 1) * nb))
            has = A[rows, :].any(axis=0) & F
            fresh = (A[rows, :] & ~pik[rows, None]).any(axis=0) & F
            sta += int(has.sum())
            dyn += int(fresh.sum())
        assert (st[k, 0], st[k, 1]) == (sta, dyn)
