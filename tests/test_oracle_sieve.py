"""Pins of the oracle directory and sieve: Eq. 4 by dense brute force, Lemma 1 and 2."""
import numpy as np
import pytest

import graphgen
import oracle


def _dense(n, src, dst):
    A = np.zeros((n, n), dtype=bool)          # A[u, v]: entry u -> v
    A[src, dst] = True
    A[dst, src] = True
    return A


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_directory_matches_dense_column_test(p):
    n = 61
    src, dst = graphgen.random_edges(n, 70, p)
    g = oracle.csr(n, src, dst)
    A = _dense(n, src, dst)
    D = oracle.cross_directory(g, p)
    for i in range(p):
        ib, il = oracle.range_begin(n, p, i), oracle.range_len(n, p, i)
        for j in range(p):
            jb, jl = oracle.range_begin(n, p, j), oracle.range_len(n, p, j)
            # block A_{i,j}: rows = destinations in range i, columns = sources in range j
            blk = A[jb:jb + jl, ib:ib + il].T
            expect = blk.any(axis=0).astype(np.uint8)
            assert (oracle.directory(g, p, i, j) == expect).all()
            assert (D[i, jb:jb + jl] == expect).all()


@pytest.mark.parametrize("seed", range(6))
def test_lemma_1_and_2_sieving_keeps_t(seed):
    """A_{i,j} (x) f_j = A_{i,j} (x) (f_j (.) V_{i,j}) for every block and random f."""
    rng = np.random.default_rng(seed)
    n, p = 80, 4
    src, dst = graphgen.random_edges(n, 90, 100 + seed)
    g = oracle.csr(n, src, dst)
    A = _dense(n, src, dst).astype(np.int64)
    D = oracle.cross_directory(g, p)
    for density in (0.05, 0.3, 0.9):
        f = (rng.random(n) < density).astype(np.int64)
        t_full = np.zeros(n, np.int64)
        t_sieved = np.zeros(n, np.int64)
        for i in range(p):
            ib, il = oracle.range_begin(n, p, i), oracle.range_len(n, p, i)
            for j in range(p):
                jb, jl = oracle.range_begin(n, p, j), oracle.range_len(n, p, j)
                blk = A[jb:jb + jl, ib:ib + il].T
                fj = f[jb:jb + jl]
                sieved = fj * D[i, jb:jb + jl]
                a = (blk @ fj) > 0
                b = (blk @ sieved) > 0
                assert (a == b).all()                     # Lemma 1, per block
                t_full[ib:ib + il] |= a
                t_sieved[ib:ib + il] |= b
        assert (t_full == t_sieved).all()                 # Lemma 2
        assert (t_full == ((A.T @ f) > 0)).all()


def test_exchange_streams_decode_to_sieved_slices():
    n, src, dst = graphgen.edges(11, 16)
    g = oracle.csr(n, src, dst)
    p = 4
    D = oracle.cross_directory(g, p)
    rng = np.random.default_rng(3)
    f = (rng.random(n) < 0.02).astype(np.uint8)
    streams, counts = oracle.level_exchange(g, p, f, oracle.COMPRESS_SIEVE, D=D)
    total = 0
    for i in range(p):
        for j in range(p):
            jb, jl = oracle.range_begin(n, p, j), oracle.range_len(n, p, j)
            dec = oracle.wah_decode(streams[i * p + j], jl)
            assert (dec == (f[jb:jb + jl] & D[i, jb:jb + jl])).all()
            assert counts[i * p + j] == int(dec.sum())
            total += int(dec.sum())
    # the sieve only removes: at most p copies of each frontier vertex survive
    assert total <= p * int(f.sum())
