"""Pins of the oracle's level-adaptive exchange format: a sieved slice goes out
as the smallest of its WAH stream (Sec. IV), its sparse vector of set-bit
offsets (Sec. II, Table 2; Sec. V-A) and its raw bitmap (Alg. 1), the lower
format number on a tie."""
import numpy as np
import pytest

import graphgen
import oracle

WAH, LIST, RAW = oracle.ADAPTIVE_WAH, oracle.ADAPTIVE_LIST, oracle.ADAPTIVE_RAW


def _bitmap(n, ones):
    b = np.zeros(n, np.uint8)
    b[list(ones)] = 1
    return b


# (bits, word width, expected format, expected elements), worked out by hand
HAND = [
    # one vertex of 1000: WAH needs fill, literal, fill, active (16 B); the vector 4 B
    (_bitmap(1000, [500]), 32, LIST, [500]),
    # 62 ones: one 1-fill word of two groups (4 B) against 8 B of raw bitmap
    (np.ones(62, np.uint8), 32, WAH, [0xC0000002]),
    # nothing to send: the empty vector (0 B)
    (np.zeros(1000, np.uint8), 32, LIST, []),
    # a tie of vector and bitmap (8 B each; WAH 12 B): the vector
    (_bitmap(64, [0, 40]), 32, LIST, [0, 40]),
    # a tie of WAH (a 32-group zero fill and the active word) and the vector (8 B each): WAH
    (_bitmap(1000, [993, 999]), 32, WAH, [0x80000020, 0x41]),
    # 64-bit words: one vertex of 1000 costs 32 B of WAH, 4 B of vector
    (_bitmap(1000, [500]), 64, LIST, [500]),
    # every other bit of 93: 3 literal words (12 B) against 3 raw words (12 B): WAH wins the tie
    (np.tile(np.array([1, 0], np.uint8), 47)[:93], 32, WAH, None),
    # every other bit of 96: WAH 3 literals + active (16 B), raw 3 words (12 B)
    (np.tile(np.array([1, 0], np.uint8), 48), 32, RAW, [0x55555555] * 3),
]


@pytest.mark.parametrize("k", range(len(HAND)))
def test_hand_worked_choices(k):
    bits, w, fmt, elems = HAND[k]
    got_fmt, got = oracle.adaptive_encode(bits, w)
    assert got_fmt == fmt
    if elems is not None:
        assert [int(x) for x in got] == elems
    back = oracle.adaptive_decode(got_fmt, got, len(bits), w)
    assert back is not None and (back == bits).all()


@pytest.mark.parametrize("w", [32, 64])
def test_choice_is_the_smallest_and_round_trips(w):
    rng = np.random.default_rng(w)
    seen = set()
    for _ in range(300):
        n = int(rng.integers(0, 3000))
        bits = (rng.random(n) < rng.choice([0.0, 0.001, 0.01, 0.05, 0.3, 0.5, 0.99])).astype(np.uint8)
        fmt, elems = oracle.adaptive_encode(bits, w)
        sizes = [len(oracle.wah_encode(bits, w)) * w // 8, 4 * int(bits.sum()), 4 * ((n + 31) // 32)]
        assert sizes[fmt] == min(sizes) and all(sizes[f] > min(sizes) for f in range(fmt))
        back = oracle.adaptive_decode(fmt, elems, n, w)
        assert back is not None and (back == bits).all()
        seen.add(fmt)
    assert seen == {WAH, LIST, RAW}


@pytest.mark.parametrize("fmt,elems,nbits", [
    (LIST, [5, 3], 10),            # not increasing
    (LIST, [3, 3], 10),            # a repeated offset
    (LIST, [10], 10),              # an offset past the slice
    (RAW, [0], 40),                # too few words
    (RAW, [0, 1 << 8], 40),        # bit 40 set in a 40-bit slice
    (WAH, [0x80000002], 31),       # a WAH stream with groups past the slice
    (3, [], 0),                    # an unknown format
])
def test_malformed_elements_are_rejected(fmt, elems, nbits):
    assert oracle.adaptive_decode(fmt, np.array(elems, np.uint64), nbits) is None


def test_search_levels_choose_by_density():
    """Alg. 3's sieved slices of one Kronecker search: the dense levels go out as
    raw bitmaps (WAH spends 32 bits on 31), the sparse ones as vectors, and the
    adaptive total is below both the all-WAH and the all-raw exchange."""
    n, src, dst = graphgen.edges(16, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    _, _, tr = oracle.dist_bfs(go, p, root, mode=oracle.COMPRESS_SIEVE, trace=True)
    tot = {"wah": 0, "raw": 0, "adaptive": 0}
    per_level = []
    for level in tr:
        counts = [0, 0, 0]
        for s, words in enumerate(level):
            nbits = oracle.range_len(n, p, s % p)
            bits = oracle.wah_decode(np.asarray(words, np.uint64), nbits)
            fmt, elems = oracle.adaptive_encode(bits)
            counts[fmt] += 1
            tot["wah"] += 4 * len(words)
            tot["raw"] += 4 * ((nbits + 31) // 32)
            tot["adaptive"] += 4 * len(elems)
        per_level.append(counts)
    assert tot["adaptive"] < min(tot["wah"], tot["raw"])
    assert any(c[RAW] == sum(c) for c in per_level)          # a dense level: every slice raw
    assert per_level[1][LIST] == sum(per_level[1])           # the root's neighbours: every slice a vector


@pytest.mark.parametrize("mode,w", [(oracle.COMPRESS_SIEVE, 32), (oracle.COMPRESS, 32), (oracle.COMPRESS_SIEVE, 64)])
def test_adaptive_trace_carries_the_same_slices(mode, w):
    """Every slot of the adaptive exchange decodes to the slice the WAH exchange
    carries: the format changes the bytes, never the frontier."""
    n, src, dst = graphgen.edges(12, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    _, _, tr = oracle.dist_bfs(go, p, root, mode=mode, w=w, trace=True)
    ad = oracle.adaptive_trace(tr, n, p, mode=mode, w=w)
    assert len(ad) == len(tr)
    for level, arow in zip(tr, ad):
        assert len(level) == len(arow) == (p * p if mode == oracle.COMPRESS_SIEVE else p)
        for s, (words, (fmt, elems)) in enumerate(zip(level, arow)):
            j = s % p if mode == oracle.COMPRESS_SIEVE else s
            nbits = oracle.range_len(n, p, j)
            want = oracle.wah_decode(np.asarray(words, np.uint64), nbits, w)
            got = oracle.adaptive_decode(fmt, elems, nbits, w)
            assert got is not None and (got == want).all()
            if fmt == WAH:
                assert (np.asarray(elems, np.uint64) == np.asarray(words, np.uint64)).all()
