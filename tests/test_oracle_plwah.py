"""Pins of the oracle's PLWAH codec (the position-list WAH that Sec. IV names
beside WAH as an alternative bitmap code).

PLWAH is WAH with one change: the literal group right after a fill run, when it
differs from the run's value in a single bit, is not written -- the run's fill
word carries that bit's position (5 bits) and its run length shrinks to 25
bits.  The pins: words worked out by hand from that definition, the same
streams obtained from the oracle's WAH code (itself pinned to Table 3) by
folding those literals into their fills, round trips, and rejection of
malformed streams.
"""
import numpy as np
import pytest

import graphgen
import oracle


def _bits(*runs):
    """Concatenate (value, length) runs into a 0/1 byte array."""
    return np.concatenate([np.full(n, v, np.uint8) for v, n in runs]) if runs else np.zeros(0, np.uint8)


def _group_with(value, odd_places):
    """One 31-bit group of `value` with the given places (1 = first bit) flipped."""
    g = np.full(31, value, np.uint8)
    for q in odd_places:
        g[q - 1] ^= 1
    return g


# words worked out by hand from the definition
HAND = [
    # a zero run of one group, then a group whose 5th bit is set: one word,
    # 1 (fill) 0 (value) 00101 (position 5) 0...01 (one group)
    (np.concatenate([_bits((0, 31)), _group_with(0, [5])]), [0x8A000001]),
    # a one run, then a group of ones but its first bit: 1 1 00001 0...01
    (np.concatenate([_bits((1, 31)), _group_with(1, [1])]), [0xC2000001]),
    # the run's last bit place (31) and a run of three groups
    (np.concatenate([_bits((0, 93)), _group_with(0, [31])]), [0x80000003 | (31 << 25)]),
    # the folded group ends the run: the zeros after it start a new fill word
    (np.concatenate([_bits((0, 31)), _group_with(0, [2]), _bits((0, 62))]), [0x84000001, 0x80000002]),
    # two odd bits: a literal word (payload bits 30-2 and 30-9: first bit most significant)
    (np.concatenate([_bits((0, 31)), _group_with(0, [3, 10])]), [0x80000001, (1 << 28) | (1 << 21)]),
    # a one-bit literal with no run before it stays a literal
    (_group_with(0, [1]), [0x40000000]),
    # Table 3's 128-bit example has no foldable literal: the WAH words unchanged
    (_bits((1, 1), (0, 20), (1, 3), (0, 79), (1, 25)), [0x40000380, 0x80000002, 0x001FFFFF, 0x0000000F]),
    # an active word after a folded group: 4 trailing bits 1011
    (np.concatenate([_bits((0, 31)), _group_with(0, [7]), np.array([1, 0, 1, 1], np.uint8)]),
     [0x8E000001, 0xB]),
]


@pytest.mark.parametrize("k", range(len(HAND)))
def test_hand_worked_words(k):
    bits, want = HAND[k]
    got = oracle.plwah_encode(bits)
    assert [int(x) for x in got] == want, [hex(int(x)) for x in got]
    back = oracle.plwah_decode(got, len(bits))
    assert back is not None and (back == bits).all()


def _fold_wah(words, nbits):
    """PLWAH from the oracle's WAH words: every literal that follows a fill word
    and differs from its value in one bit is folded into it (runs < 2^25)."""
    r = nbits % 31
    out = []
    last_fill = None
    for k, w in enumerate(int(x) for x in words):
        active = r > 0 and k == len(words) - 1
        if w >> 31 and not active:
            assert (w & 0x3FFFFFFF) < (1 << 25)
            out.append(0x80000000 | (w & 0x40000000) | (w & 0x3FFFFFFF))
            last_fill = (w >> 30) & 1
            continue
        if last_fill is not None and not active:
            diff = w ^ (0x7FFFFFFF if last_fill else 0)
            if diff and not diff & (diff - 1):
                q = 31 - diff.bit_length() + 1          # first bit of the group = place 1
                out[-1] |= q << 25
                last_fill = None
                continue
        out.append(w)
        last_fill = None
    return out


def _random_bitmap(rng, ngroups):
    """Runs of fills, one-bit-off groups, sparse and dense literals, and a tail."""
    parts = []
    for _ in range(ngroups):
        kind = rng.integers(0, 6)
        if kind == 0:
            parts.append(np.full(31 * int(rng.integers(1, 5)), int(rng.integers(0, 2)), np.uint8))
        elif kind == 1:
            parts.append(_group_with(int(rng.integers(0, 2)), [int(rng.integers(1, 32))]))
        elif kind == 2:
            parts.append(_group_with(int(rng.integers(0, 2)), list(rng.choice(np.arange(1, 32), 2, replace=False))))
        else:
            parts.append((rng.random(31) < rng.choice([0.03, 0.5, 0.97])).astype(np.uint8))
    parts.append((rng.random(int(rng.integers(0, 31))) < 0.5).astype(np.uint8))
    return np.concatenate(parts)


def test_plwah_is_wah_with_the_odd_literals_folded():
    rng = np.random.default_rng(5)
    folded_total = 0
    for _ in range(400):
        bits = _random_bitmap(rng, int(rng.integers(1, 40)))
        wah = oracle.wah_encode(bits)
        want = _fold_wah(wah, len(bits))
        got = oracle.plwah_encode(bits)
        assert [int(x) for x in got] == want
        assert len(got) <= len(wah)
        folded_total += len(wah) - len(got)
        back = oracle.plwah_decode(got, len(bits))
        assert back is not None and (back == bits).all()
    assert folded_total > 100


def test_long_runs_split_at_the_25_bit_count():
    """A run of 2^25 + 2 zero groups, then a one-bit group: the run is split
    greedily (a full word, then 3 groups) and the last word takes the position."""
    n = 31 * ((1 << 25) + 2) + 31
    bits = np.zeros(n, np.uint8)
    bits[n - 31 + 9] = 1
    got = [int(x) for x in oracle.plwah_encode(bits)]
    assert got == [0x80000000 | ((1 << 25) - 1), 0x80000000 | (10 << 25) | 3]
    back = oracle.plwah_decode(np.array(got, np.uint32), n)
    assert back is not None and (back == bits).all()


@pytest.mark.parametrize("words,nbits", [
    ([0x80000000], 31),                      # a fill of length 0
    ([0x8A000001], 31),                      # the position group lies past nbits
    ([0x80000002], 31),                      # groups past nbits
    ([0x80000001, 0x1], 31),                 # a trailing word
    ([0x80000001], 35),                      # the active word is missing
    ([0x80000001, 0x10], 35),                # the active word holds more than 4 bits
])
def test_malformed_streams_are_rejected(words, nbits):
    assert oracle.plwah_decode(np.array(words, np.uint32), nbits) is None


def test_search_streams_only_shrink():
    """The exchanged streams of Alg. 3 on a Kronecker graph: PLWAH never writes
    more words than WAH, and the sparse levels (mostly fill + one-bit literal
    pairs) shrink by about half."""
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    p = 4
    root = int(graphgen.pick_roots(n, src, dst, 1)[0])
    _, _, tr = oracle.dist_bfs(go, p, root, mode=oracle.COMPRESS_SIEVE, trace=True)
    best = 1.0
    for level in tr:
        w = pl = 0
        for s, words in enumerate(level):
            j = s % p
            nbits = oracle.range_len(n, p, j)
            bits = oracle.wah_decode(np.asarray(words, np.uint64), nbits)
            got = oracle.plwah_encode(bits)
            assert len(got) <= len(words)
            w += len(words)
            pl += len(got)
        if w >= 64:
            best = min(best, pl / w)
    assert best < 0.75
