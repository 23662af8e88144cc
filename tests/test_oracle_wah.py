"""Pins of the oracle WAH codec (Sec. IV, Table 3) beyond the printed examples.

The printed examples fix the bit order, the literal/fill/active layout and the
run merging; these tests fix the rest: round trip, the canonical form (which
makes the encoding of a bitmap unique), the size bound, length splitting and
malformed-stream rejection.
"""
import numpy as np
import pytest

import oracle


def _groups(bits, g):
    full = len(bits) // g
    gr = bits[: full * g].reshape(full, g) if full else np.zeros((0, g), np.uint8)
    return gr, len(bits) % g


def _expected_count(bits, w, fill_bit=True):
    """Closed form for the word count: literals + maximal fill runs (split at the
    largest count) + the active word."""
    g = w - 1
    gr, r = _groups(bits, g)
    s = gr.sum(axis=1) if len(gr) else np.zeros(0)
    kind = np.where(s == 0, 0, np.where((s == g) & fill_bit, 1, 2))
    maxc = (1 << (w - 2 if fill_bit else w - 1)) - 1
    words, k = 0, 0
    while k < len(kind):
        if kind[k] == 2:
            words, k = words + 1, k + 1
            continue
        e = k
        while e < len(kind) and kind[e] == kind[k]:
            e += 1
        words += -(-(e - k) // maxc)
        k = e
    return words + (1 if r else 0)


def _check_canonical(words, bits, w, fill_bit=True):
    g = w - 1
    top = 1 << (w - 1)
    maxc = (1 << (w - 2 if fill_bit else w - 1)) - 1
    cmask = maxc
    full = len(bits) // g
    body = words[: len(words) - (1 if len(bits) % g else 0)]
    prev = None
    for x in map(int, body):
        if x & top:
            val = (x >> (w - 2)) & 1 if fill_bit else 0
            cnt = x & cmask
            assert cnt >= 1
            if prev is not None and prev[0] == "fill" and prev[1] == val:
                assert prev[2] == maxc           # only a full fill may be followed by the same fill
            prev = ("fill", val, cnt)
        else:
            assert x != 0
            if fill_bit:
                assert x != (1 << g) - 1
            prev = ("lit",)
    assert len(words) <= full + 1


@pytest.mark.parametrize("w", [32, 64])
def test_round_trip_random_densities_and_lengths(w):
    rng = np.random.default_rng(w)
    g = w - 1
    for r in range(g):                       # every nbits mod g
        for density in (0.0, 0.001, 0.05, 0.5, 0.97, 1.0):
            nbits = g * int(rng.integers(0, 9)) + r
            bits = (rng.random(nbits) < density).astype(np.uint8)
            words = oracle.wah_encode(bits, w)
            assert len(words) == _expected_count(bits, w)
            assert len(words) <= nbits // g + 1
            _check_canonical(words, bits, w)
            back = oracle.wah_decode(words, nbits, w)
            assert back is not None and (back == bits).all()


@pytest.mark.parametrize("run", [30, 31, 32, 62, 63, 64, 93, 1000])
@pytest.mark.parametrize("value", [0, 1])
def test_runs_around_group_boundaries(run, value):
    w = 32
    bits = np.concatenate([np.full(5, 1 - value), np.full(run, value), np.full(40, 1 - value)]).astype(np.uint8)
    words = oracle.wah_encode(bits, w)
    assert len(words) == _expected_count(bits, w)
    _check_canonical(words, bits, w)
    assert (oracle.wah_decode(words, len(bits), w) == bits).all()


def test_structured_bitmaps():
    w = 32
    for bits in (np.zeros(31 * 100, np.uint8), np.ones(31 * 100, np.uint8), np.zeros(0, np.uint8),
                 np.tile([1, 0], 500).astype(np.uint8), np.ones(1, np.uint8)):
        words = oracle.wah_encode(bits, w)
        assert (oracle.wah_decode(words, len(bits), w) == bits).all()
    assert [int(x) for x in oracle.wah_encode(np.zeros(31 * 100, np.uint8))] == [0x80000000 | 100]
    assert [int(x) for x in oracle.wah_encode(np.ones(31 * 100, np.uint8))] == [0xC0000000 | 100]
    assert [int(x) for x in oracle.wah_encode(np.zeros(0, np.uint8))] == []
    assert [int(x) for x in oracle.wah_encode(np.ones(5, np.uint8))] == [0b11111]
    # one group of alternating bits, first bit most significant
    assert [int(x) for x in oracle.wah_encode(np.tile([1, 0], 16)[:31].astype(np.uint8))] == [0x55555555]


def test_fill_length_splits_at_count_field_limit():
    # 4-bit words without a value bit: count field of 3 bits, at most 7 groups
    words = oracle.wah_encode(np.zeros(3 * 20, np.uint8), w=4, fill_bit=False)
    assert [int(x) for x in words] == [0b1111, 0b1111, 0b1110]
    # 8-bit words with a value bit: count field of 6 bits, at most 63 groups
    words = oracle.wah_encode(np.ones(7 * 100, np.uint8), w=8, fill_bit=True)
    assert [int(x) for x in words] == [0xC0 | 63, 0xC0 | 37]
    # without a value bit, an all-one group is a literal
    assert [int(x) for x in oracle.wah_encode(np.ones(3, np.uint8), w=4, fill_bit=False)] == [0b0111]


def test_exhaustive_small_bitmaps_w4():
    """Every bitmap of up to 10 bits round-trips and is canonical (4-bit words, value bit)."""
    for nbits in range(0, 11):
        for x in range(1 << nbits):
            bits = np.array([(x >> (nbits - 1 - b)) & 1 for b in range(nbits)], dtype=np.uint8)
            for fb in (True, False):
                words = oracle.wah_encode(bits, 4, fill_bit=fb)
                assert len(words) == _expected_count(bits, 4, fb)
                assert (oracle.wah_decode(words, nbits, 4, fill_bit=fb) == bits).all()


def test_decoder_rejects_malformed_streams():
    w = 32
    bits = np.zeros(31 * 4 + 3, np.uint8)
    bits[[0, 40, 125]] = 1
    good = oracle.wah_encode(bits, w)
    assert oracle.wah_decode(good, len(bits), w) is not None
    assert oracle.wah_decode(good[:-1], len(bits), w) is None                      # truncated
    assert oracle.wah_decode(np.append(good, 0), len(bits), w) is None              # trailing word
    assert oracle.wah_decode(np.array([0x80000000, 0], np.uint64), 31, w) is None   # zero-length fill
    assert oracle.wah_decode(np.array([0x80000005], np.uint64), 31 * 4, w) is None  # fill overruns
    assert oracle.wah_decode(np.array([0x80000001, 0b1000], np.uint64), 34, w) is None  # active too wide
    assert oracle.wah_decode(np.array([0x1_0000_0000], np.uint64), 31, w) is None   # wider than w
