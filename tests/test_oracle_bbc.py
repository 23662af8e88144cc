"""The oracle's byte-aligned bitmap code (BBC, the other bitmap code Sec. IV names
beside WAH and PLWAH; the paper does not define it, the oracle's header states
the reading): hand-worked streams, round trips over every short bitmap and over
run-structured long ones, closed-form sizes, and rejection of malformed
streams."""
import itertools

import numpy as np
import pytest

import oracle


def _bits(byte_values, nbits=None):
    bits = []
    for b in byte_values:
        bits += [(b >> (7 - i)) & 1 for i in range(8)]
    bits = np.array(bits, np.uint8)
    return bits if nbits is None else bits[:nbits]


# Each stream worked out by hand from the definition:
#  header 1bFFTTTT (short fill, tail), 01bFFPPP (short fill, odd byte),
#  001bTTTT + counter (long fill, tail), 0001bPPP + counter (long fill, odd).
HAND = [
    # three 0x00 gap bytes, then 0x04 = 00000100: odd for b = 0 at position 5
    ([0x00, 0x00, 0x00, 0x04], [0x40 | (3 << 3) | 5]),
    # ten 0x00 (long fill, counter 10), tail 0x12 0x34 (neither byte is odd)
    ([0x00] * 10 + [0x12, 0x34], [0x20 | 2, 10, 0x12, 0x34]),
    # two 0xFF, then 0x7F: odd for b = 1 at position 0
    ([0xFF, 0xFF, 0x7F], [0x40 | (1 << 5) | (2 << 3) | 0]),
    # a lone map byte with five bits set: F = 0, tail of one
    ([0xAB], [0x80 | 1, 0xAB]),
    # seventeen map bytes: a run with 15 of them, then one with F = 0 and 2
    ([0x11] * 17, [0x80 | 15] + [0x11] * 15 + [0x80 | 2, 0x11, 0x11]),
    # two hundred 0x00: long fill, counter 200 = 0x48 + 1 * 128 -> C8 01
    ([0x00] * 200, [0x20, 0xC8, 0x01]),
    # five 0xFF: long fill of ones, empty tail
    ([0xFF] * 5, [0x30, 0x05]),
    # 0x01 alone: F = 0, odd for b = 0 at position 7
    ([0x01], [0x47]),
    # 0xFE alone: not odd for 0, odd for b = 1 at position 7
    ([0xFE], [0x40 | (1 << 5) | 7]),
    # 0x00 then 0xFF: two fills, empty tails
    ([0x00, 0xFF], [0x80 | (1 << 4), 0x80 | (1 << 6) | (1 << 4)]),
    # four 0xFF then 0xBF (odd at 1): long fill with odd byte
    ([0xFF] * 4 + [0xBF], [0x10 | (1 << 3) | 1, 4]),
    # 0x00 0x80 0x80: the tail has two bytes, so no odd-byte run
    ([0x00, 0x80, 0x80], [0x80 | (1 << 4) | 2, 0x80, 0x80]),
    # the 128-bit bitmap of Table 3's WAH example (1 one, 20 zeros, 3 ones, 79
    # zeros, 25 ones; Sec. IV): bytes 80 00 07 00x9 01 FF FF FF ->
    #   80 alone, odd for 0 at 0          -> 01 0 00 000        = 0x40
    #   one 00, tail 07 (three bits set)  -> 1 0 01 0001, 07    = 0x91 0x07
    #   nine 00, then 01 odd for 0 at 7   -> 0001 0 111, 9      = 0x17 0x09
    #   three FF, nothing after           -> 1 1 11 0000        = 0xF0
    # six bytes where WAH needs four 32-bit words
    ([0x80, 0x00, 0x07] + [0x00] * 9 + [0x01, 0xFF, 0xFF, 0xFF], [0x40, 0x91, 0x07, 0x17, 0x09, 0xF0]),
]


@pytest.mark.parametrize("data,stream", HAND)
def test_hand_worked_streams(data, stream):
    bits = _bits(data)
    got = oracle.bbc_encode(bits)
    assert list(got) == stream
    back = oracle.bbc_decode(np.array(stream, np.uint8), len(bits))
    assert back is not None and (back == bits).all()


def test_partial_last_byte_is_padded_with_zeros():
    # 13 bits 1111111111111: bytes FF F8 -> fill of one 0xFF, tail F8
    bits = np.ones(13, np.uint8)
    assert list(oracle.bbc_encode(bits)) == [0x80 | (1 << 6) | (1 << 4) | 1, 0xF8]
    # 9 bits 000000001: bytes 00 80 -> 0x80 is odd for 0 at position 0
    bits = np.zeros(9, np.uint8)
    bits[8] = 1
    assert list(oracle.bbc_encode(bits)) == [0x40 | (1 << 3) | 0]


def test_every_bitmap_up_to_12_bits_round_trips():
    for nbits in range(0, 13):
        for x in range(1 << nbits):
            bits = np.array([(x >> (nbits - 1 - i)) & 1 for i in range(nbits)], np.uint8)
            enc = oracle.bbc_encode(bits)
            dec = oracle.bbc_decode(enc, nbits)
            assert dec is not None and (dec == bits).all(), (nbits, x)


def test_two_byte_sequences_over_every_byte_class():
    values = [0x00, 0xFF, 0x01, 0x80, 0x7F, 0xFE, 0x10, 0xEF, 0x55, 0x33]
    for a, b in itertools.product(values, repeat=2):
        bits = _bits([a, b])
        dec = oracle.bbc_decode(oracle.bbc_encode(bits), 16)
        assert dec is not None and (dec == bits).all()


def test_run_structured_bitmaps_round_trip_and_bound():
    rng = np.random.default_rng(5)
    for trial in range(300):
        parts = []
        for _ in range(rng.integers(1, 12)):
            kind = rng.integers(0, 4)
            ln = int(rng.choice([1, 2, 3, 4, 5, 14, 15, 16, 17, 30, 31, 200, 20000]))
            if kind == 0:
                parts += [0x00] * ln
            elif kind == 1:
                parts += [0xFF] * ln
            elif kind == 2:
                parts += list(rng.integers(1, 255, ln))
            else:
                parts += [int(0x80 >> rng.integers(0, 8)) ^ (0xFF if rng.integers(0, 2) else 0)]
        nbits = 8 * len(parts) - int(rng.integers(0, 8))
        bits = _bits(parts, nbits)
        enc = oracle.bbc_encode(bits)
        nbytes = (nbits + 7) // 8
        assert len(enc) <= nbytes + nbytes // 15 + 11
        dec = oracle.bbc_decode(enc, nbits)
        assert dec is not None and (dec == bits).all(), trial


@pytest.mark.parametrize("nbytes", [1, 2, 3, 4, 127, 128, 16383, 16384, 100000])
def test_all_zero_and_all_one_sizes(nbytes):
    """A bitmap of equal gap bytes is one run: a header, plus its base-128
    counter when the fill is longer than 3 bytes."""
    counter = 0 if nbytes <= 3 else len(np.base_repr(nbytes, 2)) // 7 + (len(np.base_repr(nbytes, 2)) % 7 > 0)
    for v in (0, 1):
        bits = np.full(8 * nbytes, v, np.uint8)
        assert len(oracle.bbc_encode(bits)) == 1 + counter


def test_sparse_bitmap_sizes():
    """Isolated set bits far apart: each costs a long-fill odd-byte run (a
    header and a counter) -- the shape of a sieved frontier slice."""
    nbits = 8 * 1000
    bits = np.zeros(nbits, np.uint8)
    pos = [100, 2000, 5003, 7999]
    bits[pos] = 1
    enc = oracle.bbc_encode(bits)
    dec = oracle.bbc_decode(enc, nbits)
    assert (dec == bits).all()
    # zero bytes before each: 12, 237, 374, 373 -> counters of 1, 2, 2, 2 bytes; no trailing fill
    assert len(enc) == 4 + (1 + 2 + 2 + 2)


def test_malformed_streams_are_rejected():
    bits = _bits([0x00] * 10 + [0x12, 0x34])
    good = oracle.bbc_encode(bits)
    assert oracle.bbc_decode(good, len(bits)) is not None
    assert oracle.bbc_decode(np.array([0x05], np.uint8), 8) is None            # unused header
    assert oracle.bbc_decode(good[:1], len(bits)) is None                      # counter cut
    assert oracle.bbc_decode(good[:3], len(bits)) is None                      # tail cut
    assert oracle.bbc_decode(np.concatenate([good, [0x81, 0x11]]).astype(np.uint8), len(bits)) is None
    assert oracle.bbc_decode(good, len(bits) - 8) is None                      # past nbits
    assert oracle.bbc_decode(good, len(bits) + 8) is None                      # too short
    # padding bits set: 0xF1 in a 4-bit bitmap
    assert oracle.bbc_decode(np.array([0x81, 0xF1], np.uint8), 4) is None
    assert oracle.bbc_decode(np.array([0x20, 0x80, 0x80], np.uint8), 8) is None   # endless counter


def test_non_canonical_streams_decode():
    """Any well-formed stream decodes: a short fill written in the long form,
    a tail that holds an odd byte, a fill of length 0 in the long form."""
    bits = _bits([0x00, 0x00, 0x04])
    assert (oracle.bbc_decode(np.array([0x21, 0x02, 0x04], np.uint8), 24) == bits).all()
    assert (oracle.bbc_decode(np.array([0xA1, 0x04], np.uint8), 24) == bits).all()
    assert (oracle.bbc_decode(np.array([0x20, 0x00, 0xA1, 0x04], np.uint8), 24) == bits).all()
