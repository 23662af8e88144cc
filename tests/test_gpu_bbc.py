"""The GPU byte-aligned bitmap code (BBC, the other bitmap code Sec. IV names):
every stream byte for byte the oracle's, every decode the original bitmap, on
hand-worked cases, run-structured and random bitmaps of every length class, the
sieved slices of a real search, and large slices; malformed streams are
reported, not decoded."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
from tests.test_gpu_bfs import _lib, _run, _unpack_trace
from tests.test_oracle_bbc import HAND, _bits

pytestmark = pytest.mark.gpu


def _words(bits):
    """0/1 array -> int32 CUDA words (bit b = bit b % 32 of word b // 32)."""
    nbits = len(bits)
    padded = np.zeros(((nbits + 31) // 32) * 32, np.uint8)
    padded[:nbits] = bits
    w = np.packbits(padded.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).ravel()
    return torch.from_numpy(w.view(np.int32).copy()).cuda()


def _unwords(t, nbits):
    w = t.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(w.astype(">u4").view(np.uint8).reshape(-1, 4), axis=1).reshape(-1, 32)[:, ::-1].ravel()
    return bits[:nbits]


def _roundtrip(bfs, bits):
    nbits = len(bits)
    want = oracle.bbc_encode(bits)
    got = bfs.bbc_encode(_words(bits), nbits).cpu().numpy()
    assert len(got) == len(want) and (got == want).all(), (nbits, got[:12], want[:12])
    back = _unwords(bfs.bbc_decode(torch.from_numpy(want).cuda(), nbits), nbits)
    assert (back == bits).all()


@pytest.mark.parametrize("data,stream", HAND)
def test_hand_worked_streams(data, stream):
    bfs = _lib()
    bits = _bits(data)
    got = bfs.bbc_encode(_words(bits), len(bits)).cpu().numpy()
    assert list(got) == stream
    _roundtrip(bfs, bits)


def test_every_length_class_and_structure():
    bfs = _lib()
    rng = np.random.default_rng(9)
    for nbits in [1, 7, 8, 9, 31, 32, 33, 63, 64, 65, 120, 121, 4095, 4096, 4097, 40000, 1 << 17]:
        for density in (0.0, 1.0, 0.001, 0.02, 0.5):
            _roundtrip(bfs, (rng.random(nbits) < density).astype(np.uint8))
    for trial in range(40):                                     # runs of gap bytes, map bytes and odd bytes
        parts = []
        for _ in range(rng.integers(1, 30)):
            kind = rng.integers(0, 4)
            ln = int(rng.choice([1, 2, 3, 4, 5, 14, 15, 16, 17, 30, 31, 127, 128, 129, 5000, 70000]))
            if kind == 0:
                parts += [0x00] * ln
            elif kind == 1:
                parts += [0xFF] * ln
            elif kind == 2:
                parts += list(rng.integers(1, 255, ln))
            else:
                parts += [int(0x80 >> rng.integers(0, 8)) ^ (0xFF if rng.integers(0, 2) else 0)]
        nbits = 8 * len(parts) - int(rng.integers(0, 8))
        _roundtrip(bfs, _bits(parts, nbits))


def test_sieved_slices_of_a_search():
    """Every slice the DIR-WAH exchange of a Kronecker search carries (decoded
    from the oracle's WAH streams), sparse and dense levels, ragged ranges."""
    bfs = _lib()
    n, src, dst = graphgen.edges(16, 16)
    go = oracle.csr(n, src, dst)
    p = 5
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    _, _, tr = oracle.dist_bfs(go, p, r, mode=oracle.COMPRESS_SIEVE, trace=True)
    count = 0
    for level in tr:
        for s, words in enumerate(level):
            nbits = oracle.range_len(n, p, s % p)
            bits = oracle.wah_decode(np.asarray(words, np.uint64), nbits, 32)
            _roundtrip(bfs, bits)
            count += 1
    assert count >= 5 * p * p


def test_large_slices():
    """Slices of the bench's range size (4M bits): empty, full, sparse, dense."""
    bfs = _lib()
    rng = np.random.default_rng(3)
    nbits = 1 << 22
    for density in (0.0, 1.0, 1e-5, 0.01, 0.3):
        _roundtrip(bfs, (rng.random(nbits) < density).astype(np.uint8))


def test_malformed_streams_are_reported():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    bits = _bits([0x00] * 10 + [0x12, 0x34])
    good = oracle.bbc_encode(bits)
    bad = [
        (np.array([0x05], np.uint8), 8),                         # unused header
        (good[:1], len(bits)),                                   # counter cut
        (good[:3], len(bits)),                                   # tail cut
        (np.concatenate([good, [0x81, 0x11]]).astype(np.uint8), len(bits)),   # bytes past nbits
        (good, len(bits) + 8),                                   # too few bytes
        (np.array([0x81, 0xF1], np.uint8), 4),                   # padding bits set
        (np.array([0x20, 0x80, 0x80], np.uint8), 8),             # endless counter
    ]
    for data, nbits in bad:
        assert oracle.bbc_decode(data, nbits) is None
        with pytest.raises(BfsError, match="CORRUPT"):
            bfs.bbc_decode(torch.from_numpy(np.ascontiguousarray(data)).cuda(), nbits)
    # a stream longer than one decoding chunk whose last record is cut
    long_bits = (np.random.default_rng(1).random(80000) < 0.5).astype(np.uint8)
    s = oracle.bbc_encode(long_bits)
    with pytest.raises(BfsError, match="CORRUPT"):
        bfs.bbc_decode(torch.from_numpy(s[:-1].copy()).cuda(), len(long_bits))
    _roundtrip(bfs, long_bits)


def test_non_canonical_streams_decode():
    bfs = _lib()
    bits = _bits([0x00, 0x00, 0x04])
    for s in ([0x21, 0x02, 0x04], [0xA1, 0x04], [0x20, 0x00, 0xA1, 0x04]):
        out = _unwords(bfs.bbc_decode(torch.tensor(s, dtype=torch.uint8).cuda(), 24), 24)
        assert (out == bits).all()
