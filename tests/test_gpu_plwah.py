"""PLWAH codec on the GPU (bfs_plwah_encode / bfs_plwah_decode) against the oracle:
identical words, round trips, and rejection of malformed streams."""
import numpy as np
import pytest
import torch

import oracle
from tests.test_oracle_plwah import _group_with, _random_bitmap

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1208_5542_gb300 import bfs
    from paper_1208_5542_gb300 import build
    build.build()
    return bfs


def _dev_words(bits):
    w = oracle.pack_bits(bits)
    return torch.from_numpy(w.view(np.int32).copy()).cuda() if len(w) else torch.zeros(1, dtype=torch.int32,
                                                                                       device="cuda")


def _check(bfs, bits):
    n = len(bits)
    got = bfs.plwah_encode(_dev_words(bits), n)
    want = oracle.plwah_encode(bits)
    g = got.cpu().numpy().view(np.uint32)
    assert len(g) == len(want) and (g == want).all(), (n, [hex(int(x)) for x in g[:8]], [hex(int(x)) for x in want[:8]])
    back = bfs.plwah_decode(got, n)
    assert (oracle.unpack_bits(back.cpu().numpy().view(np.uint32), n) == bits).all()


def test_random_bitmaps_match_the_oracle():
    bfs = _lib()
    rng = np.random.default_rng(21)
    for _ in range(150):
        _check(bfs, _random_bitmap(rng, int(rng.integers(1, 60))))
    for n in (0, 1, 30, 31, 32, 62, 63, 64, 93, 1000):
        _check(bfs, (rng.random(n) < 0.5).astype(np.uint8))


def test_streams_of_several_tiles():
    """Sparse bitmaps long enough for thousands of words (the transcoding CTA
    walks the stream in tiles of 1024 words): isolated bits after zero runs
    (folded), pairs of bits (literals), dense stretches and 1-fills."""
    bfs = _lib()
    rng = np.random.default_rng(4)
    n = 400_000
    bits = np.zeros(n, np.uint8)
    bits[rng.choice(n, 6000, replace=False)] = 1
    bits[100_000:130_000] = 1
    bits[200_000:220_000] = rng.random(20_000) < 0.5
    _check(bfs, bits)
    ones = np.ones(n + 17, np.uint8)
    ones[rng.choice(n, 3000, replace=False)] = 0
    _check(bfs, ones)


@pytest.mark.parametrize("words,nbits", [
    ([0x80000000], 31),                      # a fill of length 0
    ([0x8A000001], 31),                      # the position group lies past nbits
    ([0x80000002], 31),                      # groups past nbits
    ([0x80000001, 0x1], 31),                 # a trailing word
    ([0x80000001], 35),                      # the active word is missing
    ([0x80000001, 0x10], 35),                # the active word holds more than 4 bits
])
def test_malformed_streams_raise(words, nbits):
    from paper_1208_5542_gb300 import native
    bfs = _lib()
    t = torch.from_numpy(np.array(words, np.uint32).view(np.int32)).cuda()
    with pytest.raises(native.BfsError, match="CORRUPT"):
        bfs.plwah_decode(t, nbits)


def test_size_limit_and_capacity():
    from paper_1208_5542_gb300 import native
    bfs = _lib()
    lib = native.lib()
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    limit = 31 * ((1 << 25) - 1)
    assert lib.bfs_plwah_encode(buf.data_ptr(), limit + 1, buf.data_ptr(), 1 << 30, cnt.data_ptr(), None) == 1
    assert lib.bfs_plwah_decode(buf.data_ptr(), 1, limit + 1, buf.data_ptr(), None) == 1
    assert lib.bfs_plwah_encode(buf.data_ptr(), 62, buf.data_ptr(), 2, cnt.data_ptr(), None) == 1   # bound is 3
    bits = np.concatenate([np.zeros(31, np.uint8), _group_with(0, [5])])
    got = bfs.plwah_encode(_dev_words(bits), 62)
    assert got.cpu().numpy().view(np.uint32).tolist() == [0x8A000001]
    torch.cuda.synchronize()
