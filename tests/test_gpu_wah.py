"""Bit-exact parity of the CUDA WAH codec (bfs_wah_encode / bfs_wah_decode) with the oracle codec."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1208_5542_gb300 import bfs, build
    build.build()
    return bfs


def _bitmap(rng, nbits, kind):
    if kind == "random":
        dens = rng.choice([0.0005, 0.02, 0.3, 0.7, 0.995])
        return (rng.random(nbits) < dens).astype(np.uint8)
    if kind == "zeros":
        return np.zeros(nbits, np.uint8)
    if kind == "ones":
        return np.ones(nbits, np.uint8)
    if kind == "runs":
        out = np.zeros(nbits, np.uint8)
        pos, val = 0, int(rng.integers(0, 2))
        while pos < nbits:
            ln = int(rng.choice([1, 30, 31, 32, 62, 63, 64, 93, 500, 40000]))
            out[pos:pos + ln] = val
            pos += ln
            val ^= 1
        return out
    raise ValueError(kind)


def _to_words(bits):
    return torch.from_numpy(oracle.pack_bits(bits).view(np.int32).copy()).cuda()


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("kind", ["random", "zeros", "ones", "runs"])
def test_encode_matches_oracle(w, kind):
    bfs = _lib()
    rng = np.random.default_rng(hash((w, kind)) & 0xffff)
    g = w - 1
    # every residue mod g, lengths from one word to several encoder tiles (1024 groups)
    sizes = [0, 1, g - 1, g, g + 1, 5 * g + 7] + [g * int(rng.integers(1000, 3500)) + r for r in range(0, g, 5)]
    for nbits in sizes:
        bits = _bitmap(rng, nbits, kind)
        want = oracle.wah_encode(bits, w)
        got = bfs.wah_encode(_to_words(bits), nbits, w).cpu().numpy()
        got = got.view(np.uint32 if w == 32 else np.uint64).astype(np.uint64)
        assert len(got) == len(want) and (got == want).all(), (nbits, kind)
        arr = got.astype(np.uint32).view(np.int32) if w == 32 else got.view(np.int64)
        back = bfs.wah_decode(torch.from_numpy(arr.copy()).cuda(), nbits, w).cpu().numpy()
        assert (oracle.unpack_bits(back.view(np.uint32), nbits) == bits).all(), (nbits, kind)


def test_decode_rejects_malformed_streams():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    bits = np.zeros(31 * 4 + 3, np.uint8)
    bits[[0, 40, 125]] = 1
    good = oracle.wah_encode(bits, 32).astype(np.uint32)
    t = lambda a: torch.from_numpy(np.asarray(a, np.uint32).view(np.int32).copy()).cuda()  # noqa: E731
    bfs.wah_decode(t(good), len(bits))
    for bad, nb in ((good[:-1], len(bits)), (np.append(good, 0), len(bits)), ([0x80000000, 0], 31),
                    ([0x80000005], 31 * 4), ([0x80000001, 0b1000], 34)):
        with pytest.raises(BfsError, match="CORRUPT"):
            bfs.wah_decode(t(bad), nb)
    # the oracle rejects the same streams
    for bad, nb in ((good[:-1], len(bits)), ([0x80000001, 0b1000], 34)):
        assert oracle.wah_decode(np.asarray(bad, np.uint64), nb) is None


def test_scatter_read_measurement():
    """The diagnostic entry point returns a plausible positive rate and rejects bad sizes."""
    from paper_1208_5542_gb300 import bfs, build
    from paper_1208_5542_gb300.native import BfsError
    build.build()
    r = bfs.measure_scatter_reads(512 << 10, 256)
    assert 1e9 < r < 1e14
    with pytest.raises(BfsError):
        bfs.measure_scatter_reads(100, 256)
