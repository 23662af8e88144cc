"""bfs_wah_decode_static: the decoder for callers that cannot allocate device memory.

Some callers cannot let a library call allocate: a serving process that has
handed the whole HBM budget to resident graphs, or a latency-critical thread
that must not wait on cudaFree (it synchronises the device).  The static
variant keeps its scratch in one array of static device memory.  These tests
call it through the C ABI and check that it gives exactly the output of the
allocating bfs_wah_decode, on two calls in a row (which share that array), and
that it rejects sizes past its limit.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

LIMIT_BITS = 1 << 23


def _lib():
    from paper_1208_5542_gb300 import build, native
    build.build()
    return native


def _decode(native, fn_name, words, nbits, w):
    out = torch.full((max(1, (nbits + 31) // 32),), -1, dtype=torch.int32, device="cuda")   # stale contents
    stream = torch.cuda.current_stream().cuda_stream
    fn = getattr(native.lib(), fn_name)
    rc = fn(ctypes.c_void_p(words.data_ptr()) if words.numel() else None, words.numel(), nbits, w,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    return rc, out[: (nbits + 31) // 32].cpu().numpy().view(np.uint32)


def _stream(bits, w):
    words = oracle.wah_encode(bits, w)
    arr = words.astype(np.uint32).view(np.int32) if w == 32 else words.view(np.int64)
    return torch.from_numpy(arr.copy()).cuda()


def test_static_decode_matches_allocating_decode_twice():
    native = _lib()
    rng = np.random.default_rng(2024)
    for call in range(2):
        for w in (32, 64):
            for nbits in (LIMIT_BITS - 5 - call, 1000 + 31 * call, 0):
                bits = (rng.random(nbits) < (0.01 if call == 0 else 0.6)).astype(np.uint8)
                words = _stream(bits, w)
                rc_a, ref = _decode(native, "bfs_wah_decode", words, nbits, w)
                rc_b, got = _decode(native, "bfs_wah_decode_static", words, nbits, w)
                assert rc_a == 0 and rc_b == 0
                assert (got == ref).all()
                assert (got == oracle.pack_bits(bits)).all()


def test_static_decode_limits_and_errors():
    native = _lib()
    bits = np.zeros(LIMIT_BITS + 1, np.uint8)
    bits[[3, LIMIT_BITS]] = 1
    rc, _ = _decode(native, "bfs_wah_decode_static", _stream(bits, 32), LIMIT_BITS + 1, 32)
    assert native.STATUS[rc] == "BFS_ERR_INVALID_ARG"
    bad = torch.from_numpy(np.array([0x80000005], np.uint32).view(np.int32)).cuda()   # fill past the end
    rc, _ = _decode(native, "bfs_wah_decode_static", bad, 31 * 4, 32)
    assert native.STATUS[rc] == "BFS_ERR_CORRUPT"
    # the error word left by the failed call is cleared by the next one
    good = np.zeros(100, np.uint8)
    good[[0, 50, 99]] = 1
    rc, got = _decode(native, "bfs_wah_decode_static", _stream(good, 32), 100, 32)
    assert rc == 0 and (got == oracle.pack_bits(good)).all()
