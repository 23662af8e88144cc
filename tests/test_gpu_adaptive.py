"""The level-adaptive exchange format on the GPU: every exchanged slice goes as the
smallest of its WAH stream, sparse vector and raw bitmap (Sec. II, Table 2; Sec.
V-A; Alg. 1), and format and elements of every slot equal the oracle's choice
for the same slice, level by level; levels and parents stay the oracle's."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

ORACLE_MODE = {1: oracle.COMPRESS, 2: oracle.COMPRESS_SIEVE}


def _lib():
    from paper_1208_5542_gb300 import bfs, build
    build.build()
    return bfs


def _unpack(st):
    """GPU trace -> per level, per slot: (format, elements as uint64)."""
    words = st.trace_words[: st.trace_used].cpu().numpy().view(np.uint32)
    counts = st.trace_counts.cpu().numpy()
    fmts = st.trace_formats.cpu().numpy()
    out, off = [], 0
    for k in range(counts.shape[0]):
        lv = []
        for s, c in enumerate(counts[k]):
            c = int(c)
            lv.append((int(fmts[k][s]), words[off: off + c].astype(np.uint64)))
            off += c
        out.append(lv)
    return out


def _check(gpu, want):
    assert len(gpu) == len(want)
    kinds = set()
    for k, (a, b) in enumerate(zip(gpu, want)):
        assert len(a) == len(b)
        for s, ((fa, ea), (fb, eb)) in enumerate(zip(a, b)):
            assert fa == fb, f"level {k}, slot {s}: format {fa} vs {fb}"
            assert len(ea) == len(eb) and (ea == eb).all(), f"level {k}, slot {s}: {ea[:6]} vs {eb[:6]}"
            kinds.add(fa)
    return kinds


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scale,p", [(14, 4), (14, 5), (13, 8), (12, 1)])
def test_adaptive_slices_equal_the_oracle(mode, scale, p):
    bfs = _lib()
    n, src, dst = graphgen.edges(scale, 16)
    go = oracle.csr(n, src, dst)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
    g.set_exchange_format(True)
    kinds = set()
    for r in graphgen.pick_roots(n, src, dst, 3):
        lv, pa, tr = oracle.dist_bfs(go, p, int(r), mode=ORACLE_MODE[mode], trace=True)
        want = oracle.adaptive_trace(tr, n, p, mode=ORACLE_MODE[mode])
        parent, level, st = g.run(int(r), stats=True, trace_capacity=1 << 22)
        assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
        kinds |= _check(_unpack(st), want)
        for k, ls in enumerate(st.levels):             # exchange bytes: 4 per element
            assert ls["wah_bytes"] == 4 * sum(len(e) for _, e in want[k])
        parent, level, _ = g.run(int(r))                # the graph-launched level loop
        assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
    if p > 1:
        assert oracle.ADAPTIVE_LIST in kinds


def test_adaptive_scale22_grid8_every_format():
    """Kronecker scale 22 on the 8 x 8 grid: sparse levels as vectors, dense
    levels raw; every slot of one search as the oracle chooses."""
    bfs = _lib()
    n, src, dst = graphgen.edges(22, 16)
    go = oracle.csr(n, src, dst)
    p = 8
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
    g.set_exchange_format(True)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    cap = 32 * (2 * p * p + n * p // 31 + 8)
    lv, pa, tr = oracle.dist_bfs(go, p, r, mode=oracle.COMPRESS_SIEVE, trace=True, max_levels=32, trace_cap=cap)
    want = oracle.adaptive_trace(tr, n, p)
    parent, level, st = g.run(r, stats=True, trace_capacity=2 * cap)
    assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
    kinds = _check(_unpack(st), want)
    assert kinds >= {oracle.ADAPTIVE_LIST, oracle.ADAPTIVE_RAW}


@pytest.mark.parametrize("mode", [1, 2])
def test_adaptive_with_bottom_up_levels_and_row_exchange(mode):
    """Bottom-up levels decode vector and raw slots into the stream bitmap; the
    row exchange and the ragged grid keep levels and parents the oracle's."""
    bfs = _lib()
    n, src, dst = graphgen.edges(15, 16)
    go = oracle.csr(n, src, dst)
    for p in (3, 8):
        g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
        g.set_exchange_format(True)
        for policy in (bfs.DIRECTION_HYBRID, bfs.DIRECTION_BOTTOM_UP):
            g.set_direction(policy, 4, 24)
            for r in graphgen.pick_roots(n, src, dst, 2):
                lv, pa = oracle.bfs(go, int(r))
                parent, level, _ = g.run(int(r))
                assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
                parent, level, _ = g.run(int(r), stats=True)
                assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()


def test_adaptive_dense_one_fills_and_ragged_tail():
    """A dense contiguous level-1 frontier (WAH 1-fills win) and ranges whose
    length is not a multiple of 31 or 32 (the active word, the raw tail)."""
    bfs = _lib()
    mid = np.arange(1, 4000)
    src = np.concatenate([np.zeros(len(mid), np.int64), mid]).astype(np.int32)
    dst = np.concatenate([mid, 4000 + (mid * 7) % 4001]).astype(np.int32)
    n = 8001
    go = oracle.csr(n, src, dst)
    for mode in (1, 2):
        for p in (1, 2, 3):
            g = bfs.Graph.from_edges(n, src, dst, p=p, mode=mode)
            g.set_exchange_format(True)
            lv, pa, tr = oracle.dist_bfs(go, p, 0, mode=ORACLE_MODE[mode], trace=True)
            parent, level, st = g.run(0, stats=True, trace_capacity=1 << 20)
            assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
            _check(_unpack(st), oracle.adaptive_trace(tr, n, p, mode=ORACLE_MODE[mode]))


def test_adaptive_needs_32bit_words():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(10, 16)
    g = bfs.Graph.from_edges(n, src, dst, p=2, mode=2, wah_bits=64)
    g.set_exchange_format(True)
    with pytest.raises(BfsError, match="INVALID_ARG"):
        g.run(0)
    g.set_exchange_format(False)
    g.run(0)
