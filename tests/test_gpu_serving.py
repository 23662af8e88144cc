"""Continuous-batching server: every result equals the oracle and the same query served alone."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1208_5542_gb300 import bfs, build
    build.build()
    return bfs


def test_mix_equals_alone_equals_oracle():
    bfs = _lib()
    rng = np.random.default_rng(11)
    specs = [(12, 2), (14, 4), (16, 8)]
    graphs, oracles, roots = [], [], []
    srv = bfs.Server(hbm_budget_bytes=8 << 30, max_lanes=64)
    for scale, p in specs:
        n, src, dst = graphgen.edges(scale, 16)
        g = bfs.Graph.from_edges(n, src, dst, p=p)
        gid = srv.add_graph(g)
        graphs.append((gid, n, g))
        oracles.append(oracle.csr(n, src, dst))
        roots.append(graphgen.pick_roots(n, src, dst, 64, seed=5 + scale))
    # the mix: bursts of queries arrive while earlier ones are on the GPU
    queries, tickets = [], []
    for burst in range(6):
        for _ in range(int(rng.integers(10, 60))):
            k = int(rng.integers(0, len(graphs)))
            r = int(roots[k][int(rng.integers(0, 64))])
            queries.append((k, r))
            tickets.append(srv.submit(graphs[k][0], r))
        if burst % 2:
            srv.wait(tickets[len(tickets) // 2], graphs[queries[len(tickets) // 2][0]][1])
            tickets[len(tickets) // 2] = None
    mix = {}
    for q, t in zip(queries, tickets):
        if t is not None:
            mix[q] = srv.wait(t, graphs[q[0]][1]).cpu().numpy()
    st = srv.stats()
    assert st["completed"] == len(queries) and st["peak_lanes"] > 1
    # each distinct query again, alone (one at a time), and against the oracle
    for (k, r), lv in list(mix.items())[:40]:
        alone = srv.wait(srv.submit(graphs[k][0], r), graphs[k][1]).cpu().numpy()
        assert (alone == lv).all()
        assert (lv == oracle.bfs_levels(oracles[k], r)).all()
    srv.close()


def test_budget_admission_and_errors():
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(14, 16)
    g = bfs.Graph.from_edges(n, src, dst, p=4)
    small = bfs.Server(hbm_budget_bytes=1 << 16, max_lanes=8)
    with pytest.raises(BfsError, match="OUT_OF_MEMORY"):
        small.add_graph(g)
    small.close()
    srv = bfs.Server(hbm_budget_bytes=1 << 30, max_lanes=64)
    gid = srv.add_graph(g)
    with pytest.raises(BfsError, match="BUSY"):       # the server holds the graph
        g.run(0)
    with pytest.raises(BfsError, match="NOT_FOUND"):
        srv.submit(gid + 1, 0)
    with pytest.raises(BfsError, match="INVALID_ARG"):
        srv.submit(gid, n)
    t = srv.submit(gid, int(graphgen.pick_roots(n, src, dst, 1)[0]))
    from paper_1208_5542_gb300 import native
    import ctypes
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = native.lib().bfs_server_wait(srv._h, t, 10_000_000, ctypes.c_void_p(lv.data_ptr()),
                                      ctypes.c_void_p(par.data_ptr()))
    assert native.STATUS[rc] == "BFS_ERR_INVALID_ARG"
    srv.wait(t, n)
    with pytest.raises(BfsError, match="NOT_FOUND"):
        srv.poll(t)
    srv.close()
    g.run(0)                                           # released by the server
