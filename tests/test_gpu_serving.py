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
    """Queries on four resident graphs (Kronecker scales 12-20) arrive in bursts
    while earlier ones run, half of them asking for parents; every result --
    levels, and parents where asked -- equals the oracle's, and a sample of
    them equals the same query served alone."""
    bfs = _lib()
    rng = np.random.default_rng(11)
    specs = [(12, 2), (16, 4), (18, 8), (20, 8)]
    graphs, oracles, roots = [], [], []
    srv = bfs.Server(hbm_budget_bytes=16 << 30, max_lanes=64)
    for scale, p in specs:
        n, src, dst = graphgen.edges(scale, 16)
        g = bfs.Graph.from_edges(n, src, dst, p=p)
        gid = srv.add_graph(g)
        graphs.append((gid, n, g))
        oracles.append(oracle.csr(n, src, dst))
        roots.append(graphgen.pick_roots(n, src, dst, 16, seed=5 + scale))
    # the mix: bursts of queries arrive while earlier ones are on the GPU
    queries, tickets = [], []
    for burst in range(6):
        for _ in range(int(rng.integers(10, 60))):
            k = int(rng.integers(0, len(graphs)))
            r = int(roots[k][int(rng.integers(0, len(roots[k])))])
            wp = r % 2 == 0                            # the query's root decides: a query is repeatable
            queries.append((k, r))
            tickets.append(srv.submit(graphs[k][0], r, parents=wp))
        if burst % 2:
            h = len(tickets) // 2
            k, r = queries[h]
            got = srv.wait(tickets[h], graphs[k][1], parents=r % 2 == 0)
            tickets[h] = (got[0].cpu().numpy(), got[1].cpu().numpy()) if r % 2 == 0 else (got.cpu().numpy(), None)
    mix = {}
    for q, t in zip(queries, tickets):
        if isinstance(t, tuple):
            got = t
        elif q[1] % 2 == 0:
            lv, pa = srv.wait(t, graphs[q[0]][1], parents=True)
            got = (lv.cpu().numpy(), pa.cpu().numpy())
        else:
            got = (srv.wait(t, graphs[q[0]][1]).cpu().numpy(), None)
        if q in mix:
            assert (mix[q][0] == got[0]).all() and (got[1] is None or (mix[q][1] == got[1]).all())
        mix[q] = got
    st = srv.stats()
    assert st["completed"] == len(queries) and st["peak_lanes"] > 1
    # every distinct query against the oracle; a sample again, alone
    parents_checked = 0
    for i, ((k, r), (lv, pa)) in enumerate(mix.items()):
        olv, opa = oracle.bfs(oracles[k], r)
        assert (lv == olv).all(), (k, r)
        if pa is not None:
            assert (pa == opa).all(), (k, r)
            parents_checked += 1
        if i % 4 == 0:
            alv, apa = srv.wait(srv.submit(graphs[k][0], r, parents=True), graphs[k][1], parents=True)
            assert (alv.cpu().numpy() == lv).all() and (apa.cpu().numpy() == opa).all()
    assert parents_checked > 10
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
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    t0 = srv.submit(gid, r)
    with pytest.raises(BfsError, match="INVALID_ARG"):   # submitted without parents
        srv.wait(t0, n, parents=True)
    srv.wait(t0, n)
    t = srv.submit(gid, r, parents=True)
    # host output buffers, parents only
    par = np.empty(n, np.int32)
    from paper_1208_5542_gb300 import native
    import ctypes
    native.check(native.lib().bfs_server_wait(srv._h, t, 10_000_000, None, ctypes.c_void_p(par.ctypes.data)))
    assert (par == oracle.bfs(oracle.csr(n, src, dst), r)[1]).all()
    with pytest.raises(BfsError, match="NOT_FOUND"):
        srv.poll(t)
    with pytest.raises(BfsError, match="INVALID_ARG"):
        srv.set_queue_limit(0)
    srv.close()
    g.run(0)                                           # released by the server
