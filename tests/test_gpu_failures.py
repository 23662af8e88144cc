"""Failure paths of the C ABI, made to fire from the host: a bounded wait that
runs out, a full queue, corrupt CSR inputs, injected allocation failures and
corrupted search outputs.  None of them faults or stalls the GPU: every error
is found by the host or by a device check that reports a status."""
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


def test_server_wait_times_out_then_completes():
    """A query queued behind others on a one-lane server is not done after 1 us:
    BFS_ERR_TIMEOUT; the ticket stays valid and a longer wait returns the oracle's result."""
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(18, 16)
    g = bfs.Graph.from_edges(n, src, dst, p=4)
    srv = bfs.Server(hbm_budget_bytes=4 << 30, max_lanes=1)
    srv.add_graph(g)
    roots = graphgen.pick_roots(n, src, dst, 8)
    tickets = [srv.submit(0, int(r), parents=True) for r in roots]
    with pytest.raises(BfsError, match="TIMEOUT"):
        srv.wait(tickets[-1], n, timeout_us=1)
    lv, pa = srv.wait(tickets[-1], n, timeout_s=120.0, parents=True)
    olv, opa = oracle.bfs(oracle.csr(n, src, dst), int(roots[-1]))
    assert (lv.cpu().numpy() == olv).all() and (pa.cpu().numpy() == opa).all()
    for t in tickets[:-1]:
        srv.wait(t, n, timeout_s=120.0)
    srv.close()


def test_server_queue_full_is_busy_and_counted():
    """With a queue limit of 1 and one lane, a burst of submissions is partly
    refused with BFS_ERR_BUSY; every refusal is counted, every accepted query completes."""
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(18, 16)
    g = bfs.Graph.from_edges(n, src, dst, p=4)
    srv = bfs.Server(hbm_budget_bytes=4 << 30, max_lanes=1)
    srv.add_graph(g)
    srv.set_queue_limit(1)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    accepted, busy = [], 0
    for _ in range(64):
        try:
            accepted.append(srv.submit(0, r))
        except BfsError as e:
            assert "BUSY" in str(e)
            busy += 1
    st = srv.stats()
    assert busy > 0 and st["rejected"] == busy and st["submitted"] == len(accepted)
    want = oracle.bfs_levels(oracle.csr(n, src, dst), r)
    for t in accepted:
        assert (srv.wait(t, n, timeout_s=120.0).cpu().numpy() == want).all()
    srv.close()


def test_corrupt_csr_is_rejected():
    """A row_ptr that decreases, one that does not start at 0, a column id >= n:
    BFS_ERR_INVALID_ARG from the input check; the device stays usable."""
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n = 6
    good_rp = np.array([0, 2, 3, 3, 5, 5, 6], np.int64)
    good_col = np.array([1, 2, 0, 4, 5, 3], np.int32)
    bad = [
        (np.array([0, 2, 1, 3, 5, 5, 6], np.int64), good_col),     # decreasing
        (np.array([1, 2, 3, 3, 5, 5, 6], np.int64), good_col),     # row_ptr[0] != 0
        (good_rp, np.array([1, 2, 0, 4, 6, 3], np.int32)),         # a column id == n
        (good_rp, np.array([1, 2, 0, -1, 5, 3], np.int32)),        # a negative id
    ]
    for rp, col in bad:
        with pytest.raises(BfsError, match="INVALID_ARG"):
            bfs.Graph.from_csr(n, rp, col, p=2)
        with pytest.raises(BfsError, match="INVALID_ARG"):          # device copies too
            bfs.Graph.from_csr(n, torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p=2)
    g = bfs.Graph.from_csr(n, good_rp, good_col, p=2)
    parent, level, _ = g.run(0)
    go = oracle.CSR(n, good_rp, good_col)
    lv, pa = oracle.bfs(go, 0)
    assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_leak_nothing():
    """Every device allocation of a graph build, of the first search (its
    workspace and row-exchange buffers) and of the first batch made to fail in
    turn: the call returns BFS_ERR_OUT_OF_MEMORY, releases what it allocated,
    and the same call succeeds once the injection is disarmed."""
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(14, 16)
    want_l, want_p = oracle.bfs(oracle.csr(n, src, dst), 0)
    # the same calls once without injection, so that one-time costs of the
    # process (the CUDA-graph and allocator pools, torch's cache) come before the baseline
    g = bfs.Graph.from_edges(n, src, dst, p=4)
    g.run(0, stats=True, row_trace_capacity=1 << 16)
    g.run(0)
    g.run_batch([0, 1, 2])
    g.close()
    base = _free_bytes()
    fired = 0
    try:
        for k in range(1, 64):
            bfs.debug_fail_allocation(k)
            try:
                g = bfs.Graph.from_edges(n, src, dst, p=4)
            except BfsError as e:
                assert "OUT_OF_MEMORY" in str(e)
                fired += 1
                continue
            finally:
                bfs.debug_fail_allocation(0)
            g.close()
            break
        assert fired >= 5                                  # the layout build allocates several arrays
        assert _free_bytes() >= base - (8 << 20)
        g = bfs.Graph.from_edges(n, src, dst, p=4)
        for k in (1, 2, 3):                                # the first search's lazy allocations
            bfs.debug_fail_allocation(k)
            try:
                g.run(0, stats=True, row_trace_capacity=1 << 16)
            except BfsError as e:
                assert "OUT_OF_MEMORY" in str(e)
            finally:
                bfs.debug_fail_allocation(0)
        parent, level, _ = g.run(0)
        assert (level.cpu().numpy() == want_l).all() and (parent.cpu().numpy() == want_p).all()
        bfs.debug_fail_allocation(1)                       # the batch state
        with pytest.raises(BfsError, match="OUT_OF_MEMORY"):
            g.run_batch([0, 1, 2])
        bfs.debug_fail_allocation(0)
        levels, _, _ = g.run_batch([0, 1, 2])
        assert (levels[0].cpu().numpy() == want_l).all()
        g.close()
    finally:
        bfs.debug_fail_allocation(0)
    assert _free_bytes() >= base - (8 << 20)


def test_debug_checks_and_corrupted_outputs():
    """debug_checks: searches check their outputs and pass; bfs_check_search
    reports BFS_ERR_CORRUPT for a wrong parent level, a wrong root, and an
    unreached vertex with a parent."""
    bfs = _lib()
    from paper_1208_5542_gb300.native import BfsError
    n, src, dst = graphgen.edges(14, 16)
    go = oracle.csr(n, src, dst)
    for mode in (0, 1, 2):
        g = bfs.Graph.from_edges(n, src, dst, p=4, mode=mode, debug=True)
        for r in graphgen.pick_roots(n, src, dst, 2):
            parent, level, _ = g.run(int(r))
            lv, pa = oracle.bfs(go, int(r))
            assert (level.cpu().numpy() == lv).all() and (parent.cpu().numpy() == pa).all()
            parent, level, _ = g.run(int(r), stats=True)
    r = int(graphgen.pick_roots(n, src, dst, 1)[0])
    parent, level, _ = g.run(r)
    g.check_search(r, parent, level)
    lv = level.cpu().numpy()
    v2 = int(np.nonzero(lv == 2)[0][0])
    same = int(np.nonzero(lv == 2)[0][1])
    unreached = np.nonzero(lv < 0)[0]
    cases = []
    p1 = parent.clone(); p1[v2] = same; cases.append((p1, level))          # parent on the same level
    l1 = level.clone(); l1[r] = 1; cases.append((parent, l1))               # root not at level 0
    if len(unreached):
        p2 = parent.clone(); p2[int(unreached[0])] = r; cases.append((p2, level))
    for pa_, lv_ in cases:
        with pytest.raises(BfsError, match="CORRUPT"):
            g.check_search(r, pa_, lv_)


def test_autotune_option_tunes_the_first_batch():
    bfs = _lib()
    n, src, dst = graphgen.edges(14, 16)
    roots = graphgen.pick_roots(n, src, dst, 8)
    g = bfs.Graph.from_edges(n, src, dst, p=4, autotune=True)
    levels, _, _ = g.run_batch(roots)
    go = oracle.csr(n, src, dst)
    for k, r in enumerate(roots):
        assert (levels[k].cpu().numpy() == oracle.bfs_levels(go, int(r))).all()
