"""Failure handling on the GPU, without a GPU fault.

Every failure is made on the host: a wall-clock limit far below what the
work needs, or a state imported with a planted inconsistency.  The device
loop checks its limit once per iteration and stops with a status that the
host reads (MF_ETIMEOUT); the debug_checks pass re-derives the state's
invariants at the end of the kernel and reports a mismatch (MF_ECHECK).  No
kernel traps or hangs, and the graph recovers with mf_solve."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_05895_gb300 as pkg
    return pkg


def test_time_limit_runs_out_and_the_graph_recovers(mf):
    """A static solve of a 2048^2 segmentation grid (tens of ms of device
    work) with a 1 ms limit: MF_ETIMEOUT from mf_flow_value, updates refused
    with MF_ENOTSOLVED, then mf_solve under the default limit reaches the
    oracle's value."""
    g = gen.grid_segmentation(2048, 2048, seed=61)
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, time_limit_ms=1)
    G.solve()
    with pytest.raises(mf.MFError) as ei:
        G.flow_value()
    assert ei.value.code == mf.MF_ETIMEOUT
    b = gen.grid_rect_batch(g, seed=61, index=0, side_lo=64, side_hi=64)
    with pytest.raises(mf.MFError) as ei:
        G.apply_updates(b.edge_id, b.new_cap)
    assert ei.value.code == mf.MF_ENOTSOLVED
    G.set_time_limit(0)
    G.solve()
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    G.close()


def test_time_limit_in_the_serving_loop(mf):
    """Through the server: a static recompute request of a 2048^2 grid whose
    limit is 1 ms ends with MF_ETIMEOUT (the limit is checked at the start of
    every loop iteration, and the recompute needs many); the requests of
    another graph served beside it are unaffected and equal the oracle."""
    big = gen.grid_segmentation(2048, 2048, seed=62)
    small = gen.random_graph(seed=63)
    Gb = mf.MaxFlowGraph(big.n, big.row_ptr, big.col, big.cap, big.s, big.t)
    Gs = mf.MaxFlowGraph(small.n, small.row_ptr, small.col, small.cap, small.s, small.t)
    S = None
    try:
        Gb.solve()
        Gb.flow_value()
        Gs.solve()
        Gs.flow_value()
        Gb.set_time_limit(1)
        S = mf.Server()
        ib = S.add_graph(Gb, 600_000)
        isml = S.add_graph(Gs, 1000)
        cap = small.cap.copy()
        tickets = []
        empty = np.zeros(0, np.int32)
        tb = S.submit(ib, empty, empty, recompute=True)
        for j in range(4):
            b = gen.mixed_batch(cap, 50, 1, 50, seed=63, index=j)
            gen.apply_batch(cap, b)
            tickets.append((S.submit(isml, b.edge_id, b.new_cap), cap.copy()))
        S.drain()
        done, _, code, _ = S.poll(tb)
        assert done and code == mf.MF_ETIMEOUT
        for t, c in tickets:
            done, f, code, _ = S.poll(t)
            assert done and code == mf.MF_OK
            assert f == oracle.maxflow_fifo(small.n, small.row_ptr, small.col, c, small.s, small.t)
    finally:
        if S is not None:
            S.close()   # the server first: it holds the graphs' streams
        Gb.close()
        Gs.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_debug_checks_pass_on_clean_runs(mf, mode):
    """With debug_checks every kernel re-derives e(v) from the residuals,
    checks each residual pair and the mirror, and bounds-checks its list
    entries; on correct runs nothing fires and every value is the oracle's."""
    for g in (gen.random_graph(seed=65), gen.rmat(scale=12, seed=66)):
        cap = g.cap.copy()
        G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, debug_checks=True, mode=mode)
        G.solve()
        assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        for j in range(3):
            b = gen.mixed_batch(cap, max(50, g.m // 100), 1, 50, seed=65, index=j)
            gen.apply_batch(cap, b)
            G.apply_updates(b.edge_id, b.new_cap)
            assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        G.close()


def test_debug_checks_report_a_planted_inconsistency(mf):
    """A state imported with one excess one unit above the vertex's net
    inflow: the next repair's end-of-kernel check reports MF_ECHECK (the
    kernel moves excess and residual by equal amounts, so the discrepancy
    survives), updates are refused until mf_solve, which restores the
    oracle's value."""
    g = gen.random_graph(seed=67)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, debug_checks=True)
    try:
        G.solve()
        assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        r, e, h = G.export_state()
        v = next(x for x in range(g.n) if x not in (g.s, g.t))
        e = e.copy()
        e[v] += 1
        G.import_state(r, e, h)
        b = gen.mixed_batch(cap, 50, 1, 50, seed=67, index=0)
        gen.apply_batch(cap, b)
        G.apply_updates(b.edge_id, b.new_cap)
        with pytest.raises(mf.MFError) as ei:
            G.flow_value()
        assert ei.value.code == mf.MF_ECHECK
        assert "excess differs from the net inflow" in str(ei.value)
        with pytest.raises(mf.MFError) as ei:
            G.apply_updates(b.edge_id, b.new_cap)
        assert ei.value.code == mf.MF_ENOTSOLVED
        G.solve()
        assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    finally:
        G.close()
