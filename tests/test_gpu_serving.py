"""The serving loop (mf_server_*): several resident graphs, continuous
batching, CUDA-graph-captured repairs.

Each graph's flow value after each of its batches is the same when the
batches are served alone (one graph, direct calls) and when they are served
in the mix through the server with the other graphs' batches overlapping on
the device; both equal the CPU oracle (tolerance: exact, integer flows)."""
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


def workloads():
    gs = [gen.random_graph(seed=51), gen.rmat(scale=12, seed=52), gen.rmat(scale=13, seed=53),
          gen.grid_segmentation(96, 64, seed=54)]
    seqs = []
    for gi, g in enumerate(gs):
        cap = g.cap.copy()
        bs = []
        for j in range(6):
            if g.meta.get("kind") == "grid":
                b = gen.grid_rect_batch(g, seed=54, index=j, side_lo=8, side_hi=40)
            else:
                b = gen.mixed_batch(cap, max(10, g.m // (200 if j % 2 else 20)), 1, 100, seed=gi, index=j)
            gen.apply_batch(cap, b)
            bs.append(b)
        seqs.append(bs)
    return gs, seqs


def test_results_alone_equal_results_in_the_mix(mf):
    gs, seqs = workloads()
    # alone: direct calls, one graph at a time
    alone = []
    for g, bs in zip(gs, seqs):
        G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
        G.solve()
        G.flow_value()
        fl = []
        for b in bs:
            G.apply_updates(b.edge_id, b.new_cap)
            fl.append(G.flow_value())
        alone.append(fl)
        G.close()
    # oracle on the cumulative capacities
    for g, bs, fl in zip(gs, seqs, alone):
        cap = g.cap.copy()
        for b, f in zip(bs, fl):
            gen.apply_batch(cap, b)
            assert f == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    # in the mix: four graphs on grids of 38 CTAs, all batches queued at once
    S = mf.Server(sm_slots=152)
    Gs = []
    for g, bs in zip(gs, seqs):
        G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, grid_blocks=38)
        G.solve()
        G.flow_value()
        Gs.append(G)
        S.add_graph(G, max(len(b.edge_id) for b in bs))
    rng = np.random.default_rng(0)
    order = np.concatenate([np.full(len(bs), gi) for gi, bs in enumerate(seqs)])
    rng.shuffle(order)
    nxt = [0] * len(gs)
    tickets = {}
    for gi in order:
        j = nxt[gi]
        nxt[gi] += 1
        b = seqs[gi][j]
        tickets[(gi, j)] = S.submit(int(gi), b.edge_id, b.new_cap)
    S.drain()
    for (gi, j), t in tickets.items():
        done, flow, code, lat = S.poll(t)
        assert done and code == 0
        assert flow == alone[gi][j], (gi, j)
    st = S.stats()
    assert st["completed"] == st["submitted"] == sum(len(b) for b in seqs)
    assert st["failed"] == 0 and st["max_inflight"] >= 2
    assert st["p99_us"] >= st["p50_us"] > 0
    S.close()
    for G in Gs:
        G.close()


def test_sm_slots_serialise_and_hbm_budget_admits(mf):
    g1, g2 = gen.rmat(scale=11, seed=61), gen.random_graph(seed=62)
    G1 = mf.MaxFlowGraph(g1.n, g1.row_ptr, g1.col, g1.cap, g1.s, g1.t, grid_blocks=38)
    G2 = mf.MaxFlowGraph(g2.n, g2.row_ptr, g2.col, g2.cap, g2.s, g2.t, grid_blocks=38)
    for G in (G1, G2):
        G.solve()
        G.flow_value()
    # a budget that holds one graph only
    import ctypes
    b1, b2 = ctypes.c_int64(0), ctypes.c_int64(0)
    mf.lib().mf_device_bytes(G1._h, ctypes.byref(b1))
    mf.lib().mf_device_bytes(G2._h, ctypes.byref(b2))
    staging = 4 * (4 + 2 * 4096)
    assert b2.value > 4 * staging
    S = mf.Server(hbm_budget_bytes=b1.value + 2 * staging, sm_slots=38)
    S.add_graph(G1, 4096)
    with pytest.raises(mf.MFError) as ei:
        S.add_graph(G2, 4096)
    assert ei.value.code == mf.MF_ENOMEM
    cap = g1.cap.copy()
    ts = []
    for j in range(4):
        b = gen.mixed_batch(cap, 300, 1, 100, seed=61, index=j)
        gen.apply_batch(cap, b)
        ts.append(S.submit(0, b.edge_id, b.new_cap))
    S.drain()
    assert S.poll(ts[-1])[1] == oracle.maxflow_fifo(g1.n, g1.row_ptr, g1.col, cap, g1.s, g1.t)
    assert S.stats()["max_inflight"] == 1
    S.close()
    G1.close()
    G2.close()


def test_push_pull_graphs_in_the_server(mf):
    """Push-pull graphs served by the request loop (captured repairs) give the
    oracle's values."""
    g = gen.rmat(scale=12, seed=72)
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, grid_blocks=76, mode=mf.MF_MODE_PUSH_PULL)
    G.solve()
    G.flow_value()
    S = mf.Server()
    S.add_graph(G, 2000)
    cap = g.cap.copy()
    out = []
    for j in range(5):
        b = gen.mixed_batch(cap, 500, 1, 100, seed=72, index=j)
        gen.apply_batch(cap, b)
        out.append((S.submit(0, b.edge_id, b.new_cap), oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)))
    S.drain()
    for t, want in out:
        assert S.poll(t)[1] == want
    S.close()
    G.close()


def test_cuda_graph_capture_and_recompute_requests(mf):
    """Every graph's repair is captured once per grid class (full, half,
    quarter of its grid) and its recompute once; every request -- batches of
    each class, a recompute -- is a replay of one of them, and each value is
    the oracle's.  A delta batch is launched directly (the captures read
    absolute capacities)."""
    g = gen.rmat(scale=14, seed=71)
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, grid_blocks=76)
    G.solve()
    G.flow_value()
    S = mf.Server()
    S.add_graph(G, 30_000)
    st = S.stats()
    assert st["captured_graphs"] == 4, st     # 76, 38 and 19 CTAs, plus the recompute
    cap = g.cap.copy()
    out = []
    for j, k in enumerate((500, 5000, 25_000, 800)):
        b = gen.mixed_batch(cap, k, 1, 100, seed=71, index=j)
        gen.apply_batch(cap, b)
        t = S.submit(0, b.edge_id, b.new_cap, recompute=(j == 3))
        out.append((t, oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)))
    b = gen.mixed_batch(cap, 300, 1, 100, seed=71, index=9)
    delta = (b.new_cap.astype(np.int64) - cap[b.edge_id]).astype(np.int32)
    gen.apply_batch(cap, b)
    out.append((S.submit(0, b.edge_id, delta, delta=True), oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)))
    S.drain()
    for t, want in out:
        done, f, code, _ = S.poll(t)
        assert done and code == 0 and f == want
    st = S.stats()
    assert st["replays"] == 4 and st["direct_launches"] == 1, st
    S.close()
    G.close()


def test_small_repairs_run_beside_a_large_one(mf):
    """With SM slots for one full grid, a small batch of another graph is
    admitted while a large graph's big batch is in flight: its grid class is
    a quarter of its graph's grid, which fits beside the other's half."""
    big = gen.rmat(scale=16, seed=73)
    small = gen.random_graph(seed=74)
    Gb = mf.MaxFlowGraph(big.n, big.row_ptr, big.col, big.cap, big.s, big.t, grid_blocks=100)
    Gs = mf.MaxFlowGraph(small.n, small.row_ptr, small.col, small.cap, small.s, small.t, grid_blocks=100)
    for G in (Gb, Gs):
        G.solve()
        G.flow_value()
    S = mf.Server(sm_slots=100)
    ib, isml = S.add_graph(Gb, 20_000), S.add_graph(Gs, 100)
    capb, caps = big.cap.copy(), small.cap.copy()
    out = []
    for j in range(3):
        bb = gen.mixed_batch(capb, 10_000, 1, 500, seed=73, index=j)   # half grid (50 CTAs)
        gen.apply_batch(capb, bb)
        out.append((S.submit(ib, bb.edge_id, bb.new_cap), big, capb.copy()))
        bs = gen.mixed_batch(caps, 50, 1, 50, seed=74, index=j)         # quarter grid (25 CTAs)
        gen.apply_batch(caps, bs)
        out.append((S.submit(isml, bs.edge_id, bs.new_cap), small, caps.copy()))
    S.drain()
    for t, g, c in out:
        done, f, code, _ = S.poll(t)
        assert done and code == 0 and f == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, c, g.s, g.t)
    assert S.stats()["max_inflight"] == 2
    S.close()
    Gb.close()
    Gs.close()


def test_a_graphs_requests_keep_their_order(mf):
    """A graph's batches carry absolute capacities, so they must be applied
    in submission order even when a later one's smaller grid would fit while
    an earlier one waits for SMs: with SM slots for one full grid and a
    half-grid repair of another graph in flight, a full-grid batch of graph 1
    waits, and the small batches submitted after it must wait behind it.
    Every value equals the oracle's on the capacities in submission order."""
    g1, g2 = gen.rmat(scale=14, seed=75), gen.rmat(scale=14, seed=76)
    G1 = mf.MaxFlowGraph(g1.n, g1.row_ptr, g1.col, g1.cap, g1.s, g1.t, grid_blocks=64)
    G2 = mf.MaxFlowGraph(g2.n, g2.row_ptr, g2.col, g2.cap, g2.s, g2.t, grid_blocks=64)
    for G in (G1, G2):
        G.solve()
        G.flow_value()
    S = mf.Server(sm_slots=64)
    try:
        i1, i2 = S.add_graph(G1, 30_000), S.add_graph(G2, 30_000)
        c1, c2 = g1.cap.copy(), g2.cap.copy()
        out = []
        for r in range(3):
            b = gen.mixed_batch(c2, 5000, 1, 500, seed=76, index=r)       # half grid of graph 2
            gen.apply_batch(c2, b)
            out.append((S.submit(i2, b.edge_id, b.new_cap), g2, c2.copy()))
            for j, k in enumerate((25_000, 300, 300)):                     # full, then quarter grids
                b = gen.mixed_batch(c1, k, 1, 500, seed=75, index=10 * r + j)
                gen.apply_batch(c1, b)
                out.append((S.submit(i1, b.edge_id, b.new_cap), g1, c1.copy()))
        S.drain()
        for t, g, c in out:
            done, f, code, _ = S.poll(t)
            assert done and code == 0 and f == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, c, g.s, g.t)
    finally:
        S.close()
        G1.close()
        G2.close()
