"""GPU parity: the CUDA library's int64 max-flow value equals the CPU
oracle's bit-exactly on every batch, and its final state passes the
optimality certificate (capacity feasibility, excess bookkeeping, min cut
S = {h >= n} with no residual arc leaving it, value = cut capacity, heights =
exact BFS distances to the sinks).  All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
from tests._helpers import certify_gpu
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_05895_gb300 as pkg
    return pkg


def oracle_flow(g, cap):
    return oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)


def run_batches(mf, g, batches, certify=True, **opts):
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, **opts)
    G.solve()
    f = G.flow_value()
    assert f == oracle_flow(g, cap)
    if certify:
        certify_gpu(G, g, cap, f)
    for b in batches(cap):
        G.apply_updates(b.edge_id, b.new_cap)
        gen.apply_batch(cap, b)
        f = G.flow_value()
        assert f == oracle_flow(g, cap)
        if certify:
            certify_gpu(G, g, cap, f)
    return G, cap


def mixed(g, k, lo, hi, seed, count):
    def it(cap):
        for i in range(count):
            yield gen.mixed_batch(cap, k, lo, hi, seed=seed, index=i)
    return it


@pytest.mark.parametrize("seed", range(20))
def test_config1_random_graph(mf, seed):
    """1,000 vertices / 8,000 edges, caps U[1,100]; 50-update mixed batches."""
    g = gen.random_graph(seed=seed)
    G, _ = run_batches(mf, g, mixed(g, 50, 1, 50, seed, 3))
    st = G.stats()
    assert st["batch"] == 50 and st["iterations"] >= 0
    G.close()


@pytest.mark.parametrize("mode", ["data-driven", "push-pull"])
def test_tiny_graphs_many(mf, mode):
    """Hundreds of tiny graphs with ties, zero caps, self-loops, parallel and
    antiparallel edges, in the data-driven and the push-pull mode (empty and
    one-vertex subgraphs P, s next to t, unreachable t); every state
    certified."""
    opts = {"mode": mf.MF_MODE_PUSH_PULL} if mode == "push-pull" else {}
    rng = np.random.default_rng(2024 if mode == "data-driven" else 2025)
    for trial in range(150):
        n = int(rng.integers(2, 24))
        m = int(rng.integers(1, 4 * n + 1))
        tails = rng.integers(0, n, m)
        heads = rng.integers(0, n, m)
        caps = rng.integers(0, 6, m)
        s, t = (int(x) for x in rng.choice(n, 2, replace=False))
        g = gen.from_edges(n, tails, heads, caps, s, t)

        def batches(cap, trial=trial, m=m):
            r = np.random.default_rng(trial)
            for _ in range(3):
                k = int(r.integers(0, m + 1))
                ids = r.choice(m, k, replace=False).astype(np.int32)
                yield gen.Batch(edge_id=ids, new_cap=r.integers(0, 7, k).astype(np.int32))
        G, _ = run_batches(mf, g, batches, **opts)
        G.close()


@pytest.mark.parametrize("grid_blocks", [1, 3, 37])
def test_small_launch_shapes(mf, grid_blocks):
    """Few CTAs: every phase and barrier with a ragged split of the work."""
    g = gen.random_graph(n=500, m=4000, seed=grid_blocks)
    G, _ = run_batches(mf, g, mixed(g, 40, 1, 50, grid_blocks, 3), grid_blocks=grid_blocks)
    G.close()


@pytest.mark.parametrize("mode", ["data-driven", "push-pull"])
@pytest.mark.parametrize("grid_blocks", [1, 3])
def test_few_ctas_on_a_power_law_graph(mf, mode, grid_blocks):
    """RMAT-15 on 1 or 3 CTAs: every warp serves a thousand vertices or more
    per BFS level, so its staged frontier fills and is published in the middle
    of a level many times (bottom-up and top-down), and every fixed-stride
    loop of a phase wraps around the warps many times."""
    g = gen.rmat(scale=15, seed=91)
    opts = {"grid_blocks": grid_blocks}
    if mode == "push-pull":
        opts["mode"] = mf.MF_MODE_PUSH_PULL

    def batches(cap):
        yield gen.mixed_batch(cap, g.m // 1000, 1, 500, seed=91, index=0)
        yield gen.mixed_batch(cap, g.m // 100, 1, 500, seed=91, index=1)
    G, _ = run_batches(mf, g, batches, **opts)
    G.close()


@pytest.mark.parametrize("kc", [1, 2, 64])
def test_kernel_cycles_do_not_change_the_value(mf, kc):
    g = gen.random_graph(seed=100 + kc)
    G, _ = run_batches(mf, g, mixed(g, 50, 1, 50, kc, 2), kernel_cycles=kc)
    G.close()


@pytest.mark.parametrize("scale", [12, 15])
def test_rmat_dynamic(mf, scale):
    """RMAT power-law graphs (hubs above the big-vertex threshold), batches of
    0.1 % and 1 % of the edges."""
    g = gen.rmat(scale=scale, seed=scale)
    k1, k2 = max(1, g.m // 1000), max(1, g.m // 100)

    def batches(cap):
        yield gen.mixed_batch(cap, k1, 1, 500, seed=scale, index=0)
        yield gen.mixed_batch(cap, k2, 1, 500, seed=scale, index=1)
        yield gen.mixed_batch(cap, k1, 1, 500, seed=scale, index=2)
    G, _ = run_batches(mf, g, batches)
    G.close()


def test_grid_dynamic(mf):
    """Segmentation grid: source and sink have one arc per pixel (big vertices
    split into chunks); rectangle batches rewrite terminal capacities."""
    g = gen.grid_segmentation(160, 144, seed=7)

    def batches(cap):
        for i in range(4):
            yield gen.grid_rect_batch(g, seed=7, index=i, side_lo=16, side_hi=96)
    G, _ = run_batches(mf, g, batches)
    G.close()


def test_recompute_flag_matches(mf):
    g = gen.random_graph(seed=5)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    for i in range(3):
        b = gen.mixed_batch(cap, 200, 1, 50, seed=5, index=i)
        G.apply_updates(b.edge_id, b.new_cap, recompute=True)
        gen.apply_batch(cap, b)
        f = G.flow_value()
        assert f == oracle_flow(g, cap)
        certify_gpu(G, g, cap, f)
    G.close()


def test_delta_flag(mf):
    g = gen.random_graph(seed=6)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    b = gen.mixed_batch(cap, 80, 1, 50, seed=6, index=0)
    delta = b.new_cap.astype(np.int64) - cap[b.edge_id]
    delta[::3] -= 1000            # clamped at zero
    G.apply_updates(b.edge_id, delta.astype(np.int32), delta=True)
    cap[b.edge_id] = np.maximum(0, cap[b.edge_id] + delta)
    f = G.flow_value()
    assert f == oracle_flow(g, cap)
    certify_gpu(G, g, cap, f)
    G.close()


def test_device_batch_and_torch_allocator(mf):
    import torch
    g = gen.random_graph(seed=8)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                        torch.from_numpy(cap).cuda(), g.s, g.t, torch_allocator=True)
    G.solve()
    assert G.flow_value() == oracle_flow(g, cap)
    for i in range(3):
        b = gen.mixed_batch(cap, 50, 1, 50, seed=8, index=i)
        G.apply_updates(torch.from_numpy(b.edge_id).cuda(), torch.from_numpy(b.new_cap).cuda())
        gen.apply_batch(cap, b)
        assert G.flow_value() == oracle_flow(g, cap)
    certify_gpu(G, g, cap, G.flow_value())
    G.close()


def test_empty_batch_and_degenerate_graphs(mf):
    # empty batch: value unchanged
    g = gen.random_graph(seed=9)
    G, cap = run_batches(mf, g, lambda cap: iter([gen.Batch(np.zeros(0, np.int32), np.zeros(0, np.int32))]))
    G.close()
    cases = [
        gen.from_edges(2, [0], [1], [17], 0, 1),                           # single edge
        gen.from_edges(2, [0, 0, 1], [1, 1, 0], [3, 4, 9], 0, 1),          # parallel + back edge
        gen.from_edges(5, [0, 1, 3], [1, 2, 4], [5, 5, 5], 0, 4),          # no s-t path
        gen.from_edges(4, [1, 2], [2, 3], [5, 5], 0, 3),                   # s has no out-edges
        gen.from_edges(4, [0, 1, 1, 2], [1, 1, 2, 3], [0, 7, 0, 0], 0, 3),  # zero caps + self-loop
        gen.from_edges(3, [0, 1, 2, 1], [1, 2, 0, 0], [5, 5, 5, 5], 0, 2),  # edges into s
    ]
    for g in cases:
        def batches(cap, g=g):
            yield gen.Batch(np.arange(g.m, dtype=np.int32), (cap + 3).astype(np.int32))
            yield gen.Batch(np.arange(g.m, dtype=np.int32)[::2], np.zeros((g.m + 1) // 2, np.int32))
        G, _ = run_batches(mf, g, batches)
        G.close()


def test_rejected_batches_leave_state_unchanged(mf):
    g = gen.random_graph(seed=10)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    f0 = G.flow_value()
    lim = G.cap_limit()
    bad = [
        (np.array([1, 2, 1], np.int32), np.array([5, 5, 5], np.int32)),          # duplicate id
        (np.array([3, g.m], np.int32), np.array([5, 5], np.int32)),              # id out of range
        (np.array([3, -1], np.int32), np.array([5, 5], np.int32)),               # negative id
        (np.array([3, 4], np.int32), np.array([5, -2], np.int32)),               # negative capacity
        (np.array([3], np.int32), np.array([lim + 1], np.int32) if lim < 2 ** 31 - 1 else np.array([-5], np.int32)),
    ]
    for ids, caps in bad:
        G.apply_updates(ids, caps)
        with pytest.raises(mf.MFError) as ei:
            G.sync()
        assert ei.value.code == mf.MF_EINVAL
        assert G.flow_value() == f0
    certify_gpu(G, g, cap, f0)
    b = gen.mixed_batch(cap, 50, 1, 50, seed=10, index=0)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle_flow(g, cap)
    with pytest.raises(mf.MFError):
        G.apply_updates(np.zeros(g.m + 1, np.int32), np.zeros(g.m + 1, np.int32))  # k > m, host check
    G.close()


def test_iteration_cap_reports_timeout_and_solve_recovers(mf):
    # a segmentation grid: its static solve starts with every pixel active,
    # far more than one activation-round cap can finish in one iteration
    g = gen.grid_segmentation(256, 192, seed=3)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, max_iters=1)
    G.solve()
    with pytest.raises(mf.MFError) as ei:
        G.flow_value()
    assert ei.value.code == mf.MF_ETIMEOUT
    with pytest.raises(mf.MFError) as ei:
        G.apply_updates(np.array([0], np.int32), np.array([1], np.int32))
    assert ei.value.code == mf.MF_ENOTSOLVED
    G.close()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    assert G.flow_value() == oracle_flow(g, cap)
    G.close()


def test_not_solved(mf):
    g = gen.random_graph(seed=12)
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    with pytest.raises(mf.MFError) as ei:
        G.apply_updates(np.array([0], np.int32), np.array([1], np.int32))
    assert ei.value.code == mf.MF_ENOTSOLVED
    G.close()


def test_checkpoint_resume(mf):
    g = gen.random_graph(seed=13)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    b = gen.mixed_batch(cap, 50, 1, 50, seed=13, index=0)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    f1 = G.flow_value()
    r, e, h = G.export_state()
    # resume in a fresh graph built from the current capacities
    H = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    H.import_state(r, e, h)
    assert H.flow_value() == f1
    b2 = gen.mixed_batch(cap, 50, 1, 50, seed=13, index=1)
    H.apply_updates(b2.edge_id, b2.new_cap)
    G.apply_updates(b2.edge_id, b2.new_cap)
    gen.apply_batch(cap, b2)
    want = oracle_flow(g, cap)
    assert H.flow_value() == want == G.flow_value()
    certify_gpu(H, g, cap, want)
    assert f1 >= 0
    G.close()
    H.close()


def test_min_cut_capacity_equals_flow(mf):
    g = gen.rmat(scale=13, seed=21)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    f = G.flow_value()
    side = G.min_cut()
    tails = g.tails()
    cut = int(cap[(side[tails] == 1) & (side[g.col] == 0)].astype(np.int64).sum())
    assert side[g.s] == 1 and side[g.t] == 0 and cut == f == oracle_flow(g, cap)
    G.close()


@pytest.mark.slow
def test_full_size_rmat20_bench_batches(mf):
    """RMAT scale 20 (the benchmark graph) with the benchmark's launch
    configuration: 1k and 100k mixed batches, value equal to the oracle and
    the certificate checked on the full state."""
    g = gen.rmat(scale=20, seed=1)

    def batches(cap):
        yield gen.mixed_batch(cap, 1000, 1, 500, seed=1, index=0)
        yield gen.mixed_batch(cap, 100000, 1, 500, seed=1, index=1)
    G, _ = run_batches(mf, g, batches)
    G.close()


def test_trace_records(mf):
    """Tracing: one record per grid barrier plus one per BFS level that CTA 0
    ran alone (mode 4), phases in order, BFS levels counted."""
    g = gen.rmat(scale=12, seed=31)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.trace_enable(8192)
    G.solve()
    f = G.flow_value()
    recs = G.trace()
    st = G.stats()
    solo = [r for r in recs if r["phase"] == "bfs" and r["mode"] == 4]
    assert len(recs) == st["barriers"] + len(solo) > 0
    assert {r["phase"] for r in recs} >= {"batch", "height_init", "bfs"}
    bfs = [r for r in recs if r["phase"] == "bfs" and r["mode"] in (0, 2, 4)]
    assert len(bfs) == st["bfs_levels"]
    assert all(r["ns"] >= 0 for r in recs)
    b = gen.mixed_batch(cap, 200, 1, 500, seed=31, index=0)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle_flow(g, cap)
    recs = G.trace()
    assert len(recs) == G.stats()["barriers"] + sum(r["phase"] == "bfs" and r["mode"] == 4 for r in recs)
    G.trace_enable(0)
    assert f >= 0
    G.close()


@pytest.mark.parametrize("scale", [11, 14])
def test_topology_driven_mode(mf, scale):
    """MF_MODE_TOPOLOGY (Sec. 5.2): same values, certified states."""
    g = gen.rmat(scale=scale, seed=90 + scale)
    G, _ = run_batches(mf, g, mixed(g, max(10, g.m // 200), 1, 500, scale, 3), mode=mf.MF_MODE_TOPOLOGY)
    G.close()


@pytest.mark.slow
def test_full_size_grid4096_rect_batches(mf):
    """The 4096 x 4096 segmentation grid (16.8M vertices, s and t with one
    arc per pixel) with rectangle batches of side 64-512: values equal to the
    oracle and the certificate on the full state."""
    g = gen.grid_segmentation(4096, 4096, seed=3)

    def batches(cap):
        for i in range(2):
            yield gen.grid_rect_batch(g, seed=3, index=i)
    G, _ = run_batches(mf, g, batches, kernel_cycles=4)
    G.close()


def test_clean_exit_without_final_bfs(mf):
    """When the last PushRelabel/RemoveInvalidEdges round leaves no active
    vertex the loop stops without another BFS (exit_kind 1).  A path graph
    does so deterministically (one iteration pushes everything to t); on the
    larger workloads it depends on the schedule.  Every value still equals
    the oracle's, and the certificate (which asks for the cut and exact
    heights, recomputed by one BFS) holds."""
    path = gen.from_edges(6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], [9, 7, 8, 5, 6], 0, 5, name="path")
    G = mf.MaxFlowGraph(path.n, path.row_ptr, path.col, path.cap, path.s, path.t)
    G.solve()
    assert G.flow_value() == 5 and G.stats()["exit_kind"] == 1
    certify_gpu(G, path, path.cap.copy(), 5)
    G.close()
    kinds = []
    cases = [("grid", gen.grid_segmentation(256, 192, seed=45)), ("rmat", gen.rmat(scale=13, seed=44))]
    cases += [("random", gen.random_graph(seed=70 + i)) for i in range(4)]
    for name, g in cases:
        cap = g.cap.copy()
        G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        G.solve()
        kinds.append(G.stats()["exit_kind"])
        for i in range(4):
            if name == "grid":
                b = gen.grid_rect_batch(g, seed=45, index=i, side_lo=16, side_hi=96)
            else:
                b = gen.mixed_batch(cap, max(10, g.m // (100 if i % 2 else 1000)), 1, 50, seed=44, index=i)
            G.apply_updates(b.edge_id, b.new_cap)
            gen.apply_batch(cap, b)
            f = G.flow_value()
            st = G.stats()
            kinds.append(st["exit_kind"])
            assert f == oracle_flow(g, cap)
            if st["exit_kind"] == 1 or i == 3:
                certify_gpu(G, g, cap, f)
        G.close()
    assert set(kinds) <= {0, 1}, kinds
    print("exit kinds:", kinds)


def test_pure_increment_fast_path(mf):
    """A batch that only raises capacities of arcs not going from S to T of
    the exact cut cannot change the flow value: no loop runs (exit_kind 2),
    the value is the oracle's, the state stays certified; an increment on an
    arc across the cut or any decrement takes the full repair."""
    g = gen.rmat(scale=12, seed=41)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    f0 = G.flow_value()
    side = G.min_cut()   # exact cut: recomputed by a BFS if needed
    tails = g.tails()
    crossing = (side[tails] == 1) & (side[g.col] == 0)
    rng = np.random.default_rng(41)
    off = np.flatnonzero(~crossing)
    for rep in range(2):
        ids = np.sort(rng.choice(off, 300, replace=False)).astype(np.int32)
        new = (cap[ids].astype(np.int64) + rng.integers(1, 100, ids.size)).astype(np.int32)
        G.apply_updates(ids, new)
        cap[ids] = new
        assert G.flow_value() == f0 == oracle_flow(g, cap)
        st = G.stats()
        assert st["exit_kind"] == 2 and st["bfs_levels"] == 0 and st["iterations"] == 0
    certify_gpu(G, g, cap, f0)
    xs = np.flatnonzero(crossing)
    assert xs.size > 0
    ids = xs[:4].astype(np.int32)
    new = (cap[ids].astype(np.int64) + 50).astype(np.int32)
    G.apply_updates(ids, new)
    cap[ids] = new
    f1 = G.flow_value()
    assert G.stats()["exit_kind"] != 2 and f1 == oracle_flow(g, cap) and f1 >= f0
    G.min_cut()
    ids = np.sort(rng.choice(off, 50, replace=False)).astype(np.int32)
    new = cap[ids].copy()
    new[np.flatnonzero(new > 0)[0]] -= 1      # one decrement among unchanged entries
    G.apply_updates(ids, new)
    cap[ids] = new
    assert G.flow_value() == oracle_flow(g, cap)
    assert G.stats()["exit_kind"] != 2
    certify_gpu(G, g, cap, G.flow_value())
    G.close()


@pytest.mark.parametrize("case", ["config1", "rmat12", "rmat15", "grid"])
def test_push_pull_mode(mf, case):
    """MF_MODE_PUSH_PULL (Dynamic Push-Pull, Alg. 8): every repair is a
    push-pull repair (exit_kind 3), every value equals the oracle's and every
    state passes the certificate."""
    if case == "config1":
        g = gen.random_graph(seed=81)
        mk = lambda cap, i: gen.mixed_batch(cap, 50, 1, 50, seed=81, index=i)  # noqa: E731
    elif case.startswith("rmat"):
        g = gen.rmat(scale=int(case[4:]), seed=82)
        mk = lambda cap, i: gen.mixed_batch(cap, max(10, g.m // (100 if i % 2 else 1000)), 1, 500,  # noqa: E731
                                            seed=82, index=i)
    else:
        g = gen.grid_segmentation(192, 128, seed=83)
        mk = lambda cap, i: gen.grid_rect_batch(g, seed=83, index=i, side_lo=8, side_hi=64)  # noqa: E731
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, mode=mf.MF_MODE_PUSH_PULL)
    G.solve()
    assert G.flow_value() == oracle_flow(g, cap)
    kinds = []
    for i in range(4):
        b = mk(cap, i)
        G.apply_updates(b.edge_id, b.new_cap)
        gen.apply_batch(cap, b)
        f = G.flow_value()
        kinds.append(G.stats()["exit_kind"])
        assert f == oracle_flow(g, cap), (case, i)
        if i % 2:
            certify_gpu(G, g, cap, f)
    assert set(kinds) <= {2, 3} and 3 in kinds, kinds
    G.close()


def test_push_pull_with_every_entry_point(mf):
    """A push-pull graph through the other entry points: MF_DELTA, device
    batches, a pure-increment batch off the cut (fast path), a static
    recompute, checkpoint/resume into another push-pull graph, and the
    learned policy -- every value the oracle's, states certified."""
    import torch
    g = gen.rmat(scale=12, seed=84)
    cap = g.cap.copy()
    PP = mf.MF_MODE_PUSH_PULL
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, mode=PP)
    G.solve()
    f = G.flow_value()
    assert f == oracle_flow(g, cap)
    # signed changes
    b = gen.mixed_batch(cap, 300, 1, 100, seed=84, index=0)
    delta = (b.new_cap.astype(np.int64) - cap[b.edge_id]).astype(np.int32)
    G.apply_updates(b.edge_id, delta, delta=True)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle_flow(g, cap) and G.stats()["exit_kind"] == 3
    # device batch
    b = gen.mixed_batch(cap, 300, 1, 100, seed=84, index=1)
    G.apply_updates(torch.from_numpy(b.edge_id).cuda(), torch.from_numpy(b.new_cap).cuda())
    gen.apply_batch(cap, b)
    f = G.flow_value()
    assert f == oracle_flow(g, cap)
    # increments off the exact cut: no loop, value unchanged
    side = G.min_cut()
    tails = g.tails()
    off = np.flatnonzero(~((side[tails] == 1) & (side[g.col] == 0)))
    ids = np.sort(np.random.default_rng(84).choice(off, 200, replace=False)).astype(np.int32)
    new = (cap[ids].astype(np.int64) + 7).astype(np.int32)
    G.apply_updates(ids, new)
    cap[ids] = new
    assert G.flow_value() == f == oracle_flow(g, cap) and G.stats()["exit_kind"] == 2
    # a push-pull repair right after the fast path, then a static recompute
    b = gen.mixed_batch(cap, 300, 1, 100, seed=84, index=2)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle_flow(g, cap) and G.stats()["exit_kind"] == 3
    b = gen.mixed_batch(cap, 300, 1, 100, seed=84, index=3)
    G.apply_updates(b.edge_id, b.new_cap, recompute=True)
    gen.apply_batch(cap, b)
    f = G.flow_value()
    assert f == oracle_flow(g, cap)
    certify_gpu(G, g, cap, f)
    # checkpoint into a fresh push-pull graph: its first repair falls back to
    # the plain loop (no exact cut yet), the next ones are push-pull again
    r, e, h = G.export_state()
    H = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, mode=PP)
    H.import_state(r, e, h)
    kinds = []
    for i in range(4, 7):
        b = gen.mixed_batch(cap, 300, 1, 100, seed=84, index=i)
        H.apply_updates(b.edge_id, b.new_cap)
        gen.apply_batch(cap, b)
        assert H.flow_value() == oracle_flow(g, cap)
        kinds.append(H.stats()["exit_kind"])
    assert kinds[0] != 3 and kinds[-1] == 3, kinds
    certify_gpu(H, g, cap, H.flow_value())
    # the learned policy on a push-pull graph
    from paper_2511_05895_gb300.policy import load_default_params
    H.set_policy(mf.MF_POLICY_LEARNED, load_default_params())
    for i in range(7, 9):
        b = gen.mixed_batch(cap, 300 if i == 7 else g.m // 10, 1, 100, seed=84, index=i)
        H.apply_updates(b.edge_id, b.new_cap)
        gen.apply_batch(cap, b)
        assert H.flow_value() == oracle_flow(g, cap)
    certify_gpu(H, g, cap, H.flow_value())
    G.close()
    H.close()
