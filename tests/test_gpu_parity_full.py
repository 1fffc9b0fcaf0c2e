"""Oracle parity of the remaining workloads and modes, on every batch.

* the unit-capacity bipartite assignment graph of the serving mix (s -> 2^20
  left vertices, 16M uniform left -> right edges, 2^20 right vertices -> t),
  at a reduced size and at full size, with +/-1 batches clamped at 0 -- many
  ties and s/t hubs of degree 2^20;
* RMAT scale 22 with a 10k and a 100k mixed batch;
* Dynamic Push-Pull on RMAT-20 (1k and 100k batches) and on the 4096^2
  segmentation grid (two rectangle batches);
* the topology-driven mode on RMAT-20;
* debug_checks on RMAT-20 in the data-driven and push-pull modes.

Every value is compared with the CPU oracle (FIFO push-relabel from scratch
on the cumulative capacities, bit-exact int64) and every final state is
certified (capacity feasibility, excess bookkeeping, saturated cut, value =
cut capacity, heights = BFS fixed point).  The batch sequence is generated
first and the oracle's values computed in parallel processes."""
import numpy as np
import pytest

from tests._helpers import certify_gpu, oracle_flows_parallel
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_05895_gb300 as pkg
    return pkg


def sequence(g, make):
    """Batches made by make(cap, i) applied to a host copy of the capacities;
    returns the batches and the capacities after each (initial first)."""
    cap = g.cap.copy()
    caps, bs = [cap.copy()], []
    for i, b in enumerate(make):
        if callable(b):
            b = b(cap)
        gen.apply_batch(cap, b)
        bs.append(b)
        caps.append(cap.copy())
    return bs, caps


def check_sequence(mf, g, bs, caps, certify_each=True, **opts):
    want = oracle_flows_parallel(g, caps)
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, **opts)
    G.solve()
    got = [G.flow_value()]
    if certify_each:
        certify_gpu(G, g, caps[0], got[0])
    kinds = []
    for b, cap in zip(bs, caps[1:]):
        G.apply_updates(b.edge_id, b.new_cap)
        got.append(G.flow_value())
        kinds.append(G.stats()["exit_kind"])
        if certify_each:
            certify_gpu(G, g, cap, got[-1])
    if not certify_each:
        certify_gpu(G, g, caps[-1], got[-1])
    G.close()
    assert got == want, (got, want)
    return kinds


def unit_batches(g, k, seed, count):
    return [lambda cap, i=i: gen.mixed_batch(cap, k, 1, 1, seed=seed, index=i) for i in range(count)]


@pytest.mark.parametrize("mode", [0, 2])
def test_bipartite_reduced(mf, mode):
    """2^12 + 2^12 vertices, 2^16 unit edges; +/-1 batches of 1 % and 0.1 %."""
    g = gen.bipartite(1 << 12, 1 << 12, 1 << 16, seed=81)
    bs, caps = sequence(g, [lambda cap, i=i: gen.mixed_batch(cap, g.m // (100 if i % 2 else 1000), 1, 1,
                                                           seed=81, index=i) for i in range(5)])
    check_sequence(mf, g, bs, caps, mode=mode)


@pytest.mark.slow
def test_bipartite_full_size(mf):
    """The serving mix's assignment graph at full size: 10k and 100k +/-1 batches."""
    g = gen.bipartite(seed=308)
    bs, caps = sequence(g, [lambda cap: gen.mixed_batch(cap, 10_000, 1, 1, seed=308, index=0),
                            lambda cap: gen.mixed_batch(cap, 100_000, 1, 1, seed=308, index=1)])
    check_sequence(mf, g, bs, caps, kernel_cycles=4)


@pytest.mark.slow
def test_rmat22(mf):
    """RMAT scale 22 (4.2M vertices, 67M edges): 10k and 100k mixed batches."""
    g = gen.rmat(scale=22, seed=304)
    bs, caps = sequence(g, [lambda cap: gen.mixed_batch(cap, 10_000, 1, 500, seed=304, index=0),
                            lambda cap: gen.mixed_batch(cap, 100_000, 1, 500, seed=304, index=1)])
    check_sequence(mf, g, bs, caps, certify_each=False, kernel_cycles=4)


@pytest.mark.slow
def test_push_pull_rmat20(mf):
    """Dynamic Push-Pull on the benchmark graph: 1k and 100k mixed batches,
    every repair a push-pull repair (exit kind 3)."""
    g = gen.rmat(scale=20, seed=1)
    bs, caps = sequence(g, [lambda cap: gen.mixed_batch(cap, 1000, 1, 500, seed=1, index=0),
                            lambda cap: gen.mixed_batch(cap, 100_000, 1, 500, seed=1, index=1)])
    kinds = check_sequence(mf, g, bs, caps, kernel_cycles=4, mode=mf.MF_MODE_PUSH_PULL)
    assert set(kinds) <= {2, 3}, kinds


@pytest.mark.slow
def test_push_pull_grid4096(mf):
    """Dynamic Push-Pull on the 4096^2 segmentation grid, two rectangles."""
    g = gen.grid_segmentation(4096, 4096, seed=3)
    rects = [gen.grid_rect_batch(g, seed=3, index=i) for i in range(2)]
    bs, caps = sequence(g, rects)
    kinds = check_sequence(mf, g, bs, caps, certify_each=False, kernel_cycles=4, mode=mf.MF_MODE_PUSH_PULL)
    assert set(kinds) <= {2, 3}, kinds


@pytest.mark.slow
def test_topology_mode_rmat20(mf):
    """The topology-driven mode on the benchmark graph: 1k and 100k batches."""
    g = gen.rmat(scale=20, seed=1)
    bs, caps = sequence(g, [lambda cap: gen.mixed_batch(cap, 1000, 1, 500, seed=1, index=0),
                            lambda cap: gen.mixed_batch(cap, 100_000, 1, 500, seed=1, index=1)])
    check_sequence(mf, g, bs, caps, kernel_cycles=4, mode=mf.MF_MODE_TOPOLOGY)


@pytest.mark.slow
@pytest.mark.parametrize("mode", [0, 2])
def test_debug_checks_rmat20(mf, mode):
    """debug_checks at full size: the end-of-kernel recount of every excess,
    residual pair and mirror entry, and the bounds checks of list entries,
    pass on three 100k-edge batches of the benchmark graph in the
    data-driven and the push-pull mode (a failed check makes flow_value
    raise MF_ECHECK); every value is the oracle's."""
    g = gen.rmat(scale=20, seed=1)
    bs, caps = sequence(g, [lambda cap, i=i: gen.mixed_batch(cap, 100_000, 1, 500, seed=7, index=i)
                            for i in range(3)])
    check_sequence(mf, g, bs, caps, certify_each=False, kernel_cycles=4, mode=mode, debug_checks=True)
