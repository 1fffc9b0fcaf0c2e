"""The seeded input generators: published splitmix64 outputs, determinism and
the workload shapes the parity tests and the benchmark rely on."""
import numpy as np

from workloads import generators as gen


def test_splitmix64_published_values():
    # splitmix64 seeded with state 0 (Steele, Lea, Flood 2014; the reference
    # generator of Vigna's xoshiro page) starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4.
    z = np.array([0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) % 2 ** 64], dtype=np.uint64)
    out = gen._mix64(z)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_streams_are_deterministic_and_independent():
    a = gen.Stream(7, "x").u64(1000)
    b = gen.Stream(7, "x").u64(1000)
    c = gen.Stream(7, "y").u64(1000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    st = gen.Stream(1, "z")
    first = st.u64(10)
    rest = st.u64(10)
    assert np.array_equal(np.concatenate([first, rest]), gen.Stream(1, "z").u64(20))
    ints = gen.Stream(3, "i").integers(100000, 1, 50)
    assert ints.min() == 1 and ints.max() == 50


def test_random_graph_shape():
    g = gen.random_graph(seed=2)
    tails = g.tails()
    assert g.n == 1000 and g.m == 8000 and g.s == 0 and g.t == 999
    assert not np.any(tails == g.col)
    assert g.cap.min() >= 1 and g.cap.max() <= 100
    # the guaranteed path s -> v1 -> v2 -> t
    out_s = set(g.col[g.row_ptr[g.s]:g.row_ptr[g.s + 1]].tolist())
    assert any(g.t in set(g.col[g.row_ptr[v1]:g.row_ptr[v1 + 1]].tolist()) or
               any(g.t in set(g.col[g.row_ptr[v2]:g.row_ptr[v2 + 1]].tolist())
                   for v2 in g.col[g.row_ptr[v1]:g.row_ptr[v1 + 1]]) for v1 in out_s)


def test_rmat_shape_small():
    g = gen.rmat(scale=12, seed=3)
    deg = np.diff(g.row_ptr)
    assert g.n == 4096 and g.m <= 16 * 4096 and g.m > 15 * 4096
    assert deg[g.s] == deg.max() and g.s != g.t
    assert deg[g.t] == np.sort(deg)[-2]
    assert not np.any(g.tails() == g.col)


def test_grid_shape_small():
    W, H = 40, 30
    g = gen.grid_segmentation(W, H, seed=1)
    P = W * H
    assert g.n == P + 2 and g.s == P and g.t == P + 1
    nl = 2 * (W - 1) * H + 2 * W * (H - 1)
    assert g.m == nl + 2 * P
    assert g.cap.min() >= 0 and g.cap[g.row_ptr[P]:].max() <= 1000


def test_mixed_batch_properties():
    g = gen.random_graph(seed=5)
    b = gen.mixed_batch(g.cap, 50, 1, 50, seed=5, index=0)
    assert len(np.unique(b.edge_id)) == 50
    old = g.cap[b.edge_id]
    assert np.all(b.new_cap[:25] > old[:25]) and np.all(b.new_cap[:25] - old[:25] <= 50)
    assert np.all(b.new_cap[25:] <= old[25:]) and np.all(b.new_cap[25:] >= 0)
    b2 = gen.mixed_batch(g.cap, 50, 1, 50, seed=5, index=0)
    assert np.array_equal(b.edge_id, b2.edge_id) and np.array_equal(b.new_cap, b2.new_cap)


def test_grid_rect_batch_rewrites_terminal_links_only():
    g = gen.grid_segmentation(96, 80, seed=2)
    b = gen.grid_rect_batch(g, seed=2, index=0, side_lo=8, side_hi=32)
    tails = g.tails()
    P = 96 * 80
    ids = b.edge_id.astype(np.int64)
    assert len(np.unique(ids)) == len(ids)
    term = (tails[ids] == g.s) | (g.col[ids] == g.t)
    assert term.all()
    assert b.new_cap.min() >= 0 and b.new_cap.max() <= 1000
    k = len(ids) // 2
    assert np.array_equal(g.col[ids[:k]], tails[ids[k:]])   # same pixels, s-links then t-links
    assert P > 0
