"""Pins of the CPU oracle against things other than itself.

Each pin would fail for a plausible bug in the oracle: a dropped reverse arc,
a wrong sign in a push, a transposed edge direction, a global relabel that
walks arcs the wrong way, or a certificate check that accepts a bad state.

* brute-force enumeration of every s-t cut (max-flow = min-cut), written here
  in Python, independent of the oracle's C code;
* scipy.sparse.csgraph.maximum_flow (a library routine);
* closed forms: path, disjoint paths, grid with no n-links, unit bipartite
  graph (= maximum matching, scipy's Hopcroft-Karp), disconnected graphs;
* textbook flow networks with published values (tests/golden/);
* certificate self-check of the oracle's own final state, and planted
  mistakes that each certificate bit must catch;
* BFS heights against scipy's unweighted shortest paths.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import maximum_bipartite_matching, maximum_flow, shortest_path

import oracle
from workloads import generators as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_mincut_py(n, tails, heads, caps, s, t):
    others = [v for v in range(n) if v not in (s, t)]
    best = None
    for bits in itertools.product((0, 1), repeat=len(others)):
        S = {s} | {v for v, b in zip(others, bits) if b}
        c = sum(int(cp) for u, v, cp in zip(tails, heads, caps) if u in S and v not in S)
        best = c if best is None else min(best, c)
    return best


def scipy_flow(g):
    M = sp.csr_matrix((g.cap.astype(np.int64), (g.tails(), g.col.astype(np.int64))), shape=(g.n, g.n))
    M.sum_duplicates()
    M.setdiag(0)
    M.eliminate_zeros()
    return int(maximum_flow(M.astype(np.int32), g.s, g.t).flow_value)


def tiny_graph(rng, n, m, cap_hi):
    tails = rng.integers(0, n, m)
    heads = rng.integers(0, n, m)      # self-loops allowed: they must be ignored
    caps = rng.integers(0, cap_hi + 1, m)
    s, t = rng.choice(n, 2, replace=False)
    return gen.from_edges(n, tails, heads, caps, int(s), int(t))


def test_tiny_graphs_vs_python_bruteforce():
    rng = np.random.default_rng(12345)
    for trial in range(600):
        n = int(rng.integers(2, 9))
        m = int(rng.integers(0, 3 * n + 1))
        g = tiny_graph(rng, n, m, 5)
        tails = g.tails()
        want = brute_mincut_py(g.n, tails, g.col, g.cap, g.s, g.t)
        assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want, trial
        assert oracle.maxflow_ek(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want, trial
        assert oracle.mincut_brute(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want, trial


def test_small_graphs_c_bruteforce():
    rng = np.random.default_rng(7)
    for trial in range(100):
        n = int(rng.integers(10, 15))
        g = tiny_graph(rng, n, int(rng.integers(n, 5 * n)), 9)
        want = oracle.mincut_brute(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
        assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want


@pytest.mark.parametrize("seed", range(8))
def test_random_graph_vs_scipy(seed):
    g = gen.random_graph(seed=seed)
    want = scipy_flow(g)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want
    assert oracle.maxflow_ek(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want


@pytest.mark.parametrize("scale,seed", [(10, 1), (12, 2)])
def test_rmat_vs_scipy(scale, seed):
    g = gen.rmat(scale=scale, seed=seed)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == scipy_flow(g)


def test_grid_vs_scipy():
    g = gen.grid_segmentation(48, 40, seed=3)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == scipy_flow(g)


def test_closed_form_path():
    caps = [7, 3, 9, 4, 11]
    n = len(caps) + 1
    g = gen.from_edges(n, range(n - 1), range(1, n), caps, 0, n - 1)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == min(caps)


def test_closed_form_disjoint_paths():
    rng = np.random.default_rng(3)
    tails, heads, caps, want = [], [], [], 0
    n, s, t = 2, 0, 1
    for _ in range(12):
        L = int(rng.integers(1, 6))
        cs = rng.integers(1, 50, L + 1)
        verts = [s] + list(range(n, n + L)) + [t]
        n += L
        for a, b, c in zip(verts[:-1], verts[1:], cs):
            tails.append(a); heads.append(b); caps.append(int(c))
        want += int(cs.min())
    g = gen.from_edges(n, tails, heads, caps, s, t)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want
    assert oracle.maxflow_ek(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want


def test_closed_form_grid_without_nlinks():
    g = gen.grid_segmentation(64, 48, seed=5)
    tails = g.tails()
    P = g.meta["W"] * g.meta["H"]
    nlink = (tails < P) & (g.col < P)
    cap = g.cap.copy()
    cap[nlink] = 0
    cap_t = np.zeros(P, np.int64)
    cap_s = np.zeros(P, np.int64)
    tl = (tails < P) & (g.col == g.t)
    cap_t[tails[tl]] = cap[tl]
    sl = tails == g.s
    cap_s[g.col[sl]] = cap[sl]
    want = int(np.minimum(cap_s, cap_t).sum())
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t) == want


def test_closed_form_unit_bipartite_matching():
    rng = np.random.default_rng(11)
    L, R, E = 300, 280, 1200
    lu = rng.integers(0, L, E)
    rv = rng.integers(0, R, E)
    s, t = L + R, L + R + 1
    tails = np.concatenate([np.full(L, s), lu, L + np.arange(R)])
    heads = np.concatenate([np.arange(L), L + rv, np.full(R, t)])
    g = gen.from_edges(L + R + 2, tails, heads, np.ones(len(tails), np.int64), s, t)
    B = sp.csr_matrix((np.ones(E, np.int8), (lu, rv)), shape=(L, R))
    B.sum_duplicates()
    match = maximum_bipartite_matching(B, perm_type="column")
    want = int((match >= 0).sum())
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want


def test_closed_form_no_path_and_zero_caps():
    g = gen.from_edges(5, [0, 1, 3], [1, 2, 4], [5, 5, 5], 0, 4)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == 0
    g = gen.from_edges(3, [0, 1], [1, 2], [0, 0], 0, 2)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == 0
    g = gen.from_edges(2, [0, 0, 0, 1], [1, 1, 0, 0], [3, 4, 9, 8], 0, 1)   # parallel + loop + back
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == 7


def read_golden(name):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    n, s, t, want = map(int, rows[0])
    e = np.array([list(map(int, r)) for r in rows[1:]], dtype=np.int64)
    return gen.from_edges(n, e[:, 0], e[:, 1], e[:, 2], s, t), want


@pytest.mark.parametrize("name", ["clrs_fig26_1.txt", "ff_worst_case.txt"])
def test_golden_textbook_networks(name):
    g, want = read_golden(name)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want
    assert oracle.maxflow_ek(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want
    assert oracle.mincut_brute(g.n, g.row_ptr, g.col, g.cap, g.s, g.t) == want


def _oracle_state(g):
    f, st = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, want_state=True)
    side = (st.height >= g.n).astype(np.uint8)
    return f, st, side


def _cert(g, st, side, f, height=None, cap=None):
    return oracle.certify(g.n, g.row_ptr, g.col, g.cap if cap is None else cap, g.s, g.t,
                          st.arc_row, st.head, st.rev, st.cap, st.r, st.excess, side, f, height)


@pytest.mark.parametrize("seed", range(4))
def test_certificate_accepts_oracle_state(seed):
    g = gen.random_graph(seed=seed)
    f, st, side = _oracle_state(g)
    assert _cert(g, st, side, f, st.height)[0] == 0


def test_certificate_catches_planted_mistakes():
    g = gen.random_graph(seed=1)
    f, st, side = _oracle_state(g)
    # wrong value
    assert "VALUE" in _cert(g, st, side, f + 1)[2]
    # residual below zero / not conserving the pair
    bad = oracle.OracleState(**{k: v.copy() for k, v in st.__dict__.items()})
    a = int(np.flatnonzero(bad.r > 0)[0])
    bad.r[a] += 1
    assert "RESID" in _cert(g, bad, side, f)[2]
    # excess bookkeeping
    bad = oracle.OracleState(**{k: v.copy() for k, v in st.__dict__.items()})
    v = next(x for x in range(g.n) if x not in (g.s, g.t))
    bad.excess[v] += 1
    assert "EXCESS" in _cert(g, bad, side, f)[2]
    # arc capacity disagreeing with the edge list
    cap2 = g.cap.copy()
    cap2[5] += 1
    assert "CAPS" in _cert(g, st, side, f, cap=cap2)[2]
    # a T vertex that still has a residual arc from S: move t's predecessor set
    side2 = side.copy()
    side2[g.t] = 1
    assert "CUT" in _cert(g, st, side2, f)[2]
    # moving a source-side vertex with excess into T breaks the sign condition
    # or the cut; both are failures
    sv = [v for v in range(g.n) if side[v] and v != g.s and st.excess[v] > 0]
    if sv:
        side3 = side.copy()
        side3[sv[0]] = 0
        assert _cert(g, st, side3, f)[0] != 0
    # heights that are not the BFS fixed point
    h2 = st.height.copy()
    w = next(x for x in range(g.n) if x not in (g.s, g.t))
    h2[w] = h2[w] + 1 if h2[w] < g.n else 1
    assert "HEIGHTS" in _cert(g, st, side, f, h2)[2]
    # broken pairing
    bad = oracle.OracleState(**{k: v.copy() for k, v in st.__dict__.items()})
    bad.rev[0], bad.rev[1] = bad.rev[1], bad.rev[0]
    assert "STRUCT" in _cert(g, bad, side, f)[2]


def _hand_state(n, tails, heads, caps, s, t, flow_on_edge):
    """A state written out by hand: one arc pair per input edge (tail -> head
    listed first), the given flow on each edge, residuals and excesses derived
    from it (excess = inflow - outflow)."""
    g = gen.from_edges(n, tails, heads, caps, s, t)
    out = [[] for _ in range(n)]
    for i, (u, v, c, f) in enumerate(zip(tails, heads, caps, flow_on_edge)):
        out[u].append((v, c - f, c, 2 * i))       # forward arc: residual c - f
        out[v].append((u, f, 0, 2 * i + 1))       # reverse arc: residual f
    arc_row = np.zeros(n + 1, np.int64)
    head, r, capa, key = [], [], [], []
    for u in range(n):
        for v, res, c, k in out[u]:
            head.append(v); r.append(res); capa.append(c); key.append(k)
        arc_row[u + 1] = len(head)
    pos = {k: a for a, k in enumerate(key)}
    rev = np.array([pos[k ^ 1] for k in key], np.int64)
    ex = np.zeros(n, np.int64)
    for u, v, f in zip(tails, heads, flow_on_edge):
        ex[v] += f
        ex[u] -= f
    st = oracle.OracleState(arc_row=arc_row, head=np.array(head, np.int32), rev=rev,
                            cap=np.array(capa, np.int64), r=np.array(r, np.int64), excess=ex,
                            height=np.zeros(n, np.int32))
    return g, st


def test_certificate_signs_bit_alone():
    """States whose only defect is the sign condition: every other bit holds
    (residual pairs, excess = net inflow with sum 0, no residual arc from S to
    T, value = sum over T of the excess = capacity of the cut)."""
    # a deficit on the source side: s -> a (5), a -> t (1) carrying flow 0 and
    # 1; S = {s, a}: e(a) = -1, e(t) = 1 = C(S, T)
    g, st = _hand_state(3, [0, 1], [1, 2], [5, 1], 0, 2, [0, 1])
    side = np.array([1, 1, 0], np.uint8)
    bits, _, names = _cert(g, st, side, 1)
    assert names == ["SIGNS"], names
    # an excess on the sink side: s -> a (1), a -> t (5) carrying flow 1 and
    # 0; S = {s}: e(a) = 1 sits in T, sum over T = 1 = C(S, T)
    g, st = _hand_state(3, [0, 1], [1, 2], [1, 5], 0, 2, [1, 0])
    side = np.array([1, 0, 0], np.uint8)
    bits, _, names = _cert(g, st, side, 1)
    assert names == ["SIGNS"], names
    # the same graphs with the flow completed are certified
    g, st = _hand_state(3, [0, 1], [1, 2], [5, 1], 0, 2, [1, 1])
    assert _cert(g, st, np.array([1, 1, 0], np.uint8), 1)[0] == 0


def test_bfs_heights_vs_scipy():
    rng = np.random.default_rng(5)
    g = gen.random_graph(n=300, m=1500, seed=9)
    f, st = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, want_state=True)
    root = np.zeros(g.n, np.uint8)
    root[g.t] = 1
    root[rng.choice(g.n, 5, replace=False)] = 1
    root[g.s] = 0
    h = oracle.bfs_heights(g.n, st.arc_row, st.head, st.rev, st.r, root, g.s)
    # distances to roots in the residual graph without s: reverse the residual arcs and
    # run an unweighted shortest path from a super-root joined to every root
    A = st.head.shape[0]
    tails = np.repeat(np.arange(g.n), np.diff(st.arc_row))
    keep = (st.r > 0) & (tails != g.s) & (st.head != g.s)
    rows = np.concatenate([st.head[keep], np.full(int(root.sum()), g.n)])
    cols = np.concatenate([tails[keep], np.flatnonzero(root)])
    R = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(g.n + 1, g.n + 1))
    d = shortest_path(R, unweighted=True, indices=g.n)
    want = np.where(np.isinf(d[:g.n]), g.n, d[:g.n] - 1).astype(np.int64)
    want[g.s] = g.n
    assert A > 0 and np.array_equal(h.astype(np.int64), want)


def test_update_monotonicity_bounds():
    """F_old - sum|dec| <= F_new <= F_old + sum inc, and a pure increment batch
    never lowers F (capacities only grow), a pure decrement never raises it."""
    g = gen.random_graph(seed=4)
    cap = g.cap.copy()
    f_old = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    for idx in range(6):
        b = gen.mixed_batch(cap, 50, 1, 50, seed=4, index=idx)
        old = cap[b.edge_id].astype(np.int64)
        inc = np.maximum(b.new_cap - old, 0).sum()
        dec = np.maximum(old - b.new_cap, 0).sum()
        gen.apply_batch(cap, b)
        f_new = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        assert f_old - dec <= f_new <= f_old + inc
        f_old = f_new
    up = cap.copy()
    up[::7] += 5
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, up, g.s, g.t) >= f_old
    down = cap.copy()
    down[::7] = np.maximum(down[::7] - 5, 0)
    assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, down, g.s, g.t) <= f_old


def test_increments_off_the_min_cut_leave_the_value():
    """Raising capacities of edges that do not go from S to T of a minimum cut
    (S = vertices that cannot reach t in the final residual graph, found here
    by scipy's BFS) leaves the maximum flow unchanged; raising one edge that
    does cross can raise it, never by more than the increment."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    for seed in range(4):
        g = gen.rmat(scale=9, seed=300 + seed)
        cap = g.cap.copy()
        f, st = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t, want_state=True)
        tails = np.repeat(np.arange(g.n), np.diff(st.arc_row))
        res = st.r > 0
        # reverse residual graph: who can reach t
        R = csr_matrix((np.ones(int(res.sum())), (st.head[res], tails[res])), shape=(g.n, g.n))
        reach = np.zeros(g.n, bool)
        reach[breadth_first_order(R, g.t, directed=True, return_predecessors=False)] = True
        S = ~reach
        assert S[g.s] and not S[g.t]
        et = g.tails()
        crossing = S[et] & ~S[g.col]
        assert int(cap[crossing].astype(np.int64).sum()) == f      # it is a minimum cut
        rng = np.random.default_rng(seed)
        up = cap.copy()
        off = np.flatnonzero(~crossing)
        pick = rng.choice(off, min(200, off.size), replace=False)
        up[pick] += rng.integers(1, 1000, pick.size).astype(np.int32)
        assert oracle.maxflow_fifo(g.n, g.row_ptr, g.col, up, g.s, g.t) == f
        e = np.flatnonzero(crossing)[0]
        up = cap.copy()
        up[e] += 7
        f2 = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, up, g.s, g.t)
        assert f <= f2 <= f + 7


# ---- the policy network oracle -------------------------------------------
from oracle import mlp as omlp  # noqa: E402


def _mlp_case(seed, n=40):
    rng = np.random.default_rng(seed)
    P = omlp.init_params(rng, mu=rng.normal(0, 1, 12), sd=rng.uniform(0.5, 2.0, 12))
    P[omlp.O_B1:omlp.O_W2] = rng.normal(0, 0.1, 64)   # biases away from 0 (ReLU kinks)
    P[omlp.O_B2:omlp.O_W3] = rng.normal(0, 0.1, 64)
    X = rng.normal(0, 1.5, (n, 12))
    T0 = (rng.uniform(size=n) < 0.5).astype(np.float64)
    T1 = rng.uniform(0, 5, n)
    T2 = rng.integers(0, omlp.K_MODES, n).astype(np.float64)
    return P, X, T0, T1, T2


def test_mlp_gradient_matches_central_differences():
    P, X, T0, T1, T2 = _mlp_case(1)
    L, g = omlp.loss_and_grad(P, X, T0, T1, T2, 0.3, 0.7)
    assert abs(L - omlp.loss(P, X, T0, T1, T2, 0.3, 0.7)) < 1e-12
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(omlp.N_TRAINED, 120, replace=False),
                          np.arange(omlp.O_W3, omlp.O_B3, 13),   # weights of every output
                          np.arange(omlp.O_B3, omlp.N_TRAINED)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (omlp.loss(Pp, X, T0, T1, T2, 0.3, 0.7) - omlp.loss(Pm, X, T0, T1, T2, 0.3, 0.7)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_closed_form_with_zero_output_weights():
    """With W3 = 0 the outputs are the biases: the loss and the gradient of b3
    have closed forms."""
    P, X, T0, T1, T2 = _mlp_case(3)
    P[omlp.O_W3:omlp.O_B3] = 0.0
    c0, c1 = 0.7, -1.2
    cm = np.array([0.3, -0.4, 1.1])               # the mode logits
    P[omlp.O_B3:omlp.N_TRAINED] = [c0, c1, *cm]
    wm = 0.5
    L, g = omlp.loss_and_grad(P, X, T0, T1, T2, 2.0, wm)
    # closed form of the cross-entropy of constant logits: log-sum-exp minus
    # the mean logit of the target classes; its gradient is the softmax
    # minus the class frequencies
    lse = np.log(np.exp(cm).sum())
    freq = np.array([np.mean(T2 == c) for c in range(3)])
    want = (np.log1p(np.exp(c0)) - T0.mean() * c0 + 0.5 * 2.0 * np.mean((c1 - T1) ** 2)
            + wm * (lse - (freq * cm).sum()))
    assert abs(L - want) < 1e-12
    assert abs(g[omlp.O_B3] - (1 / (1 + np.exp(-c0)) - T0.mean())) < 1e-12
    assert abs(g[omlp.O_B3 + 1] - 2.0 * np.mean(c1 - T1)) < 1e-12
    assert np.allclose(g[omlp.O_B3 + 2:omlp.N_TRAINED], wm * (np.exp(cm) / np.exp(cm).sum() - freq), atol=1e-12)
    assert np.all(g[:omlp.O_W3] == 0.0)          # nothing reaches the hidden layers
