"""The learned batch policy on the GPU.

* the CUDA training kernels' loss and gradient equal the float64 oracle's
  (oracle/mlp.py, itself pinned by finite differences);
* training reduces the loss;
* the device features equal their definition computed here from the batch;
* the plain rule and the network choose repair or recompute, KERNELCYCLES
  and the processing mode as specified, fall back on out-of-range inputs,
  and every solve stays exact (oracle value on every batch);
* on the committed log of the method's own runs, the trained network's
  decisions cost less time on held-out workloads than the plain rule's and
  than the best fixed processing mode.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from workloads import generators as gen

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2511_05895_gb300",
                    "policy_log.npz")


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_05895_gb300 as pkg
    return pkg


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def test_mlp_grad_and_forward_match_oracle(mf):
    import torch
    L = mf.lib()
    rng = np.random.default_rng(5)
    n = 700
    P = omlp.init_params(rng, mu=rng.normal(0, 1, 12), sd=rng.uniform(0.5, 2, 12))
    P[omlp.O_B1:omlp.O_W2] = rng.normal(0, 0.1, 64)
    X = rng.normal(0, 1.5, (n, 12))
    T0 = (rng.uniform(size=n) < 0.4).astype(np.float64)
    T1 = rng.uniform(0, 4, n)
    T2 = rng.integers(0, omlp.K_MODES, n).astype(np.float64)
    wkc, wmode = 0.5, 0.7
    P32 = P.astype(np.float32)
    tP, tX, tT0, tT1, tT2 = _dev(P32), _dev(X), _dev(T0), _dev(T1), _dev(T2)
    g = torch.zeros(omlp.N_TRAINED, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(int(L.mf_mlp_workspace_bytes(n)) // 4 + 1, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mf_mlp_grad(p(tP), p(tX), p(tT0), p(tT1), p(tT2), n, wkc, wmode, p(g), p(loss), p(ws), st) == 0
    torch.cuda.synchronize()
    # the oracle sees the same float32-rounded parameters and inputs
    Lw, gw = omlp.loss_and_grad(P32.astype(np.float64), X.astype(np.float32).astype(np.float64),
                                T0, T1.astype(np.float32).astype(np.float64), T2, wkc, wmode)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - Lw) <= 1e-5 * max(1.0, abs(Lw))
    assert np.max(np.abs(gg - gw)) <= 1e-4 * np.max(np.abs(gw)) + 1e-7
    from paper_2511_05895_gb300 import policy
    Y = policy.forward(P32, X.astype(np.float32))
    Yw = omlp.forward(P32.astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(Y - Yw)) <= 1e-4 * (1 + np.max(np.abs(Yw)))


def test_mlp_training_reduces_loss(mf):
    from paper_2511_05895_gb300 import policy
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, (2048, 12)).astype(np.float32)
    T0 = (X[:, 0] + 0.5 * X[:, 3] > 0).astype(np.float32)
    T1 = np.clip(2 + X[:, 1], 0, 4).astype(np.float32)
    T2 = np.where(X[:, 2] > 0.5, 2, np.where(X[:, 4] > 0, 1, 0)).astype(np.float32)
    P, hist = policy.train(X, T0, T1, T2, steps=1500, batch=128, lr=3e-3, wkc=0.5, wmode=0.5, seed=1)
    assert hist[-100:].mean() < 0.5 * hist[:20].mean()
    Y = policy.forward(P, X)
    assert np.mean((Y[:, 0] > 0) == (T0 > 0.5)) > 0.9
    assert np.mean(Y[:, 2:5].argmax(axis=1) == T2) > 0.9


def test_policy_features_match_their_definition(mf):
    g = gen.rmat(scale=12, seed=7)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    flow = G.flow_value()
    st = G.stats()
    b = gen.mixed_batch(cap, 500, 1, 500, seed=7, index=0)
    f = G.policy_features(b.edge_id, b.new_cap)
    tails = g.tails()
    ids = b.edge_id.astype(np.int64)
    old = cap[ids].astype(np.int64)
    new = b.new_cap.astype(np.int64)
    touch = (tails[ids] == g.s) | (g.col[ids] == g.t)
    B = mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    A = B["head"].shape[0]
    want = np.array([np.log2(g.n), np.log2(g.m), np.log2(1 + 500), 500 / g.m, np.mean(new > old),
                     np.mean(touch), np.log2(1 + np.abs(new - old).sum()), np.log2(1 + flow), A / g.n,
                     np.log2(1 + np.diff(B["arc_row"]).max()), st["iterations"],
                     st["bfs_vertices"] / ((st["iterations"] + 1) * g.n)], np.float64)
    assert np.allclose(f, want, rtol=1e-5, atol=1e-5), (f, want)
    G.close()


def test_plain_and_learned_decisions_stay_exact(mf):
    g = gen.rmat(scale=12, seed=8)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    G.solve()
    G.set_policy(mf.MF_POLICY_PLAIN)
    small = gen.mixed_batch(cap, g.m // 200, 1, 500, seed=8, index=0)
    G.apply_updates(small.edge_id, small.new_cap)
    gen.apply_batch(cap, small)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    s = G.stats()
    assert s["policy_kind"] == 0 and s["policy_kernel_cycles"] == s["kernel_cycles"]
    big = gen.mixed_batch(cap, g.m // 20, 1, 500, seed=8, index=1)
    G.apply_updates(big.edge_id, big.new_cap)
    gen.apply_batch(cap, big)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    assert G.stats()["policy_kind"] == 1
    # a network whose outputs are its last biases: recompute, KERNELCYCLES 2^3
    P = np.zeros(omlp.N_TOTAL, np.float32)
    P[omlp.O_B3:omlp.N_TRAINED] = [-4.0, 3.2, 0.0, 1.0, 0.5]   # mode: topology-driven
    P[omlp.O_SD:] = 1e6                       # every feature normalises to ~0
    G.set_policy(mf.MF_POLICY_LEARNED, P)
    b = gen.mixed_batch(cap, 50, 1, 500, seed=8, index=2)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    s = G.stats()
    assert (s["policy_kind"], s["policy_kernel_cycles"], s["policy_fallback"]) == (1, 8, 0)
    # repair (logit > 0), KERNELCYCLES 2, topology-driven: exact as well
    P[omlp.O_B3:omlp.N_TRAINED] = [4.0, 1.0, 0.0, 1.0, 0.5]
    G.set_policy(mf.MF_POLICY_LEARNED, P)
    b = gen.mixed_batch(cap, 50, 1, 500, seed=8, index=4)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    s = G.stats()
    assert (s["policy_kind"], s["policy_kernel_cycles"], s["policy_mode"]) == (0, 2, mf.MF_MODE_TOPOLOGY)
    # push-pull chosen on a graph without the push-pull state: the better of
    # the other two (here data-driven)
    P[omlp.O_B3:omlp.N_TRAINED] = [4.0, 1.0, 0.7, 0.2, 3.0]
    G.set_policy(mf.MF_POLICY_LEARNED, P)
    b = gen.mixed_batch(cap, 50, 1, 500, seed=8, index=5)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    assert G.stats()["policy_mode"] == mf.MF_MODE_DATA_DRIVEN
    # out-of-range input: fall back to the plain rule
    P[omlp.O_SD:] = 1e-6
    G.set_policy(mf.MF_POLICY_LEARNED, P)
    b = gen.mixed_batch(cap, 50, 1, 500, seed=8, index=3)
    G.apply_updates(b.edge_id, b.new_cap)
    gen.apply_batch(cap, b)
    assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
    s = G.stats()
    assert s["policy_fallback"] == 1 and s["policy_kind"] == 0
    G.close()


def test_learned_mode_choice_on_a_push_pull_graph(mf):
    """On a graph created with MF_MODE_PUSH_PULL the network's mode output
    picks any of the three modes per batch; every value is the oracle's and
    the chosen mode is reported (a push-pull repair ends with exit kind 3)."""
    g = gen.rmat(scale=12, seed=10)
    cap = g.cap.copy()
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, mode=mf.MF_MODE_PUSH_PULL)
    G.solve()
    P = np.zeros(omlp.N_TOTAL, np.float32)
    P[omlp.O_SD:] = 1e6
    for j, mode in enumerate([2, 0, 1, 2, 1, 0]):
        logits = [0.0, 0.0, 0.0]
        logits[mode] = 2.0
        P[omlp.O_B3:omlp.N_TRAINED] = [4.0, 2.0, *logits]
        G.set_policy(mf.MF_POLICY_LEARNED, P)
        b = gen.mixed_batch(cap, g.m // 300, 1, 500, seed=10, index=j)
        G.apply_updates(b.edge_id, b.new_cap)
        gen.apply_batch(cap, b)
        assert G.flow_value() == oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        s = G.stats()
        assert s["policy_mode"] == mode and s["policy_fallback"] == 0
        if mode == 2:
            assert s["exit_kind"] in (2, 3)
    G.close()


@pytest.mark.skipif(not os.path.exists(DATA), reason="no committed policy log")
def test_trained_policy_beats_plain_rule_on_held_out_workloads(mf):
    """Train on the committed log (every 4th workload held out) with the CUDA
    kernels and replay the held-out batches: the network's choices must cost
    less device time than the plain rule's and than always repairing in the
    best fixed processing mode."""
    from paper_2511_05895_gb300 import policy
    d = np.load(DATA)
    if "t_pp" not in d:
        pytest.skip("the committed log predates the mode output")
    held = d["group"] % 4 == 3
    T0, T1, T2 = policy.labels(d)
    P, hist = policy.train(d["X"][~held], T0[~held], T1[~held], T2[~held], steps=6000, seed=0)
    r = policy.evaluate({k: d[k][held] for k in policy.LOG_KEYS}, P)
    assert r["learned_ms"] < r["plain_ms"], r
    assert r["learned_ms"] < r["best_fixed_mode_ms"], r
    assert r["learned_ms"] >= r["best_ms"]
