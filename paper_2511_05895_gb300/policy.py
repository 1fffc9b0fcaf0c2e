"""The learned batch policy: logging, training and evaluation.

The paper observes that the dynamic repair wins for small batches and a
static recompute wins past a crossover (Sec. 6.5), that KERNELCYCLES trades
pushes against global relabels (Note 2 of Sec. 3), and that the processing
mode matters: topology-driven processing can beat the worklist when many
vertices are active, and push-pull helps on large graphs (Sec. 6.5).  A small
network (csrc/mf_mlp.cuh) predicts the three choices from 12 batch features
(mf_policy_features); the library evaluates it on the device before each
repair when the graph's policy is MF_POLICY_LEARNED, and falls back to the
plain rule on unusual inputs.

* ``collect``  runs the method itself on seeded workloads and logs, per
  batch, the features and the device time of the data-driven repair at each
  KERNELCYCLES value of ``KC_CHOICES``, of the topology-driven and the
  Dynamic Push-Pull repair (KERNELCYCLES 4), and of a static recompute;
* ``train``    fits the network with the library's own CUDA kernels
  (mf_mlp_train: forward, backward and Adam on the GPU);
* ``evaluate`` replays logged batches: total time of the decisions of the
  learned policy against the plain rule (and the best possible choice).

Every repair and recompute during collection is still an exact solve; the
flow values of all instances are compared batch by batch.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native
from ._native import MaxFlowGraph, lib

KC_CHOICES = (1, 2, 4, 8, 16)
KC_STATIC = 4
MODE_NAMES = ("data-driven", "topology", "push-pull")   # network outputs 2, 3, 4 (MF_MODE_*)
PARAMS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy_params.npy")
N_IN = 12


def sizes():
    a, b, c, d = (ctypes.c_int32() for _ in range(4))
    lib().mf_mlp_sizes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return a.value, b.value, c.value, d.value


def load_default_params():
    """The committed trained parameters, or None."""
    return np.load(PARAMS_PATH).astype(np.float32) if os.path.exists(PARAMS_PATH) else None


# ---------------------------------------------------------------- logging --
def _time_apply(G, ids, caps, recompute=False):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    G.apply_updates(ids, caps, recompute=recompute)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def collect_graph(g, batches, group, log):
    """Run every batch of ``batches`` (iterable of workloads.generators.Batch,
    applied cumulatively) through one data-driven graph instance per KC
    choice, a topology-driven and a Dynamic Push-Pull instance, and a
    static-recompute instance; append rows to ``log`` (dict of lists)."""
    import torch
    from ._native import MF_MODE_PUSH_PULL, MF_MODE_TOPOLOGY
    inst = [MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=kc) for kc in KC_CHOICES]
    topo = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=KC_STATIC, mode=MF_MODE_TOPOLOGY)
    pp = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=KC_STATIC, mode=MF_MODE_PUSH_PULL)
    stat = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=KC_STATIC)
    every = inst + [topo, pp, stat]
    for G in every:
        G.solve()
    flows = {G.flow_value() for G in every}
    assert len(flows) == 1, flows
    observer = inst[KC_CHOICES.index(4)]
    for b in batches:
        ids = torch.from_numpy(b.edge_id).cuda()
        caps = torch.from_numpy(b.new_cap).cuda()
        feats = observer.policy_features(ids, caps)
        t_dyn = [_time_apply(G, ids, caps) for G in inst]
        t_topo = _time_apply(topo, ids, caps)
        t_pp = _time_apply(pp, ids, caps)
        t_st = _time_apply(stat, ids, caps, recompute=True)
        flows = {G.flow_value() for G in every}
        assert len(flows) == 1, flows                 # every choice is exact
        log["X"].append(feats)
        log["t_dyn"].append(t_dyn)
        log["t_topo"].append(t_topo)
        log["t_pp"].append(t_pp)
        log["t_static"].append(t_st)
        log["group"].append(group)
        log["k"].append(len(b.edge_id))
    for G in every:
        G.close()


LOG_KEYS = ("X", "t_dyn", "t_topo", "t_pp", "t_static")


def mode_times(data):
    """[n x 3] repair times per mode: data-driven at its best KERNELCYCLES,
    topology-driven and push-pull at KC_STATIC."""
    return np.stack([data["t_dyn"].min(axis=1), data["t_topo"], data["t_pp"]], axis=1)


def labels(data):
    """Targets: T0 = 1 if the best repair (any mode, any logged KC) beats the
    static recompute, T1 = log2 of the best KERNELCYCLES of the data-driven
    repair, T2 = the index of the fastest mode."""
    mt = mode_times(data)
    T0 = (mt.min(axis=1) < data["t_static"]).astype(np.float32)
    T1 = np.log2(np.asarray(KC_CHOICES, np.float32)[data["t_dyn"].argmin(axis=1)])
    T2 = mt.argmin(axis=1).astype(np.float32)
    return T0, T1, T2


# --------------------------------------------------------------- training --
def train(X, T0, T1, T2=None, steps=6000, batch=256, lr=2e-3, wkc=0.25, wmode=0.5, seed=0):
    """Fit the network on the GPU with mf_mlp_train; returns float32 params.
    T2 (the mode class) may be None: the mode outputs are then not trained."""
    import torch
    n_in, n_out, n_tr, n_tot = sizes()
    X = np.asarray(X, np.float32)
    if T2 is None:
        T2, wmode = np.zeros(X.shape[0], np.float32), 0.0
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    X, T0, T1 = X[perm], np.asarray(T0, np.float32)[perm], np.asarray(T1, np.float32)[perm]
    T2 = np.asarray(T2, np.float32)[perm]
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd < 1e-3] = 1.0
    P = np.zeros(n_tot, np.float32)
    # He initialisation of the layers (the layout is that of csrc/mf_mlp.cuh)
    o = 0
    for (fan_out, fan_in), gain in (((64, 12), 2.0), ((64, 64), 2.0), ((n_out, 64), 1.0)):
        P[o:o + fan_out * fan_in] = rng.normal(0, np.sqrt(gain / fan_in), fan_out * fan_in)
        o += fan_out * fan_in + fan_out
    P[n_tr:n_tr + n_in] = mu
    P[n_tr + n_in:] = sd
    dev = torch.device("cuda")
    tP = torch.from_numpy(P).to(dev)
    tM = torch.zeros(n_tr, device=dev)
    tV = torch.zeros(n_tr, device=dev)
    tX = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    tT0 = torch.from_numpy(np.ascontiguousarray(T0)).to(dev)
    tT1 = torch.from_numpy(np.ascontiguousarray(T1)).to(dev)
    tT2 = torch.from_numpy(np.ascontiguousarray(T2)).to(dev)
    B = min(batch, X.shape[0])
    ws = torch.empty(int(lib().mf_mlp_workspace_bytes(B)) // 4 + 1, device=dev)
    hist = torch.zeros(steps, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = lib().mf_mlp_train(p(tP), p(tM), p(tV), p(tX), p(tT0), p(tT1), p(tT2), X.shape[0], steps, B, lr, wkc,
                            wmode, 0, p(hist), p(ws), st)
    if rc != 0:
        raise _native.MFError(rc, "mf_mlp_train")
    torch.cuda.synchronize()
    return tP.cpu().numpy(), hist.cpu().numpy()


def forward(P, X):
    """Network outputs for X through mf_mlp_forward (GPU)."""
    import torch
    dev = torch.device("cuda")
    tP = torch.from_numpy(np.ascontiguousarray(P, np.float32)).to(dev)
    tX = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    tY = torch.zeros((tX.shape[0], sizes()[1]), device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().mf_mlp_forward(ctypes.c_void_p(tP.data_ptr()), ctypes.c_void_p(tX.data_ptr()), tX.shape[0],
                              ctypes.c_void_p(tY.data_ptr()), st)
    if rc != 0:
        raise _native.MFError(rc, "mf_mlp_forward")
    return tY.cpu().numpy()


# ------------------------------------------------------------- evaluation --
def _kc_index(kc):
    kc = np.asarray(kc)
    return np.abs(np.log2(kc)[:, None] - np.log2(np.asarray(KC_CHOICES))[None, :]).argmin(axis=1)


def decide_plain(X):
    """The plain rule: repair iff k <= 1 % of m; KERNELCYCLES = average degree
    (feature 8 is the average Bi-CSR degree, about 2 m / n); data-driven."""
    X = np.asarray(X)
    repair = X[:, 3] <= 0.01
    m, n = 2.0 ** X[:, 1], 2.0 ** X[:, 0]
    kc = np.maximum(1, np.rint(m / n))
    return repair, kc, np.zeros(X.shape[0], np.int64)


def decide_learned(P, X):
    """Decisions of the device kernel (k_policy), from the same outputs (on a
    graph that can repair by push-pull)."""
    Y = forward(P, X)
    repair = Y[:, 0] > 0
    kc = 2.0 ** np.clip(np.rint(Y[:, 1]), 0, 6)
    mode = Y[:, 2:5].argmax(axis=1)
    return repair, kc, mode


def cost(repair, kc, mode, data):
    """Device time of the decisions: the data-driven repair at the KC choice
    nearest kc, the topology-driven or push-pull repair (KC_STATIC), or the
    static recompute."""
    idx = _kc_index(kc)
    r = np.arange(len(idx))
    rep = np.where(mode == 0, data["t_dyn"][r, idx], np.where(mode == 1, data["t_topo"], data["t_pp"]))
    return np.where(repair, rep, data["t_static"])


def evaluate(data, P):
    """Total device time on the logged batches of: the plain rule; every
    fixed mode (always repair, the graph's default KC); the learned policy
    with one, two and all three of its outputs used (the others held at the
    plain rule's repair decision, the default KC, the data-driven mode); and
    the best possible choice."""
    X = data["X"]
    rp, kp, mp = decide_plain(X)
    rl, kl, ml = decide_learned(P, X)
    always = np.ones_like(rp)
    best = np.minimum(mode_times(data).min(axis=1), data["t_static"])
    out = {"batches": int(X.shape[0]), "plain_ms": float(cost(rp, kp, mp, data).sum())}
    for m, name in enumerate(MODE_NAMES):
        out[f"always_{name}_ms"] = float(cost(always, kp, np.full_like(mp, m), data).sum())
    out["best_fixed_mode_ms"] = min(out[f"always_{name}_ms"] for name in MODE_NAMES)
    out["learned_repair_only_ms"] = float(cost(rl, kp, mp, data).sum())
    out["learned_repair_kc_ms"] = float(cost(rl, kl, mp, data).sum())
    out["learned_repair_mode_ms"] = float(cost(rl, kp, ml, data).sum())
    out["learned_ms"] = float(cost(rl, kl, ml, data).sum())
    out["best_ms"] = float(best.sum())
    out["mode_choices"] = {name: int((ml[rl] == m).sum()) for m, name in enumerate(MODE_NAMES)}
    return out


# -------------------------------------------------------------------- CLI --
def _specs():
    """Seeded workloads of the logging run: (name, group, graph factory,
    batch factory (cap, i, rng) -> Batch, number of batches)."""
    from workloads import generators as gen

    def mixed(lo, hi, kmin, kmax_frac):
        def make(g, cap, i, rng):
            k = int(np.exp(rng.uniform(np.log(kmin), np.log(max(kmin + 1, kmax_frac * g.m)))))
            return gen.mixed_batch(cap, min(k, g.m), lo, hi, seed=int(rng.integers(1 << 30)), index=i)
        return make

    def rect(side_lo, side_hi):
        def make(g, cap, i, rng):
            return gen.grid_rect_batch(g, seed=int(rng.integers(1 << 30)), index=i, side_lo=side_lo,
                                       side_hi=side_hi)
        return make

    out = []
    for s in range(200):
        out.append((f"random_s{s}", len(out), lambda s=s: gen.random_graph(seed=s), mixed(1, 50, 5, 0.5), 150))
    for sc, seeds, nb in ((14, 40, 200), (16, 20, 150), (18, 8, 100), (20, 4, 60)):
        for s in range(seeds):
            out.append((f"rmat{sc}_s{s}", len(out), lambda sc=sc, s=s: gen.rmat(scale=sc, seed=100 + s),
                        mixed(1, 500, 100, 0.08), nb))
    for L, seeds, nb in ((1 << 12, 8, 100), (1 << 14, 4, 100)):
        for s in range(seeds):
            out.append((f"bipartite{L}_s{s}", len(out),
                        lambda L=L, s=s: gen.bipartite(L, L, 16 * L, seed=300 + s), mixed(1, 1, 10, 0.08), nb))
    for W, seeds, nb, lo, hi in ((512, 16, 80, 16, 128), (1024, 8, 50, 32, 256), (2048, 2, 30, 64, 512),
                                 (4096, 1, 15, 64, 512)):
        for s in range(seeds):
            out.append((f"grid{W}_s{s}", len(out), lambda W=W, s=s: gen.grid_segmentation(W, W, seed=200 + s),
                        rect(lo, hi), nb))
    return out


def main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", required=True)
    c.add_argument("--limit", type=int, default=0, help="only the first N workloads")
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", default=PARAMS_PATH)
    t.add_argument("--steps", type=int, default=6000)
    e = sub.add_parser("eval")
    e.add_argument("--data", required=True)
    e.add_argument("--params", default=PARAMS_PATH)
    args = ap.parse_args(argv)
    if args.cmd == "collect":
        log = {"X": [], "t_dyn": [], "t_topo": [], "t_pp": [], "t_static": [], "group": [], "k": []}
        names = []
        t0 = time.time()
        specs = _specs()[: args.limit or None]
        for name, group, make_graph, make_batch, nb in specs:
            g = make_graph()
            cap = g.cap.copy()
            rng = np.random.default_rng(1000 + group)

            def batches(g=g, cap=cap, rng=rng, make_batch=make_batch, nb=nb):
                from workloads import generators as gen
                for i in range(nb):
                    b = make_batch(g, cap, i, rng)
                    gen.apply_batch(cap, b)
                    yield b
            collect_graph(g, batches(), group, log)
            names.append(name)
            print(json.dumps({"workload": name, "rows": len(log["k"]), "s": round(time.time() - t0, 1)}), flush=True)
        np.savez_compressed(args.out, X=np.asarray(log["X"], np.float32), t_dyn=np.asarray(log["t_dyn"], np.float32),
                            t_topo=np.asarray(log["t_topo"], np.float32), t_pp=np.asarray(log["t_pp"], np.float32),
                            t_static=np.asarray(log["t_static"], np.float32), group=np.asarray(log["group"], np.int32),
                            k=np.asarray(log["k"], np.int64), names=np.asarray(names), kc=np.asarray(KC_CHOICES))
    elif args.cmd == "train":
        d = np.load(args.data)
        train_rows = d["group"] % 4 != 3            # every 4th workload is held out
        T0, T1, T2 = labels(d)
        P, hist = train(d["X"][train_rows], T0[train_rows], T1[train_rows], T2[train_rows], steps=args.steps)
        np.save(args.out, P)
        print(json.dumps({"train_rows": int(train_rows.sum()), "loss_first": float(hist[:50].mean()),
                          "loss_last": float(hist[-50:].mean())}))
    else:
        d = np.load(args.data)
        held = d["group"] % 4 == 3
        P = np.load(args.params)
        sub_d = {k: d[k][held] for k in LOG_KEYS}
        print(json.dumps({"held_out": evaluate(sub_d, P), "all": evaluate({k: d[k] for k in sub_d}, P)}))


if __name__ == "__main__":
    main()
