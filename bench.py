#!/usr/bin/env python3
"""Benchmark: dynamic max-flow repair on an RMAT scale-20 graph (GB300).

Workload (one GPU): RMAT power-law graph, 2^20 vertices, 16.7M directed edges
(a, b, c, d = 0.57, 0.19, 0.19, 0.05), int32 capacities U[1, 1000], s and t the
two vertices of highest out-degree.  One step = one mixed batch of
--batch distinct uniformly chosen edges (half +U[1,500], half -U[1,500]
clamped at 0) applied to the resident residual graph and repaired by the
dynamic push-relabel kernel (validate, apply, clamp, re-saturate, then BFS /
push-relabel / remove-invalid until no vertex is active).

value      batches repaired per second, batch already resident in HBM,
           device time of the repair kernel (CUDA events, L2 flushed between
           steps by writing a 512 MiB buffer outside the timed region)
e2e        the same through the C ABI with pinned HOST batch buffers: the
           host->device batch copy, the repair and the device->host read of the
           flow value and status are inside the timed region
sizes      dynamic repair vs static GPU recompute (solve from zero flow on the
           same capacities) for 1k / 10k / 100k / 1M-edge batches
config1    the small configuration (1,000 vertices, 50-update batches) over 100
           seeds, every value checked against the CPU oracle
grid       the same comparison on the 4096^2 segmentation grid with
           rectangle batches (terminal-capacity rewrites)
serving    the request loop over eight resident graphs at two offered rates
roofline   algorithmic bytes of the repair kernel (per-unit figures x device
           counters) / its measured duration / measured HBM peak
cpu_baseline  the CPU oracle (FIFO push-relabel, from scratch) on a bounded
           sample of the same batches, timed on this host

--impl reference runs that oracle arm alone.  Under torchrun every rank runs an
independent replica of the workload on its own GPU (the method has no
exchange step); value = batches of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import generators as gen  # noqa: E402

METRIC = "update-batch latency & speedup vs static GPU push-relabel; HBM GB/s frac"
UNIT = "batches/s"
SCALE = 20
SEED = 1

# Algorithmic bytes per unit of work of the repair kernel: the per-unit
# figures of the method's memory accesses, each random 4-byte gather counted
# as 4 bytes and an atomic read-modify-write as its operand size.
BYTES = {
    "bfs_arcs": 12,       # head 4 + mirrored residual 4 + height of the head 4
    "bfs_vertices": 12,   # row offsets 8 + height write 4
    "height_init": 12,    # per vertex per BFS: excess 8 + height write 4 (+ 8 per vertex for
                          # the deficit recount of a loop that ends without a final BFS)
    "pr_arcs": 12,        # residual 4 + head 4 + height of the head 4 (one scan per step)
    "pushes": 28,         # residual 4 + reverse residual 4 + reverse arc 4 + excess of u 8 + of v 8
    "relabels": 4,
    "ri_arcs": 12,
    "ri_moves": 28,
    "worklist": 8,        # worklist write + read
    "batch": 32,          # id + cap 8, cap_edge 4, arc map 4, residual RMW 8, arc capacity RMW 8
    "clamped": 24,        # reverse residual 4 + reverse arc 4 + two int64 excesses 16
    "resat_arcs": 4,
}


def algorithmic_bytes(st: dict, n: int) -> int:
    b = 0
    for k, w in BYTES.items():
        if k == "height_init":
            bfs_runs = st["iterations"] + (1 if st["exit_kind"] == 0 else 0)
            b += w * n * bfs_runs + (8 * n if st["exit_kind"] == 1 else 0)
        else:
            b += w * st[k]
    return int(b)


def kernel_source_hash() -> str:
    """sha256[:16] of mf_gpu.cu without its comments and blank space: the
    same hash means the same compiled kernel."""
    p = os.path.join(ROOT, "paper_2511_05895_gb300", "csrc", "mf_gpu.cu")
    src = open(p).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", " ", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def recorded_traffic(kernel_hash: str, profile: str):
    """DRAM bytes per launch of k_solve from the committed ncu summary
    profiles/<profile>, if it was taken on this exact kernel source (recorded
    by an earlier capture, not measured in this run); else None."""
    p = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", txt)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9]+)", txt)
    if h and t and h.group(1) == kernel_hash:
        return int(t.group(1))
    return None
    txt = open(p).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", txt)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9]+)", txt)
    if h and t and h.group(1) == kernel_hash:
        return int(t.group(1))
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names[1:], r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_batches(cap: np.ndarray, k: int, count: int, index0: int):
    out = []
    for i in range(count):
        b = gen.mixed_batch(cap, k, 1, 500, seed=SEED, index=index0 + i)
        gen.apply_batch(cap, b)
        out.append(b)
    return out


def run_reference(args, rank: int, world: int) -> None:
    """The oracle arm: FIFO push-relabel from scratch after each batch."""
    if rank != 0:
        return
    import oracle
    g = gen.rmat(scale=SCALE, seed=SEED)
    cap = g.cap.copy()
    batches = make_batches(cap.copy(), args.batch, args.warmup + args.steps, 10_000)
    cur = g.cap.copy()
    times = []
    for i, b in enumerate(batches):
        gen.apply_batch(cur, b)
        t0 = time.perf_counter()
        oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cur, g.s, g.t)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": workload_config(args, g),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} consecutive {args.batch}-edge mixed batches, "
                                   "FIFO push-relabel from scratch per batch, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SERVE_GRAPHS = "RMAT scales 16, 18, 20, 22 (caps U[1,1000]); segmentation grids 1024^2, 2048^2, 4096^2; " \
               "unit bipartite graph 2^20 + 2^20 vertices, 16M edges"


def serving_measurement(rates, duration_s: float, seed: int = 5) -> dict:
    """Serving loop on eight resident graphs (RMAT scales 16-22, segmentation
    grids 1024^2-4096^2, a unit bipartite assignment graph of 2^20 + 2^20
    vertices and 16M edges): for each offered rate, Poisson arrivals for
    `duration_s`, batch sizes log-uniform in [100, 100k] (grids: the pixels of
    a rectangle of that many terminal arcs), served by mf_server with per-graph
    grids of 19 to 152 CTAs, every graph repaired by Dynamic Push-Pull.  Reports
    p50/p99 submit-to-completion latency and the completed batches per second
    at each rate.  Each request's repair runs on a grid sized to its batch
    (the graph's full grid, half or a quarter; see mf_server)."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2511_05895_gb300 import MF_MODE_PUSH_PULL, MaxFlowGraph, Server
    makers = [(lambda: gen.rmat(scale=16, seed=301), 19), (lambda: gen.rmat(scale=18, seed=302), 38),
              (lambda: gen.rmat(scale=20, seed=303), 76), (lambda: gen.rmat(scale=22, seed=304), 152),
              (lambda: gen.grid_segmentation(1024, 1024, seed=305), 38),
              (lambda: gen.grid_segmentation(2048, 2048, seed=306), 76),
              (lambda: gen.grid_segmentation(4096, 4096, seed=307), 152),
              (lambda: gen.bipartite(1 << 20, 1 << 20, 1 << 24, seed=308), 76)]
    t_setup = time.perf_counter()
    with ThreadPoolExecutor(max_workers=4) as ex:      # numpy releases the GIL
        graphs = list(ex.map(lambda mk: mk[0](), makers))
    S = Server()
    Gs, caps = [], []
    for g, (_, grid) in zip(graphs, makers):
        G = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=4, grid_blocks=grid,
                         mode=MF_MODE_PUSH_PULL)
        G.solve()
        G.flow_value()
        S.add_graph(G, 100_000)
        Gs.append(G)
        caps.append(g.cap.copy())
    t_setup = time.perf_counter() - t_setup
    rng = np.random.default_rng(seed)
    runs = []
    idx = 0
    for rate in rates:
        n_req = max(8, int(rate * duration_s))
        plan = []
        for _ in range(n_req):
            gi = int(rng.integers(len(graphs)))
            g = graphs[gi]
            k = int(np.exp(rng.uniform(np.log(100), np.log(min(100_000, g.m // 10)))))
            if g.meta.get("kind") == "grid":
                side = max(8, int(np.sqrt(k / 2)))        # 2 side^2 <= k terminal arcs
                b = gen.grid_rect_batch(g, seed=seed, index=idx, side_lo=side, side_hi=side)
            else:
                hi = 1 if g.meta.get("kind") == "bipartite" else 500
                b = gen.mixed_batch(caps[gi], k, 1, hi, seed=seed, index=idx)
            idx += 1
            gen.apply_batch(caps[gi], b)
            plan.append((gi, b))
        gaps = rng.exponential(1.0 / rate, n_req)
        S.reset_stats()
        t_next = time.perf_counter()
        for (gi, b), gap in zip(plan, gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                pass
            S.submit(gi, b.edge_id, b.new_cap)
        S.drain()
        st = S.stats()
        runs.append({"offered_rate_per_s": rate, "requests": st["completed"],
                     "batches_per_s": round(st["completed"] / max(st["makespan_s"], 1e-9), 1),
                     "p50_ms": round(st["p50_us"] / 1000, 3), "p99_ms": round(st["p99_us"] / 1000, 3),
                     "max_inflight": st["max_inflight"], "captured_graphs": st["captured_graphs"],
                     "replays": st["replays"], "direct_launches": st["direct_launches"],
                     "failed": st["failed"]})
    # every graph's final value against a fresh static solve of its final
    # capacities; where the two differ, the CPU oracle says which is right
    exact, per_graph = True, []
    for G, g, cap in zip(Gs, graphs, caps):
        H = MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, kernel_cycles=4)
        H.solve()
        served, static = G.flow_value(), H.flow_value()
        H.close()
        row = {"graph": g.name or g.meta.get("kind", "?"), "served": served, "static": static}
        if served != static:
            import oracle
            row["oracle"] = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        exact = exact and served == static
        per_graph.append(row)
    S.close()
    for G in Gs:
        G.close()
    return {"graphs": SERVE_GRAPHS, "mode": "push-pull", "setup_s": round(t_setup, 1), "runs": runs,
            "final_values_equal_static_recompute": exact, "final_values": per_graph}


def config1_measurement(seeds: int = 100) -> dict:
    """The small configuration: 1,000-vertex / 8,000-edge random graphs (caps
    U[1,100], a guaranteed s-t path), one static solve, then one 50-update
    mixed batch (25 x +U[1,50], 25 x -U[1,50] clamped) and a dynamic re-solve,
    over `seeds` seeds.  Every value is checked against the CPU oracle; the
    graphs fit in L2, so only latencies are reported (device time, median)."""
    import oracle
    import torch
    from paper_2511_05895_gb300 import MaxFlowGraph
    stream = torch.cuda.current_stream()
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    dyn, sta, orc, exact = [], [], [], True
    for seed in range(seeds):
        g = gen.random_graph(seed=seed)
        cap = g.cap.copy()
        G = MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        G.solve()
        G.flow_value()
        b = gen.mixed_batch(cap, 50, 1, 50, seed=seed, index=0)
        gen.apply_batch(cap, b)
        ids, cp = torch.from_numpy(b.edge_id).cuda(), torch.from_numpy(b.new_cap).cuda()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        G.apply_updates(ids, cp)
        ev[1].record(stream)
        ev[1].synchronize()
        f = G.flow_value()
        ev[2].record(stream)
        G.apply_updates(empty, empty, recompute=True)
        ev[3].record(stream)
        ev[3].synchronize()
        t0 = time.perf_counter()
        want = oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t)
        orc.append(time.perf_counter() - t0)
        exact = exact and f == want == G.flow_value()
        dyn.append(ev[0].elapsed_time(ev[1]))
        sta.append(ev[2].elapsed_time(ev[3]))
        G.close()
    d, s_ = statistics.median(dyn), statistics.median(sta)
    return {"workload": "random graphs n=1000 m=8000 caps U[1,100], one 50-update mixed batch each",
            "seeds": seeds, "dynamic_ms": round(d, 4), "static_recompute_ms": round(s_, 4),
            "speedup": round(s_ / d, 3), "oracle_ms_one_core": round(1000 * statistics.median(orc), 3),
            "values_equal_oracle": exact}


def grid_measurement(batches: int, flush, peak: float, seed: int = 3, side: int = 4096) -> dict:
    """The side x side segmentation grid (4096: 16.8M vertices, 67M n-link
    arcs plus one s- and one t-arc per pixel): each batch rewrites the
    terminal capacities of a random rectangle of side 64-512; dynamic repair
    vs static GPU recompute of the same capacities (median ms), the repair's
    share of measured HBM bandwidth, and a check that both give the same
    value."""
    import torch
    from paper_2511_05895_gb300 import MaxFlowGraph
    from paper_2511_05895_gb300 import MF_MODE_PUSH_PULL
    g = gen.grid_segmentation(side, side, seed=seed)
    G = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=4)
    G.solve()
    G.flow_value()
    Gp = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=4, mode=MF_MODE_PUSH_PULL)
    Gp.solve()
    stream = torch.cuda.current_stream()
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    dyn, sta, ks, fr, ppt = [], [], [], [], []
    equal = True
    for i in range(batches):
        b = gen.grid_rect_batch(g, seed=seed, index=i)
        ids = torch.from_numpy(b.edge_id).cuda()
        cp = torch.from_numpy(b.new_cap).cuda()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        flush.zero_()
        ev[0].record(stream)
        G.apply_updates(ids, cp)
        ev[1].record(stream)
        ev[1].synchronize()
        f_dyn = G.flow_value()
        st = G.stats()
        flush.zero_()
        ev[2].record(stream)
        G.apply_updates(empty, empty, recompute=True)
        ev[3].record(stream)
        ev[3].synchronize()
        equal = equal and G.flow_value() == f_dyn
        ppt.append(time_repairs(Gp, [(ids, cp)], 0, flush, stream)[0][0])
        equal = equal and Gp.flow_value() == f_dyn
        d, s_ = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        dyn.append(d)
        sta.append(s_)
        ks.append(len(b.edge_id))
        fr.append(algorithmic_bytes(st, g.n) / (d * 1e-3) / 1e9 / peak)
    G.close()
    Gp.close()
    d, s_, pm = statistics.median(dyn), statistics.median(sta), statistics.median(ppt)
    return {"workload": f"segmentation grid {side}^2 (n={g.n}, m={g.m}), rectangle batches of side 64-512 "
                        "rewriting terminal capacities", "batches": batches,
            "entries_median": int(statistics.median(ks)), "dynamic_ms": round(d, 3),
            "push_pull_ms": round(pm, 3), "static_recompute_ms": round(s_, 3), "speedup": round(s_ / d, 3),
            "push_pull_speedup": round(s_ / pm, 3), "dynamic_spread_ms": spread(dyn),
            "push_pull_spread_ms": spread(ppt), "static_spread_ms": spread(sta),
            "hbm_frac_of_measured": round(statistics.median(fr), 4), "values_equal": equal}


MODES = {"data-driven": 0, "topology": 1, "push-pull": 2}


def certify_state(G, g, cap, flow) -> bool:
    """The optimality certificate of the GPU state (capacity feasibility,
    excess bookkeeping, a cut with no residual arc from S to T, signs, value =
    cut capacity, heights = BFS fixed point), checked by the oracle's C
    checker on the host."""
    import oracle
    st = G.export_graph()
    r, e, h = G.export_state()
    side = G.min_cut()
    bits, _, _ = oracle.certify(g.n, g.row_ptr, g.col, cap, g.s, g.t, st["arc_row"], st["head"],
                                st["rev"].astype(np.int64), st["cap"], r, e, side, flow, h)
    return bits == 0


def spread(xs) -> dict:
    """min / median / max of a sample (ms)."""
    return {"min": round(min(xs), 4), "median": round(statistics.median(xs), 4), "max": round(max(xs), 4)}


def time_repairs(G, dev, warmup, flush, stream):
    """Apply dev[:warmup] untimed, then time each remaining batch on the
    device (L2 flushed before each); returns (ms list, stats list)."""
    import torch
    for ids, caps in dev[:warmup]:
        G.apply_updates(ids, caps)
    G.sync()
    ms, sts = [], []
    for ids, caps in dev[warmup:]:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.apply_updates(ids, caps)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        sts.append(G.stats())
    return ms, sts


def _oracle_warm(_):
    import oracle
    oracle.lib()
    return os.getpid()


def _oracle_recompute(job):
    """One oracle recompute in a worker process (graph and capacities read
    from .npy files); returns (flow, seconds)."""
    import oracle
    rp, col, capf, s, t = job
    row_ptr = np.load(rp, mmap_mode="r")
    cols = np.load(col, mmap_mode="r")
    cap = np.load(capf)
    t0 = time.perf_counter()
    f = oracle.maxflow_fifo(row_ptr.shape[0] - 1, row_ptr, cols, cap, s, t)
    return f, time.perf_counter() - t0


def cpu_oracle_sample(g, args) -> dict:
    """The CPU oracle (FIFO push-relabel from scratch, one thread per
    recompute) on the host cores: one recompute per core, each on the
    cumulative capacities after a different 100k-edge batch of the benchmark
    sequence, run as parallel processes (the recomputes are independent)."""
    import multiprocessing
    cores = args.cpu_sample if args.cpu_sample > 0 else (os.cpu_count() or 1)
    cur = g.cap.copy()
    jobs = []
    with tempfile.TemporaryDirectory() as tmp:
        rp, col = os.path.join(tmp, "row_ptr.npy"), os.path.join(tmp, "col.npy")
        np.save(rp, g.row_ptr)
        np.save(col, g.col)
        # the batches are drawn on a copy (make_batches applies them as it
        # draws), then applied one by one: job i sees batches 0 .. i
        for i, b in enumerate(make_batches(cur.copy(), args.batch, cores, 0)):
            gen.apply_batch(cur, b)
            cf = os.path.join(tmp, f"cap{i}.npy")
            np.save(cf, cur)   # the capacities after batches 0 .. i
            jobs.append((rp, col, cf, g.s, g.t))
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=cores, mp_context=multiprocessing.get_context("spawn")) as ex:
            list(ex.map(_oracle_warm, range(cores)))      # workers started, oracle loaded
            t0 = time.perf_counter()
            res = list(ex.map(_oracle_recompute, jobs))
            wall = time.perf_counter() - t0
    per = [sec for _, sec in res]
    return {"value": len(jobs) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "flows": [f for f, _ in res],
            "seconds_per_batch_one_core": round(statistics.mean(per), 3),
            "sample": f"{len(jobs)} recomputes from scratch (FIFO push-relabel, one thread each) of the "
                      f"RMAT-20 graph after {args.batch}-edge batches, as {cores} parallel processes "
                      f"on {os.cpu_count()} host cores"}


def workload_config(args, g) -> dict:
    return {"workload": f"RMAT scale {SCALE} (n={g.n}, m={g.m}, a=0.57 b=0.19 c=0.19), caps U[1,1000], "
                        f"mixed batches of {args.batch} edges (+/-U[1,500])",
            "n": g.n, "m": g.m, "batch_edges": args.batch, "seed": SEED,
            "kernel_cycles": args.kc, "policy": args.policy,
            "mode": "chosen per batch by the learned policy" if args.policy == "learned" else args.mode,
            "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=100_000)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-sizes", action="store_true", help="skip the per-size dynamic/static comparison")
    ap.add_argument("--cpu-sample", type=int, default=-1,
                    help="batches (= parallel processes) of the CPU-oracle sample; -1: one per host core, 0: skip")
    ap.add_argument("--kc", type=int, default=4, help="KERNELCYCLES of the repair (0 = average degree)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-grid", action="store_true", help="skip the 4096^2 segmentation-grid measurement")
    ap.add_argument("--policy", default="fixed", choices=["fixed", "plain", "learned"],
                    help="batch policy: fixed repair, the plain rule, or the trained network")
    ap.add_argument("--mode", default="data-driven", choices=list(MODES),
                    help="processing mode of the timed repairs (Sec. 5.2 / 5.3 / Alg. 8); with --policy learned "
                         "the network chooses it per batch")
    ap.add_argument("--no-pp", action="store_true", help="skip the Dynamic Push-Pull comparison")
    ap.add_argument("--size-batches", type=int, default=20, help="batches per size in the dynamic/static sweep")
    ap.add_argument("--grid-batches", type=int, default=20, help="rectangle batches on the segmentation grid")
    ap.add_argument("--grid-side", type=int, default=4096, help="side of the segmentation grid")
    ap.add_argument("--only-serve", action="store_true",
                    help="run only the serving measurement (prints its JSON)")
    ap.add_argument("--only-grid", action="store_true",
                    help="run only the segmentation-grid measurement (a profiling case; prints its JSON)")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_05895_gb300 import MaxFlowGraph, replicas

    if args.only_serve:
        print(json.dumps({"serving": serving_measurement((100.0, 300.0, 600.0, 1000.0), 3.0)}), flush=True)
        return

    if args.only_grid:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peak = float(json.load(open(peaks_path))["hbm_gbs"]) if os.path.exists(peaks_path) else 6800.0
        print(json.dumps({"grid": grid_measurement(args.grid_batches, flush, peak, side=args.grid_side)}), flush=True)
        return

    g = gen.rmat(scale=SCALE, seed=SEED + 1000 * rank)
    cap = g.cap.copy()
    # the learned policy picks the processing mode per batch: the graph keeps
    # the push-pull state (and the exact cut) so that all three are open
    gmode = MODES["push-pull"] if args.policy == "learned" else MODES[args.mode]
    G = MaxFlowGraph(g.n, g.row_ptr, g.col, cap, g.s, g.t, kernel_cycles=args.kc, mode=gmode)
    G.solve()
    flow0 = G.flow_value()
    if args.policy != "fixed":
        from paper_2511_05895_gb300 import MF_POLICY_LEARNED, MF_POLICY_PLAIN
        from paper_2511_05895_gb300.policy import load_default_params
        if args.policy == "plain":
            G.set_policy(MF_POLICY_PLAIN)
        else:
            G.set_policy(MF_POLICY_LEARNED, load_default_params())

    host_cap = cap.copy()
    batches = make_batches(host_cap, args.batch, args.warmup + args.steps, 0)
    dev = [(torch.from_numpy(b.edge_id).cuda(), torch.from_numpy(b.new_cap).cuda()) for b in batches]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed_step(ids, caps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.apply_updates(ids, caps)
        e1.record(stream)
        return e0, e1

    flows = []   # the GPU's value after each batch (warm-up and timed), read outside the timing
    for i in range(args.warmup):
        a, b = timed_step(*dev[i])
        b.synchronize()
        flows.append(G.flow_value())
    G.sync()
    stats_acc = {k: 0 for k in [b for b in BYTES if b != "height_init"] +
                 ["iterations", "bfs_levels", "t_batch_ns", "t_reset_ns", "t_bfs_ns", "t_pr_ns",
                  "t_hub_ns", "t_ri_ns", "hub_cycles", "barriers", "bfs_bottom_up_levels", "pr_rounds",
                  "clean_exits"]}
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    events, per_step_bytes, chosen = [], [], []
    for i in range(args.warmup, args.warmup + args.steps):
        ev = timed_step(*dev[i])
        events.append(ev)
        # device counters of this launch (read after it completes; outside the timing)
        ev[1].synchronize()
        st = G.stats()
        flows.append(G.flow_value())
        per_step_bytes.append(algorithmic_bytes(st, g.n))
        for k in stats_acc:
            stats_acc[k] += st[k] if k != "clean_exits" else int(st["exit_kind"] == 1)
        chosen.append((st["policy_kind"], st["policy_kernel_cycles"], st["policy_mode"]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in events]          # ms
    t_total = replicas.max_over_ranks(sum(times) / 1000.0, device="cuda")
    if dist:
        dist.barrier()
    G.sync()
    flow_after = G.flow_value()

    # certificate of the final state (optimality proof; the oracle's checker)
    certified = certify_state(G, g, host_cap, flow_after)

    # ---- the same batches repaired by Dynamic Push-Pull (Alg. 8) ----------
    pp, Gp = None, None
    if not args.no_pp and args.mode != "push-pull" and args.policy == "fixed":
        from paper_2511_05895_gb300 import MF_MODE_PUSH_PULL
        Gp = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=args.kc, mode=MF_MODE_PUSH_PULL)
        Gp.solve()
        pms, psts = time_repairs(Gp, dev, args.warmup, flush, stream)
        p_ms = sum(pms) / len(pms)
        p_bytes = sum(algorithmic_bytes(st, g.n) for st in psts) / len(psts)
        pp = {"mode": "push-pull (MF_MODE_PUSH_PULL, Alg. 8)", "ms_per_step": round(p_ms, 4),
              "value": round(1000.0 / p_ms, 2), "unit": UNIT,
              "speedup_vs_headline_mode": round((1000.0 * t_total / args.steps) / p_ms, 3),
              "hbm_frac_of_measured": None, "algorithmic_bytes_per_launch": int(p_bytes),
              "exit_kinds": sorted({st["exit_kind"] for st in psts}),
              "value_equal": Gp.flow_value() == flow_after}

    # ---- the same batches under the learned batch policy --------------------
    # (the library as a user runs it: the network picks repair or recompute,
    # KERNELCYCLES and the mode per batch, on a graph that keeps the push-pull
    # state so that all three modes are open)
    learned = None
    if not args.no_pp and args.policy == "fixed":
        from paper_2511_05895_gb300 import MF_MODE_PUSH_PULL, MF_POLICY_LEARNED
        from paper_2511_05895_gb300.policy import load_default_params
        Gl = MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, kernel_cycles=args.kc, mode=MF_MODE_PUSH_PULL)
        Gl.solve()
        Gl.set_policy(MF_POLICY_LEARNED, load_default_params())
        lms, lsts = time_repairs(Gl, dev, args.warmup, flush, stream)
        l_ms = sum(lms) / len(lms)
        learned = {"policy": "learned (MF_POLICY_LEARNED, the committed parameters)", "ms_per_step": round(l_ms, 4),
                   "value": round(1000.0 / l_ms, 2), "unit": UNIT,
                   "speedup_vs_headline_mode": round((1000.0 * t_total / args.steps) / l_ms, 3),
                   "algorithmic_bytes_per_launch": int(sum(algorithmic_bytes(st, g.n) for st in lsts) / len(lsts)),
                   "hbm_frac_of_measured": None,
                   "choices": {"recompute": sum(st["policy_kind"] for st in lsts),
                               "kernel_cycles": sorted({st["policy_kernel_cycles"] for st in lsts}),
                               "modes": {name: sum(st["policy_mode"] == m for st in lsts)
                                         for name, m in MODES.items()}},
                   "value_equal": Gl.flow_value() == flow_after}
        Gl.close()

    # ---- e2e through the C ABI with pinned host buffers ------------------
    e2e_batches = make_batches(host_cap, args.batch, args.steps, 5_000)
    pinned = [(torch.from_numpy(b.edge_id).pin_memory(), torch.from_numpy(b.new_cap).pin_memory()) for b in e2e_batches]
    torch.cuda.synchronize()
    t_e2e = 0.0
    for ids, caps in pinned:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.apply_updates(ids, caps)
        G.flow_value()
        t_e2e += time.perf_counter() - t0
    e2e_value = replicas.whole_job_rate(args.steps, t_e2e, device="cuda")
    if Gp is not None:   # keep the push-pull instance on the same capacities
        for ids, caps in pinned:
            Gp.apply_updates(ids, caps)

    # ---- dynamic vs static recompute per batch size ----------------------
    sizes = {}
    if not args.no_sizes:
        empty = (torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
        for j, k in enumerate((1_000, 10_000, 100_000, 1_000_000)):
            bs = make_batches(host_cap, k, args.size_batches, 20_000 + 100 * j)
            dyn, sta, ppt = [], [], []
            for b in bs:
                ids = torch.from_numpy(b.edge_id).cuda()
                cp = torch.from_numpy(b.new_cap).cuda()
                a0, a1 = timed_step(ids, cp)
                a1.synchronize()
                dyn.append(a0.elapsed_time(a1))
                if Gp is not None:
                    ppt.append(time_repairs(Gp, [(ids, cp)], 0, flush, stream)[0][0])
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                s0.record(stream)
                G.apply_updates(empty[0], empty[1], recompute=True)    # static recompute, same caps
                s1.record(stream)
                s1.synchronize()
                sta.append(s0.elapsed_time(s1))
            G.sync()
            d, s = statistics.median(dyn), statistics.median(sta)
            sizes[str(k)] = {"batches": len(bs), "dynamic_ms": round(d, 4), "static_recompute_ms": round(s, 4),
                             "speedup": round(s / d, 3), "frac_of_edges": round(k / g.m, 6),
                             "dynamic_spread_ms": spread(dyn), "static_spread_ms": spread(sta)}
            if ppt:
                pm = statistics.median(ppt)
                sizes[str(k)].update(push_pull_ms=round(pm, 4), push_pull_speedup=round(s / pm, 3),
                                     push_pull_spread_ms=spread(ppt))
    if Gp is not None:
        Gp.close()

    # ---- CPU oracle on a bounded sample ----------------------------------
    cpu = None
    if rank == 0 and world >= 1 and args.cpu_sample != 0:
        cpu = cpu_oracle_sample(g, args)
        # the sample recomputes the values after the first batches of the same
        # sequence the GPU repaired: compare them one by one
        want = cpu.pop("flows")
        cpu["values_equal_oracle"] = all(flows[i] == f for i, f in enumerate(want) if i < len(flows))
        cpu["values_compared"] = min(len(want), len(flows))

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"

    if pp is not None:
        pp["hbm_frac_of_measured"] = round(pp["algorithmic_bytes_per_launch"] / (pp["ms_per_step"] * 1e-3) / 1e9 / peak, 4)
    if learned is not None:
        learned["hbm_frac_of_measured"] = round(
            learned["algorithmic_bytes_per_launch"] / (learned["ms_per_step"] * 1e-3) / 1e9 / peak, 4)

    config1 = config1_measurement() if rank == 0 and not args.no_sizes else None

    grid = None
    if not args.no_grid and rank == 0:
        grid = grid_measurement(args.grid_batches, flush, peak)

    serving = None
    if not args.no_serve and rank == 0:
        serving = serving_measurement((100.0, 300.0, 600.0, 1000.0), 3.0)

    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return

    mean_ms = 1000.0 * sum(times) / 1000.0 / len(times)
    mean_bytes = sum(per_step_bytes) / len(per_step_bytes)
    achieved = mean_bytes / (mean_ms / 1000.0) / 1e9
    khash = kernel_source_hash()
    # the capture of the workload the timed repairs ran: the data-driven
    # repair, or the push-pull one (fixed mode, or every batch's choice);
    # none for other modes
    pp_steps = args.mode == "push-pull" if args.policy == "fixed" else \
        all(c[2] == MODES["push-pull"] for c in chosen)
    profile = "k_solve_pushpull_rmat20_batch100k.md" if pp_steps else "k_solve_rmat20_batch100k.md"
    dd_steps = args.policy == "fixed" and args.mode == "data-driven"
    traffic = recorded_traffic(khash, profile) if (pp_steps or dd_steps) else None
    value = world * args.steps / t_total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(args, g),
        "latency_ms": {"p50": statistics.median(times), "p99": float(np.percentile(times, 99)),
                       "min": min(times), "max": max(times)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "traffic_source": ("recorded: an ncu capture of this kernel source "
                                        f"(profiles/{profile}), not measured in this run")
                     if traffic is not None else None,
                     "peak_source": peak_src, "kernel": "k_solve",
                     "algorithmic_bytes_per_launch": int(mean_bytes), "kernel_source": khash},
        "counters_per_step": {k: v / args.steps for k, v in stats_acc.items()},
        "policy_choices": None if args.policy == "fixed" else {
            "recompute": sum(c[0] for c in chosen),
            "kernel_cycles": sorted({c[1] for c in chosen}),
            "modes": {name: sum(c[2] == m for c in chosen) for name, m in MODES.items()}},
        "sizes": sizes,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * args.batch,
                "d2h_bytes_per_step": 16},
        "gpu_launches": args.steps * (2 if args.policy != "fixed" else 1),   # k_solve (+ k_policy) per step
        "clocks": clk,
        "cpu_baseline": cpu,
        "checks": {"flow_initial": flow0, "flow_final": flow_after, "certified": certified},
        "push_pull": pp,
        "learned_policy": learned,
        "config1": config1,
        "grid": grid,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
