"""Shared test helpers: certificate check of a GPU graph's state."""
import numpy as np

import oracle


def certify_gpu(G, g, cap, flow):
    """Check the GPU state against the optimality certificate (capacity
    feasibility, excess bookkeeping, cut with no residual arc S->T, signs,
    value = cut capacity, heights = BFS fixed point).  Raises on failure."""
    st = G.export_graph()
    r, e, h = G.export_state()
    side = G.min_cut()
    bits, where, names = oracle.certify(g.n, g.row_ptr, g.col, cap, g.s, g.t, st["arc_row"],
                                        st["head"], st["rev"].astype(np.int64), st["cap"], r, e,
                                        side, flow, h)
    assert bits == 0, f"certificate failed: {names} at {where}"
    return side


def _oracle_job(job):
    rp, col, capf, s, t = job
    row_ptr = np.load(rp, mmap_mode="r")
    c = np.load(col, mmap_mode="r")
    return oracle.maxflow_fifo(row_ptr.shape[0] - 1, row_ptr, c, np.load(capf), s, t)


def oracle_flows_parallel(g, caps_list, workers=8):
    """The oracle's value for each capacity vector of caps_list, computed in
    parallel worker processes (started with spawn: the test process has an
    initialised CUDA context, which a fork would copy)."""
    import multiprocessing
    import os
    import tempfile
    from concurrent.futures import ProcessPoolExecutor
    with tempfile.TemporaryDirectory() as tmp:
        rp, col = os.path.join(tmp, "row_ptr.npy"), os.path.join(tmp, "col.npy")
        np.save(rp, g.row_ptr)
        np.save(col, g.col)
        jobs = []
        for i, cap in enumerate(caps_list):
            cf = os.path.join(tmp, f"cap{i}.npy")
            np.save(cf, cap)
            jobs.append((rp, col, cf, g.s, g.t))
        n = max(1, min(workers, len(jobs), os.cpu_count() or 1))
        with ProcessPoolExecutor(max_workers=n, mp_context=multiprocessing.get_context("spawn")) as ex:
            return list(ex.map(_oracle_job, jobs))
