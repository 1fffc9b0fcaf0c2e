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
