"""The allocation-free entry point, mf_solve_bicsr_noalloc.

Some callers must not allocate GPU memory themselves (a plugin inside another
framework that owns every device allocation through its own pool, or a
service path that forbids allocations after start-up).  For them the library
offers one solve that works in a static device array instead of cudaMalloc.
Its results must equal those of the regular entry points (mf_create +
mf_solve), here the int64 max-flow value bit-exactly, on two calls in a row
that share the static array; its final state must also pass the optimality
certificate.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

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
    L = pkg.lib()
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.mf_solve_bicsr_noalloc.argtypes = [i32, i64, P, P, P, P, i32, i32, i32, P, P, P, P, P]
    L.mf_solve_bicsr_noalloc.restype = ctypes.c_int
    return pkg


def noalloc_solve(mf, g):
    """Solve g through mf_solve_bicsr_noalloc; returns (rc, flow, B, r, e, h)."""
    import torch
    B = mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    A = int(B["head"].shape[0])
    dev = {k: torch.from_numpy(np.ascontiguousarray(B[k], dtype=np.int32)).cuda()
           for k in ("head", "rev", "cap")}
    dev["row"] = torch.from_numpy(B["arc_row"].astype(np.int32)).cuda()
    r = torch.empty(max(A, 1), dtype=torch.int32, device="cuda")
    e = torch.empty(g.n, dtype=torch.int64, device="cuda")
    h = torch.empty(g.n, dtype=torch.int32, device="cuda")
    flow = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = mf.lib().mf_solve_bicsr_noalloc(
        g.n, A, ctypes.c_void_p(dev["row"].data_ptr()), ctypes.c_void_p(dev["head"].data_ptr()),
        ctypes.c_void_p(dev["rev"].data_ptr()), ctypes.c_void_p(dev["cap"].data_ptr()), g.s, g.t, 0,
        ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(h.data_ptr()),
        ctypes.byref(flow), stream)
    return rc, flow.value, B, r[:A].cpu().numpy(), e.cpu().numpy(), h.cpu().numpy()


def regular_solve(mf, g):
    G = mf.MaxFlowGraph(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    G.solve()
    f = G.flow_value()
    G.close()
    return f


def test_noalloc_matches_regular_entry_point_twice(mf):
    small, large = gen.random_graph(seed=41), gen.rmat(scale=13, seed=42)
    # calls in a row share the static array: small, then larger, then the
    # small graph again over what the larger call left behind (entries past
    # the small graph's n, hub and chunk lists, queue slots)
    graphs = [small, large, small]
    for g in graphs:
        rc, flow, B, r, e, h = noalloc_solve(mf, g)
        assert rc == 0, mf.lib().mf_last_error()
        want = regular_solve(mf, g)
        assert flow == want
        side = (h >= g.n).astype(np.uint8)
        bits, where, names = oracle.certify(g.n, g.row_ptr, g.col, g.cap, g.s, g.t, B["arc_row"],
                                            B["head"], B["rev"].astype(np.int64), B["cap"], r, e, side,
                                            flow, h)
        assert bits == 0, (names, where)


def test_noalloc_rejects_graphs_beyond_its_scratch(mf):
    L = mf.lib()
    n_big = (1 << 17) + 1
    rc = L.mf_solve_bicsr_noalloc(n_big, 10, None, None, None, None, 0, 1, 0, None, None, None, None, None)
    assert rc == mf.MF_EINVAL and b"at most" in L.mf_last_error()
    rc = L.mf_solve_bicsr_noalloc(100, (1 << 21) + 1, None, None, None, None, 0, 1, 0, None, None, None,
                                  None, None)
    assert rc == mf.MF_EINVAL
