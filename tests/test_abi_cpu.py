"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/mf.h declares, and its host-side Bi-CSR builder (Sec. 5.1) is right.
No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

from workloads import generators as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_05895_gb300 as pkg
    return pkg


def header_functions():
    text = open(os.path.join(ROOT, "include", "mf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(mf):
    L = mf.lib()
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    from paper_2511_05895_gb300 import _native
    assert sorted(_native.EXPORTED) == names


def test_strerror_and_version(mf):
    L = mf.lib()
    assert L.mf_version() == b"0.1.0"
    assert L.mf_strerror(0) == b"ok" and L.mf_strerror(1) == b"invalid argument"
    assert L.mf_strerror(5) == b"device loop timeout"


def test_options_default(mf):
    from paper_2511_05895_gb300._native import Options
    o = Options()
    o.kernel_cycles = 99
    assert mf.lib().mf_options_default(ctypes.byref(o)) == 0
    assert o.kernel_cycles == 0 and o.max_iters == 0 and o.grid_blocks == 0


def test_null_arguments_rejected(mf):
    L = mf.lib()
    assert L.mf_solve(None, None) == 1
    assert L.mf_flow_value(None, None) == 1
    assert L.mf_sync(None) == 1
    L.mf_destroy(None)


def _check_bicsr(g, B):
    tails = g.tails()
    A = B["head"].shape[0]
    arc_tail = np.repeat(np.arange(g.n), np.diff(B["arc_row"]))
    # pairing
    assert np.array_equal(B["rev"][B["rev"]], np.arange(A))
    assert np.array_equal(B["head"][B["rev"]], arc_tail)
    # one arc per distinct neighbour, sorted by head within each vertex
    both = np.concatenate([np.stack([tails, g.col], 1), np.stack([g.col, tails], 1)])
    pairs = np.unique(both, axis=0)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    assert A == pairs.shape[0]
    assert np.array_equal(np.stack([arc_tail, B["head"]], 1), pairs)
    # capacities: per arc, sum of its edges; edge map points at the right arc
    want = np.zeros(A, np.int64)
    nl = tails != g.col
    np.add.at(want, B["arc_of_edge"][nl], g.cap[nl])
    assert np.array_equal(B["cap"].astype(np.int64), want)
    assert np.all(B["arc_of_edge"][~nl] == -1)
    assert np.array_equal(arc_tail[B["arc_of_edge"][nl]], tails[nl])
    assert np.array_equal(B["head"][B["arc_of_edge"][nl]], g.col[nl])


@pytest.mark.parametrize("seed", range(3))
def test_bicsr_random(mf, seed):
    g = gen.random_graph(n=200, m=3000, seed=seed)   # many parallel/antiparallel pairs
    _check_bicsr(g, mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, g.s, g.t))


def test_bicsr_rmat_and_grid(mf):
    for g in (gen.rmat(scale=12, seed=4), gen.grid_segmentation(33, 17, seed=4)):
        _check_bicsr(g, mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, g.s, g.t))


def test_bicsr_self_loops_and_limits(mf):
    g = gen.from_edges(4, [0, 1, 1, 2, 2, 2], [1, 1, 2, 3, 3, 1], [5, 9, 3, 4, 6, 2], 0, 3)
    B = mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, g.s, g.t)
    _check_bicsr(g, B)
    # pair (1,2) carries edges 1->2 and 2->1, pair (2,3) two parallel edges
    assert B["cap_limit"] == (2 ** 31 - 1) // 2
    with pytest.raises(Exception):
        mf.bicsr_host(g.n, g.row_ptr, g.col, np.array([5, 9, 3, 2 ** 30, 2 ** 30, 2], np.int32), g.s, g.t)
    with pytest.raises(Exception):
        mf.bicsr_host(g.n, g.row_ptr, g.col, g.cap, 1, 1)          # s == t
    with pytest.raises(Exception):
        mf.bicsr_host(g.n, g.row_ptr, g.col, np.array([5, -1, 3, 4, 6, 2], np.int32), 0, 3)


def test_product_path_has_no_fallback(mf, tmp_path, monkeypatch):
    """Without the built library the binding raises instead of computing."""
    from paper_2511_05895_gb300 import _native, _build
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _native.lib()


def test_header_constants_match_binding(mf):
    """Every MF_* constant the binding defines has the value include/mf.h gives it."""
    from paper_2511_05895_gb300 import _native
    text = open(os.path.join(ROOT, "include", "mf.h")).read()
    defs = dict(re.findall(r"#define\s+(MF_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)", text))
    checked = 0
    for name, val in defs.items():
        if hasattr(_native, name):
            assert getattr(_native, name) == int(val, 0), name
            checked += 1
    assert checked >= 15, checked
