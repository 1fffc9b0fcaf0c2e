"""CPU oracle for the dynamic max-flow path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` import this package.  The CUDA
library (``paper_2511_05895_gb300``) never imports it and shares no code with
it; the two meet only in the seeded inputs of ``workloads.generators``.

The arithmetic lives in ``mf_oracle.c`` (plain C, one thread), loaded here
through ctypes:

* ``maxflow_fifo``  -- FIFO push-relabel with exact global relabelling
  (Goldberg-Tarjan, recalled in Sec. 2.2), the oracle proper.  It recomputes
  the max-flow value of the current capacities from scratch; the dynamic
  method reaches exactly this value (closing theorem of Sec. 4.1).
* ``maxflow_ek``    -- Edmonds-Karp (Sec. 2.2), a cross-check.
* ``mincut_brute``  -- minimum cut by enumeration (max-flow = min-cut).
* ``certify``       -- optimality certificate of any solver's final state
  (Theorem 3.2's cut argument and the pseudo-flow theorem of Sec. 4.1).
* ``bfs_heights``   -- exact backward BFS distances (global relabel, Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")

CERT_BITS = {
    0: "STRUCT", 1: "CAPS", 2: "RESID", 3: "EXCESS", 4: "CUT", 5: "SIGNS", 6: "VALUE", 7: "HEIGHTS",
}


def build(force: bool = False) -> str:
    """Compile mf_oracle.c into oracle/_lib/liborc.so (gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.orc_maxflow_fifo.argtypes = [i32, i64, P, P, P, i32, i32, P, P, P, P, P, P, P, P]
        L.orc_maxflow_fifo.restype = ctypes.c_int
        L.orc_maxflow_ek.argtypes = [i32, i64, P, P, P, i32, i32, P]
        L.orc_maxflow_ek.restype = ctypes.c_int
        L.orc_mincut_brute.argtypes = [i32, i64, P, P, P, i32, i32, P]
        L.orc_mincut_brute.restype = ctypes.c_int
        L.orc_arc_count.argtypes = [i32, P, P]
        L.orc_arc_count.restype = i64
        L.orc_bfs_heights.argtypes = [i32, P, P, P, P, P, i32, P]
        L.orc_bfs_heights.restype = ctypes.c_int
        L.orc_certify.argtypes = [i32, i64, P, P, P, i32, i32, P, P, P, P, P, P, P, P, i64, P, P]
        L.orc_certify.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col, cap):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(cap, dtype=np.int32))


@dataclass
class OracleState:
    """Final residual state of the FIFO oracle (unmerged arc pairs)."""
    arc_row: np.ndarray
    head: np.ndarray
    rev: np.ndarray
    cap: np.ndarray
    r: np.ndarray
    excess: np.ndarray
    height: np.ndarray


def maxflow_fifo(n, row_ptr, col, cap, s, t, want_state: bool = False):
    """Max-flow value (int) by FIFO push-relabel; optionally the final state."""
    row_ptr, col, cap = _csr(row_ptr, col, cap)
    L = lib()
    flow = np.zeros(1, dtype=np.int64)
    st = None
    if want_state:
        na = int(L.orc_arc_count(n, _p(row_ptr), _p(col)))
        st = OracleState(arc_row=np.zeros(n + 1, np.int64), head=np.zeros(max(na, 1), np.int32),
                         rev=np.zeros(max(na, 1), np.int64), cap=np.zeros(max(na, 1), np.int64),
                         r=np.zeros(max(na, 1), np.int64), excess=np.zeros(n, np.int64),
                         height=np.zeros(n, np.int32))
        rc = L.orc_maxflow_fifo(n, col.shape[0], _p(row_ptr), _p(col), _p(cap), s, t, _p(flow),
                                _p(st.arc_row), _p(st.head), _p(st.rev), _p(st.cap), _p(st.r),
                                _p(st.excess), _p(st.height))
        for f in ("head", "rev", "cap", "r"):
            setattr(st, f, getattr(st, f)[:na])
    else:
        rc = L.orc_maxflow_fifo(n, col.shape[0], _p(row_ptr), _p(col), _p(cap), s, t, _p(flow),
                                None, None, None, None, None, None, None)
    if rc != 0:
        raise ValueError(f"orc_maxflow_fifo failed: {rc}")
    return (int(flow[0]), st) if want_state else int(flow[0])


def maxflow_ek(n, row_ptr, col, cap, s, t) -> int:
    row_ptr, col, cap = _csr(row_ptr, col, cap)
    flow = np.zeros(1, dtype=np.int64)
    rc = lib().orc_maxflow_ek(n, col.shape[0], _p(row_ptr), _p(col), _p(cap), s, t, _p(flow))
    if rc != 0:
        raise ValueError(f"orc_maxflow_ek failed: {rc}")
    return int(flow[0])


def mincut_brute(n, row_ptr, col, cap, s, t) -> int:
    row_ptr, col, cap = _csr(row_ptr, col, cap)
    out = np.zeros(1, dtype=np.int64)
    rc = lib().orc_mincut_brute(n, col.shape[0], _p(row_ptr), _p(col), _p(cap), s, t, _p(out))
    if rc != 0:
        raise ValueError(f"orc_mincut_brute failed: {rc}")
    return int(out[0])


def bfs_heights(n, arc_row, head, rev, r, root, s) -> np.ndarray:
    arc_row = np.ascontiguousarray(arc_row, dtype=np.int64)
    head = np.ascontiguousarray(head, dtype=np.int32)
    rev = np.ascontiguousarray(rev, dtype=np.int64)
    r = np.ascontiguousarray(r, dtype=np.int64)
    root = np.ascontiguousarray(root, dtype=np.uint8)
    h = np.zeros(n, dtype=np.int32)
    rc = lib().orc_bfs_heights(n, _p(arc_row), _p(head), _p(rev), _p(r), _p(root), s, _p(h))
    if rc != 0:
        raise ValueError(f"orc_bfs_heights failed: {rc}")
    return h


def certify(n, row_ptr, col, cap, s, t, arc_row, head, rev, arc_cap, r, excess, side,
            flow, height=None):
    """Return (fail_bits, where, names).  fail_bits == 0 means the state is a
    certified maximum flow of value ``flow`` for the edge capacities given."""
    row_ptr, col, cap = _csr(row_ptr, col, cap)
    arc_row = np.ascontiguousarray(arc_row, dtype=np.int64)
    head = np.ascontiguousarray(head, dtype=np.int32)
    rev = np.ascontiguousarray(rev, dtype=np.int64)
    arc_cap = np.ascontiguousarray(arc_cap, dtype=np.int64)
    r = np.ascontiguousarray(r, dtype=np.int64)
    excess = np.ascontiguousarray(excess, dtype=np.int64)
    side = np.ascontiguousarray(side, dtype=np.uint8)
    if height is not None:
        height = np.ascontiguousarray(height, dtype=np.int32)
    bits = np.zeros(1, dtype=np.uint32)
    where = np.zeros(1, dtype=np.int64)
    rc = lib().orc_certify(n, col.shape[0], _p(row_ptr), _p(col), _p(cap), s, t, _p(arc_row),
                           _p(head), _p(rev), _p(arc_cap), _p(r), _p(excess), _p(side),
                           _p(height), int(flow), _p(bits), _p(where))
    if rc != 0:
        raise ValueError(f"orc_certify failed: {rc}")
    b = int(bits[0])
    return b, int(where[0]), [CERT_BITS[i] for i in range(8) if b >> i & 1]
