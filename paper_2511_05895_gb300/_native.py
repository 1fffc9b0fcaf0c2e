"""ctypes binding of libmfgpu.so (the C ABI declared in include/mf.h).

Argument marshalling only: every step of the solve and of the dynamic repair
runs in the library's CUDA kernels.  There is no CPU fallback -- if the
library is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_ENOTSOLVED, MF_ETIMEOUT, MF_ECHECK = range(7)
MF_HOST_PTRS, MF_DEVICE_PTRS, MF_DELTA, MF_RECOMPUTE = 0x0, 0x1, 0x2, 0x4
MF_POLICY_FIXED, MF_POLICY_PLAIN, MF_POLICY_LEARNED = 0, 1, 2
MF_MODE_DATA_DRIVEN, MF_MODE_TOPOLOGY, MF_MODE_PUSH_PULL = 0, 1, 2

ERROR_NAMES = {MF_EINVAL: "MF_EINVAL", MF_ENOMEM: "MF_ENOMEM", MF_ECUDA: "MF_ECUDA",
               MF_ENOTSOLVED: "MF_ENOTSOLVED", MF_ETIMEOUT: "MF_ETIMEOUT", MF_ECHECK: "MF_ECHECK"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("kernel_cycles", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("max_iters", ctypes.c_int64), ("grid_blocks", ctypes.c_int32),
                ("time_limit_ms", ctypes.c_int32), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("debug_checks", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "flow", "iterations", "bfs_levels", "bfs_vertices", "bfs_arcs", "worklist", "pr_arcs",
        "pushes", "relabels", "ri_arcs", "ri_moves", "batch", "clamped", "resat_arcs", "n", "m",
        "arcs", "t_batch_ns", "t_reset_ns", "t_bfs_ns", "t_pr_ns", "t_hub_ns", "t_ri_ns",
        "hub_cycles", "barriers", "bfs_bottom_up_levels", "pr_rounds")] + [
        (f, ctypes.c_int32) for f in ("policy_kind", "policy_kernel_cycles", "policy_fallback",
                                      "exit_kind")] + [(f, ctypes.c_int32) for f in ("status", "kernel_cycles", "grid_blocks",
                                                   "block_threads", "policy_mode", "reserved0")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved0"}


# every symbol include/mf.h declares (checked by the CPU test suite)
EXPORTED = ["mf_options_default", "mf_create", "mf_cap_limit", "mf_solve", "mf_apply_updates",
            "mf_sync", "mf_flow_value", "mf_min_cut", "mf_stats_get", "mf_sizes",
            "mf_export_graph", "mf_export_state", "mf_import_state", "mf_destroy",
            "mf_strerror", "mf_version", "mf_last_error", "mf_bicsr_host", "mf_solve_bicsr_noalloc",
            "mf_trace_enable", "mf_trace_read", "mf_set_time_limit", "mf_set_policy", "mf_policy_features",
            "mf_mlp_sizes", "mf_mlp_workspace_bytes", "mf_mlp_forward", "mf_mlp_grad", "mf_mlp_train",
            "mf_apply_updates_dev", "mf_flow_value_async", "mf_set_stream", "mf_device_bytes", "mf_grid_blocks", "mf_set_grid_blocks",
            "mf_server_options_default", "mf_server_create", "mf_server_add_graph", "mf_server_submit",
            "mf_server_poll", "mf_server_drain", "mf_server_stats_get", "mf_server_reset_stats",
            "mf_server_destroy"]


class TraceRec(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int16), ("mode", ctypes.c_int16), ("iter", ctypes.c_int32),
                ("step", ctypes.c_int32), ("count", ctypes.c_int32), ("ns", ctypes.c_int64)]


PHASES = ["batch", "height_init", "bfs", "push_relabel", "hub", "remove_invalid"]


class MFError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)} {detail}".strip())


_lib = None


def lib(build_if_missing: bool = False):
    """Load libmfgpu.so.  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"{_build.LIB} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(_build.LIB)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "mf_options_default": ([P], ctypes.c_int),
        "mf_create": ([i32, i64, P, P, P, i32, i32, P, P, P], ctypes.c_int),
        "mf_cap_limit": ([P, P], ctypes.c_int),
        "mf_solve": ([P, P], ctypes.c_int),
        "mf_apply_updates": ([P, i64, P, P, i32, P], ctypes.c_int),
        "mf_sync": ([P], ctypes.c_int),
        "mf_flow_value": ([P, P], ctypes.c_int),
        "mf_min_cut": ([P, P, i32], ctypes.c_int),
        "mf_stats_get": ([P, P], ctypes.c_int),
        "mf_sizes": ([P, P, P, P], ctypes.c_int),
        "mf_export_graph": ([P, P, P, P, P], ctypes.c_int),
        "mf_export_state": ([P, P, P, P, i32], ctypes.c_int),
        "mf_import_state": ([P, P, P, P, i32], ctypes.c_int),
        "mf_destroy": ([P], None),
        "mf_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "mf_version": ([], ctypes.c_char_p),
        "mf_last_error": ([], ctypes.c_char_p),
        "mf_bicsr_host": ([i32, i64, P, P, P, i32, i32, P, P, P, P, P, P, P], ctypes.c_int),
        "mf_solve_bicsr_noalloc": ([i32, i64, P, P, P, P, i32, i32, i32, P, P, P, P, P], ctypes.c_int),
        "mf_trace_enable": ([P, i32], ctypes.c_int),
        "mf_set_time_limit": ([P, i32], ctypes.c_int),
        "mf_trace_read": ([P, P, i32, P], ctypes.c_int),
        "mf_set_policy": ([P, i32, P], ctypes.c_int),
        "mf_policy_features": ([P, i64, P, P, i32, P], ctypes.c_int),
        "mf_mlp_sizes": ([P, P, P, P], ctypes.c_int),
        "mf_mlp_workspace_bytes": ([i32], i64),
        "mf_mlp_forward": ([P, P, i32, P, P], ctypes.c_int),
        "mf_mlp_grad": ([P, P, P, P, P, i32, ctypes.c_float, ctypes.c_float, P, P, P, P], ctypes.c_int),
        "mf_mlp_train": ([P, P, P, P, P, P, P, i32, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32,
                          P, P, P], ctypes.c_int),
        "mf_apply_updates_dev": ([P, P, i64, P, P, i32, P], ctypes.c_int),
        "mf_flow_value_async": ([P, P, P], ctypes.c_int),
        "mf_set_stream": ([P, P], ctypes.c_int),
        "mf_device_bytes": ([P, P], ctypes.c_int),
        "mf_grid_blocks": ([P, P], ctypes.c_int),
        "mf_set_grid_blocks": ([P, i32], ctypes.c_int),
        "mf_server_options_default": ([P], ctypes.c_int),
        "mf_server_create": ([P, P], ctypes.c_int),
        "mf_server_add_graph": ([P, P, i64, P], ctypes.c_int),
        "mf_server_submit": ([P, i32, i64, P, P, i32, P], ctypes.c_int),
        "mf_server_poll": ([P, i64, P, P, P, P], ctypes.c_int),
        "mf_server_drain": ([P], ctypes.c_int),
        "mf_server_stats_get": ([P, P], ctypes.c_int),
        "mf_server_reset_stats": ([P], None),
        "mf_server_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc, where):
    if rc != MF_OK:
        raise MFError(rc, where, lib().mf_last_error().decode(errors="replace"))


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def bicsr_host(n, row_ptr, col, cap, s, t):
    """Host-only Bi-CSR construction (no GPU needed): returns a dict with
    arc_row, head, rev, cap, arc_of_edge and cap_limit."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    cap = np.ascontiguousarray(cap, dtype=np.int32)
    L = lib()
    arcs = ctypes.c_int64(0)
    _check(L.mf_bicsr_host(n, col.shape[0], _np_ptr(row_ptr), _np_ptr(col), _np_ptr(cap), s, t,
                           ctypes.byref(arcs), None, None, None, None, None, None), "mf_bicsr_host")
    A = arcs.value
    out = dict(arc_row=np.zeros(n + 1, np.int64), head=np.zeros(max(A, 1), np.int32),
               rev=np.zeros(max(A, 1), np.int32), cap=np.zeros(max(A, 1), np.int32),
               arc_of_edge=np.zeros(max(col.shape[0], 1), np.int32))
    lim = ctypes.c_int32(0)
    _check(L.mf_bicsr_host(n, col.shape[0], _np_ptr(row_ptr), _np_ptr(col), _np_ptr(cap), s, t,
                           ctypes.byref(arcs), _np_ptr(out["arc_row"]), _np_ptr(out["head"]),
                           _np_ptr(out["rev"]), _np_ptr(out["cap"]), _np_ptr(out["arc_of_edge"]),
                           ctypes.byref(lim)), "mf_bicsr_host")
    for k in ("head", "rev", "cap"):
        out[k] = out[k][:A]
    out["arc_of_edge"] = out["arc_of_edge"][:col.shape[0]]
    out["cap_limit"] = lim.value
    return out


def _torch():
    import torch
    return torch


def _current_stream():
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _array_arg(x, dtype):
    """(pointer, flags, keepalive) for a numpy array or a torch tensor."""
    try:
        torch = _torch()
        if isinstance(x, torch.Tensor):
            want = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
            if x.dtype != want or not x.is_contiguous():
                x = x.to(want).contiguous()
            return ctypes.c_void_p(x.data_ptr()), (MF_DEVICE_PTRS if x.is_cuda else 0), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return _np_ptr(a), 0, a


class MaxFlowGraph:
    """A flow network resident on the current CUDA device.

    Thin wrapper over mf_create / mf_solve / mf_apply_updates / mf_flow_value
    / mf_min_cut (include/mf.h).  Arrays may be numpy arrays or torch tensors
    (CPU or CUDA); the stream defaults to torch's current stream."""

    def __init__(self, n, row_ptr, col, cap, s, t, *, kernel_cycles=0, max_iters=0,
                 grid_blocks=0, time_limit_ms=0, mode=MF_MODE_DATA_DRIVEN, torch_allocator=False,
                 debug_checks=False, stream=None):
        L = lib()
        self._opt = Options()
        L.mf_options_default(ctypes.byref(self._opt))
        self._opt.kernel_cycles = kernel_cycles
        self._opt.max_iters = max_iters
        self._opt.grid_blocks = grid_blocks
        self._opt.time_limit_ms = time_limit_ms
        self._opt.mode = mode
        self._opt.debug_checks = 1 if debug_checks else 0
        self._keep = []
        if torch_allocator:
            torch = _torch()
            dev = torch.cuda.current_device()

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
                except RuntimeError:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._keep += [ALLOC_FN(_alloc), FREE_FN(_free)]
            self._opt.alloc, self._opt.free = self._keep[0], self._keep[1]
        rp, _, k1 = _array_arg(row_ptr, np.int64)
        cp, _, k2 = _array_arg(col, np.int32)
        kp, _, k3 = _array_arg(cap, np.int32)
        self.n, self.s, self.t = int(n), int(s), int(t)
        self.m = int(k2.shape[0]) if hasattr(k2, "shape") else int(len(k2))
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        _check(L.mf_create(self.n, self.m, rp, cp, kp, self.s, self.t, ctypes.byref(self._opt), st,
                           ctypes.byref(h)), "mf_create")
        self._h = h

    # -- lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().mf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- operations -------------------------------------------------------------
    def solve(self, stream=None):
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        _check(lib().mf_solve(self._h, st), "mf_solve")

    def apply_updates(self, edge_id, new_cap, *, delta=False, recompute=False, stream=None):
        ip, f1, k1 = _array_arg(edge_id, np.int32)
        cp, f2, k2 = _array_arg(new_cap, np.int32)
        if f1 != f2:
            raise ValueError("edge_id and new_cap must both be host or both be device arrays")
        k = int(k1.shape[0]) if hasattr(k1, "shape") else len(k1)
        flags = f1 | (MF_DELTA if delta else 0) | (MF_RECOMPUTE if recompute else 0)
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        _check(lib().mf_apply_updates(self._h, k, ip, cp, flags, st), "mf_apply_updates")
        self._keep_batch = (k1, k2)   # host buffers must outlive the async copy

    def sync(self):
        _check(lib().mf_sync(self._h), "mf_sync")

    def set_time_limit(self, time_limit_ms):
        """Wall-clock limit of the following solve/repair kernels (0 = 60 s)."""
        _check(lib().mf_set_time_limit(self._h, int(time_limit_ms)), "mf_set_time_limit")

    def flow_value(self) -> int:
        out = ctypes.c_int64(0)
        _check(lib().mf_flow_value(self._h, ctypes.byref(out)), "mf_flow_value")
        return out.value

    def min_cut(self) -> np.ndarray:
        side = np.zeros(self.n, dtype=np.uint8)
        _check(lib().mf_min_cut(self._h, _np_ptr(side), MF_HOST_PTRS), "mf_min_cut")
        return side

    def stats(self) -> dict:
        s = Stats()
        _check(lib().mf_stats_get(self._h, ctypes.byref(s)), "mf_stats_get")
        return s.as_dict()

    def trace_enable(self, capacity=4096):
        _check(lib().mf_trace_enable(self._h, int(capacity)), "mf_trace_enable")

    def trace(self, max_records=4096):
        """Records of the last solve/repair: a list of dicts (phase name, mode,
        iter, step, count, ns)."""
        buf = (TraceRec * max_records)()
        cnt = ctypes.c_int32(0)
        _check(lib().mf_trace_read(self._h, buf, max_records, ctypes.byref(cnt)), "mf_trace_read")
        return [dict(phase=PHASES[r.phase], mode=r.mode, iter=r.iter, step=r.step, count=r.count, ns=r.ns)
                for r in buf[:min(cnt.value, max_records)]]

    def set_policy(self, mode, params=None):
        """mode: MF_POLICY_FIXED / _PLAIN / _LEARNED; params: float32 network
        parameters (numpy, mf_mlp_sizes' n_total) for the learned policy."""
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().mf_set_policy(self._h, int(mode), None if p is None else _np_ptr(p)), "mf_set_policy")

    def policy_features(self, edge_id, new_cap, *, delta=False):
        ip, f1, k1 = _array_arg(edge_id, np.int32)
        cp, f2, k2 = _array_arg(new_cap, np.int32)
        k = int(k1.shape[0]) if hasattr(k1, "shape") else len(k1)
        out = np.zeros(12, np.float32)
        _check(lib().mf_policy_features(self._h, k, ip, cp, f1 | (MF_DELTA if delta else 0), _np_ptr(out)),
               "mf_policy_features")
        return out

    def cap_limit(self) -> int:
        v = ctypes.c_int32(0)
        _check(lib().mf_cap_limit(self._h, ctypes.byref(v)), "mf_cap_limit")
        return v.value

    def sizes(self):
        n, m, a = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().mf_sizes(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(a)), "mf_sizes")
        return n.value, m.value, a.value

    def export_graph(self) -> dict:
        n, m, A = self.sizes()
        out = dict(arc_row=np.zeros(n + 1, np.int64), head=np.zeros(max(A, 1), np.int32),
                   rev=np.zeros(max(A, 1), np.int32), cap=np.zeros(max(A, 1), np.int32))
        _check(lib().mf_export_graph(self._h, _np_ptr(out["arc_row"]), _np_ptr(out["head"]),
                                     _np_ptr(out["rev"]), _np_ptr(out["cap"])), "mf_export_graph")
        for k in ("head", "rev", "cap"):
            out[k] = out[k][:A]
        return out

    def export_state(self):
        n, m, A = self.sizes()
        r = np.zeros(max(A, 1), np.int32)
        e = np.zeros(n, np.int64)
        h = np.zeros(n, np.int32)
        _check(lib().mf_export_state(self._h, _np_ptr(r), _np_ptr(e), _np_ptr(h), MF_HOST_PTRS),
               "mf_export_state")
        return r[:A], e, h

    def import_state(self, r, e, h):
        r = np.ascontiguousarray(r, np.int32)
        e = np.ascontiguousarray(e, np.int64)
        h = np.ascontiguousarray(h, np.int32)
        _check(lib().mf_import_state(self._h, _np_ptr(r), _np_ptr(e), _np_ptr(h), MF_HOST_PTRS),
               "mf_import_state")


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("sm_slots", ctypes.c_int32),
                ("use_cuda_graphs", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("max_inflight", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("captured_graphs", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("makespan_s", ctypes.c_double), ("replays", ctypes.c_int64), ("direct_launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Server:
    """Continuous-batching server over several resident graphs (mf_server_*).

    Graphs are added once solved; afterwards only the server drives them."""

    def __init__(self, hbm_budget_bytes=0, sm_slots=0, use_cuda_graphs=True):
        L = lib()
        o = ServerOptions()
        L.mf_server_options_default(ctypes.byref(o))
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        o.sm_slots = int(sm_slots)
        o.use_cuda_graphs = 1 if use_cuda_graphs else 0
        h = ctypes.c_void_p()
        _check(L.mf_server_create(ctypes.byref(o), ctypes.byref(h)), "mf_server_create")
        self._h = h
        self._graphs = []

    def add_graph(self, G, max_batch):
        idx = ctypes.c_int32(-1)
        _check(lib().mf_server_add_graph(self._h, G._h, int(max_batch), ctypes.byref(idx)), "mf_server_add_graph")
        self._graphs.append(G)
        return idx.value

    def submit(self, graph, edge_id, new_cap, *, delta=False, recompute=False):
        ids = np.ascontiguousarray(edge_id, np.int32)
        caps = np.ascontiguousarray(new_cap, np.int32)
        t = ctypes.c_int64(0)
        flags = (MF_DELTA if delta else 0) | (MF_RECOMPUTE if recompute else 0)
        _check(lib().mf_server_submit(self._h, int(graph), ids.shape[0], _np_ptr(ids), _np_ptr(caps), flags,
                                      ctypes.byref(t)), "mf_server_submit")
        return t.value

    def poll(self, ticket):
        d, c = ctypes.c_int32(0), ctypes.c_int32(0)
        f = ctypes.c_int64(0)
        lat = ctypes.c_double(0)
        _check(lib().mf_server_poll(self._h, int(ticket), ctypes.byref(d), ctypes.byref(f), ctypes.byref(c),
                                    ctypes.byref(lat)), "mf_server_poll")
        return bool(d.value), f.value, c.value, lat.value

    def drain(self):
        _check(lib().mf_server_drain(self._h), "mf_server_drain")

    def stats(self):
        s = ServerStats()
        _check(lib().mf_server_stats_get(self._h, ctypes.byref(s)), "mf_server_stats_get")
        return s.as_dict()

    def reset_stats(self):
        lib().mf_server_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().mf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
