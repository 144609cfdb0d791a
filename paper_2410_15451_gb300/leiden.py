"""Python binding of the C ABI in include/leiden_gb300.h (ctypes; argument
marshalling only -- every step of the computation runs in the CUDA library).

The functions keep the C names.  Host arrays are numpy; device arrays may be
anything exposing ``data_ptr()`` (e.g. torch CUDA tensors) or a raw int
pointer.  Loading fails loudly when ``libleiden_gb300.so`` has not been
built (see ``paper_2410_15451_gb300._build.build``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LEIDEN_OK, LEIDEN_ERR_ARG, LEIDEN_ERR_BATCH, LEIDEN_ERR_OOM = 0, 1, 2, 3
LEIDEN_ERR_CUDA, LEIDEN_ERR_TIMEOUT, LEIDEN_ERR_STATE = 4, 5, 6
LEIDEN_ND, LEIDEN_DS, LEIDEN_DF = 0, 1, 2
TRACE_WORDS = 2 + 10 * 25

_lib = None


class leiden_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tau_drop", ctypes.c_double), ("tau_refine", ctypes.c_double),
                ("max_iterations", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("classes", ctypes.c_int32),
                ("slack", ctypes.c_double), ("min_slack", ctypes.c_int32), ("collect_stats", ctypes.c_int32),
                ("split_all", ctypes.c_int32), ("converge_any", ctypes.c_int32), ("arena_log2", ctypes.c_int32)]


class leiden_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "passes", "lm_iterations", "lm_vertices", "lm_arcs", "lm_moves", "refine_vertices", "refine_arcs",
        "aggregate_arcs", "affected", "communities", "batch_arcs")] + [(k, ctypes.c_double) for k in (
        "ms_total", "ms_batch", "ms_move", "ms_refine", "ms_aggregate", "ms_track")] + [
        (k, ctypes.c_int64 * 3) for k in ("lmk_launches", "lmk_vertices", "lmk_arcs", "lmk_bytes")] + [
        ("lmk_ms", ctypes.c_double * 3), ("rebuilds", ctypes.c_int64), ("phase_ms", ctypes.c_double * 6),
        ("phase_bytes", ctypes.c_int64 * 6), ("xk_launches", ctypes.c_int64 * 3), ("xk_bytes", ctypes.c_int64 * 3),
        ("xk_ms", ctypes.c_double * 3), ("agg_tables", ctypes.c_int64 * 2)]

PHASES = ("batch", "move", "split", "refine", "aggregate", "track")


class leiden_tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("tiny_max", "warp_max", "block_max", "warp_blocks_per_sm",
                                              "block_blocks_per_sm", "hub_blocks_per_sm", "overlap")]


class leiden_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "graphs_resident", "graphs_waiting", "requests_queued", "requests_running", "requests_done", "bytes_used",
        "bytes_budget")]


class LeidenError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"leiden status {status}: {message}")
        self.status = status


def library_path() -> str:
    """The library this process loads: libleiden_gb300.so, or the checked
    build libleiden_gb300_checked.so when LEIDEN_GB300_CHECKED=1."""
    return _build.LIB_PATH_CHECKED if os.environ.get("LEIDEN_GB300_CHECKED") == "1" else _build.LIB_PATH


def load():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_2410_15451_gb300._build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    P = ctypes.POINTER
    lib.leiden_default_params.argtypes = [P(leiden_params)]
    lib.leiden_default_params.restype = None
    lib.leiden_create.argtypes = [P(leiden_params), i64, vp, vp, vp, vp, P(vp)]
    lib.leiden_static.argtypes = [vp, vp]
    lib.leiden_update.argtypes = [vp, vp, i64, vp, i64, ctypes.c_int, vp]
    lib.leiden_update_device.argtypes = [vp, vp, i64, vp, i64, ctypes.c_int, vp]
    lib.leiden_modularity.argtypes = [vp, vp, P(ctypes.c_double)]
    lib.leiden_membership_device.argtypes = [vp, P(vp)]
    lib.leiden_modularity_noalloc.argtypes = [i64, vp, vp, vp, vp, vp, P(ctypes.c_double)]
    lib.leiden_modularity_noalloc.restype = ctypes.c_int
    lib.leiden_get_state.argtypes = [vp, vp, vp, vp, vp, P(i64)]
    lib.leiden_import_state.argtypes = [vp, vp, vp]
    lib.leiden_import_state.restype = ctypes.c_int
    lib.leiden_graph_arcs.argtypes = [vp]
    lib.leiden_graph_arcs.restype = i64
    lib.leiden_get_graph.argtypes = [vp, vp, vp, vp]
    lib.leiden_get_affected.argtypes = [vp, vp]
    lib.leiden_get_trace.argtypes = [vp, vp]
    lib.leiden_get_stats.argtypes = [vp, P(leiden_stats)]
    lib.leiden_create_batched.argtypes = [P(leiden_params), i32, vp, vp, vp, vp, vp, P(vp)]
    lib.leiden_create_batched.restype = ctypes.c_int
    lib.leiden_batch_graphs.argtypes = [vp]
    lib.leiden_batch_graphs.restype = i32
    lib.leiden_batch_trace.argtypes = [vp, i32, vp]
    lib.leiden_batch_trace.restype = ctypes.c_int
    lib.leiden_batch_modularity.argtypes = [vp, vp]
    lib.leiden_batch_modularity.restype = ctypes.c_int
    lib.leiden_default_tuning.argtypes = [P(leiden_tuning)]
    lib.leiden_default_tuning.restype = None
    lib.leiden_set_tuning.argtypes = [vp, P(leiden_tuning)]
    lib.leiden_set_tuning.restype = ctypes.c_int
    lib.leiden_footprint_bytes.argtypes = [P(leiden_params), i64, vp]
    lib.leiden_footprint_bytes.restype = i64
    lib.leiden_transient_bytes.argtypes = [i64, vp]
    lib.leiden_transient_bytes.restype = i64
    d = ctypes.c_double
    for name, args in (("leiden_server_create", [P(leiden_params), i64, i32, P(vp)]),
                       ("leiden_server_add_graph", [vp, i64, vp, vp, vp, P(i32)]),
                       ("leiden_server_submit", [vp, i32, vp, i64, vp, i64, ctypes.c_int, i32, P(i64)]),
                       ("leiden_server_wait", [vp, i64, vp, P(d), P(d)]),
                       ("leiden_server_wait_for", [vp, i64, d, vp, P(d), P(d)]),
                       ("leiden_server_membership", [vp, i32, vp]),
                       ("leiden_server_remove_graph", [vp, i32]),
                       ("leiden_server_get_stats", [vp, P(leiden_server_stats)])):
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = ctypes.c_int
    lib.leiden_server_last_error.argtypes = [vp]
    lib.leiden_server_last_error.restype = ctypes.c_char_p
    lib.leiden_server_destroy.argtypes = [vp]
    lib.leiden_server_destroy.restype = None
    lib.leiden_kernel_launches.argtypes = []
    lib.leiden_kernel_launches.restype = i64
    lib.leiden_checked_build.argtypes = []
    lib.leiden_checked_build.restype = i32
    lib.leiden_check_selftest.argtypes = [vp]
    lib.leiden_check_selftest.restype = i32
    lib.leiden_last_error.argtypes = [vp]
    lib.leiden_last_error.restype = ctypes.c_char_p
    lib.leiden_destroy.argtypes = [vp]
    lib.leiden_destroy.restype = None
    for f in ("leiden_create", "leiden_static", "leiden_update", "leiden_update_device", "leiden_modularity",
              "leiden_membership_device", "leiden_get_state", "leiden_get_graph", "leiden_get_affected",
              "leiden_get_trace", "leiden_get_stats"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _check(h, st):
    if st != LEIDEN_OK:
        msg = load().leiden_last_error(h)
        raise LeidenError(st, msg.decode() if msg else "")


# ---- C-named functions ---------------------------------------------------------------

def leiden_default_params() -> leiden_params:
    p = leiden_params()
    load().leiden_default_params(ctypes.byref(p))
    return p


def leiden_create(params, n, offsets, cols, weights=None, cuda_stream=None) -> int:
    lib = load()
    offsets = np.ascontiguousarray(offsets, np.int64)
    cols = np.ascontiguousarray(cols, np.int32)
    weights = None if weights is None else np.ascontiguousarray(weights, np.int32)
    h = ctypes.c_void_p()
    st = lib.leiden_create(ctypes.byref(params) if params is not None else None, int(n), _ptr(offsets), _ptr(cols),
                           _ptr(weights), cuda_stream, ctypes.byref(h))
    _check(None, st)
    return h.value


def leiden_static(h, membership_out=None):
    _check(h, load().leiden_static(h, _ptr(membership_out)))


def leiden_update(h, dels, ins, mode, membership_out=None):
    dels = np.ascontiguousarray(np.asarray(dels, np.int32).reshape(-1, 3))
    ins = np.ascontiguousarray(np.asarray(ins, np.int32).reshape(-1, 3))
    _check(h, load().leiden_update(h, _ptr(dels), len(dels), _ptr(ins), len(ins), int(mode), _ptr(membership_out)))


def leiden_update_device(h, d_dels, n_del, d_ins, n_ins, mode, d_membership_out=None):
    _check(h, load().leiden_update_device(h, _ptr(d_dels), int(n_del), _ptr(d_ins), int(n_ins), int(mode),
                                          _ptr(d_membership_out)))


def leiden_modularity(h, membership=None) -> float:
    q = ctypes.c_double()
    m = None if membership is None else np.ascontiguousarray(membership, np.int32)
    _check(h, load().leiden_modularity(h, _ptr(m), ctypes.byref(q)))
    return q.value


def leiden_modularity_noalloc(n, d_offsets, d_cols, d_weights, d_membership, cuda_stream=None) -> float:
    """Modularity on a caller-owned device CSR without any device allocation
    (for callers that may not allocate; see the C header for the limits)."""
    q = ctypes.c_double()
    _check(None, load().leiden_modularity_noalloc(int(n), _ptr(d_offsets), _ptr(d_cols), _ptr(d_weights),
                                                  _ptr(d_membership), cuda_stream, ctypes.byref(q)))
    return q.value


def leiden_membership_device(h) -> int:
    p = ctypes.c_void_p()
    _check(h, load().leiden_membership_device(h, ctypes.byref(p)))
    return p.value


def leiden_get_state(h, n):
    C = np.zeros(n, np.int32)
    K = np.zeros(n, np.int64)
    S = np.zeros(n, np.int64)
    dS = np.zeros(n, np.int64)
    m2 = ctypes.c_int64()
    _check(h, load().leiden_get_state(h, _ptr(C), _ptr(K), _ptr(S), _ptr(dS), ctypes.byref(m2)))
    return dict(C=C, K=K, Sigma=S, dSigma=dS, m2=m2.value)


def leiden_import_state(h, C, dSigma):
    C = np.ascontiguousarray(C, np.int32)
    dS = np.ascontiguousarray(dSigma, np.int64)
    _check(h, load().leiden_import_state(h, _ptr(C), _ptr(dS)))


def leiden_graph_arcs(h) -> int:
    return int(load().leiden_graph_arcs(h))


def leiden_get_graph(h, n):
    arcs = leiden_graph_arcs(h)
    off = np.zeros(n + 1, np.int64)
    col = np.zeros(max(arcs, 1), np.int32)
    w = np.zeros(max(arcs, 1), np.int64)
    _check(h, load().leiden_get_graph(h, _ptr(off), _ptr(col), _ptr(w)))
    return off, col[:arcs], w[:arcs]


def leiden_get_affected(h, n):
    dV = np.zeros(n, np.uint8)
    _check(h, load().leiden_get_affected(h, _ptr(dV)))
    return dV


def leiden_get_trace(h) -> dict:
    t = np.zeros(TRACE_WORDS, np.int64)
    _check(h, load().leiden_get_trace(h, _ptr(t)))
    return _trace_dict(t)


def _trace_dict(t) -> dict:
    passes = []
    for p in range(int(t[0])):
        r = t[2 + p * 25: 2 + (p + 1) * 25]
        passes.append(dict(n=int(r[0]), iterations=int(r[1]), communities=int(r[2]), refined_any=int(r[3]),
                           refine_rounds=int(r[4]), moves=[int(x) for x in r[5:5 + min(int(r[1]), 20)]]))
    return dict(passes=passes, affected=int(t[1]))


def leiden_get_stats(h) -> dict:
    s = leiden_stats()
    _check(h, load().leiden_get_stats(h, ctypes.byref(s)))
    out = {}
    for k, _ in leiden_stats._fields_:
        v = getattr(s, k)
        out[k] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def leiden_create_batched(params, vertex_offsets, offsets, cols, weights=None, cuda_stream=None) -> int:
    lib = load()
    vo = np.ascontiguousarray(vertex_offsets, np.int64)
    offsets = np.ascontiguousarray(offsets, np.int64)
    cols = np.ascontiguousarray(cols, np.int32)
    weights = None if weights is None else np.ascontiguousarray(weights, np.int32)
    h = ctypes.c_void_p()
    st = lib.leiden_create_batched(ctypes.byref(params) if params is not None else None, len(vo) - 1, _ptr(vo),
                                   _ptr(offsets), _ptr(cols), _ptr(weights), cuda_stream, ctypes.byref(h))
    _check(None, st)
    return h.value


def leiden_batch_graphs(h) -> int:
    return int(load().leiden_batch_graphs(h))


def leiden_batch_trace(h, graph) -> dict:
    t = np.zeros(TRACE_WORDS, np.int64)
    _check(h, load().leiden_batch_trace(h, int(graph), _ptr(t)))
    return _trace_dict(t)


def leiden_batch_modularity(h) -> np.ndarray:
    q = np.zeros(leiden_batch_graphs(h), np.float64)
    _check(h, load().leiden_batch_modularity(h, _ptr(q)))
    return q


def leiden_default_tuning() -> leiden_tuning:
    t = leiden_tuning()
    load().leiden_default_tuning(ctypes.byref(t))
    return t


def leiden_set_tuning(h, **fields):
    """Set launch shapes (defaults for the fields not given)."""
    t = leiden_default_tuning()
    for k, v in fields.items():
        setattr(t, k, int(v))
    _check(h, load().leiden_set_tuning(h, ctypes.byref(t)))


def leiden_kernel_launches() -> int:
    return int(load().leiden_kernel_launches())


def leiden_checked_build() -> bool:
    return bool(load().leiden_checked_build())


def leiden_check_selftest(cuda_stream=None) -> int:
    return int(load().leiden_check_selftest(cuda_stream))


def leiden_last_error(h=None) -> str:
    m = load().leiden_last_error(h)
    return m.decode() if m else ""


def leiden_destroy(h):
    if h:
        load().leiden_destroy(h)


class Leiden:
    """Owning wrapper of a handle: ``Leiden(n, off, col, w).static()``, ``.update(dels, ins, mode)``."""

    def __init__(self, n, off, col, w=None, deterministic=True, cuda_stream=None, **params):
        p = leiden_default_params()
        p.deterministic = 1 if deterministic else 0
        for k, v in params.items():
            setattr(p, k, v)
        self.n = int(n)
        self.h = leiden_create(p, n, off, col, w, cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            leiden_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def static(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        leiden_static(self.h, out)
        return out

    def update(self, dels, ins, mode) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        leiden_update(self.h, dels, ins, mode, out)
        return out

    def modularity(self, membership=None) -> float:
        return leiden_modularity(self.h, membership)

    def state(self):
        return leiden_get_state(self.h, self.n)

    def graph(self):
        return leiden_get_graph(self.h, self.n)

    def affected(self):
        return leiden_get_affected(self.h, self.n)

    def trace(self):
        return leiden_get_trace(self.h)

    def stats(self):
        return leiden_get_stats(self.h)


class LeidenBatch:
    """G graphs in one batched handle (``leiden_create_batched``).

    ``graphs`` is a list of ``(n, off, col, w)`` CSRs; they are concatenated
    with vertex offsets ``self.voff``.  Memberships and batches use the
    concatenated ids; ``local(arr, g)`` gives graph g's slice shifted back to
    its own ids.
    """

    def __init__(self, graphs, cuda_stream=None, **params):
        p = leiden_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        sizes = [int(g[0]) for g in graphs]
        self.voff = np.zeros(len(graphs) + 1, np.int64)
        self.voff[1:] = np.cumsum(sizes)
        offs, cols, ws = [np.zeros(1, np.int64)], [], []
        arc_base = 0
        for (n, off, col, w), v0 in zip(graphs, self.voff[:-1]):
            off = np.asarray(off, np.int64)
            offs.append(off[1:] + arc_base)
            arc_base += int(off[-1])
            cols.append(np.asarray(col, np.int64) + v0)
            ws.append(np.ones(int(off[-1]), np.int32) if w is None else np.asarray(w, np.int32))
        self.n = int(self.voff[-1])
        self.off = np.concatenate(offs)
        self.col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
        self.w = np.concatenate(ws) if ws else np.zeros(0, np.int32)
        self.h = leiden_create_batched(p, self.voff, self.off, self.col, self.w, cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            leiden_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def to_global(self, edges, g):
        """Edge triples of graph g in its own ids -> concatenated ids."""
        e = np.array(edges, np.int32).reshape(-1, 3)
        e[:, :2] += self.voff[g]
        return e

    def local(self, arr, g):
        a, b = int(self.voff[g]), int(self.voff[g + 1])
        return np.asarray(arr)[a:b] - a

    def static(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        leiden_static(self.h, out)
        return out

    def update(self, dels, ins, mode) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        leiden_update(self.h, dels, ins, mode, out)
        return out

    def modularity(self) -> np.ndarray:
        return leiden_batch_modularity(self.h)

    def trace(self, g) -> dict:
        return leiden_batch_trace(self.h, g)

    def state(self):
        return leiden_get_state(self.h, self.n)


def leiden_footprint_bytes(n, offsets, params=None) -> int:
    off = np.ascontiguousarray(offsets, np.int64)
    return int(load().leiden_footprint_bytes(ctypes.byref(params) if params is not None else None, int(n), _ptr(off)))


def leiden_transient_bytes(n, offsets) -> int:
    off = np.ascontiguousarray(offsets, np.int64)
    return int(load().leiden_transient_bytes(int(n), _ptr(off)))


class LeidenServer:
    """Resident graphs and concurrent update requests (``leiden_server_*``)."""

    def __init__(self, device_bytes, slots=4, **params):
        p = leiden_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        self.p = p
        s = ctypes.c_void_p()
        self._check(load().leiden_server_create(ctypes.byref(p), int(device_bytes), int(slots), ctypes.byref(s)),
                    None)
        self.s = s.value
        self.sizes = {}

    def _check(self, st, s):
        if st != LEIDEN_OK:
            msg = load().leiden_server_last_error(s)
            raise LeidenError(st, msg.decode() if msg else "")

    def add_graph(self, n, off, col, w=None) -> int:
        off = np.ascontiguousarray(off, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        w = None if w is None else np.ascontiguousarray(w, np.int32)
        g = ctypes.c_int32()
        self._check(load().leiden_server_add_graph(self.s, int(n), _ptr(off), _ptr(col), _ptr(w), ctypes.byref(g)),
                    self.s)
        self.sizes[g.value] = int(n)
        return g.value

    def submit(self, graph, dels, ins, mode=LEIDEN_DF, keep_membership=False) -> int:
        dels = np.ascontiguousarray(np.asarray(dels, np.int32).reshape(-1, 3))
        ins = np.ascontiguousarray(np.asarray(ins, np.int32).reshape(-1, 3))
        t = ctypes.c_int64()
        self._check(load().leiden_server_submit(self.s, int(graph), _ptr(dels), len(dels), _ptr(ins), len(ins),
                                                int(mode), 1 if keep_membership else 0, ctypes.byref(t)), self.s)
        return (t.value, int(graph), bool(keep_membership))

    def wait(self, ticket):
        """-> (membership or None, latency ms, service ms)"""
        t, graph, keep = ticket
        out = np.zeros(self.sizes[graph], np.int32) if keep else None
        lat, svc = ctypes.c_double(), ctypes.c_double()
        self._check(load().leiden_server_wait(self.s, t, _ptr(out), ctypes.byref(lat), ctypes.byref(svc)), self.s)
        return out, lat.value, svc.value

    def wait_for(self, ticket, timeout_ms):
        """-> (membership or None, latency ms, service ms); LeidenError with
        LEIDEN_ERR_TIMEOUT if not done in time (the ticket stays valid)."""
        t, graph, keep = ticket
        out = np.zeros(self.sizes[graph], np.int32) if keep else None
        lat, svc = ctypes.c_double(), ctypes.c_double()
        self._check(load().leiden_server_wait_for(self.s, t, float(timeout_ms), _ptr(out), ctypes.byref(lat),
                                                  ctypes.byref(svc)), self.s)
        return out, lat.value, svc.value

    def membership(self, graph) -> np.ndarray:
        out = np.zeros(self.sizes[graph], np.int32)
        self._check(load().leiden_server_membership(self.s, int(graph), _ptr(out)), self.s)
        return out

    def remove_graph(self, graph):
        self._check(load().leiden_server_remove_graph(self.s, int(graph)), self.s)

    def stats(self) -> dict:
        st = leiden_server_stats()
        self._check(load().leiden_server_get_stats(self.s, ctypes.byref(st)), self.s)
        return {k: getattr(st, k) for k, _ in leiden_server_stats._fields_}

    def close(self):
        if getattr(self, "s", None):
            load().leiden_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
