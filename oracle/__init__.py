"""CPU oracle for dynamic Leiden -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``liboracle.so`` (plain sequential C, see
leiden_oracle.c).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the product path
(``paper_2410_15451_gb300``) never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

SEQ, SYNC = 0, 1
ND, DS, DF = 0, 1, 2
OK, ERR_ARG, ERR_BATCH, ERR_OOM, ERR_STATE = 0, 1, 2, 3, 6
TRACE_PASS = 25
TRACE_WORDS = 2 + 10 * TRACE_PASS


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "leiden_oracle.c")
    hdr = os.path.join(_HERE, "leiden_oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tau_drop", ctypes.c_double), ("tau_refine", ctypes.c_double),
                ("max_iterations", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("classes", ctypes.c_int32),
                ("split_all", ctypes.c_int32), ("converge_any", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_create.argtypes = [ctypes.POINTER(_Params), i64, vp, vp, vp]
        lib.oracle_create.restype = vp
        lib.oracle_destroy.argtypes = [vp]
        lib.oracle_destroy.restype = None
        lib.oracle_static.argtypes = [vp, vp]
        lib.oracle_update.argtypes = [vp, vp, i64, vp, i64, ctypes.c_int, vp]
        lib.oracle_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.oracle_graph_arcs.argtypes = [vp]
        lib.oracle_graph_arcs.restype = i64
        lib.oracle_get_graph.argtypes = [vp, vp, vp, vp]
        lib.oracle_get_affected.argtypes = [vp, vp]
        lib.oracle_get_trace.argtypes = [vp, vp]
        lib.oracle_modularity.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        lib.oracle_move_gain.argtypes = [i64, vp, vp, vp, vp, i64, i32, vp]
        lib.oracle_aggregate.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.oracle_aggregate.restype = i64
        lib.oracle_split.argtypes = [i64, vp, vp, vp, vp]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def params(schedule=SYNC, tau=1e-2, tau_drop=10.0, tau_refine=0.6, max_iterations=20, max_passes=10,
           classes=4, split_all=0, converge_any=0):
    return _Params(tau, tau_drop, tau_refine, max_iterations, max_passes, schedule, classes, split_all, converge_any)


def _i128(lo, hi) -> int:
    return (int(hi) << 64) | (int(lo) & ((1 << 64) - 1))


def modularity(off, col, w, C) -> tuple[float, int]:
    """Eq. 1 -> (Q as double, exact numerator 2m*sum sigma_c - sum Sigma_c^2)."""
    lib = _load()
    off = np.ascontiguousarray(off, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.int64)
    C = np.ascontiguousarray(C, np.int32)
    q = ctypes.c_double()
    num = np.zeros(2, np.int64)
    rc = lib.oracle_modularity(len(off) - 1, _p(off), _p(col), _p(w), _p(C), ctypes.byref(q), _p(num))
    if rc != OK:
        raise ValueError(f"oracle_modularity rc={rc}")
    return q.value, _i128(num[0], num[1])


def move_gain(off, col, w, C, i, c) -> int:
    """Eq. 2 times 2m^2 as an exact integer."""
    lib = _load()
    off = np.ascontiguousarray(off, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.int64)
    C = np.ascontiguousarray(C, np.int32)
    out = np.zeros(2, np.int64)
    rc = lib.oracle_move_gain(len(off) - 1, _p(off), _p(col), _p(w), _p(C), int(i), int(c), _p(out))
    if rc != OK:
        raise ValueError(f"oracle_move_gain rc={rc}")
    return _i128(out[0], out[1])


def aggregate(off, col, w, C, ncomm):
    lib = _load()
    off = np.ascontiguousarray(off, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.int64)
    C = np.ascontiguousarray(C, np.int32)
    cap = max(int(off[-1]), 1)
    yo = np.zeros(ncomm + 1, np.int64)
    yc = np.zeros(cap, np.int32)
    yw = np.zeros(cap, np.int64)
    arcs = lib.oracle_aggregate(len(off) - 1, _p(off), _p(col), _p(w), _p(C), int(ncomm), _p(yo), _p(yc), _p(yw))
    if arcs < 0:
        raise ValueError("oracle_aggregate failed")
    return yo, yc[:arcs].copy(), yw[:arcs].copy()


def split(off, col, C, split_c):
    lib = _load()
    off = np.ascontiguousarray(off, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    C = np.array(C, np.int32, copy=True)
    split_c = np.ascontiguousarray(split_c, np.uint8)
    rc = lib.oracle_split(len(off) - 1, _p(off), _p(col), _p(C), _p(split_c))
    if rc != OK:
        raise ValueError(f"oracle_split rc={rc}")
    return C


class Oracle:
    """Stateful oracle mirroring the C-ABI of the CUDA library."""

    def __init__(self, n, off, col, w=None, schedule=SYNC, **kw):
        lib = _load()
        self.n = int(n)
        self._off = np.ascontiguousarray(off, np.int64)
        self._col = np.ascontiguousarray(col, np.int32)
        self._w = None if w is None else np.ascontiguousarray(w, np.int32)
        self._params = params(schedule=schedule, **kw)
        h = lib.oracle_create(ctypes.byref(self._params), self.n, _p(self._off), _p(self._col), _p(self._w))
        if not h:
            raise ValueError("oracle_create rejected the graph")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _load().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def static(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        rc = _load().oracle_static(self._h, _p(out))
        if rc != OK:
            raise RuntimeError(f"oracle_static rc={rc}")
        return out

    def update(self, dels, ins, mode) -> np.ndarray:
        dels = np.ascontiguousarray(np.asarray(dels, np.int32).reshape(-1, 3))
        ins = np.ascontiguousarray(np.asarray(ins, np.int32).reshape(-1, 3))
        out = np.zeros(self.n, np.int32)
        rc = _load().oracle_update(self._h, _p(dels), len(dels), _p(ins), len(ins), int(mode), _p(out))
        if rc != OK:
            raise OracleError(rc)
        return out

    def state(self):
        C = np.zeros(self.n, np.int32)
        K = np.zeros(self.n, np.int64)
        S = np.zeros(self.n, np.int64)
        dS = np.zeros(self.n, np.int64)
        m2 = ctypes.c_int64()
        _load().oracle_get_state(self._h, _p(C), _p(K), _p(S), _p(dS), ctypes.byref(m2))
        return dict(C=C, K=K, Sigma=S, dSigma=dS, m2=m2.value)

    def graph(self):
        lib = _load()
        arcs = lib.oracle_graph_arcs(self._h)
        off = np.zeros(self.n + 1, np.int64)
        col = np.zeros(max(arcs, 1), np.int32)
        w = np.zeros(max(arcs, 1), np.int64)
        lib.oracle_get_graph(self._h, _p(off), _p(col), _p(w))
        return off, col[:arcs], w[:arcs]

    def affected(self) -> np.ndarray:
        dV = np.zeros(self.n, np.uint8)
        _load().oracle_get_affected(self._h, _p(dV))
        return dV

    def trace(self) -> dict:
        t = np.zeros(TRACE_WORDS, np.int64)
        _load().oracle_get_trace(self._h, _p(t))
        passes = []
        for p in range(int(t[0])):
            r = t[2 + p * TRACE_PASS: 2 + (p + 1) * TRACE_PASS]
            passes.append(dict(n=int(r[0]), iterations=int(r[1]), communities=int(r[2]),
                               refined_any=int(r[3]), refine_rounds=int(r[4]),
                               moves=[int(x) for x in r[5:5 + min(int(r[1]), 20)]]))
        return dict(passes=passes, affected=int(t[1]))

    def modularity(self, C=None) -> float:
        off, col, w = self.graph()
        st = self.state()
        return modularity(off, col, w, st["C"] if C is None else C)[0]


class OracleError(RuntimeError):
    def __init__(self, rc):
        super().__init__(f"oracle status {rc}")
        self.rc = rc
