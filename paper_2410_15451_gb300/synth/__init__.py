"""Seeded synthetic graphs and batch updates (no community-detection arithmetic).

The workloads stand in for the paper's SuiteSparse graphs and random batch
updates (Evaluation, "Batch generation": 80% insertions of uniformly chosen
vertex pairs, 20% deletions of uniformly chosen existing edges, unit weights,
undirected, no new vertices).  Generation runs in ``libsynth.so`` (plain C,
SplitMix64 counter-based draws), so the same seed gives the same bytes on any
host.  Both the CUDA path's tests/benchmark and the CPU oracle take their
inputs from here; nothing here is used by either implementation's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

BASE_SEED = 2410154510


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (host code only, portable C11)."""
    import subprocess

    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        out_args = [P(P(i64)), P(P(i32)), P(P(i32)), P(i64)]
        lib.synth_planted_partition.argtypes = [i64, i64, dbl, dbl, u64] + out_args
        lib.synth_planted_partition.restype = ctypes.c_int
        lib.synth_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64] + out_args
        lib.synth_rmat.restype = ctypes.c_int
        lib.synth_dcpp.argtypes = [i64, dbl, dbl, dbl, dbl, i64, i64, dbl, i32, u64] + out_args
        lib.synth_dcpp.restype = ctypes.c_int
        lib.synth_batch.argtypes = [i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, i64, i64,
                                    i32, i32, u64, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_batch.restype = ctypes.c_int
        lib.synth_uniform.argtypes = [u64, u64, i64, u64, ctypes.c_void_p]
        lib.synth_uniform.restype = None
        lib.synth_free.argtypes = [ctypes.c_void_p]
        lib.synth_free.restype = None
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Symmetric CSR: ``off`` int64[n+1], ``col`` int32[arcs], ``w`` int32[arcs]."""

    n: int
    off: np.ndarray
    col: np.ndarray
    w: np.ndarray

    @property
    def arcs(self) -> int:
        return int(self.off[-1])

    @property
    def edges(self) -> int:
        return self.arcs // 2


def _take_csr(lib, n, off_p, col_p, w_p, arcs):
    a = int(arcs.value)
    off = np.ctypeslib.as_array(off_p, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(col_p, shape=(max(a, 1),))[:a].copy()
    w = np.ctypeslib.as_array(w_p, shape=(max(a, 1),))[:a].copy()
    for p in (off_p, col_p, w_p):
        lib.synth_free(ctypes.cast(p, ctypes.c_void_p))
    return Graph(n, off, col, w)


def _csr_call(fn, n, *args):
    lib = _load()
    P = ctypes.POINTER
    off_p, col_p, w_p = P(ctypes.c_int64)(), P(ctypes.c_int32)(), P(ctypes.c_int32)()
    arcs = ctypes.c_int64()
    rc = fn(*args, ctypes.byref(off_p), ctypes.byref(col_p), ctypes.byref(w_p), ctypes.byref(arcs))
    if rc != 0:
        raise RuntimeError(f"synthetic graph generation failed (rc={rc})")
    return _take_csr(lib, n, off_p, col_p, w_p, arcs)


def planted_partition(n: int, blocks: int, avg_deg: float, mu: float, seed: int) -> Graph:
    """n vertices in `blocks` equal blocks, mean degree ~avg_deg, mixing mu, unit weights."""
    lib = _load()
    return _csr_call(lib.synth_planted_partition, n, n, blocks, float(avg_deg), float(mu), seed)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = BASE_SEED + 1) -> Graph:
    """R-MAT graph, symmetrised and deduplicated, vertex IDs randomly permuted, unit weights."""
    lib = _load()
    return _csr_call(lib.synth_rmat, 1 << scale, scale, edge_factor, float(a), float(b), float(c), seed)


def dcpp(n: int, avg_deg: float = 66.7, deg_exp: float = 2.1, max_deg: float = 1e6, comm_exp: float = 1.5,
         cmin: int = 10, cmax: int = 100000, mu: float = 0.3, wmax: int = 8, seed: int = BASE_SEED + 2) -> Graph:
    """Degree-corrected planted partition: power-law expected degrees (exponent
    deg_exp, bounded by max_deg, mean avg_deg), power-law community sizes
    (exponent comm_exp in [cmin, cmax]), mixing mu, weights 1..wmax."""
    lib = _load()
    return _csr_call(lib.synth_dcpp, n, n, float(avg_deg), float(deg_exp), float(max_deg), float(comm_exp),
                     int(cmin), int(cmax), float(mu), int(wmax), seed)


def random_batch(g: Graph, n_edges: int, seed: int, frac_ins: float = 0.8,
                 w_lo: int = 1, w_hi: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Random batch of `n_edges` undirected edges: round(frac_ins*n) insertions of
    uniform non-edge pairs and the rest deletions of uniform existing edges.
    Returns (deletions, insertions) as int32 arrays of shape (k, 3) = (u, v, w)."""
    lib = _load()
    n_ins = int(round(frac_ins * n_edges))
    n_del = int(n_edges) - n_ins
    dels = np.zeros((max(n_del, 0), 3), dtype=np.int32)
    ins = np.zeros((max(n_ins, 0), 3), dtype=np.int32)
    rc = lib.synth_batch(g.n, g.off.ctypes.data, g.col.ctypes.data, g.w.ctypes.data, n_del, n_ins,
                         w_lo, w_hi, seed, dels.ctypes.data, ins.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"batch generation failed (rc={rc})")
    return dels, ins


def uniform_ints(seed: int, stream: int, count: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(count, dtype=np.int64)
    lib.synth_uniform(seed, stream, count, n, out.ctypes.data)
    return out


def apply_batch_numpy(g: Graph, dels: np.ndarray, ins: np.ndarray) -> Graph:
    """Edge-set bookkeeping for test fixtures: the graph after removing `dels`
    and adding `ins` (weights of an existing edge add up).  Used to chain
    batches in generators; holds no community arithmetic."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    key = src * g.n + g.col.astype(np.int64)
    wt = g.w.astype(np.int64)
    if len(dels):
        d = np.concatenate([dels[:, 0].astype(np.int64) * g.n + dels[:, 1],
                            dels[:, 1].astype(np.int64) * g.n + dels[:, 0]])
        keep = ~np.isin(key, d)
        key, wt = key[keep], wt[keep]
    if len(ins):
        ik = np.concatenate([ins[:, 0].astype(np.int64) * g.n + ins[:, 1],
                             ins[:, 1].astype(np.int64) * g.n + ins[:, 0]])
        iw = np.concatenate([ins[:, 2], ins[:, 2]]).astype(np.int64)
        key = np.concatenate([key, ik])
        wt = np.concatenate([wt, iw])
    order = np.argsort(key, kind="stable")
    key, wt = key[order], wt[order]
    uk, first = np.unique(key, return_index=True)
    uw = np.add.reduceat(wt, first) if len(key) else wt
    rows = uk // g.n
    off = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(off, rows + 1, 1)
    off = np.cumsum(off)
    return Graph(g.n, off, (uk % g.n).astype(np.int32), uw.astype(np.int32))


# --- the workloads (shapes of the paper's experiments, seeds fixed) ---------------------

def workload_small(seed: int = BASE_SEED + 0) -> Graph:
    """Planted partition: 10,000 vertices in 100 blocks of 100, mean degree 16, mixing 0.2."""
    return planted_partition(10_000, 100, 16.0, 0.2, seed)


def workload_rmat22(seed: int = BASE_SEED + 1) -> Graph:
    """R-MAT scale 22 (4.19M vertices, edge factor 16, a=0.57 b=c=0.19 d=0.05)."""
    return rmat(22, 16, 0.57, 0.19, 0.19, seed)
