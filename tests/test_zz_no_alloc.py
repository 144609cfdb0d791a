"""The allocation-free modularity entry point, through the C ABI.

Some callers cannot allocate device memory while they run: a serving loop
that reserved all device memory up front, code whose device memory belongs
to another allocator (a framework's caching pool), or a latency-critical path
that cannot take the implicit synchronisation of cudaMalloc and cudaFree.
For them leiden_modularity_noalloc computes Eq. 1 with a fixed scratch array
in the library's own device memory.  It must give the same Q as the regular
entry point and as the CPU oracle, call after call, although every call
reuses that one array, and it must leave the device's free memory unchanged.

This file is collected last (its name sorts after the others), so that a run
that stops at the first failure has run every other test before it.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import leiden as L
from paper_2410_15451_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15451_gb300 import _build

    _build.build()
    L.load()
    return torch


def _device_csr(torch, g):
    return (torch.from_numpy(g.off).cuda(), torch.from_numpy(g.col).cuda(), torch.from_numpy(g.w).cuda())


def test_noalloc_modularity_matches_regular_entry_point_twice(torch_cuda):
    """Two calls in a row for each membership: the second must not see the
    first one's leftovers in the shared scratch."""
    torch = torch_cuda
    g = synth.rmat(14, seed=71)
    h = L.Leiden(g.n, g.off, g.col, g.w)
    C = h.static()
    d_off, d_col, d_w = _device_csr(torch, g)
    rng = np.random.default_rng(5)
    memberships = [C, rng.integers(0, 300, g.n).astype(np.int32)]
    for C_k in memberships:
        expect = h.modularity(C_k)
        d_C = torch.from_numpy(C_k).cuda()
        q1 = L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, d_C)
        q2 = L.leiden_modularity_noalloc(g.n, d_off, d_col, None if np.all(g.w == 1) else d_w, d_C)
        assert q1 == expect
        assert q2 == expect
    h.close()


def test_noalloc_modularity_matches_the_oracle(torch_cuda):
    """Weighted graph, several memberships: the same double as the oracle's
    Eq. 1 (exact numerator, one division)."""
    torch = torch_cuda
    g0 = synth.planted_partition(3000, 15, 12, 0.3, 41)
    src = np.repeat(np.arange(g0.n), np.diff(g0.off)).astype(np.int64)
    a, b = np.minimum(src, g0.col), np.maximum(src, g0.col)
    g = synth.Graph(g0.n, g0.off, g0.col, ((a * 2654435761 + b * 40503) % 8 + 1).astype(np.int32))
    d_off, d_col, d_w = _device_csr(torch, g)
    rng = np.random.default_rng(6)
    for C_k in (np.arange(g.n, dtype=np.int32), np.zeros(g.n, np.int32),
                rng.integers(0, 40, g.n).astype(np.int32), (np.arange(g.n) // 200).astype(np.int32)):
        q_or, _ = oracle.modularity(g.off, g.col, g.w.astype(np.int64), C_k)
        for _ in range(2):
            assert L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, torch.from_numpy(C_k).cuda()) == q_or


def test_noalloc_graph_without_arcs(torch_cuda):
    torch = torch_cuda
    n = 50
    d_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    d_col = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_C = torch.arange(n, dtype=torch.int32, device="cuda")
    assert L.leiden_modularity_noalloc(n, d_off, d_col, None, d_C) == 0.0


def test_noalloc_rejects_bad_ids_then_works(torch_cuda):
    """A membership id of -1 or n, or a column id of n, is found by the
    kernels and returns LEIDEN_ERR_ARG; the next correct call is exact."""
    torch = torch_cuda
    g = synth.rmat(12, seed=72)
    d_off, d_col, d_w = _device_csr(torch, g)
    C = np.zeros(g.n, np.int32)
    q_or, _ = oracle.modularity(g.off, g.col, g.w.astype(np.int64), C)
    for bad in (-1, g.n):
        Cb = C.copy()
        Cb[g.n // 2] = bad
        with pytest.raises(L.LeidenError) as e:
            L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, torch.from_numpy(Cb).cuda())
        assert e.value.status == L.LEIDEN_ERR_ARG
        assert "membership" in L.leiden_last_error(None)
        assert L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, torch.from_numpy(C).cuda()) == q_or
    col_bad = g.col.copy()
    col_bad[5] = g.n
    with pytest.raises(L.LeidenError) as e:
        L.leiden_modularity_noalloc(g.n, d_off, torch.from_numpy(col_bad).cuda(), d_w, torch.from_numpy(C).cuda())
    assert e.value.status == L.LEIDEN_ERR_ARG
    assert "column" in L.leiden_last_error(None)
    assert L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, torch.from_numpy(C).cuda()) == q_or


def test_noalloc_rejects_oversized_input_and_null_columns(torch_cuda):
    torch = torch_cuda
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(L.LeidenError) as e:
        L.leiden_modularity_noalloc((1 << 22) + 1, d, d, None, d)
    assert e.value.status == L.LEIDEN_ERR_ARG
    assert "4194304" in L.leiden_last_error(None)
    with pytest.raises(L.LeidenError) as e:
        L.leiden_modularity_noalloc(3, d, None, None, d)
    assert e.value.status == L.LEIDEN_ERR_ARG


def test_noalloc_leaves_free_device_memory_unchanged(torch_cuda):
    """The reason for the entry point: after a first call (which loads the
    library's kernels), further calls take no device memory."""
    torch = torch_cuda
    g = synth.rmat(13, seed=73)
    d_off, d_col, d_w = _device_csr(torch, g)
    d_C = torch.from_numpy((np.arange(g.n) % 97).astype(np.int32)).cuda()
    q0 = L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, d_C)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, d_C) == q0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
