"""The allocation-free modularity entry point (for callers that may not
allocate device memory: a serving loop that reserved all memory up front, a
framework that owns the device allocator, a latency path that cannot afford
cudaMalloc's implicit synchronisation) must give the same Q as the regular
entry point, call after call, even though every call reuses one fixed
scratch array.  This file is collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

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


def test_noalloc_modularity_matches_regular_entry_point_twice(torch_cuda):
    torch = torch_cuda
    g = synth.rmat(14, seed=71)
    h = L.Leiden(g.n, g.off, g.col, g.w)
    C = h.static()
    d_off = torch.from_numpy(g.off).cuda()
    d_col = torch.from_numpy(g.col).cuda()
    d_w = torch.from_numpy(g.w).cuda()
    rng = np.random.default_rng(5)
    memberships = [C, rng.integers(0, 300, g.n).astype(np.int32)]
    for C_k in memberships:
        expect = h.modularity(C_k)
        d_C = torch.from_numpy(C_k).cuda()
        # two calls in a row: the second must not see the first one's leftovers
        q1 = L.leiden_modularity_noalloc(g.n, d_off, d_col, d_w, d_C)
        q2 = L.leiden_modularity_noalloc(g.n, d_off, d_col, None if np.all(g.w == 1) else d_w, d_C)
        assert q1 == expect
        assert q2 == expect
    h.close()


def test_noalloc_rejects_oversized_input(torch_cuda):
    torch = torch_cuda
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(L.LeidenError) as e:
        L.leiden_modularity_noalloc((1 << 22) + 1, d, d, None, d)
    assert e.value.status == L.LEIDEN_ERR_ARG
    assert "4194304" in L.leiden_last_error(None)
