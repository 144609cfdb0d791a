"""State export / import (checkpoint and resume) and the delete-then-reinsert
protocol of the paper's stability discussion (needs a GB300)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import leiden as L
from paper_2410_15451_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15451_gb300 import _build

    _build.build()
    L.load()


def _same_state(a, b):
    sa, sb = a.state(), b.state()
    for k in ("C", "K", "Sigma", "dSigma"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["m2"] == sb["m2"]


@pytest.mark.parametrize("mode", [L.LEIDEN_DF, L.LEIDEN_DS, L.LEIDEN_ND], ids=["DF", "DS", "ND"])
def test_export_import_resumes_exactly(mode):
    g = synth.rmat(13, seed=101)
    a = L.Leiden(g.n, g.off, g.col, g.w)
    a.static()
    cur = g
    for k in range(2):
        d, i = synth.random_batch(cur, 300, seed=102 + k)
        a.update(d, i, L.LEIDEN_DF)
        cur = synth.apply_batch_numpy(cur, d, i)
    off, col, w = a.graph()
    st = a.state()
    b = L.Leiden(g.n, off, col, w.astype(np.int32))
    L.leiden_import_state(b.h, st["C"], st["dSigma"])
    _same_state(a, b)
    assert a.modularity() == b.modularity()
    d, i = synth.random_batch(cur, 500, seed=110)
    ca, cb = a.update(d, i, mode), b.update(d, i, mode)
    assert np.array_equal(ca, cb)
    assert a.trace()["passes"] == b.trace()["passes"]
    _same_state(a, b)


def test_import_rejects_ids_out_of_range():
    g = synth.planted_partition(500, 5, 8, 0.2, 111)
    h = L.Leiden(g.n, g.off, g.col, g.w)
    C = np.arange(g.n, dtype=np.int32)
    C[3] = g.n
    with pytest.raises(L.LeidenError) as e:
        L.leiden_import_state(h.h, C, np.zeros(g.n, np.int64))
    assert e.value.status == L.LEIDEN_ERR_ARG


def test_delete_then_reinsert_matches_the_oracle():
    """The stability protocol (delete a batch, insert it back) on the CUDA
    path equals the oracle's, and most memberships come back."""
    g = synth.planted_partition(3000, 30, 12, 0.2, 121)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    c0 = gpu.static()
    ref.static()
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    keep = src < g.col
    edges = np.stack([src[keep], g.col[keep], g.w[keep]], 1).astype(np.int32)
    pick = np.random.default_rng(122).choice(len(edges), 60, replace=False)
    batch = edges[pick]
    none = np.zeros((0, 3), np.int32)
    assert np.array_equal(gpu.update(batch, none, L.LEIDEN_DF), ref.update(batch, none, oracle.DF))
    c2 = gpu.update(none, batch, L.LEIDEN_DF)
    assert np.array_equal(c2, ref.update(none, batch, oracle.DF))
    assert np.mean(c2 == c0) > 0.5
