"""Batched handles (many graphs, one launch per kernel for all of them)
against one handle per graph and against the oracle (needs a GB300).

Each graph of a batch must come out exactly as it does alone: membership
(offset by its vertex offset), per-graph trace, K / Sigma / Delta Sigma and
per-graph modularity, for static Leiden and for ND / DS / DF updates, with
graphs of very different sizes, some with empty batches.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import leiden as L
from paper_2410_15451_gb300 import synth
from tests.helpers import csr_from_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15451_gb300 import _build

    _build.build()
    L.load()


def _path(n):
    edges = [(i, i + 1) for i in range(n - 1)]
    off, col, w = csr_from_edges(n, edges)
    return synth.Graph(n, off, col, w.astype(np.int32))


def _weighted(g):
    src = np.repeat(np.arange(g.n), np.diff(g.off)).astype(np.int64)
    a, b = np.minimum(src, g.col), np.maximum(src, g.col)
    w = ((a * 2654435761 + b * 40503) % 8 + 1).astype(np.int32)
    return synth.Graph(g.n, g.off, g.col, w)


def graphs():
    return [
        synth.planted_partition(1500, 15, 10, 0.2, 71),
        synth.rmat(11, seed=72),
        _path(7),
        synth.rmat(9, seed=73),
        _weighted(synth.planted_partition(900, 9, 12, 0.3, 74)),
        synth.planted_partition(4000, 40, 14, 0.25, 75),
        synth.rmat(12, seed=76),
    ]


def _singles(gs):
    return [L.Leiden(g.n, g.off, g.col, g.w) for g in gs]


def _same(batch, singles, cb, cs_list):
    for k, (s, cs) in enumerate(zip(singles, cs_list)):
        assert np.array_equal(batch.local(cb, k), cs), f"graph {k} membership"
        assert batch.trace(k)["passes"] == s.trace()["passes"], f"graph {k} trace"
    st = batch.state()
    for k, s in enumerate(singles):
        ss = s.state()
        a, b = int(batch.voff[k]), int(batch.voff[k + 1])
        for key in ("K", "Sigma", "dSigma"):
            assert np.array_equal(st[key][a:b], ss[key]), f"graph {k} {key}"
    q = batch.modularity()
    for k, s in enumerate(singles):
        assert q[k] == s.modularity(), f"graph {k} modularity"


def test_batched_static_matches_single_handles_and_oracle():
    gs = graphs()
    batch = L.LeidenBatch([(g.n, g.off, g.col, g.w) for g in gs])
    assert L.leiden_batch_graphs(batch.h) == len(gs)
    singles = _singles(gs)
    cb = batch.static()
    cs = [s.static() for s in singles]
    _same(batch, singles, cb, cs)
    for k in (0, 2, 4):
        ref = oracle.Oracle(gs[k].n, gs[k].off, gs[k].col, gs[k].w, schedule=oracle.SYNC)
        assert np.array_equal(batch.local(cb, k), ref.static())


@pytest.mark.parametrize("mode", [L.LEIDEN_DF, L.LEIDEN_DS, L.LEIDEN_ND], ids=["DF", "DS", "ND"])
def test_batched_updates_match_single_handles(mode):
    gs = graphs()
    batch = L.LeidenBatch([(g.n, g.off, g.col, g.w) for g in gs])
    singles = _singles(gs)
    batch.static()
    for s in singles:
        s.static()
    cur = list(gs)
    for step, frac in enumerate([0.002, 0.02]):
        dels_all, ins_all, cs = [], [], []
        for k, (g, s) in enumerate(zip(cur, singles)):
            size = 0 if (k + step) % 3 == 2 else max(1, int(frac * g.off[-1] / 2))  # some graphs idle
            if size and g.off[-1] > 2:
                d, i = synth.random_batch(g, size, seed=900 + 10 * step + k, w_lo=1, w_hi=3 if k == 4 else 1)
            else:
                d, i = np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32)
            cs.append(s.update(d, i, mode))
            dels_all.append(batch.to_global(d, k))
            ins_all.append(batch.to_global(i, k))
            cur[k] = synth.apply_batch_numpy(g, d, i)
        cb = batch.update(np.concatenate(dels_all), np.concatenate(ins_all), mode)
        _same(batch, singles, cb, cs)


def test_batched_df_update_matches_oracle():
    gs = graphs()[:4]
    batch = L.LeidenBatch([(g.n, g.off, g.col, g.w) for g in gs])
    refs = [oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC) for g in gs]
    batch.static()
    for r in refs:
        r.static()
    dels_all, ins_all, want = [], [], []
    for k, (g, r) in enumerate(zip(gs, refs)):
        d, i = synth.random_batch(g, 40, seed=950 + k) if g.off[-1] > 80 else (np.zeros((0, 3), np.int32),) * 2
        want.append(r.update(d, i, oracle.DF))
        dels_all.append(batch.to_global(d, k))
        ins_all.append(batch.to_global(i, k))
    cb = batch.update(np.concatenate(dels_all), np.concatenate(ins_all), L.LEIDEN_DF)
    for k, w in enumerate(want):
        assert np.array_equal(batch.local(cb, k), w), f"graph {k}"


def test_batched_rejects_an_edge_between_graphs():
    gs = graphs()[:3]
    batch = L.LeidenBatch([(g.n, g.off, g.col, g.w) for g in gs])
    before = batch.static()
    bad = np.array([[0, int(batch.voff[1]), 1]], np.int32)  # graph 0 to graph 1
    with pytest.raises(L.LeidenError) as e:
        batch.update(np.zeros((0, 3), np.int32), bad, L.LEIDEN_DF)
    assert e.value.status == L.LEIDEN_ERR_BATCH
    assert np.array_equal(batch.update(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32), L.LEIDEN_DF), before)
