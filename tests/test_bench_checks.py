"""The full-size checks of `bench.py --large` restate connectivity and Eq. 1
without the oracle (scipy components, exact integers); here they are held
against the oracle's component labelling and modularity on small graphs,
including memberships with a disconnected community."""
from __future__ import annotations

import numpy as np
import pytest

import bench
import oracle
from paper_2410_15451_gb300 import synth
from tests.helpers import csr_from_edges

pytest.importorskip("scipy")


def row_sums(g):
    K = np.add.reduceat(np.append(g.w.astype(np.int64), 0), g.off[:-1])
    K[np.diff(g.off) == 0] = 0
    return K


@pytest.mark.parametrize("chunk", [7, 1000, 1 << 20])
def test_components_and_modularity_match_the_oracle(chunk):
    g = synth.rmat(12, 16, 0.57, 0.19, 0.19, 11)
    C = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC).static()
    ncc, q = bench.intra_community_checks(g.off, g.col, g.w, C, row_sums(g), rows_per_chunk=chunk)
    labels = oracle.split(g.off, g.col, C, np.ones(g.n, np.uint8))
    assert ncc == len(np.unique(labels)) == len(np.unique(C))
    q_or, _ = oracle.modularity(g.off, g.col, g.w, C)
    assert abs(q - q_or) <= 1e-12


def test_a_disconnected_community_is_found():
    # a ring of eight 5-cliques, one community per clique, then cliques 0
    # and 2 (which share no edge) under one id
    L, k = 8, 5
    edges = [(c * k + i, c * k + j) for c in range(L) for i in range(k) for j in range(i + 1, k)]
    edges += [(c * k, ((c + 1) % L) * k + 1) for c in range(L)]
    off, col, w = csr_from_edges(L * k, edges)
    C = np.repeat(np.arange(L, dtype=np.int32), k)
    K = np.add.reduceat(w, off[:-1])
    for C2, extra in ((C, 0), (np.where(C == 2, 0, C).astype(np.int32), 1)):
        ncc, q = bench.intra_community_checks(off, col, w, C2, K, rows_per_chunk=3)
        labels = oracle.split(off, col, C2, np.ones(L * k, np.uint8))
        assert ncc == len(np.unique(labels)) == len(np.unique(C2)) + extra
        q_or, _ = oracle.modularity(off, col, w, C2)
        assert abs(q - q_or) <= 1e-12
