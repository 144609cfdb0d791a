"""Full-size checks at the benchmark's configuration (needs a GB300).

R-MAT scale 22 (4,194,304 vertices, 64,154,367 edges after deduplication),
static Leiden, then DF updates of 1e-3|E| edges (80% insertions) through the
device entry point with the default parameters and launch shapes: the
launches that the benchmark times.  At this size the oracle cannot run the
whole algorithm in seconds, so the results are checked by what it computes
exactly on the GPU's own output and by properties that hold at any size:

- the affected set equals the DF marking (Alg. "frontier") of each batch on
  the previous membership: endpoints of deletions inside a community and of
  insertions across communities;
- the applied graph: rows of sampled touched vertices equal the batches
  applied on the host, and K, Sigma and 2m equal their definitions on the
  final graph and membership;
- every community is connected (the oracle's component labelling finds one
  component per community), as refinement and splitting guarantee;
- Q equals the oracle's Eq. 1 on the same membership, to the last bit;
- DF quality: Q of static Leiden on the final graph exceeds the DF result by
  at most 0.005.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import leiden as L
from paper_2410_15451_gb300 import synth

pytestmark = pytest.mark.gpu

SCALE = 22
BATCHES = 3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15451_gb300 import _build

    _build.build()
    L.load()


def df_marking(dels, ins, C):
    """Alg. "frontier" initial marking: deletions with both endpoints in one
    community, insertions whose endpoints lie in different communities."""
    dV = np.zeros(len(C), np.uint8)
    for e, same_wanted in ((dels, True), (ins, False)):
        if len(e) == 0:
            continue
        u, v = e[:, 0], e[:, 1]
        hit = (C[u] == C[v]) == same_wanted
        dV[u[hit]] = 1
        dV[v[hit]] = 1
    return dV


def test_rmat22_df_updates_at_full_size():
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    seed = synth.BASE_SEED + 1
    g = synth.rmat(SCALE, 16, 0.57, 0.19, 0.19, seed)
    n, E = g.n, g.edges
    size = max(1, int(round(1e-3 * E)))
    n_ins = int(round(0.8 * size))
    n_del = size - n_ins
    dels, ins = synth.random_batch(g, BATCHES * size, seed=seed + 5, frac_ins=n_ins / size)
    batches = [(np.ascontiguousarray(dels[k * n_del:(k + 1) * n_del]),
                np.ascontiguousarray(ins[k * n_ins:(k + 1) * n_ins])) for k in range(BATCHES)]

    # rows of sampled touched vertices in G^0
    touched = np.unique(np.concatenate([dels[:, 0], dels[:, 1], ins[:, 0], ins[:, 1]]))
    sample = np.random.default_rng(seed).choice(touched, min(2000, len(touched)), replace=False)
    rows = {int(v): dict(zip(g.col[g.off[v]:g.off[v + 1]].tolist(), g.w[g.off[v]:g.off[v + 1]].tolist()))
            for v in sample}

    h = L.Leiden(n, g.off, g.col, g.w, cuda_stream=stream.cuda_stream)
    C_prev = h.static()
    d_out = torch.empty(n, dtype=torch.int32, device=dev)
    for k, (d, i) in enumerate(batches):
        dd, di = torch.from_numpy(d).to(dev), torch.from_numpy(i).to(dev)
        L.leiden_update_device(h.h, dd, d.shape[0], di, i.shape[0], L.LEIDEN_DF, d_out)
        torch.cuda.synchronize()
        C = d_out.cpu().numpy()
        assert np.array_equal(h.affected(), df_marking(d, i, C_prev)), f"batch {k}: affected set"
        assert C.min() >= 0 and C.max() < n
        C_prev = C
        for (u, v, _) in d.tolist():
            for a, b in ((u, v), (v, u)):
                if a in rows:
                    rows[a].pop(b, None)
        for (u, v, wt) in i.tolist():
            for a, b in ((u, v), (v, u)):
                if a in rows:
                    rows[a][b] = rows[a].get(b, 0) + wt

    st = h.state()
    assert np.array_equal(st["C"], C_prev)
    q_df = h.modularity()
    off, col, w = h.graph()
    h.close()
    del g

    for v, row in rows.items():
        got = dict(zip(col[off[v]:off[v + 1]].tolist(), w[off[v]:off[v + 1]].tolist()))
        assert got == row, f"row {v}"
    assert int(off[-1]) == 2 * (E - BATCHES * n_del + BATCHES * n_ins)  # insertions are non-edges

    K = np.add.reduceat(np.append(w.astype(np.int64), 0), off[:-1])
    K[np.diff(off) == 0] = 0
    assert np.array_equal(K, st["K"])
    assert int(K.sum()) == st["m2"]
    Sig = np.bincount(st["C"], K.astype(np.float64), n).astype(np.int64)  # sums below 2^53: exact
    assert np.array_equal(Sig, st["Sigma"])

    labels = oracle.split(off, col, st["C"], np.ones(n, np.uint8))
    assert len(np.unique(labels)) == len(np.unique(st["C"])), "a community is disconnected"

    q_or, _ = oracle.modularity(off, col, w, st["C"])
    assert q_df == q_or

    s = L.Leiden(n, off, col, w.astype(np.int32), cuda_stream=stream.cuda_stream)
    s.static()
    q_static = s.modularity()
    s.close()
    assert q_static - q_df <= 0.005, (q_static, q_df)
