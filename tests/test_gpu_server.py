"""Serving runtime (needs a GB300): resident graphs, footprint admission,
requests from several threads at once; every result must equal the one the
graph gets alone and the CPU oracle's, bit for bit (deterministic schedule)."""
from __future__ import annotations

import threading
import time

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


def _weighted(g):
    src = np.repeat(np.arange(g.n), np.diff(g.off)).astype(np.int64)
    a, b = np.minimum(src, g.col), np.maximum(src, g.col)
    return synth.Graph(g.n, g.off, g.col, ((a * 2654435761 + b * 40503) % 8 + 1).astype(np.int32))


def _workload():
    gs = [synth.planted_partition(1500, 15, 10, 0.2, 81), synth.rmat(10, seed=82), synth.rmat(11, seed=83),
          synth.planted_partition(3000, 30, 12, 0.25, 84), _weighted(synth.planted_partition(900, 9, 12, 0.3, 85)),
          synth.rmat(12, seed=86)]
    modes = [L.LEIDEN_DF, L.LEIDEN_DS, L.LEIDEN_DF, L.LEIDEN_ND]
    reqs = []  # per graph: list of (dels, ins, mode)
    for k, g in enumerate(gs):
        cur, lst = g, []
        for step, size in enumerate([30, 200, 5, 60]):
            d, i = synth.random_batch(cur, size, seed=1200 + 10 * k + step, w_hi=3 if k == 4 else 1)
            lst.append((d, i, modes[step]))
            cur = synth.apply_batch_numpy(cur, d, i)
        reqs.append(lst)
    return gs, reqs


def _alone(g, lst):
    h = L.Leiden(g.n, g.off, g.col, g.w)
    h.static()
    out = [h.update(d, i, m) for d, i, m in lst]
    h.close()
    return out


ORACLE_MODE = {L.LEIDEN_ND: oracle.ND, L.LEIDEN_DS: oracle.DS, L.LEIDEN_DF: oracle.DF}


def _oracle(g, lst):
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    o.static()
    return [o.update(d, i, ORACLE_MODE[m]) for d, i, m in lst]


def test_server_results_equal_results_alone():
    gs, reqs = _workload()
    expected = [_oracle(g, lst) for g, lst in zip(gs, reqs)]
    for k, (g, lst) in enumerate(zip(gs, reqs)):  # each graph alone on the GPU equals the oracle
        for step, c in enumerate(_alone(g, lst)):
            assert np.array_equal(c, expected[k][step]), (k, step)
    fp = [L.leiden_footprint_bytes(g.n, g.off) for g in gs]
    tr = [L.leiden_transient_bytes(g.n, g.off) for g in gs]
    # graphs 4 and 5 wait for memory; room for three slots' aggregation buffers
    budget = sum(fp[:4]) + 3 * max(tr) + 1
    assert budget < sum(fp[:5]) + 3 * max(tr)
    srv = L.LeidenServer(budget, slots=3)
    ids = [srv.add_graph(g.n, g.off, g.col, g.w) for g in gs]
    tickets = {k: [None] * len(reqs[k]) for k in range(len(gs))}
    lock = threading.Lock()

    def submitter(graphs):
        # interleave graphs, each graph's requests in order
        for step in range(4):
            for k in graphs:
                d, i, m = reqs[k][step]
                t = srv.submit(ids[k], d, i, m, keep_membership=True)
                with lock:
                    tickets[k][step] = t
                time.sleep(0.001)

    threads = [threading.Thread(target=submitter, args=(part,)) for part in ([0, 3], [1, 4], [2, 5])]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for k in range(4):
        for step in range(4):
            memb, lat, svc = srv.wait(tickets[k][step])
            assert lat >= svc >= 0.0
            assert np.array_equal(memb, expected[k][step]), (k, step)
    st = srv.stats()
    assert st["graphs_resident"] == 4 and st["graphs_waiting"] == 2
    assert st["bytes_used"] <= st["bytes_budget"]
    # freeing memory admits the waiting graphs, whose queued requests then run
    for k in range(4):
        srv.remove_graph(ids[k])
    for k in (4, 5):
        for step in range(4):
            memb, _, _ = srv.wait(tickets[k][step])
            assert np.array_equal(memb, expected[k][step]), (k, step)
        assert np.array_equal(srv.membership(ids[k]), expected[k][-1])
    srv.close()


def test_server_bad_batch_leaves_the_graph_unchanged():
    g = synth.planted_partition(1200, 12, 10, 0.2, 91)
    srv = L.LeidenServer(10 * (L.leiden_footprint_bytes(g.n, g.off) + L.leiden_transient_bytes(g.n, g.off)), slots=2)
    gid = srv.add_graph(g.n, g.off, g.col, g.w)
    before = srv.membership(gid)
    bad = np.array([[0, 1, 1]], np.int32) if not np.any(g.col[g.off[0]:g.off[1]] == 1) else np.array([[0, 0, 1]],
                                                                                                     np.int32)
    t = srv.submit(gid, bad, np.zeros((0, 3), np.int32), L.LEIDEN_DF)
    with pytest.raises(L.LeidenError) as e:
        srv.wait(t)
    assert e.value.status in (L.LEIDEN_ERR_BATCH, L.LEIDEN_ERR_ARG)
    assert np.array_equal(srv.membership(gid), before)
    d, i = synth.random_batch(g, 50, seed=92)
    memb, _, _ = srv.wait(srv.submit(gid, d, i, L.LEIDEN_DF, keep_membership=True))
    assert np.array_equal(memb, _oracle(g, [(d, i, L.LEIDEN_DF)])[0])
    srv.close()


def test_server_wait_for_times_out_then_the_ticket_completes():
    """A bounded wait on a request of a graph still waiting for memory gives
    up with LEIDEN_ERR_TIMEOUT and leaves the ticket valid; once memory is
    freed the graph is admitted and the same ticket completes with the
    oracle's result.  The failure is made on the host (no GPU fault)."""
    g1 = synth.planted_partition(1500, 15, 10, 0.2, 93)
    g2 = synth.planted_partition(1200, 12, 10, 0.2, 94)
    fp1, fp2 = L.leiden_footprint_bytes(g1.n, g1.off), L.leiden_footprint_bytes(g2.n, g2.off)
    tr = max(L.leiden_transient_bytes(g1.n, g1.off), L.leiden_transient_bytes(g2.n, g2.off))
    assert fp2 <= fp1
    srv = L.LeidenServer(fp1 + fp2 + 2 * tr - 1, slots=2)  # each fits alone, not both
    id1 = srv.add_graph(g1.n, g1.off, g1.col, g1.w)
    while srv.stats()["graphs_resident"] < 1:
        time.sleep(0.01)
    id2 = srv.add_graph(g2.n, g2.off, g2.col, g2.w)
    d, i = synth.random_batch(g2, 40, seed=95)
    t = srv.submit(id2, d, i, L.LEIDEN_DF, keep_membership=True)
    for _ in range(2):
        with pytest.raises(L.LeidenError) as e:
            srv.wait_for(t, 50.0)
        assert e.value.status == L.LEIDEN_ERR_TIMEOUT
    assert srv.stats()["graphs_waiting"] == 1
    srv.remove_graph(id1)
    memb, lat, svc = srv.wait_for(t, 120000.0)
    assert lat >= svc >= 0.0
    assert np.array_equal(memb, _oracle(g2, [(d, i, L.LEIDEN_DF)])[0])
    srv.close()
