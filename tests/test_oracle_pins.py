"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test names what it pins; none re-types the oracle's own code.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import synth
from tests.helpers import (components, csr_from_edges, disconnected_communities, newman_numerator,
                           set_partitions)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHEDULES = [oracle.SEQ, oracle.SYNC]


def clique_edges(base, k):
    return [(base + a, base + b) for a in range(k) for b in range(a + 1, k)]


def random_graph(n, p, seed, wmax=1, loops=False):
    rng = np.random.default_rng(seed)
    edges, ws = [], []
    for u in range(n):
        for v in range(u + (0 if loops else 1), n):
            if rng.random() < p:
                edges.append((u, v))
                ws.append(int(rng.integers(1, wmax + 1)))
    return csr_from_edges(n, edges, ws)


# ---------------------------------------------------------------- Eq. 1

def _closed_form_cases():
    with open(os.path.join(GOLDEN, "modularity_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            fam, n, k, num, den = line.split()
            yield fam, int(n), int(k), Fraction(int(num), int(den))


@pytest.mark.parametrize("case", list(_closed_form_cases()), ids=lambda c: f"{c[0]}-{c[1]}x{c[2]}")
def test_modularity_closed_forms(case):
    """Eq. 1 on disjoint cliques (1 - 1/n) and rings of cliques (L/(L+1) - 1/n)."""
    fam, n, k, expect = case
    edges = []
    for c in range(n):
        edges += clique_edges(c * k, k)
    if fam == "ring":
        for c in range(n):
            edges.append((c * k, ((c + 1) % n) * k + 1))
    off, col, w = csr_from_edges(n * k, edges)
    C = np.repeat(np.arange(n), k).astype(np.int32) * k  # community id = first vertex
    q, num = oracle.modularity(off, col, w, C)
    m2 = int(w.sum())
    assert Fraction(num, m2 * m2) == expect
    assert q == pytest.approx(float(expect), abs=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_modularity_matches_newman_pairwise_form(seed):
    """Eq. 1 equals Newman's pairwise form, exactly, with weights and self-loops."""
    n = 12
    off, col, w = random_graph(n, 0.35, seed, wmax=5, loops=True)
    rng = np.random.default_rng(100 + seed)
    C = rng.integers(0, 4, n).astype(np.int32)
    q, num = oracle.modularity(off, col, w, C)
    assert num == newman_numerator(off, col, w, C)
    assert -0.5 <= q <= 1.0  # range stated in Preliminaries, "Modularity"


# ---------------------------------------------------------------- Eq. 2

@pytest.mark.parametrize("seed", range(5))
def test_delta_modularity_is_exact_change_of_q(seed):
    """dQ of Eq. 2 (times 2m^2) equals Q(after) - Q(before) for every single
    move, in exact integers: 2 g = numerator(after) - numerator(before).
    Uses self-loops so that K_{i->c} must exclude i itself."""
    n = 10
    off, col, w = random_graph(n, 0.4, seed, wmax=4, loops=True)
    rng = np.random.default_rng(200 + seed)
    C = rng.integers(0, 4, n).astype(np.int32)
    before = newman_numerator(off, col, w, C)
    for i in range(n):
        for c in range(4):
            g = oracle.move_gain(off, col, w, C, i, c)
            C2 = C.copy()
            C2[i] = c
            assert 2 * g == newman_numerator(off, col, w, C2) - before


# ------------------------------------------------- optimum on tiny graphs

TINY = {
    "two_triangles_bridge": (6, [(0, 1), (0, 2), (1, 2), (3, 4), (3, 5), (4, 5), (2, 3)]),
    "two_k4_bridge": (8, clique_edges(0, 4) + clique_edges(4, 4) + [(3, 4)]),
    "three_k3_ring": (9, clique_edges(0, 3) + clique_edges(3, 3) + clique_edges(6, 3) + [(0, 3), (3, 6), (6, 0)]),
}


def brute_force_best(off, col, w):
    n = len(off) - 1
    m2 = int(w.sum())
    best = None
    for part in set_partitions(n):
        num = newman_numerator(off, col, w, part)
        if best is None or num > best:
            best = num
    return Fraction(best, m2 * m2)


@pytest.mark.parametrize("name", sorted(TINY))
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_static_reaches_brute_force_optimum_on_easy_graphs(name, schedule):
    """Leiden's result never beats the optimum and reaches it on these graphs."""
    n, edges = TINY[name]
    off, col, w = csr_from_edges(n, edges)
    opt = brute_force_best(off, col, w)
    o = oracle.Oracle(n, off, col, w.astype(np.int32), schedule=schedule)
    C = o.static()
    _, num = oracle.modularity(off, col, w, C)
    m2 = int(w.sum())
    assert Fraction(num, m2 * m2) == opt


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_static_never_exceeds_optimum(seed, schedule):
    n = 8
    off, col, w = random_graph(n, 0.45, seed, wmax=3)
    if w.sum() == 0:
        pytest.skip("empty graph")
    opt = brute_force_best(off, col, w)
    o = oracle.Oracle(n, off, col, w.astype(np.int32), schedule=schedule)
    C = o.static()
    _, num = oracle.modularity(off, col, w, C)
    m2 = int(w.sum())
    got = Fraction(num, m2 * m2)
    assert got <= opt
    assert got >= opt - Fraction(1, 5)  # heuristic, but not far off on 8 vertices


# ----------------------------------------------- aggregation (Alg. leidenag)

@pytest.mark.parametrize("seed", range(4))
def test_aggregation_preserves_modularity(seed):
    """Q(G', singletons) == Q(G, C) exactly, and total weight is preserved."""
    g = synth.planted_partition(300, 6, 10, 0.3, seed + 7)
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 25, g.n).astype(np.int32)
    uniq, C = np.unique(C, return_inverse=True)
    C = C.astype(np.int32)
    w = g.w.astype(np.int64)
    _, num = oracle.modularity(g.off, g.col, w, C)
    yo, yc, yw = oracle.aggregate(g.off, g.col, w, C, len(uniq))
    _, num2 = oracle.modularity(yo, yc, yw, np.arange(len(uniq), dtype=np.int32))
    assert num == num2
    assert yw.sum() == w.sum()
    # rows sorted, no duplicate neighbours
    for c in range(len(uniq)):
        r = yc[yo[c]:yo[c + 1]]
        assert np.all(np.diff(r) > 0)


# --------------------------------------------------- splitting (Alg. leidensp)

def test_split_caption_example():
    """The split example of the figure on disconnected communities (golden)."""
    spec = {}
    with open(os.path.join(GOLDEN, "split_caption_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            spec[key] = vals
    n = int(spec["n"][0])
    edges = [tuple(int(x) for x in e.split("-")) for e in spec["edges"]]
    off, col, _ = csr_from_edges(n, edges)
    C = np.array([int(x) for x in spec["membership"]], np.int32)
    flags = np.zeros(n, np.uint8)
    flags[int(spec["split_flag_community"][0])] = 1
    got = oracle.split(off, col, C, flags)
    assert got.tolist() == [int(x) for x in spec["expected"]]


@pytest.mark.parametrize("seed", range(5))
def test_split_equals_bfs_components(seed):
    """Split labels equal the connected components (min vertex id) found by
    an independent BFS over each flagged community."""
    n = 60
    off, col, _ = random_graph(n, 0.05, seed)
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 5, n).astype(np.int32)
    flags = np.zeros(n, np.uint8)
    flags[[0, 2, 3]] = 1
    got = oracle.split(off, col, C, flags)
    expect = C.copy()
    for c in (0, 2, 3):
        members = set(np.flatnonzero(C == c).tolist())
        for comp in components(off, col, members):
            expect[comp] = min(comp)
    assert got.tolist() == expect.tolist()


# -------------------------------------------------- static Leiden end to end

@pytest.mark.parametrize("schedule", SCHEDULES)
def test_planted_partition_recovered(schedule):
    """10k-vertex planted partition, 100 blocks, mixing 0.2: the planted
    partition has Q = (1 - mu) - 1/100 = 0.79 in expectation; Leiden finds
    100 communities, all connected, at that Q."""
    g = synth.workload_small()
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=schedule)
    C = o.static()
    q = o.modularity()
    assert abs(q - 0.79) < 0.01
    assert len(np.unique(C)) == 100
    assert disconnected_communities(g.off, g.col, C) == 0
    blocks = np.arange(g.n) // 100
    # every found community is one planted block
    for c in np.unique(C):
        assert len(np.unique(blocks[C == c])) == 1


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_static_ids_follow_tracking_rule(schedule):
    """Static Leiden tracks against singletons (Alg. leiden calls leidenTrack),
    so each community's id is its member of largest degree (ties: lowest)."""
    g = synth.rmat(10, seed=11)
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=schedule)
    C = o.static()
    K = np.diff(g.off)  # unit weights
    for c in np.unique(C):
        mem = np.flatnonzero(C == c)
        best = mem[np.argmax(K[mem])]  # argmax returns the first (lowest id) on ties
        assert c == best


# ---------------------------------------------------- dynamic: ND / DS / DF

def _dyn_setup(seed=3, n_edges=60, schedule=oracle.SYNC):
    g = synth.planted_partition(2000, 20, 12, 0.3, 900 + seed)
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=schedule)
    o.static()
    dels, ins = synth.random_batch(g, n_edges, seed=1000 + seed)
    return g, o, dels, ins


@pytest.mark.parametrize("mode", [oracle.ND, oracle.DS, oracle.DF])
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_update_keeps_auxiliary_state_exact(mode, schedule):
    """After an update: G^t equals an independent edge-set update, K^t equals
    the row sums of G^t, Sigma^t the member sums, sum Sigma = 2m (Alg. update)."""
    g, o, dels, ins = _dyn_setup(schedule=schedule)
    o.update(dels, ins, mode)
    off, col, w = o.graph()
    g2 = synth.apply_batch_numpy(g, dels, ins)
    assert np.array_equal(off, g2.off)
    assert np.array_equal(col, g2.col)
    assert np.array_equal(w, g2.w.astype(np.int64))
    st = o.state()
    rows = np.add.reduceat(w, off[:-1]) if len(w) else np.zeros(g.n)
    rows[np.diff(off) == 0] = 0
    assert np.array_equal(st["K"], rows)
    S = np.zeros(g.n, np.int64)
    np.add.at(S, st["C"], st["K"])
    assert np.array_equal(st["Sigma"], S)
    assert st["m2"] == int(w.sum()) == int(S.sum())
    assert disconnected_communities(off, col, st["C"]) == 0


def _df_reference_marks(g_prev_C, dels, ins, n):
    """Alg. frontier's marking loops written out: endpoints of same-community
    deletions and of cross-community insertions."""
    dV = np.zeros(n, np.uint8)
    for u, v, _ in dels:
        if g_prev_C[u] == g_prev_C[v]:
            dV[u] = dV[v] = 1
    for u, v, _ in ins:
        if g_prev_C[u] != g_prev_C[v]:
            dV[u] = dV[v] = 1
    return dV


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_marking_set_algebra(schedule):
    """ND marks all; DF marks exactly the endpoint rule; DF is a subset of DS;
    DS contains the members of communities hit by same-community deletions."""
    res = {}
    for mode in (oracle.ND, oracle.DS, oracle.DF):
        g, o, dels, ins = _dyn_setup(schedule=schedule)
        Cprev = o.state()["C"]
        o.update(dels, ins, mode)
        res[mode] = o.affected().astype(bool)
    assert res[oracle.ND].all()
    assert np.array_equal(res[oracle.DF], _df_reference_marks(Cprev, dels, ins, g.n).astype(bool))
    assert np.all(res[oracle.DS] | ~res[oracle.DF])
    for u, v, _ in dels:
        if Cprev[u] == Cprev[v]:
            assert res[oracle.DS][Cprev == Cprev[u]].all()
    assert res[oracle.DF].sum() < res[oracle.DS].sum() <= g.n


@pytest.mark.parametrize("mode", [oracle.ND, oracle.DS, oracle.DF])
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_empty_batch_changes_nothing(mode, schedule):
    """DS and DF mark nothing on an empty batch and return C^{t-1} unchanged;
    ND re-processes every vertex (Preliminaries, the Naive-dynamic approach), so it may still improve Q."""
    g, o, _, _ = _dyn_setup(schedule=schedule)
    before = o.state()
    q0 = o.modularity()
    C = o.update(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32), mode)
    after = o.state()
    assert np.array_equal(before["K"], after["K"])
    if mode == oracle.ND:
        assert o.affected().all()
        assert o.modularity() > q0 - 1e-3
        return
    assert o.affected().sum() == 0
    assert np.array_equal(C, before["C"])
    for k in ("Sigma", "dSigma"):
        assert np.array_equal(before[k], after[k])


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_delete_then_reinsert_tracks_ids(schedule):
    """The stability protocol of Approach, "Improving stability": delete a batch, reinsert it; with
    tracking, most vertices keep the community id they had before."""
    g = synth.planted_partition(3000, 30, 14, 0.2, 77)
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=schedule)
    C0 = o.static()
    dels, _ = synth.random_batch(g, 150, seed=78, frac_ins=0.0)
    o.update(dels, np.zeros((0, 3), np.int32), oracle.DF)
    C2 = o.update(np.zeros((0, 3), np.int32), dels, oracle.DF)
    assert (C2 == C0).mean() > 0.95
    off, col, _ = o.graph()
    assert np.array_equal(off, g.off) and np.array_equal(col, g.col)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_refinement_threshold_rule(schedule):
    """Alg. leidenmk with tau_re = 0.6 (Approach, "Minimizing communities to refine"): deletions inside a
    community add to its cumulative change dSigma (both directions count);
    the community is marked for refinement in the batch where
    dSigma/Sigma first exceeds 0.6, and its dSigma then resets to 0."""
    # two 6-cliques joined by the edge 5-6: community A = {0..5} has
    # Sigma = 6*5 + 1 = 31.  Deleting k edges inside A gives dSigma = 2k,
    # Sigma = 31 - 2k, and 2k/(31-2k) > 0.6 first holds at k = 6.
    edges = clique_edges(0, 6) + clique_edges(6, 6) + [(5, 6)]
    off, col, w = csr_from_edges(12, edges)
    o = oracle.Oracle(12, off, col, w.astype(np.int32), schedule=schedule)
    C = o.static()
    assert len(np.unique(C)) == 2
    cA = C[0]
    assert o.state()["Sigma"][cA] == 31
    inner = [(0, 1), (2, 3), (0, 4), (1, 2), (3, 4), (0, 2)]
    for k, (u, v) in enumerate(inner, start=1):
        o.update(np.array([[u, v, 1]], np.int32), np.zeros((0, 3), np.int32), oracle.DF)
        st = o.state()
        assert st["C"][0] == cA
        refined = o.trace()["passes"][0]["refined_any"]
        assert st["Sigma"][cA] == 31 - 2 * k
        if k < 6:
            assert refined == 0 and st["dSigma"][cA] == 2 * k
        else:
            assert refined == 1 and st["dSigma"][cA] == 0


def test_invalid_batches_rejected_without_change():
    g, o, dels, ins = _dyn_setup()
    before = o.state()
    bad = [
        (np.array([[0, 0, 1]], np.int32), np.zeros((0, 3), np.int32)),       # self-loop deletion
        (np.zeros((0, 3), np.int32), np.array([[5, 5, 1]], np.int32)),       # self-loop insertion
        (np.zeros((0, 3), np.int32), np.array([[1, 2, 0]], np.int32)),       # zero weight
        (np.zeros((0, 3), np.int32), np.array([[1, g.n, 1]], np.int32)),     # out of range
    ]
    # a deletion of an absent edge
    for v in range(1, g.n):
        if v not in g.col[g.off[0]:g.off[1]]:
            bad.append((np.array([[0, v, 1]], np.int32), np.zeros((0, 3), np.int32)))
            break
    for d, i in bad:
        with pytest.raises(oracle.OracleError) as e:
            o.update(d, i, oracle.DF)
        assert e.value.rc == oracle.ERR_BATCH
    after = o.state()
    for k in ("C", "K", "Sigma", "dSigma"):
        assert np.array_equal(before[k], after[k])


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_dynamic_quality_close_to_static(schedule):
    """Evaluation, "Performance comparison": the dynamic result stays close to static Leiden's Q."""
    g = synth.planted_partition(4000, 40, 14, 0.3, 55)
    dels, ins = synth.random_batch(g, 400, seed=56)
    g2 = synth.apply_batch_numpy(g, dels, ins)
    qs = {}
    for mode in (oracle.ND, oracle.DS, oracle.DF):
        o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=schedule)
        o.static()
        o.update(dels, ins, mode)
        qs[mode] = o.modularity()
    s = oracle.Oracle(g2.n, g2.off, g2.col, g2.w, schedule=schedule)
    s.static()
    qstat = s.modularity()
    for mode, q in qs.items():
        assert q > qstat - 0.005, (mode, q, qstat)


@pytest.mark.parametrize("scale,seed", [(12, 21), (12, 22), (12, 23), (13, 21), (13, 22), (13, 23)])
def test_sync_and_seq_agree_in_quality(scale, seed):
    """The snapshot schedule loses little against the paper's in-order loop:
    static Leiden on R-MAT graphs of scale 12 and 13 ends within 0.005 in Q
    (the largest gap measured over these six graphs is 0.0044), with every
    community connected under both schedules."""
    g = synth.rmat(scale, seed=seed)
    q = {}
    for sch in SCHEDULES:
        o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=sch)
        C = o.static()
        q[sch] = o.modularity()
        assert disconnected_communities(g.off, g.col, C) == 0
    assert abs(q[oracle.SEQ] - q[oracle.SYNC]) < 0.005


def test_sync_and_seq_agree_on_planted_partition():
    g = synth.planted_partition(4000, 40, 14, 0.3, 55)
    q = {}
    for sch in SCHEDULES:
        o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=sch)
        o.static()
        q[sch] = o.modularity()
    assert abs(q[oracle.SEQ] - q[oracle.SYNC]) < 0.002


# ---- ablation switches (Approach, "Minimizing communities to split": the
# convergence test of Alg. "leiden" read with AND, as printed, or OR)

def test_split_all_changes_nothing_in_static_leiden():
    """Static Leiden refines every community, and a refined community is
    never split, so splitting 'all' communities is the same computation."""
    g = synth.planted_partition(2000, 20, 10, 0.3, 301)
    a = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    b = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC, split_all=1)
    assert np.array_equal(a.static(), b.static())
    assert a.trace() == b.trace()


def test_split_all_keeps_communities_connected_after_updates():
    g = synth.rmat(11, seed=302)
    o = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC, split_all=1)
    o.static()
    cur = g
    for k in range(2):
        d, i = synth.random_batch(cur, 150, seed=303 + k)
        C = o.update(d, i, oracle.DF)
        cur = synth.apply_batch_numpy(cur, d, i)
        assert disconnected_communities(cur.off, cur.col, C) == 0


def test_converge_any_stops_no_later_than_the_printed_test():
    """OR is implied by AND at every pass, so the text's reading never runs
    more passes; the first pass is identical."""
    for g in (synth.planted_partition(2000, 20, 10, 0.3, 304), synth.rmat(11, seed=305)):
        a = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
        b = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC, converge_any=1)
        a.static()
        b.static()
        ta, tb = a.trace(), b.trace()
        assert len(tb["passes"]) <= len(ta["passes"])
        assert ta["passes"][0] == tb["passes"][0]


def test_dcpp_generator_shape():
    """The degree-corrected planted-partition input: symmetric, weights 1..8
    from the unordered pair, a heavy degree tail, seeded bytes."""
    g = synth.dcpp(30000, avg_deg=40, max_deg=5000, cmax=5000, seed=7)
    d = np.diff(g.off)
    src = np.repeat(np.arange(g.n), d)
    fwd = dict(zip(zip(src.tolist(), g.col.tolist()), g.w.tolist()))
    assert all(fwd[(v, u)] == w for (u, v), w in list(fwd.items())[:20000])
    assert g.w.min() >= 1 and g.w.max() <= 8
    assert d.max() > 20 * d.mean()
    h = synth.dcpp(30000, avg_deg=40, max_deg=5000, cmax=5000, seed=7)
    assert np.array_equal(g.col, h.col) and np.array_equal(g.w, h.w)


@pytest.mark.parametrize("schedule", [oracle.SEQ, oracle.SYNC])
def test_graphs_without_edges(schedule):
    """2m = 0: no vertex has a positive gain, so every vertex stays alone and
    Q is 0 by convention; an update that deletes every edge of a community
    leaves its vertices alone, with K, Sigma and 2m all zero."""
    off = np.zeros(6, np.int64)
    o = oracle.Oracle(5, off, np.zeros(0, np.int32), np.zeros(0, np.int64), schedule=schedule)
    assert np.array_equal(o.static(), np.arange(5))
    assert o.modularity() == 0.0
    # one edge: joining gives Q = 0 against -1/2 apart, so the pair merges
    off, col, w = csr_from_edges(2, [(0, 1)])
    o = oracle.Oracle(2, off, col, w, schedule=schedule)
    assert np.array_equal(o.static(), [0, 0])
    assert o.modularity() == 0.0
    # a triangle and an isolated vertex; then every edge deleted
    off, col, w = csr_from_edges(4, [(0, 1), (1, 2), (0, 2)])
    o = oracle.Oracle(4, off, col, w, schedule=schedule)
    assert np.array_equal(o.static(), [0, 0, 0, 3])
    dels = np.array([[0, 1, 1], [1, 2, 1], [0, 2, 1]], np.int32)
    c = o.update(dels, np.zeros((0, 3), np.int32), oracle.DF)
    assert len(np.unique(c)) == 4
    assert c[0] == 0 and c[3] == 3  # the old ids stay with their vertices where they can
    st = o.state()
    assert st["m2"] == 0 and not st["K"].any() and not st["Sigma"].any()
    assert o.modularity() == 0.0


# ---- Alg. "delta", insertion side: the community c* a source marks
#
# Gain of Eq. 2 times 2m^2 for moving i to c with K_{i->c} = H[c] (the
# inserted weight from i to c) and K_{i->d} = 0, on the state before the
# batch (marking precedes updateWeights in Alg. "delta"):
#     g(c) = 2m * H[c] - K_i (K_i + Sigma_c - Sigma_d)
# The term in Sigma_d is the same for every c, so c* maximises
# 2m * H[c] - K_i * Sigma_c, ties to the lower community id.

def _ds_graph(k, first, second):
    """Clique X on 0..k-1, then two blocks, each a clique with one pendant
    vertex hung on the clique's first vertex.  Returns the CSR and, per
    block, (first clique vertex, clique size, pendant)."""
    edges = clique_edges(0, k)
    blocks, base = [], k
    for s in (first, second):
        edges += clique_edges(base, s) + [(base, base + s)]
        blocks.append((base, s, base + s))
        base += s + 1
    off, col, w = csr_from_edges(base, edges)
    return base, off, col, w.astype(np.int32), blocks


def _ds_marks(k, first, second, h_first, h_second, schedule):
    """Static Leiden, then one DS update inserting (0, pendant) edges of
    weights h_first and h_second.  Returns the blocks, C^{t-1}, the state
    before the batch and dV."""
    n, off, col, w, blocks = _ds_graph(k, first, second)
    o = oracle.Oracle(n, off, col, w, schedule=schedule)
    C = o.static()
    st = o.state()
    ins = np.array([[0, blocks[0][2], h_first], [0, blocks[1][2], h_second]], np.int32)
    o.update(np.zeros((0, 3), np.int32), ins, oracle.DS)
    return blocks, C, st, o.affected().astype(bool)


def _interior(block):
    """Clique vertices of a block other than the one the pendant hangs on:
    DS marks them only through the community c* (neither they nor their
    neighbours are a source of the batch)."""
    b, s, _ = block
    return list(range(b + 1, b + s))


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_ds_best_community_beats_larger_inserted_weight(schedule):
    """X = K10 (K_0 = 9, Sigma_X = 90), A = K10 + pendant (Sigma_A = 92),
    B = K3 + pendant (Sigma_B = 8), 2m = 190; insert (0, pA) with weight 2
    and (0, pB) with weight 1.  g(A) - g(B) = 190 * (2 - 1) - 9 * (92 - 8)
    = -566 < 0, so c* = B although more weight goes to A: B is marked whole,
    the interior of A is not."""
    (A, B), C, st, dV = _ds_marks(10, 10, 3, 2, 1, schedule)
    assert len(np.unique(C)) == 3
    assert st["K"][0] == 9 and st["m2"] == 190
    assert st["Sigma"][C[A[0]]] == 92 and st["Sigma"][C[B[0]]] == 8
    assert dV[_interior(B)].all()
    assert not dV[_interior(A)].any()
    assert dV[:10].all()  # X: the pendants' c* is the community of vertex 0


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_ds_best_community_uses_the_state_before_the_batch(schedule):
    """X = K4 (K_0 = 3), A = K5 + pendant (Sigma_A = 22), B = K4 + pendant
    (Sigma_B = 14), 2m = 48; insert weights 11 (to A) and 10 (to B).
    Before the batch: g(A) - g(B) = 48 * 1 - 3 * (22 - 14) = 24 > 0, c* = A.
    With the totals after the batch (K_0 = 24, Sigma_A = 33, Sigma_B = 24,
    2m = 90) it would be 90 - 24 * 9 < 0, i.e. B: A must be marked, B not."""
    (A, B), C, st, dV = _ds_marks(4, 5, 4, 11, 10, schedule)
    assert st["K"][0] == 3 and st["m2"] == 48
    assert st["Sigma"][C[A[0]]] == 22 and st["Sigma"][C[B[0]]] == 14
    assert dV[_interior(A)].all()
    assert not dV[_interior(B)].any()


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("swap", [False, True])
def test_ds_best_community_tie_goes_to_the_lower_id(schedule, swap):
    """Two identical blocks (K5 + pendant, Sigma 22 each) receive weight 1
    each: equal gains, so c* is the block whose community id is lower --
    the one laid out first, whichever insertion is listed first."""
    n, off, col, w, blocks = _ds_graph(4, 5, 5)
    o = oracle.Oracle(n, off, col, w, schedule=schedule)
    C = o.static()
    first, second = blocks
    assert C[first[0]] < C[second[0]]
    pair = [[0, first[2], 1], [0, second[2], 1]]
    if swap:
        pair = pair[::-1]
    o.update(np.zeros((0, 3), np.int32), np.array(pair, np.int32), oracle.DS)
    dV = o.affected().astype(bool)
    assert dV[_interior(first)].all()
    assert not dV[_interior(second)].any()


# ---- Alg. "leidentr": ids of communities no old community is matched to

def _tracking_graph():
    """S = K3 on 0..2; Q = K4 on 3..6 with a pendant 7 on vertex 4; P = the
    cliques P1 = K6 on 8..13, P2 = K3 on 14..16 and P3 = K4 on 17..20 with
    every P1-P2 and P1-P3 pair joined; R = K6 on 21..26."""
    edges = (clique_edges(0, 3) + clique_edges(3, 4) + [(4, 7)] + clique_edges(8, 6) + clique_edges(14, 3)
             + clique_edges(17, 4) + clique_edges(21, 6))
    bridges = [(u, v) for u in range(8, 14) for v in range(14, 21)]
    off, col, w = csr_from_edges(27, edges + bridges)
    return off, col, w.astype(np.int32), bridges


@pytest.mark.parametrize("mode", [oracle.ND, oracle.DS, oracle.DF])
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_tracking_gives_free_ids_in_order(mode, schedule):
    """Static Leiden takes each community's member of largest degree as its
    id (ties to the lower vertex): S -> 0, Q -> 4 (vertex 4 carries the
    pendant), P -> 8 (P1's vertices have degree 12), R -> 21.  The batch
    deletes every P1-P2 / P1-P3 edge and inserts every S-R pair.  Then
    * S and R merge; R carries the larger overlap, so the merged community
      keeps 21, and S's old id 0 stays reserved (not handed out again);
    * P falls apart into P1, P2, P3 (splitting labels each part by its
      smallest vertex: 8, 14, 17); P1 carries the largest overlap and keeps 8;
    * P2 and P3 match no old community: in ascending order of their labels
      they take the smallest ids no old community used -- 1, then 2 -- not
      by size (P3 is the larger) and skipping the reserved 0.
    tau_re = 2 keeps P out of refinement (dSigma/Sigma = 84/48 for P), so
    the pass loop ends after one pass with the split labels."""
    off, col, w, bridges = _tracking_graph()
    o = oracle.Oracle(27, off, col, w, schedule=schedule, tau_refine=2.0)
    C = o.static()
    expect0 = [0] * 3 + [4] * 5 + [8] * 13 + [21] * 6
    assert C.tolist() == expect0
    dels = np.array([[u, v, 1] for u, v in bridges], np.int32)
    ins = np.array([[u, v, 1] for u in range(0, 3) for v in range(21, 27)], np.int32)
    C2 = o.update(dels, ins, mode)
    expect = [21] * 3 + [4] * 5 + [8] * 6 + [1] * 3 + [2] * 4 + [21] * 6
    assert C2.tolist() == expect
    assert o.trace()["passes"][0]["refined_any"] == 0
