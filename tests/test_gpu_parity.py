"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Deterministic mode must equal the oracle's SYNC schedule bit for bit: the
applied CSR, the affected set, K / Sigma / Delta Sigma / 2m, the per-pass
trace (iterations, moves per iteration, communities, refinement rounds),
the final membership and Q (same double).  Asynchronous mode must give
connected communities within 0.005 of the oracle's SEQ modularity.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_15451_gb300 import leiden as L
from paper_2410_15451_gb300 import synth
from tests.helpers import csr_from_edges, disconnected_communities

pytestmark = pytest.mark.gpu

MODES = [(L.LEIDEN_ND, oracle.ND), (L.LEIDEN_DS, oracle.DS), (L.LEIDEN_DF, oracle.DF)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15451_gb300 import _build

    _build.build()
    L.load()


def hub_graph(seed=5):
    """Planted partition plus a hub joined to 3000 vertices (degree > 2048)
    and a star of 40 leaves: exercises the global-table bins."""
    g = synth.planted_partition(6000, 30, 10, 0.25, seed)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    keep = src < g.col
    edges = list(zip(src[keep].tolist(), g.col[keep].tolist()))
    rng = np.random.default_rng(seed)
    hub = 17
    for v in rng.choice(np.arange(200, 6000), 3000, replace=False):
        edges.append((hub, int(v)))
    for leaf in range(6000, 6040):
        edges.append((6040, leaf))
    edges = sorted({(min(a, b), max(a, b)) for a, b in edges if a != b})
    off, col, w = csr_from_edges(6041 + 5, edges)  # 5 isolated vertices at the end
    return synth.Graph(6046, off, col, w.astype(np.int32))


GRAPHS = {
    "planted10k": lambda: synth.workload_small(),
    "rmat12": lambda: synth.rmat(12, seed=31),
    "rmat14": lambda: synth.rmat(14, seed=32),
    "hubs": lambda: hub_graph(),
    "weighted": lambda: _weighted(synth.planted_partition(3000, 15, 12, 0.3, 41)),
    # degree-corrected planted partition: power-law degrees and community sizes, weights 1..8
    "dcpp": lambda: synth.dcpp(20000, avg_deg=30, max_deg=3000, cmax=3000, seed=42),
}


def _weighted(g):
    # symmetric weights 1..8 from the smaller endpoint pair
    src = np.repeat(np.arange(g.n), np.diff(g.off)).astype(np.int64)
    a, b = np.minimum(src, g.col), np.maximum(src, g.col)
    w = ((a * 2654435761 + b * 40503) % 8 + 1).astype(np.int32)
    return synth.Graph(g.n, g.off, g.col, w)


def _heavy(g):
    # symmetric weights just below 2^30: one warp's sum for one community
    # passes 2^32 in the hub scan's 32-bit tables
    src = np.repeat(np.arange(g.n), np.diff(g.off)).astype(np.int64)
    a, b = np.minimum(src, g.col), np.maximum(src, g.col)
    w = ((1 << 30) - (a * 2654435761 + b * 40503) % 4096).astype(np.int32)
    return synth.Graph(g.n, g.off, g.col, w)


def assert_same_state(gpu, ref):
    gs, rs = gpu.state(), ref.state()
    for k in ("C", "K", "Sigma", "dSigma"):
        assert np.array_equal(gs[k], rs[k]), k
    assert gs["m2"] == rs["m2"]


def assert_same_trace(gpu, ref):
    tg, tr = gpu.trace(), ref.trace()
    assert tg["affected"] == tr["affected"]
    assert len(tg["passes"]) == len(tr["passes"])
    for pg, pr in zip(tg["passes"], tr["passes"]):
        assert pg == pr, (pg, pr)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_static_bit_exact(name):
    g = GRAPHS[name]()
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    cg, cr = gpu.static(), ref.static()
    assert_same_trace(gpu, ref)
    assert np.array_equal(cg, cr)
    assert_same_state(gpu, ref)
    assert gpu.modularity() == ref.modularity()
    assert disconnected_communities(g.off, g.col, cg) == 0


@pytest.mark.parametrize("name", ["planted10k", "rmat14", "hubs", "weighted", "dcpp"])
@pytest.mark.parametrize("mode", MODES, ids=["ND", "DS", "DF"])
def test_updates_bit_exact(name, mode):
    gm, om = mode
    g = GRAPHS[name]()
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    gpu.static()
    ref.static()
    cur = g
    for k, size in enumerate([7, 150, 1200, 4000]):  # the last sorts > 2048 arcs by radix passes
        dels, ins = synth.random_batch(cur, size, seed=500 + k, w_lo=1, w_hi=8 if name in ("weighted", "dcpp") else 1)
        cg = gpu.update(dels, ins, gm)
        cr = ref.update(dels, ins, om)
        cur = synth.apply_batch_numpy(cur, dels, ins)
        og, rg = gpu.graph(), ref.graph()
        for a, b in zip(og, rg):
            assert np.array_equal(a, b)
        assert np.array_equal(gpu.affected(), ref.affected())
        assert_same_trace(gpu, ref)
        assert np.array_equal(cg, cr), f"batch {k}"
        assert_same_state(gpu, ref)
        assert gpu.modularity() == ref.modularity()


def test_heavy_weights_bit_exact():
    """Weights near 2^30 on the hub graph: the 32-bit warp sums of the hub
    scan carry past 2^32 and must stay exact, in static Leiden (local moving
    and refinement) and in a DF update with heavy insertions."""
    g = _heavy(hub_graph())
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    for step in range(2):
        if step == 0:
            cg, cr = gpu.static(), ref.static()
        else:
            dels, ins = synth.random_batch(g, 300, seed=91, w_lo=1 << 29, w_hi=1 << 30)
            cg, cr = gpu.update(dels, ins, L.LEIDEN_DF), ref.update(dels, ins, oracle.DF)
        assert_same_trace(gpu, ref)
        assert np.array_equal(cg, cr), f"step {step}"
        assert_same_state(gpu, ref)
        assert gpu.modularity() == ref.modularity()


def test_batch_edge_cases_bit_exact():
    """Insertion of an existing edge (weights add), delete + reinsert of the
    same edge, repeated insertions (add up) and repeated deletions (collapse),
    isolating a vertex, and rows that outgrow their slack (rebuild)."""
    g = synth.planted_partition(2000, 20, 10, 0.2, 61)
    gpu = L.Leiden(g.n, g.off, g.col, g.w, slack=0.0, min_slack=1)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    gpu.static()
    ref.static()
    u = 5
    nb = g.col[g.off[u]:g.off[u + 1]]
    v0, v1 = int(nb[0]), int(nb[1])
    dels = np.array([[u, v0, 1], [v0, u, 1], [u, v1, 9]], np.int32)          # repeated deletion
    ins = np.array([[u, v1, 3],                                              # delete + reinsert
                    [u, int(nb[2]), 2], [u, int(nb[2]), 1],                  # existing edge, twice
                    [u, 1500, 1], [u, 1501, 1], [u, 1502, 1], [1500, 1501, 4]], np.int32)
    cg = gpu.update(dels, ins, L.LEIDEN_DF)
    cr = ref.update(dels, ins, oracle.DF)
    for a, b in zip(gpu.graph(), ref.graph()):
        assert np.array_equal(a, b)
    assert np.array_equal(cg, cr)
    assert_same_state(gpu, ref)
    # isolate vertex 7 entirely
    nb7 = g.col[g.off[7]:g.off[8]]
    d2 = np.array([[7, int(v), 1] for v in nb7], np.int32)
    cg = gpu.update(d2, np.zeros((0, 3), np.int32), L.LEIDEN_DS)
    cr = ref.update(d2, np.zeros((0, 3), np.int32), oracle.DS)
    assert np.array_equal(cg, cr)
    assert_same_state(gpu, ref)


def test_empty_batch_and_invalid_batches():
    g = synth.planted_partition(2000, 20, 10, 0.2, 62)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    gpu.static()
    before = gpu.state()
    c = gpu.update(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32), L.LEIDEN_DF)
    assert np.array_equal(c, before["C"])
    assert gpu.affected().sum() == 0
    absent = next(v for v in range(1, g.n) if v not in g.col[g.off[0]:g.off[1]])
    bad = [
        (np.array([[0, absent, 1]], np.int32), np.zeros((0, 3), np.int32)),
        (np.zeros((0, 3), np.int32), np.array([[3, 3, 1]], np.int32)),
        (np.zeros((0, 3), np.int32), np.array([[1, 2, 0]], np.int32)),
        (np.zeros((0, 3), np.int32), np.array([[1, g.n, 1]], np.int32)),
    ]
    for d, i in bad:
        with pytest.raises(L.LeidenError) as e:
            gpu.update(d, i, L.LEIDEN_DF)
        assert e.value.status == L.LEIDEN_ERR_BATCH
        after = gpu.state()
        for k in ("C", "K", "Sigma", "dSigma"):
            assert np.array_equal(before[k], after[k])
        og = gpu.graph()
        assert np.array_equal(og[0], g.off) and np.array_equal(og[1], g.col)


def test_update_before_static_is_rejected():
    g = synth.planted_partition(500, 5, 8, 0.2, 63)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    with pytest.raises(L.LeidenError) as e:
        gpu.update(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32), L.LEIDEN_DF)
    assert e.value.status == L.LEIDEN_ERR_STATE


@pytest.mark.parametrize("name", ["planted10k", "rmat14", "hubs"])
def test_async_mode_quality(name):
    """In-place moves: connected communities, Q within 0.005 of the oracle's
    SEQ schedule (static and after a DF update)."""
    g = GRAPHS[name]()
    gpu = L.Leiden(g.n, g.off, g.col, g.w, deterministic=False)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SEQ)
    cg = gpu.static()
    ref.static()
    assert disconnected_communities(g.off, g.col, cg) == 0
    assert gpu.modularity() >= ref.modularity() - 0.005
    dels, ins = synth.random_batch(g, 300, seed=77)
    cg = gpu.update(dels, ins, L.LEIDEN_DF)
    ref.update(dels, ins, oracle.DF)
    off, col, _ = gpu.graph()
    assert disconnected_communities(off, col, cg) == 0
    assert gpu.modularity() >= ref.modularity() - 0.005


def test_modularity_of_given_membership_matches_oracle():
    g = synth.rmat(12, seed=33)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    rng = np.random.default_rng(3)
    for _ in range(3):
        C = rng.integers(0, 50, g.n).astype(np.int32)
        q, _ = oracle.modularity(g.off, g.col, g.w.astype(np.int64), C)
        assert gpu.modularity(C) == q


def test_device_entry_point_matches_host_entry_point():
    import torch

    g = synth.rmat(13, seed=34)
    dels, ins = synth.random_batch(g, 400, seed=35)
    a = L.Leiden(g.n, g.off, g.col, g.w)
    b = L.Leiden(g.n, g.off, g.col, g.w)
    a.static()
    b.static()
    ca = a.update(dels, ins, L.LEIDEN_DF)
    dd = torch.from_numpy(dels).cuda()
    di = torch.from_numpy(ins).cuda()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    L.leiden_update_device(b.h, dd, len(dels), di, len(ins), L.LEIDEN_DF, out)
    assert np.array_equal(out.cpu().numpy(), ca)


def test_stats_timers_and_launch_counter_leave_results_unchanged():
    """collect_stats (phase events, per-launch events of the warp-bin
    local-moving kernel) only observes: the result is the same bit for bit;
    the launch counter counts this library's kernels."""
    g = synth.rmat(14, seed=36)
    a = L.Leiden(g.n, g.off, g.col, g.w, collect_stats=3)
    b = L.Leiden(g.n, g.off, g.col, g.w)
    assert np.array_equal(a.static(), b.static())
    dels, ins = synth.random_batch(g, 500, seed=37)
    n0 = L.leiden_kernel_launches()
    ca = a.update(dels, ins, L.LEIDEN_DF)
    n1 = L.leiden_kernel_launches()
    cb = b.update(dels, ins, L.LEIDEN_DF)
    assert np.array_equal(ca, cb)
    assert n1 - n0 >= 10
    s = a.stats()
    assert s["lmk_launches"][0] > 0 and s["lmk_ms"][0] > 0 and s["ms_move"] > 0
    # phase times from events at the phase boundaries, bytes from the counters
    assert all(x >= 0 for x in s["phase_ms"]) and s["phase_ms"][L.PHASES.index("move")] == s["ms_move"]
    assert abs(sum(s["phase_ms"]) - s["ms_total"]) < 1e-9 * max(1.0, s["ms_total"])
    assert all(b > 0 for b in s["phase_bytes"])
    assert s["phase_bytes"][L.PHASES.index("move")] >= sum(s["lmk_bytes"])
    assert s["affected"] == a.trace()["affected"]
    assert b.stats()["phase_bytes"] == s["phase_bytes"] and b.stats()["phase_ms"] == [0.0] * 6
    # the other timed kernels: split sampling runs in every DF update that splits
    assert s["xk_launches"][0] > 0 and s["xk_ms"][0] > 0 and s["xk_bytes"][0] > 0
    assert b.stats()["xk_bytes"] == s["xk_bytes"] and b.stats()["xk_launches"] == [0, 0, 0]
    v, e = s["lmk_vertices"], s["lmk_arcs"]
    # every visit of a vertex with arcs goes through one of the three kernels
    assert v[0] + v[1] + v[2] <= s["lm_vertices"] and e[0] + e[1] + e[2] == s["lm_arcs"]
    for k in range(3):
        lo = (40 * v[k] if k < 2 else 0) + 12 * e[k]
        assert lo <= s["lmk_bytes"][k] <= lo + 4 * e[k]


@pytest.mark.parametrize("flags", [dict(split_all=1), dict(converge_any=1), dict(tau_refine=0.2),
                                   dict(tau_refine=2.0)], ids=["split_all", "converge_any", "tau_re0.2", "tau_re2"])
def test_ablation_switches_bit_exact(flags):
    """The ablation switches (split every unrefined community, the OR reading
    of the convergence test, other tau_re) match the oracle bit for bit."""
    g = synth.rmat(13, seed=306)
    gpu = L.Leiden(g.n, g.off, g.col, g.w, **flags)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC, **flags)
    assert np.array_equal(gpu.static(), ref.static())
    assert_same_trace(gpu, ref)
    cur = g
    for k in range(2):
        d, i = synth.random_batch(cur, 400, seed=307 + k)
        cg, cr = gpu.update(d, i, L.LEIDEN_DF), ref.update(d, i, oracle.DF)
        cur = synth.apply_batch_numpy(cur, d, i)
        assert_same_trace(gpu, ref)
        assert np.array_equal(cg, cr)
        assert_same_state(gpu, ref)


@pytest.mark.parametrize("tuning", [dict(tiny_max=0), dict(tiny_max=4, warp_max=32, block_max=256),
                                    dict(warp_max=64, block_max=512, warp_blocks_per_sm=2, block_blocks_per_sm=3,
                                         hub_blocks_per_sm=4), dict(overlap=0)],
                         ids=["no-tiny", "small-bins", "mixed", "one-stream"])
def test_launch_shapes_do_not_change_results(tuning):
    """Bin thresholds, grid sizes and the side streams only move work
    between kernels and streams."""
    g = GRAPHS["hubs"]()
    a = L.Leiden(g.n, g.off, g.col, g.w)
    b = L.Leiden(g.n, g.off, g.col, g.w)
    L.leiden_set_tuning(b.h, **tuning)
    assert np.array_equal(a.static(), b.static())
    for k in range(2):
        d, i = synth.random_batch(synth.Graph(g.n, *a.graph()[:2], a.graph()[2].astype(np.int32)), 300,
                                  seed=311 + k)
        assert np.array_equal(a.update(d, i, L.LEIDEN_DF), b.update(d, i, L.LEIDEN_DF))
        assert a.trace()["passes"] == b.trace()["passes"]
    with pytest.raises(L.LeidenError):
        L.leiden_set_tuning(b.h, warp_max=200)
    with pytest.raises(L.LeidenError):
        L.leiden_set_tuning(b.h, overlap=2)


def test_full_rebuild_when_the_spill_arena_fills():
    """Rows that outgrow their slack move to the spill arena; once it is full
    the whole CSR is rebuilt.  Both paths keep the result bit-exact."""
    g = synth.planted_partition(2000, 20, 10, 0.2, 62)
    gpu = L.Leiden(g.n, g.off, g.col, g.w, slack=0.0, min_slack=1, arena_log2=0)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    gpu.static()
    ref.static()
    cur, rebuilds = g, 0
    for k in range(4):
        dels, ins = synth.random_batch(cur, 800, seed=600 + k)
        cg, cr = gpu.update(dels, ins, L.LEIDEN_DF), ref.update(dels, ins, oracle.DF)
        rebuilds += gpu.stats()["rebuilds"]
        cur = synth.apply_batch_numpy(cur, dels, ins)
        for a, b in zip(gpu.graph(), ref.graph()):
            assert np.array_equal(a, b)
        assert np.array_equal(cg, cr)
        assert_same_state(gpu, ref)
    assert rebuilds >= 1


def long_rows_graph(seed=8):
    """Planted partition plus two hubs of degree 7000 and 5000, longer than
    the 4096 arcs a block merges in shared memory, so batches that touch them
    take the chunked merge over all SMs (and, without slack, the move of a
    long row to the spill arena)."""
    g = synth.planted_partition(12000, 60, 10, 0.25, seed)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    keep = src < g.col
    edges = set(zip(src[keep].tolist(), g.col[keep].tolist()))
    rng = np.random.default_rng(seed)
    for hub, deg in ((3, 7000), (11000, 5000)):
        for v in rng.choice(np.arange(100, 11900), deg, replace=False):
            if int(v) != hub:
                edges.add((min(hub, int(v)), max(hub, int(v))))
    off, col, w = csr_from_edges(g.n, sorted(edges))
    return synth.Graph(g.n, off, col, w.astype(np.int32))


@pytest.mark.parametrize("slack", [0.25, 0.0])
@pytest.mark.parametrize("mode", MODES, ids=["ND", "DS", "DF"])
def test_long_rows_merge_bit_exact(slack, mode):
    """Batches that delete and insert arcs of rows longer than 4096: the
    chunked merge must give the oracle's CSR exactly, and the update the
    oracle's membership, trace and state."""
    gm, om = mode
    g = long_rows_graph()
    gpu = L.Leiden(g.n, g.off, g.col, g.w, slack=slack, min_slack=1)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    gpu.static()
    ref.static()
    cur = g
    rng = np.random.default_rng(9)
    for k in range(3):
        dels, ins = synth.random_batch(cur, 600, seed=700 + k)
        # plus edits on the hubs: delete 300 of their arcs, insert 400 new ones
        extra_d, extra_i = [], []
        for hub in (3, 11000):
            nb = cur.col[cur.off[hub]:cur.off[hub + 1]]
            taken = set(map(tuple, np.sort(dels[:, :2], axis=1).tolist())) | set(
                map(tuple, np.sort(ins[:, :2], axis=1).tolist()))
            for v in rng.choice(nb, 150, replace=False):
                e = (min(hub, int(v)), max(hub, int(v)))
                if e not in taken:
                    extra_d.append([hub, int(v), 1])
                    taken.add(e)
            non = np.setdiff1d(np.arange(cur.n), np.append(nb, hub))
            for v in rng.choice(non, 200, replace=False):
                e = (min(hub, int(v)), max(hub, int(v)))
                if e not in taken:
                    extra_i.append([int(v), hub, 1])
                    taken.add(e)
        dels = np.concatenate([dels, np.array(extra_d, np.int32).reshape(-1, 3)])
        ins = np.concatenate([ins, np.array(extra_i, np.int32).reshape(-1, 3)])
        cg = gpu.update(dels, ins, gm)
        cr = ref.update(dels, ins, om)
        cur = synth.apply_batch_numpy(cur, dels, ins)
        for a, b in zip(gpu.graph(), ref.graph()):
            assert np.array_equal(a, b), f"batch {k}"
        assert np.array_equal(gpu.affected(), ref.affected())
        assert_same_trace(gpu, ref)
        assert np.array_equal(cg, cr), f"batch {k}"
        assert_same_state(gpu, ref)
    assert np.diff(cur.off)[3] > 4096


def cliques_graph(triangles, seed=12):
    """Four 60-cliques, each with three arcs to other vertices, and
    `triangles` disjoint triangles.  A clique's refined communities hold more
    than 1024 member arcs, so aggregation sums them in global tables of their
    own: with 20000 triangles the level has more communities than twice those
    arcs and the tables are hashed; with 30 a table has a slot per community
    and is indexed by the community id."""
    rng = np.random.default_rng(seed)
    edges = []
    for t in range(triangles):
        a = 3 * t
        edges += [(a, a + 1), (a, a + 2), (a + 1, a + 2)]
    base = 3 * triangles
    for q in range(4):
        mem = list(range(base + 60 * q, base + 60 * q + 60))
        edges += [(a, b) for i, a in enumerate(mem) for b in mem[i + 1:]]
        for v in rng.choice(base + 240, 3, replace=False):
            if not (mem[0] <= v <= mem[-1]):
                edges.append((min(mem[0], int(v)), max(mem[0], int(v))))
    edges = sorted(set(edges))
    off, col, w = csr_from_edges(base + 240, edges)
    return synth.Graph(base + 240, off, col, w.astype(np.int32))


@pytest.mark.parametrize("triangles,table", [(20000, 0), (30, 1)], ids=["hashed", "indexed"])
def test_giant_community_aggregation_tables_bit_exact(triangles, table):
    """Both kinds of global table of the chunked aggregation (hashed, and
    indexed by the community id) give the oracle's result bit for bit: the
    static run that builds them, then DF and ND updates."""
    g = cliques_graph(triangles)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    assert np.array_equal(gpu.static(), ref.static())
    assert gpu.stats()["agg_tables"][table] > 0
    assert_same_trace(gpu, ref)
    assert_same_state(gpu, ref)
    cur = g
    for k, (gm, om) in enumerate((MODES[2], MODES[0])):
        dels, ins = synth.random_batch(cur, 150, seed=1300 + k)
        assert np.array_equal(gpu.update(dels, ins, gm), ref.update(dels, ins, om)), k
        cur = synth.apply_batch_numpy(cur, dels, ins)
        assert_same_trace(gpu, ref)
        assert_same_state(gpu, ref)


@pytest.mark.parametrize("case", ["gain_order", "state_before_batch", "tie"])
def test_ds_best_community_pin_graphs_bit_exact(case):
    """The hand-derived Delta-screening cases of the oracle pins (the
    community c* a source of insertions marks) on the CUDA path."""
    from tests.test_oracle_pins import _ds_graph

    k, a, b, ha, hb = {"gain_order": (10, 10, 3, 2, 1), "state_before_batch": (4, 5, 4, 11, 10),
                       "tie": (4, 5, 5, 1, 1)}[case]
    n, off, col, w, blocks = _ds_graph(k, a, b)
    gpu = L.Leiden(n, off, col, w)
    ref = oracle.Oracle(n, off, col, w, schedule=oracle.SYNC)
    assert np.array_equal(gpu.static(), ref.static())
    ins = np.array([[0, blocks[0][2], ha], [0, blocks[1][2], hb]], np.int32)
    cg = gpu.update(np.zeros((0, 3), np.int32), ins, L.LEIDEN_DS)
    cr = ref.update(np.zeros((0, 3), np.int32), ins, oracle.DS)
    assert np.array_equal(gpu.affected(), ref.affected())
    assert np.array_equal(cg, cr)
    assert_same_state(gpu, ref)


@pytest.mark.parametrize("mode", MODES, ids=["ND", "DS", "DF"])
def test_tracking_pin_graph_bit_exact(mode):
    """The hand-derived tracking case of the oracle pins (a merge that keeps
    the larger overlap's id, a split whose unmatched parts take the smallest
    free ids in ascending order) on the CUDA path."""
    from tests.test_oracle_pins import _tracking_graph

    gm, om = mode
    off, col, w, bridges = _tracking_graph()
    gpu = L.Leiden(27, off, col, w, tau_refine=2.0)
    ref = oracle.Oracle(27, off, col, w, schedule=oracle.SYNC, tau_refine=2.0)
    assert np.array_equal(gpu.static(), ref.static())
    dels = np.array([[u, v, 1] for u, v in bridges], np.int32)
    ins = np.array([[u, v, 1] for u in range(0, 3) for v in range(21, 27)], np.int32)
    cg = gpu.update(dels, ins, gm)
    assert np.array_equal(cg, ref.update(dels, ins, om))
    assert cg.tolist() == [21] * 3 + [4] * 5 + [8] * 6 + [1] * 3 + [2] * 4 + [21] * 6


def _async_run(g, ref, updates=3):
    """Static Leiden and `updates` DF updates of 1e-3|E| in the in-place mode
    and in the oracle; yields (GPU Q, oracle Q) after each step, with every
    community checked for connectivity."""
    gpu = L.Leiden(g.n, g.off, g.col, g.w, deterministic=False)
    cg = gpu.static()
    ref.static()
    assert disconnected_communities(g.off, g.col, cg) == 0
    yield gpu.modularity(), ref.modularity()
    cur = g
    for k in range(updates):
        dels, ins = synth.random_batch(cur, int(1e-3 * cur.edges), seed=78 + k)
        cg = gpu.update(dels, ins, L.LEIDEN_DF)
        ref.update(dels, ins, oracle.DF)
        cur = synth.apply_batch_numpy(cur, dels, ins)
        assert disconnected_communities(cur.off, cur.col, cg) == 0
        yield gpu.modularity(), ref.modularity()


def test_async_mode_quality_rmat17_against_the_sequential_oracle():
    """In-place moves on R-MAT scale 17: connected communities and Q within
    0.005 of the oracle's SEQ schedule (the paper's loop order), for static
    Leiden and three DF updates."""
    g = synth.rmat(17, seed=41)
    for q_gpu, q_seq in _async_run(g, oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SEQ)):
        assert q_gpu >= q_seq - 0.005


@pytest.mark.parametrize("seed", [38, 39, 40])
def test_async_mode_quality_rmat16_against_the_snapshot_oracle(seed):
    """In-place moves on R-MAT scale 16: connected communities and Q within
    0.005 of the oracle's snapshot schedule (the schedule the deterministic
    mode reproduces bit for bit), for static Leiden and three DF updates."""
    g = synth.rmat(16, seed=seed)
    for q_gpu, q_sync in _async_run(g, oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)):
        assert q_gpu >= q_sync - 0.005


@pytest.mark.parametrize("mode", MODES, ids=["ND", "DS", "DF"])
def test_insertion_heavy_batch_that_aggregates_bit_exact(mode):
    """A batch that adds far more arcs than it removes and marks a community
    for refinement (its Delta Sigma passes tau_re * Sigma), so the update
    aggregates a graph with more arcs than before the batch: the aggregated
    levels must fit, and the result must be the oracle's."""
    gm, om = mode
    g = synth.planted_partition(2000, 20, 8, 0.2, 64)
    gpu = L.Leiden(g.n, g.off, g.col, g.w)
    ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
    gpu.static()
    ref.static()
    C = ref.state()["C"]
    members = np.nonzero(C == C[0])[0]
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    existing = set(zip(src.tolist(), g.col.tolist()))
    rng = np.random.default_rng(65)
    ins, seen = [], set()
    while len(ins) < 6 * len(members):
        u, v = (int(x) for x in rng.choice(members, 2, replace=False))
        if (u, v) in existing or (min(u, v), max(u, v)) in seen:
            continue
        seen.add((min(u, v), max(u, v)))
        ins.append([u, v, 1])
    # plus new edges all over the graph, so that the arcs grow everywhere
    while len(ins) < 6 * len(members) + 3000:
        u, v = (int(x) for x in rng.integers(0, g.n, 2))
        if u == v or (u, v) in existing or (min(u, v), max(u, v)) in seen:
            continue
        seen.add((min(u, v), max(u, v)))
        ins.append([u, v, 1])
    ins = np.array(ins, np.int32)
    dels = np.zeros((0, 3), np.int32)
    cg = gpu.update(dels, ins, gm)
    cr = ref.update(dels, ins, om)
    tr = ref.trace()
    assert tr["passes"][0]["refined_any"] == 1 and len(tr["passes"]) >= 2  # it aggregated
    assert_same_trace(gpu, ref)
    assert np.array_equal(cg, cr)
    assert_same_state(gpu, ref)
    assert gpu.modularity() == ref.modularity()
