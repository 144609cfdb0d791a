"""The full-size checks of the benchmark restate connectivity and Eq. 1
without the oracle (label propagation in torch, exact integers); here they
are held against the oracle's component labelling and modularity on small
graphs, including memberships with a disconnected community."""
from __future__ import annotations

import os

import numpy as np
import pytest

import bench
import oracle
from paper_2410_15451_gb300 import synth
from tests.helpers import csr_from_edges


@pytest.mark.parametrize("chunk", [7, 1000, 1 << 28])
def test_components_and_modularity_match_the_oracle(chunk):
    g = synth.rmat(12, 16, 0.57, 0.19, 0.19, 11)
    C = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC).static()
    r = bench.community_checks(g.off, g.col, g.w, C, "cpu", chunk_arcs=chunk)
    labels = oracle.split(g.off, g.col, C, np.ones(g.n, np.uint8))
    assert r["components"] == len(np.unique(labels)) == len(np.unique(C)) == r["communities"]
    assert r["connected"]
    q_or, num = oracle.modularity(g.off, g.col, g.w, C)
    assert r["m2"] * r["intra"] - num == sum(int(x) ** 2 for x in np.bincount(C, np.diff(g.off).astype(float)))
    assert abs(r["q"] - q_or) <= 1e-12


def test_a_disconnected_community_is_found():
    # a ring of eight 5-cliques, one community per clique, then cliques 0
    # and 2 (which share no edge) under one id
    L, k = 8, 5
    edges = [(c * k + i, c * k + j) for c in range(L) for i in range(k) for j in range(i + 1, k)]
    edges += [(c * k, ((c + 1) % L) * k + 1) for c in range(L)]
    off, col, w = csr_from_edges(L * k, edges)
    C = np.repeat(np.arange(L, dtype=np.int32), k)
    for C2, extra in ((C, 0), (np.where(C == 2, 0, C).astype(np.int32), 1)):
        r = bench.community_checks(off, col, w, C2, "cpu", chunk_arcs=3)
        labels = oracle.split(off, col, C2, np.ones(L * k, np.uint8))
        assert r["components"] == len(np.unique(labels)) == len(np.unique(C2)) + extra
        assert r["connected"] == (extra == 0)
        q_or, _ = oracle.modularity(off, col, w, C2)
        assert abs(r["q"] - q_or) <= 1e-12


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys and the config of the main line."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--scale", "15"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["host_cores"] >= 1
    assert "R-MAT scale 15" in d["cpu_baseline"]["sample"] and "batches 2..3" in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--scale", "15"]
        defaults = bench.parse()
    finally:
        sys.argv = argv
    assert d["config"] == bench.main_config(defaults, 1)


def test_oracle_baseline_runs_in_a_spawned_process():
    """The main line's oracle timing: a spawned process on the same graph and
    batch stream as the GPU arm; the result names the sample it timed."""
    import argparse

    args = argparse.Namespace(scale=13, batch_frac=1e-3, warmup=2, steps=3)
    cb = bench.OracleBaseline(args, warmup=1, steps=2, budget_s=60).result(timeout=600)
    assert "error" not in cb, cb
    assert cb["value"] > 0 and cb["unit"] == "edges/s" and cb["cores"] == 1
    assert "R-MAT scale 13" in cb["sample"] and "batches 2..3" in cb["sample"]
    # the same numbers of batches as the GPU arm draws, hence the same batches
    assert bench.stream_batches(args) == 2 + 2 * 3 + 2 * (bench.ND_DS_STEPS + 1) + bench.ISO_STEPS


def test_ncu_summary_reads_the_capture_csv(tmp_path):
    """--ncu-summary: per-kernel launches, time and DRAM bytes from an ncu
    CSV (units normalised), the local-moving launches (template kind 0) per
    launch, and the source hashes the roofline's traffic is keyed to."""
    import json

    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",'
           '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    rows = []
    launches = [("void <unnamed>::k_decide_block<int, 0>(<unnamed>::Args)", 10.0, 2.0, 0.5),
                ("void <unnamed>::k_decide_block<long, 0>(<unnamed>::Args)", 20.0, 4.0, 1.5),
                ("void <unnamed>::k_decide_block<int, 1>(<unnamed>::Args)", 5.0, 1.0, 0.0),
                ("void <unnamed>::k_expand(const leiden_edge *, long)", 3.0, 0.25, 0.25)]
    for i, (name, us, rd, wr) in enumerate(launches):
        for metric, unit, val in (("dram__bytes_read.sum", "Mbyte", rd), ("dram__bytes_write.sum", "Mbyte", wr),
                                  ("gpu__time_duration.sum", "usecond", us)):
            rows.append(f'"{i}","1","python","h","{name}","1","7","(128, 1, 1)","(1064, 1, 1)","0","10.3",'
                        f'"Command line profiler metrics","{metric}","{unit}","{val:,}"')
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text("==PROF== Connected\n" + hdr + "\n" + "\n".join(rows) + "\n")
    out = bench.ncu_summary(str(csv_path), "ncu ...", out_json=str(tmp_path / "t.json"),
                            out_md=str(tmp_path / "t.md"))
    lm = out["local_moving"]["k_decide_block"]
    assert lm["launches"] == 2
    assert lm["traffic_bytes_per_launch"] == (2.5e6 + 5.5e6) / 2
    assert out["kernels"]["k_decide_block<int, 1>"]["launches"] == 1
    assert abs(sum(k["share"] for k in out["kernels"].values()) - 1) < 1e-12
    assert json.loads((tmp_path / "t.json").read_text())["source_sha256"]["move.cu"] == \
        bench.source_code_sha256(os.path.join(bench.CSRC, "move.cu"))
    assert "| k_expand | 1 |" in (tmp_path / "t.md").read_text()
