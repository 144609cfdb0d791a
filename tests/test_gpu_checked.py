"""The checked build (-DLEIDEN_CHECKED) on the GPU: its kernels test their
invariants (probes end within their tables, ids in range) and report a
failed test as a status.  On tiny and small cases it must give the oracle's
results bit for bit with every test passing, and a test failed on purpose
must come back to the host as its code.  The checked library runs in a
child process (a process loads one build of the library)."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

from paper_2410_15451_gb300 import leiden as L

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import oracle
from paper_2410_15451_gb300 import _build, leiden as L, synth
from tests.helpers import csr_from_edges
from tests.test_gpu_parity import hub_graph, long_rows_graph, _weighted

_build.build(checked=True)
assert L.library_path().endswith("_checked.so")
assert L.leiden_checked_build()
assert L.leiden_check_selftest() == 0x5e1f   # failed on purpose, read back
assert L.leiden_check_selftest() == 0x5e1f   # the word was cleared in between, and is set again
modes = [(L.LEIDEN_ND, oracle.ND), (L.LEIDEN_DS, oracle.DS), (L.LEIDEN_DF, oracle.DF)]
tri = csr_from_edges(4, [(0, 1), (1, 2), (0, 2)])
cases = [("triangle", synth.Graph(4, tri[0], tri[1], tri[2].astype(np.int32))), ("hubs", hub_graph()),
         ("long_rows", long_rows_graph()), ("weighted", _weighted(synth.planted_partition(3000, 15, 12, 0.3, 41)))]
for name, g in cases:
    for gm, om in modes:
        gpu = L.Leiden(g.n, g.off, g.col, g.w)
        ref = oracle.Oracle(g.n, g.off, g.col, g.w, schedule=oracle.SYNC)
        assert np.array_equal(gpu.static(), ref.static()), name
        if g.n > 10:
            d, i = synth.random_batch(g, 300, seed=17, w_hi=8 if name == "weighted" else 1)
        else:
            d, i = np.array([[0, 1, 1]], np.int32), np.array([[1, 3, 2]], np.int32)
        assert np.array_equal(gpu.update(d, i, gm), ref.update(d, i, om)), (name, gm)
        assert gpu.modularity() == ref.modularity()
        gpu.close()
print("checked build ok")
'''


def test_default_build_has_no_checks():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert not L.leiden_checked_build()
    assert L.leiden_check_selftest() == 0


def test_checked_build_matches_the_oracle_and_reports_a_failed_check():
    env = dict(os.environ, LEIDEN_GB300_CHECKED="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "checked build ok" in out.stdout
