"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h (no GPU needed; no compute call is made)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_2410_15451_gb300 import _build
from paper_2410_15451_gb300 import leiden as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("leiden_") and name not in names:
                names.append(name)
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("leiden_create", "leiden_static", "leiden_update", "leiden_modularity", "leiden_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_match_the_paper(lib):
    p = L.leiden_default_params()
    assert p.tau == 1e-2 and p.tau_drop == 10.0 and p.tau_refine == 0.6
    assert p.max_iterations == 20 and p.max_passes == 10
    assert p.deterministic == 1 and p.classes == 4


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/leiden_gb300.h as a C
    compiler lays it out (gcc, host ABI)."""
    import subprocess
    import tempfile

    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"leiden_gb300.h\"\nint main(void) {\n"
    src += f'  printf("%zu\\n", sizeof({struct}));\n'
    for f in fields:
        src += f'  printf("%zu\\n", offsetof({struct}, {f}));\n'
    src += "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    return out[0], out[1:]


@pytest.mark.parametrize("struct,cls", [("leiden_params", "leiden_params"), ("leiden_stats", "leiden_stats"),
                                        ("leiden_tuning", "leiden_tuning"),
                                        ("leiden_server_stats", "leiden_server_stats")])
def test_struct_layouts_match_the_c_header(struct, cls):
    """The binding's ctypes structures have the header's size and field
    offsets (compiled with gcc)."""
    ct = getattr(L, cls)
    names = [f for f, _ in ct._fields_]
    size, offsets = _c_layout(struct, names)
    assert ctypes.sizeof(ct) == size
    assert [getattr(ct, f).offset for f in names] == offsets


def test_create_rejects_bad_input_without_touching_the_gpu(lib):
    import numpy as np

    off = np.array([0, 1, 1], np.int64)
    col = np.array([0], np.int32)  # self-loop
    with pytest.raises(L.LeidenError) as e:
        L.leiden_create(None, 2, off, col)
    assert e.value.status == L.LEIDEN_ERR_ARG
    assert "self-loop" in L.leiden_last_error(None)


def test_create_batched_rejects_bad_input_without_touching_the_gpu(lib):
    import numpy as np

    # two graphs of 2 vertices; an arc from graph 0 into graph 1
    off = np.array([0, 1, 2, 3, 4], np.int64)
    col = np.array([2, 0, 0, 2], np.int32)
    with pytest.raises(L.LeidenError) as e:
        L.leiden_create_batched(None, np.array([0, 2, 4], np.int64), off, col)
    assert e.value.status == L.LEIDEN_ERR_ARG
    assert "two graphs" in L.leiden_last_error(None)
    with pytest.raises(L.LeidenError) as e:  # an empty graph
        L.leiden_create_batched(None, np.array([0, 2, 2, 4], np.int64), off, col)
    assert e.value.status == L.LEIDEN_ERR_ARG
    p = L.leiden_default_params()
    p.deterministic = 0
    with pytest.raises(L.LeidenError) as e:  # batched handles run the snapshot schedule
        L.leiden_create_batched(p, np.array([0, 2, 4], np.int64), off, np.array([1, 0, 3, 2], np.int32))
    assert e.value.status == L.LEIDEN_ERR_ARG


def test_footprint_estimate_grows_with_the_graph(lib):
    import numpy as np

    small = L.leiden_footprint_bytes(1000, np.arange(0, 10 * 1001, 10, dtype=np.int64))
    big = L.leiden_footprint_bytes(100000, np.arange(0, 10 * 100001, 10, dtype=np.int64))
    assert 0 < small < big
    # at least the CSR with slack: 8 bytes per arc
    assert big > 8 * 10 * 100000
    assert L.load().leiden_footprint_bytes(None, 0, None) == -1


def test_default_tuning(lib):
    t = L.leiden_default_tuning()
    assert (t.tiny_max, t.warp_max, t.block_max, t.overlap) == (8, 128, 1024, 1)
    assert ctypes.sizeof(L.leiden_tuning) == 7 * 4
