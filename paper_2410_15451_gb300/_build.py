"""Build of libleiden_gb300.so: nvcc for sm_103a, one process per .cu file,
objects under _build/, the shared library next to this file.  build(checked=True)
makes the checked variant libleiden_gb300_checked.so (-DLEIDEN_CHECKED: the
kernels test their invariants and report a failed test as a status), with its
objects under _build/checked/."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libleiden_gb300.so")
LIB_PATH_CHECKED = os.path.join(HERE, "libleiden_gb300_checked.so")
SOURCES = ["prims.cu", "batch.cu", "move.cu", "phases.cu", "track.cu", "api.cu", "noalloc.cu", "server.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "leiden_gb300.h"))
    return files


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_path = LIB_PATH_CHECKED if checked else LIB_PATH
    out_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    newest = max(os.path.getmtime(f) for f in _inputs())
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [NVCC, *ARCH, *FLAGS, *(["-DLEIDEN_CHECKED"] if checked else []), "-c", os.path.join(CSRC, src),
               "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib_path + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread"])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
