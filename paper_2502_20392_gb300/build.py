"""Builds libsigk.so in-tree (paper_2502_20392_gb300/_build/) with nvcc for
sm_103a only.  One translation unit per (edge degree P, ring count NR) is
compiled in parallel, then everything is linked into one shared library with
a C ABI (include/sigk.h).

build(debug=True) builds the same library with -DSIGK_DEBUG into
paper_2502_20392_gb300/_build_debug/: every work item checks that the buffer
regions it is about to touch lie inside their buffers and, if not, records
SIGK_ERR_BOUNDS (with the check site, offset and limit) instead of touching
them.  Load it with sigk.load(path) or the SIGK_LIB environment variable."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsigk.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libsigk.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ORDERS = (4, 6, 8, 10, 12, 14, 16)
RINGS = (2, 4, 6, 8)
ODD_RINGS = (3, 5, 7)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _sources():
    files = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")))
    files += ["../../include/sigk.h"]
    return [os.path.normpath(os.path.join(CSRC, f)) for f in files]


def _digest(extra=()) -> str:
    """Hash of the sources and flags, independent of where the repository
    lives (paths relative to its root), so a figure recorded for one build
    can be matched on another machine."""
    root = os.path.dirname(HERE)
    h = hashlib.sha256()
    for f in _sources():
        with open(f, "rb") as fh:
            h.update(os.path.relpath(f, root).encode() + b"\0" + fh.read())
    flags = [os.path.relpath(x, root) if x == INCLUDE else x for x in ARCH + FLAGS + list(extra)]
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def _units():
    units = [("sigk_capi", os.path.join(CSRC, "sigk_capi.cu"), []),
             ("sigk_tune", os.path.join(CSRC, "sigk_tune.cu"), [])]
    for P in ORDERS:
        for NR in RINGS:
            if NR <= P:
                units.append((f"sigk_fwd_P{P}_R{NR}", os.path.join(CSRC, "sigk_fwd_inst.cu"),
                              [f"-DSIGK_P={P}", f"-DSIGK_NR={NR}"]))
        # odd ring counts serve the FP32 solvers only, which launch with the
        # order clamped to twice the rings
        for NR in ODD_RINGS:
            if NR <= P <= 2 * NR:
                units.append((f"sigk_fwd_P{P}_R{NR}", os.path.join(CSRC, "sigk_fwd_inst.cu"),
                              [f"-DSIGK_P={P}", f"-DSIGK_NR={NR}"]))
    for f in sorted(os.listdir(CSRC)):
        if f.endswith("_inst2.cu"):
            units.append((f[:-3], os.path.join(CSRC, f), []))
    return units


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    dflags = ["-DSIGK_DEBUG"] if debug else []
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "libsigk.sha256")
    dig = _digest(dflags)
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return lib
    units = _units()

    def compile_one(u):
        name, src, extra = u
        obj = os.path.join(bdir, name + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *dflags, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    workers = min(len(units), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig)
    return lib


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force=True), f"{time.time() - t:.1f}s")
