"""Host-side checks of the C-ABI that need no GPU: the shared library builds
for sm_103a, loads, and exports every function declared in include/sigk.h."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_20392_gb300 import build, sigk
    build.build()
    return sigk.load()


def test_exports_every_declared_symbol(lib):
    from paper_2502_20392_gb300 import sigk
    names = sigk.exported_functions()
    assert {"sigk_pairs", "sigk_gram", "sigk_mmd", "sigk_workspace_size"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", sigk._LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_version_and_errors_without_gpu(lib):
    from paper_2502_20392_gb300 import sigk
    assert b"sm_103a" in lib.sigk_version()
    # argument validation happens on the host before any CUDA call
    o = sigk.Opts(order=99).c()
    assert lib.sigk_workspace_size(0, 4, 4, 4, ctypes.byref(o)) == 0
    st = lib.sigk_pairs(None, None, None, None, 3, 4, None, None, 0, None, None)
    assert st == -1  # SIGK_ERR_ARG: null output
    assert b"NULL" in lib.sigk_last_error() or b"null" in lib.sigk_last_error()


def test_training_calls_validate_without_gpu(lib):
    # the split training entry points reject bad arguments on the host
    from paper_2502_20392_gb300 import sigk
    o = sigk.Opts().c()
    assert lib.sigk_adjoint(7, 4, 4, 4, None, None, None, None, 0, None, ctypes.byref(o)) == -1
    assert lib.sigk_adjoint(0, 4, 4, 4, None, None, None, None, 0, None, ctypes.byref(o)) == -1
    assert b"grad_out" in lib.sigk_last_error()
    assert lib.sigk_forward_train(9, None, None, 4, None, None, 4, 4, None, None, 0, None,
                                  ctypes.byref(o)) == -1
    # a Gram training forward needs X
    assert lib.sigk_forward_train(1, None, None, 4, None, None, 0, 4, None, None, 0, None,
                                  ctypes.byref(o)) == -1
    bad = sigk.Opts(order=99).c()
    assert lib.sigk_backward_workspace_size(1, 4, 0, 4, ctypes.byref(bad)) == 0


def test_no_cpu_fallback_in_product_path():
    # the product package must not import the oracle
    pkg = os.path.join(ROOT, "paper_2502_20392_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_wait_budget_is_validated_without_gpu(lib):
    # the bounded-wait budget must lie in 1..600000 ms (0 selects 4000 ms);
    # out-of-range budgets are rejected on the host before any CUDA call
    from paper_2502_20392_gb300 import sigk
    for bad in (-1, 600001):
        o = sigk.Opts(wait_ms=bad).c()
        assert lib.sigk_workspace_size(0, 4, 4, 4, ctypes.byref(o)) == 0
        nz = ctypes.c_void_p(256)  # never dereferenced: the options are checked first
        st = lib.sigk_pairs(nz, nz, nz, nz, 3, 4, nz, nz, 1 << 20, None, ctypes.byref(o))
        assert st == -1 and b"sigk_opts" in lib.sigk_last_error()


def test_tuning_cache_without_gpu(lib, tmp_path):
    # shape-class keys and the cache's lookup, merge and file round trip are
    # host code (no GPU)
    from paper_2502_20392_gb300 import sigk
    sigk.tune_cache_clear()
    o = sigk.Opts(order=12, rings=6, max_len=1000, flags=sigk.FLAG_INCREMENTS)
    k1 = sigk.tune_key(sigk.OP_GRAM, 64, 0, 16, o)
    # the swept-length bound is bucketed by powers of two; the tuned flags
    # and the grid are not part of the class, the problem flags are
    assert k1 == sigk.tune_key(sigk.OP_GRAM, 64, 0, 16, sigk.Opts(order=12, rings=6, max_len=1024,
                                                                   flags=sigk.FLAG_INCREMENTS | sigk.FLAG_PAIR_MAJOR,
                                                                   grid_ctas=300))
    assert k1 != sigk.tune_key(sigk.OP_GRAM, 64, 0, 16, sigk.Opts(order=12, rings=6, max_len=1025,
                                                                   flags=sigk.FLAG_INCREMENTS))
    assert k1 != sigk.tune_key(sigk.OP_GRAM, 64, 0, 16, sigk.Opts(order=12, rings=6, max_len=1000))
    assert k1 != sigk.tune_key(sigk.OP_PAIRS, 64, 64, 16, o)
    assert sigk.tune_cache_get(k1, o) is None
    sigk.tune_cache_put(k1, 456, sigk.FLAG_PAIR_MAJOR | sigk.FLAG_FP64, 3.25)
    got, ms = sigk.tune_cache_get(k1, o)
    # only the layout fields are merged: grid, schedule and Gram-path flags
    assert got.grid_ctas == 456 and got.flags == sigk.FLAG_INCREMENTS | sigk.FLAG_PAIR_MAJOR
    assert (got.order, got.rings, got.max_len) == (12, 6, 1000) and ms == 3.25
    k2 = sigk.tune_key(sigk.OP_PAIRS, 512, 512, 256, sigk.Opts(order=14, rings=6, max_len=8193))
    sigk.tune_cache_put(k2, 0, sigk.FLAG_NO_TENSOR, 1.5)
    path = str(tmp_path / "tune.txt")
    sigk.tune_cache_save(path)
    sigk.tune_cache_clear()
    assert sigk.tune_cache_size() == 0
    sigk.tune_cache_load(path)
    assert sigk.tune_cache_size() == 2
    got2, ms2 = sigk.tune_cache_get(k2, sigk.Opts(order=14, rings=6, max_len=8193))
    assert got2.flags == sigk.FLAG_NO_TENSOR and got2.grid_ctas == 0 and ms2 == 1.5
    with open(path, "a") as f:
        f.write("bad line\n")
    with pytest.raises(sigk.SigkError):
        sigk.tune_cache_load(path)
    sigk.tune_cache_clear()
