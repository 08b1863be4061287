"""The bounds-checked build (SIGK_DEBUG): every work item of every solver
kernel checks that the buffer regions it is about to touch lie inside their
buffers and records SIGK_ERR_BOUNDS instead of touching them.  The forward
parity tests and the small bench case run against that build in a child
process; any violation would surface as an error status there."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def debug_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20392_gb300 import build
    build.build()
    return build.build(debug=True)


def _env(lib):
    env = dict(os.environ)
    env["SIGK_LIB"] = lib
    return env


def test_forward_parity_under_bounds_checks(debug_lib):
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu",
                        os.path.join(ROOT, "tests", "test_gpu_forward.py")],
                       cwd=ROOT, env=_env(debug_lib), capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])


def test_small_bench_case_under_bounds_checks(debug_lib):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--case", "small", "--steps", "1",
                        "--warmup", "1", "--no-cpu-baseline"],
                       cwd=ROOT, env=_env(debug_lib), capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["value"] > 0 and line["fwd_bwd"]["value"] > 0
