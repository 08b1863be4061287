"""Host-side checks of bench.py: the flop model behind the roofline figures,
and the reference arm's JSON line (it runs the FP64 oracle on the host)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_flop_model():
    import bench
    # per-tile FP32 operations (FMA = 2) of the solver and of the adjoint
    # kept entries of the truncation 2m + k <= 2n + 1, m + k <= P, written out:
    # P = 8, n = 4: ring 1 offsets 0..7, ring 2 0..5, ring 3 0..3, ring 4 0..1,
    # each off-diagonal offset on both sides of the diagonal
    assert bench.kept_entries(8, 4, 4) == (1 + 2 * 7) + (1 + 2 * 5) + (1 + 2 * 3) + (1 + 2 * 1) == 36
    assert bench.kept_entries(12, 6, 6) == sum(1 + 2 * (13 - 2 * m) for m in range(1, 7)) == 78
    # no kept entry reaches a degree above 2n: a larger order adds nothing
    assert bench.kept_entries(16, 6, 6) == bench.kept_entries(12, 6, 6)
    assert bench.launch_order(16, 6) == 12 and bench.launch_order(8, 4) == 8
    # the square truncation (the whole (P+1)^2 matrix up to ring n) as a bound
    assert bench.kept_entries(8, 4, 4) < sum(2 * (8 - m) + 1 for m in range(1, 5)) == 48
    assert bench.tile_flops(8, 4, 16) == 2 * 3 + 2 * 4 + 4 * 36 + 2 * 8 + 28 + 2 * 16 == 234
    assert bench.tile_flops(12, 6, 16) == 2 * 5 + 2 * 6 + 4 * 78 + 2 * 12 + 28 + 2 * 16 == 418
    assert bench.adjoint_tile_flops(8, 4, 16, replay=False) == 480
    for P, nr, d in ((8, 4, 16), (12, 6, 4), (16, 8, 8)):
        # the replayed pass adds exactly one forward tile
        assert (bench.adjoint_tile_flops(P, nr, d) - bench.adjoint_tile_flops(P, nr, d, replay=False)
                == bench.tile_flops(P, nr, d))
    # rings beyond the order add nothing
    assert bench.tile_flops(4, 8, 4) == bench.tile_flops(4, 4, 4)


def test_useful_work_model():
    import bench
    # algorithmic FMAs per tile: d + sum_{m=1..n} (2(P - m) + 1) + 2P, written
    # out for the bench's two launches (P = 8, n = 4 and P = 16, n = 6, d = 16)
    assert bench.useful_tile_fma(8, 4, 16) == 16 + (15 + 13 + 11 + 9) + 16 == 80
    assert bench.useful_tile_fma(16, 6, 16) == 16 + (31 + 29 + 27 + 25 + 23 + 21) + 32 == 204
    assert bench.useful_tile_fma(12, 6, 16) == 16 + (23 + 21 + 19 + 17 + 15 + 13) + 24 == 148
    assert bench.useful_tile_flops(8, 4, 16) == 160
    assert bench.useful_tile_flops(8, 4, 16, adjoint=True) == 320
    # the executed count is never below the useful one
    for P, nr, d in ((4, 2, 4), (8, 4, 16), (16, 6, 16), (14, 6, 256)):
        assert bench.tile_flops(P, nr, d) >= bench.useful_tile_flops(P, nr, d)


def test_accuracy_sample_spans_the_gram():
    import bench
    idx = bench.sample_pairs(16, 11)
    assert len(set(idx)) == 16 and all(a <= b for a, b in idx)
    assert len({a for a, _ in idx}) > 4  # not one row of the Gram


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "config", "e2e", "cpu_baseline"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
