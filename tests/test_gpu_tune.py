"""The autotuner (sigk_autotune): on two shape classes it picks a launch
layout that is never slower than the default one, its results equal the
default layout's (the layouts change the schedule, not the arithmetic), and
a later plan of the same class carries the tuned layout."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20392_gb300 import build, sigk
    build.build()
    sigk.load()
    return sigk


def _time(fn, reps=7):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    fn()
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


@pytest.mark.parametrize("shape", ["gram_d16", "pairs_d64"])
def test_tuned_layout_never_slower(S, shape):
    from paper_2502_20392_gb300 import synth
    dev = torch.device("cuda:0")
    S.tune_cache_clear()
    if shape == "gram_d16":
        pts, lens = synth.brownian(24, 700, 16, 1.0, seed=501)
        X, L = torch.from_numpy(pts).to(dev), torch.from_numpy(lens).to(dev)
        op, args = S.OP_GRAM, (X, L, None, None)
        o = S.Opts(order=8, rings=4, max_len=700)
        call = lambda oo: S.gram(X, L, opts=oo, check=False)
    else:
        (X, lx), (Y, ly) = synth.ragged_pairs(40, 200, 900, 64, 0.5, 1.0, seed=502)
        a = [torch.from_numpy(v).to(dev) for v in (X, lx, Y, ly)]
        op, args = S.OP_PAIRS, tuple(a)
        o = S.Opts(order=10, rings=6, max_len=900)
        call = lambda oo: S.pairs(*a, opts=oo, check=False)
    tuned, ms = S.autotune(op, *args, opts=o)
    assert ms > 0
    base = call(o).clone()
    got = call(tuned)
    torch.cuda.synchronize()
    assert torch.equal(base, got), (o, tuned)
    t_def = _time(lambda: call(o))
    t_tun = _time(lambda: call(tuned))
    assert t_tun <= 1.05 * t_def, (t_tun, t_def, tuned)
    # the cache now holds the class; a plan of it carries the layout
    assert S.tune_cache_size() == 1
    key = S.tune_key(op, len(args[1]), 0 if args[2] is None else len(args[3]), X.shape[1], o)
    assert S.tune_cache_get(key, o) is not None
    S.tune_cache_clear()
