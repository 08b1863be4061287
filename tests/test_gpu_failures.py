"""Failure detection on the GPU, in forms that fault, trap or hang nothing:

* a bounded inter-warp wait that runs out: the test hook
  SIGK_FLAG_TEST_WITHHOLD_SEAM keeps the first work item from publishing its
  seam, so its consumer's wait (budget wait_ms) expires; the kernel records
  SIGK_ERR_TIMEOUT, every warp returns, the host reads the status, and the
  context stays usable for the next call;
* non-finite input data: the final value of the affected pair is not finite,
  the kernel records SIGK_ERR_NONFINITE, the other pairs are unaffected."""
import time

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


def dev():
    return torch.device("cuda:0")


def _pairs_case():
    from paper_2502_20392_gb300 import synth
    # pair 0 has x of 600 points (several strips: its strips hand seams on)
    (X, lx), (Y, ly) = synth.ragged_pairs(3, 40, 90, 4, 0.7, 1.2, seed=211)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    xs[0] = synth.brownian(1, 599, 4, 1.0, seed=212)[0]
    X, lx = synth.pack(xs)
    return X, lx, Y, ly, xs, ys


def test_bounded_wait_times_out_and_reports(S, orc):
    X, lx, Y, ly, xs, ys = _pairs_case()
    a = [torch.from_numpy(v).to(dev()) for v in (X, lx, Y, ly)]
    ws = S.Workspace()
    o = S.Opts(order=8, rings=4, max_len=128, wait_ms=200, flags=S.FLAG_TEST_WITHHOLD_SEAM)
    t0 = time.perf_counter()
    S.pairs(*a, opts=o, ws=ws, check=False)
    with pytest.raises(S.SigkError) as ei:
        S.sync_status(ws)
    assert ei.value.status == -6  # SIGK_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the status was read and cleared; the context and the workspace serve the
    # next call, whose results are right
    o2 = S.Opts(order=8, rings=4, max_len=128, wait_ms=200)
    k = S.pairs(*a, opts=o2, ws=ws).cpu().numpy()
    ref = orc.series_pairs([np.diff(x.astype(np.float64), axis=0) for x in xs],
                           [np.diff(y.astype(np.float64), axis=0) for y in ys])
    np.testing.assert_allclose(k, ref, rtol=1e-5)


def test_nonfinite_input_is_reported(S, orc):
    X, lx, Y, ly, xs, ys = _pairs_case()
    for bad in (np.nan, np.inf):
        Xb = X.copy()
        Xb[int(lx[0]) + 5, 2] = bad  # a point of pair 1's x
        a = [torch.from_numpy(v).to(dev()) for v in (Xb, lx, Y, ly)]
        ws = S.Workspace()
        k = S.pairs(*a, opts=S.Opts(order=8, rings=4, max_len=128), ws=ws, check=False)
        with pytest.raises(S.SigkError) as ei:
            S.sync_status(ws)
        assert ei.value.status == -3  # SIGK_ERR_NONFINITE
        k = k.cpu().numpy()
        assert not np.isfinite(k[1])
        ref = orc.series_pairs([np.diff(xs[p].astype(np.float64), axis=0) for p in (0, 2)],
                               [np.diff(ys[p].astype(np.float64), axis=0) for p in (0, 2)])
        np.testing.assert_allclose(k[[0, 2]], ref, rtol=1e-5)
