"""CPU checks of the synthetic input generators (no method arithmetic)."""
import numpy as np
import pytest

from paper_2502_20392_gb300 import synth


@pytest.mark.parametrize("hurst", [0.5, 0.4, 0.05, 0.7])
def test_fbm_increment_autocovariance(hurst):
    # Davies-Harte is exact in distribution: the normalised increments are
    # fractional Gaussian noise with gamma(k) = (|k+1|^2H - 2|k|^2H + |k-1|^2H)/2
    n, N = 64, 4000
    pts, lens = synth.fbm(N, n, 1, hurst, seed=11)
    assert pts.dtype == np.float32 and (lens == n + 1).all()
    inc = np.diff(pts.reshape(N, n + 1).astype(np.float64), axis=1) * n ** hurst
    emp = np.array([np.mean(inc[:, :n - k] * inc[:, k:]) for k in range(4)])
    ref = synth.fgn_autocov(4, hurst)
    # standard error of a lag-k mean over N*(n-k) correlated products is ~1/sqrt(N*n)
    np.testing.assert_allclose(emp, ref, atol=6.0 / np.sqrt(N * n))
    if hurst == 0.5:
        np.testing.assert_allclose(ref, [1.0, 0.0, 0.0, 0.0], atol=1e-15)


def test_fbm_scaling_and_independent_coordinates():
    n, N = 50, 3000
    pts, _ = synth.fbm(N, n, 2, 0.1, seed=12)
    inc = np.diff(pts.reshape(N, n + 1, 2).astype(np.float64), axis=1)
    var = inc.var(axis=(0, 1))
    np.testing.assert_allclose(var, n ** (-0.2), rtol=0.05)
    corr = np.mean(inc[..., 0] * inc[..., 1]) / np.sqrt(var[0] * var[1])
    assert abs(corr) < 0.03
