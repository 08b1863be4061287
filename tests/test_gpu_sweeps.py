"""GPU parity across the sweeps that widen the tested range: path roughness
(fractional Brownian motion down to H = 0.005), dimension (d = 2 .. 8192) and
length (self-kernels up to 2^12 + 1 points, O(L) workspace).  Errors use the
Cauchy-Schwarz rule for cross kernels near zero (|dk| / sqrt(k(x,x) k(y,y)))."""
import math

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


def to_dev(*arrs):
    return [torch.from_numpy(a).to(dev()) for a in arrs]


def _order(dx, dy, tol=1e-12):
    # oracle truncation from the pair's own coupling: L C^{N+1}/((N+1)!)^2 <= tol
    c = dx @ dy.T
    C = max(np.abs(np.cumsum(c, 1)).max(), np.abs(np.cumsum(c, 0)).max(), 1e-30)
    L = max(len(dx), len(dy))
    N = 8
    while N < 56 and L * C ** (N + 1) / math.factorial(N + 1) ** 2 > tol:
        N += 1
    return N


def _errors(orc, xs, ys, k, idx):
    out = []
    for p in idx:
        dx = np.diff(xs[p].astype(np.float64), axis=0)
        dy = np.diff(ys[p].astype(np.float64), axis=0)
        r = orc.series_pair(dx, dy, N=_order(dx, dy))
        kx = orc.series_pair(dx, dx, N=_order(dx, dx))
        ky = orc.series_pair(dy, dy, N=_order(dy, dy))
        cs = math.sqrt(abs(kx)) * math.sqrt(abs(ky))
        out.append(abs(k[p] - r) / (cs if abs(r) < 1e-2 * cs else abs(r)))
    return np.array(out)


@pytest.mark.parametrize("hurst", [0.4, 0.2, 0.1, 0.05, 0.01, 0.005])
def test_roughness_sweep_fbm(S, orc, hurst):
    # 2-D fBM pairs of 51 points: as H falls the increments approach O(1) per
    # step, tiles get |c| ~ 1 and the plan refines.  FP64 meets 1e-5 on every
    # pair; FP32 meets it on the typical pair and stays within its rounding
    # level on the roughest.
    from paper_2502_20392_gb300 import synth
    n = 64
    X, lx = synth.fbm(n, 50, 2, hurst, seed=6000 + int(hurst * 1000))
    Y, ly = synth.fbm(n, 50, 2, hurst, seed=7000 + int(hurst * 1000))
    args = to_dev(X, lx, Y, ly)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    o64 = S.plan(S.OP_PAIRS, *args, tol=1e-5, opts=S.Opts(max_len=4096, flags=S.FLAG_FP64))
    k64 = S.pairs(*args, opts=o64).cpu().numpy()
    e64 = _errors(orc, xs, ys, k64, range(n))
    assert e64.max() < 1e-5, (hurst, o64, e64.max())
    o32 = S.plan(S.OP_PAIRS, *args, tol=1e-5, opts=S.Opts(max_len=4096))
    k32 = S.pairs(*args, opts=o32).cpu().numpy()
    e32 = _errors(orc, xs, ys, k32, range(n))
    assert np.median(e32) < 1e-5 and e32.max() < 1e-3, (hurst, o32, np.median(e32), e32.max())


@pytest.mark.parametrize("d", [2, 17, 64, 1000, 8192])
def test_dimension_sweep(S, orc, d):
    # register kernel (d <= 16) and two-phase kernel (d > 16) up to d = 8192;
    # Brownian increments N(0, 1/L) per coordinate, so |c| grows like sqrt(d)/L
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(6, 40, 130, d, 0.5, 1.5, seed=8100 + d)
    args = to_dev(X, lx, Y, ly)
    o = S.plan(S.OP_PAIRS, *args, tol=1e-6, opts=S.Opts(max_len=20000))
    k = S.pairs(*args, opts=o).cpu().numpy()
    e = _errors(orc, synth.split(X, lx), synth.split(Y, ly), k, range(6))
    assert e.max() < 1e-5, (d, o, e)


@pytest.mark.parametrize("k", [6, 8, 10, 12])
def test_length_sweep_self_kernel(S, orc, k):
    # 2-D Brownian self-kernels k(x, x) of 2^k + 1 points
    from paper_2502_20392_gb300 import synth
    n = 2 ** k
    pts, lens = synth.brownian(2, n, 2, 1.0, seed=9000 + k)
    X, L = to_dev(pts, lens)
    o = S.plan(S.OP_GRAM, X, L, None, None, tol=1e-6, opts=S.Opts(max_len=n + 1))
    G = S.gram(X, L, opts=o).cpu().numpy()
    paths = synth.split(pts, lens)
    for p in range(2):
        dx = np.diff(paths[p].astype(np.float64), axis=0)
        r = orc.series_pair(dx, dx, N=_order(dx, dx))
        assert abs(G[p, p] - r) / r < 1e-5, (k, p, G[p, p], r)


def test_workspace_is_linear_in_length(S):
    # O(L) device memory for one pair: doubling the swept length at most
    # doubles the workspace (plus a constant)
    sizes = [S.workspace_size(S.OP_PAIRS, 1, 1, 8, S.Opts(max_len=L, flags=S.FLAG_PAIR_MAJOR))
             for L in (2 ** 16, 2 ** 17, 2 ** 18, 2 ** 19)]
    for a, b in zip(sizes, sizes[1:]):
        assert b <= 2 * a + (1 << 20), sizes
