"""The tensor-core increment Gram (d > 16, FP32 solve): exact 8-bit digit
products accumulated on tcgen05, coefficients carried as float-float pairs
into the FP32 sweep.  Parity against the FP64 oracle on ragged pairs (strips
padded to blocks of 128 rows, swept lengths that are not multiples of the
32-column chunks, one-point paths, refined rough paths, points and increments
inputs), agreement with the FP32 FMA micro-GEMM path (SIGK_FLAG_NO_TENSOR),
and the Gram's mirror and full forms."""
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


def to_dev(*a):
    return [torch.from_numpy(v).to(dev()) for v in a]


def incs(pts, lens):
    from paper_2502_20392_gb300 import synth
    return [np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens)]


def rel_err(k, ref, kxx, kyy):
    # plain relative error, or on the Cauchy-Schwarz scale for near-zero
    # cross kernels
    scale = np.sqrt(np.abs(kxx * kyy))
    den = np.where(np.abs(ref) < 1e-2 * scale, scale, np.abs(ref))
    return np.abs(k - ref) / den


def _order(dx, dy, tol=1e-13):
    # oracle truncation from the pair's own coupling: L C^{N+1}/((N+1)!)^2 <= tol
    if len(dx) == 0 or len(dy) == 0:
        return 8
    c = dx @ dy.T
    C = max(np.abs(np.cumsum(c, 1)).max(), np.abs(np.cumsum(c, 0)).max(), 1e-30)
    L = max(len(dx), len(dy))
    N = 8
    while N < 60 and L * C ** (N + 1) / math.factorial(N + 1) ** 2 > tol:
        N += 1
    return N


def oracle3(orc, ix, iy):
    """k(x_p, y_p), k(x_p, x_p), k(y_p, y_p) with per-pair coupling orders."""
    f = lambda a, b: orc.series_pair(a, b, N=_order(a, b))
    return (np.array([f(a, b) for a, b in zip(ix, iy)]), np.array([f(a, a) for a in ix]),
            np.array([f(b, b) for b in iy]))


def _case(d, seed, s_hi=1.0):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(7, 40, 300, d, 0.5, s_hi, seed=seed)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    xs[2] = xs[2][:1]                                     # a one-point path: k = 1
    ys[4] = synth.brownian(1, 333, d, 1.0, seed=seed + 1)[0]  # 333 columns: ragged last chunk
    X, lx = synth.pack(xs)
    Y, ly = synth.pack(ys)
    return X, lx, Y, ly


@pytest.mark.parametrize("d,seed", [(17, 310), (64, 311), (256, 312), (1000, 313)])
def test_tensor_core_pairs_match_oracle(S, orc, d, seed):
    X, lx, Y, ly = _case(d, seed)
    ix, iy = incs(X, lx), incs(Y, ly)
    ref, kxx, kyy = oracle3(orc, ix, iy)
    a = to_dev(X, lx, Y, ly)
    o = S.plan(S.OP_PAIRS, *a, tol=1e-7, opts=S.Opts(max_len=20000))
    k = S.pairs(*a, opts=o).cpu().numpy()
    assert k[2] == 1.0
    e = rel_err(k, ref, kxx, kyy)
    assert e.max() < 2e-6, (d, o, e)
    # the FMA micro-GEMM path (FP32 coefficients) agrees to its own rounding
    o2 = S.Opts(order=o.order, rings=o.rings, refine_c=o.refine_c, max_len=o.max_len,
                flags=S.FLAG_NO_TENSOR)
    k2 = S.pairs(*a, opts=o2).cpu().numpy()
    assert rel_err(k2, ref, kxx, kyy).max() < 1e-5


def test_tensor_core_refined_increments(S, orc):
    # rough short paths (sigma up to 4, d = 256) need refinement; increments
    # input; refined rows take their digits from the segment with the
    # exponent lowered by log2 of the refinement factor
    X, lx, Y, ly = _case(256, 314, s_hi=3.0)
    ix, iy = incs(X, lx), incs(Y, ly)
    IX = [v.astype(np.float32) for v in ix]
    IY = [v.astype(np.float32) for v in iy]
    from paper_2502_20392_gb300 import synth
    PX, lpx = synth.pack(IX)
    PY, lpy = synth.pack(IY)
    ix = [v.astype(np.float64) for v in IX]
    iy = [v.astype(np.float64) for v in IY]
    ref, kxx, kyy = oracle3(orc, ix, iy)
    a = to_dev(PX, lpx, PY, lpy)
    o = S.plan(S.OP_PAIRS, *a, tol=1e-7, opts=S.Opts(max_len=20000, flags=S.FLAG_INCREMENTS))
    assert o.refine_c > 0
    k = S.pairs(*a, opts=o).cpu().numpy()
    e = rel_err(k, ref, kxx, kyy)
    # rough pairs (refined tiles up to |c| = 1): the ragged d = 256 workload's
    # tolerance
    assert e.max() < 1e-5, (o, e)


def test_tensor_core_gram_mirror_and_full(S, orc):
    from paper_2502_20392_gb300 import synth
    # common time step 1/300 (a short path is a short piece of Brownian
    # motion, so no single tile carries |c| ~ d)
    segs = np.array([100, 37, 260, 64, 129, 1])
    pts, lens = synth.brownian(6, segs, 96, 0.5 * np.sqrt(segs / 300), seed=315)
    X, L = to_dev(pts, lens)
    o = S.Opts(order=12, rings=8, max_len=300)
    G = S.gram(X, L, opts=o).cpu().numpy()
    Gf = S.gram(X, L, opts=S.Opts(order=12, rings=8, max_len=300, flags=S.FLAG_GRAM_FULL)).cpu().numpy()
    np.testing.assert_array_equal(G, G.T)
    np.testing.assert_allclose(Gf, G, rtol=2e-6)
    zs = incs(pts, lens)
    ref = orc.series_gram(zs, N=40)
    dg = np.sqrt(np.abs(np.diag(ref)))
    e = np.abs(G - ref) / np.maximum(np.abs(ref), 1e-2 * dg[:, None] * dg[None, :])
    assert e.max() < 1e-5, e.max()


def test_adaptive_ring_count(S, orc):
    # ring_tol (tensor-core path): each warp step keeps only the rings its
    # tiles need (first dropped ring |c|^(n+1)/((n+1)!)^2 <= ring_tol); the
    # result stays within the tolerance, every tile is counted once in the
    # ring histogram, and the smooth pairs use fewer rings than the fixed count
    from paper_2502_20392_gb300 import synth
    X, lx, Y, ly = _case(64, 316, s_hi=1.0)
    ix, iy = incs(X, lx), incs(Y, ly)
    ref, kxx, kyy = oracle3(orc, ix, iy)
    a = to_dev(X, lx, Y, ly)
    ws = S.Workspace()
    cells = max(len(u) * len(v) for u, v in zip(ix, iy))
    o = S.Opts(order=12, rings=8, max_len=20000, ring_tol=1e-8 / cells)
    k = S.pairs(*a, opts=o, ws=ws).cpu().numpy()
    e = rel_err(k, ref, kxx, kyy)
    assert e.max() < 2e-6, e
    h = S.ring_histogram(ws)
    tiles = sum(len(u) * len(v) for u, v in zip(ix, iy))
    assert sum(h) == tiles, (h, tiles)
    assert sum(h[:3]) > 0, h  # some warp steps kept fewer than 8 rings
    # the plan sets a ring tolerance and meets its own bound
    op = S.plan(S.OP_PAIRS, *a, tol=1e-6, opts=S.Opts(max_len=20000))
    assert op.ring_tol > 0
    k2 = S.pairs(*a, opts=op).cpu().numpy()
    assert rel_err(k2, ref, kxx, kyy).max() < 2e-6
