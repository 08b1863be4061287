"""GPU parity of the forward solver (through the C-ABI) against the FP64 oracle
and closed forms.  Sizes span several 128-row strips with ragged tails; the
tolerances are the per-workload relative tolerances (1e-6 for the 256-segment
pair, 1e-5 for Gram entries), with the Cauchy-Schwarz-scaled error
|dk| / sqrt(k(x,x) k(y,y)) used for near-zero cross entries."""
import math

import numpy as np
import pytest
from scipy.special import i0, j0

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


def incs(pts, lens):
    from paper_2502_20392_gb300 import synth
    return [np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens)]


def to_dev(pts, lens):
    return torch.from_numpy(pts).to(dev()), torch.from_numpy(lens).to(dev())


def rel_err(k, ref, kxx=None, kyy=None):
    e = np.abs(k - ref) / np.maximum(np.abs(ref), 1e-300)
    if kxx is not None:
        scale = np.sqrt(np.abs(kxx)) * np.sqrt(np.abs(kyy))  # no overflow for huge self-kernels
        cs = np.abs(k - ref) / scale
        small = np.abs(ref) < 1e-2 * scale
        e = np.where(small, np.minimum(e, cs), e)
    return e


def test_single_segment_closed_form(S):
    from paper_2502_20392_gb300 import synth
    cs = [-4.0, -0.5, 0.01, 0.5, 4.0, 0.0]
    (X, lx), (Y, ly) = synth.single_segment_pairs(cs)
    nr = 8
    k = S.pairs(*to_dev(X, lx), *to_dev(Y, ly), opts=S.Opts(order=16, rings=nr)).cpu().numpy()
    for kc, c in zip(k, cs):
        # one tile with nr Neumann rings is the Bessel partial sum up to c^nr/(nr!)^2
        terms = [c**m / math.factorial(m) ** 2 for m in range(nr + 1)]
        fp32 = 4e-7 * sum(abs(t) for t in terms)  # a few FP32 roundings of the largest terms
        assert abs(kc - sum(terms)) <= fp32, (c, kc, sum(terms))
        bessel = i0(2 * math.sqrt(c)) if c >= 0 else j0(2 * math.sqrt(-c))
        tail = abs(c) ** (nr + 1) / math.factorial(nr + 1) ** 2 * 1.01
        assert abs(kc - bessel) <= tail + fp32, (c, kc, bessel)


def test_pair_256_d4(S, orc):
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.workload_pair_256()
    dx, dy = incs(pts, lens)
    ref = orc.series_pair(dx, dy)
    X, L = to_dev(pts, lens)
    xs, ys = X[:257], X[257:]
    lx, ly = L[:1], L[1:]
    k = S.pairs(xs, lx, ys, ly, opts=S.Opts(order=8, rings=4)).cpu().numpy()[0]
    assert abs(k - ref) / abs(ref) < 1e-6, (k, ref)


# odd ring counts (3, 5, 7) are FP32-only instantiations at P <= 2 rings
@pytest.mark.parametrize("sigma,order,rings", [(1.0, 8, 4), (4.0, 16, 6), (2.0, 10, 5), (4.0, 14, 7)])
def test_gram_ragged_d16(S, orc, sigma, order, rings):
    from paper_2502_20392_gb300 import synth
    # common time step 1/300: a short path is a short piece of Brownian motion
    # (one 1-segment path would otherwise carry a tile with c ~ 16 sigma^2)
    segs = np.array([300, 129, 1, 257, 64, 200])
    pts, lens = synth.brownian(len(segs), segs, 16, sigma * np.sqrt(segs / 300), seed=77 + int(sigma))
    ref = orc.series_gram(incs(pts, lens), N=28)
    G = S.gram(*to_dev(pts, lens), opts=S.Opts(order=order, rings=rings)).cpu().numpy()
    dg = np.diag(ref)
    e = rel_err(G, ref, dg[:, None], dg[None, :])
    assert e.max() < 1e-5, e.max()
    np.testing.assert_array_equal(G, G.T)


def test_gram_full_matches_mirrored(S):
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(5, [90, 200, 33, 150, 7], 8, 1.0, seed=5)
    X, L = to_dev(pts, lens)
    G1 = S.gram(X, L, opts=S.Opts(order=8, rings=4)).cpu().numpy()
    G2 = S.gram(X, L, opts=S.Opts(order=8, rings=4, flags=S.FLAG_GRAM_FULL)).cpu().numpy()
    # both triangles computed independently (grid transposed for the lower one)
    np.testing.assert_allclose(G2, G2.T, rtol=1e-6)
    np.testing.assert_allclose(G1, G2, rtol=1e-6)


def test_gram_xy_and_pairs_ragged(S, orc):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(12, 1, 700, 8, 0.5, 2.0, seed=13)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    xs[3] = xs[3][:1]  # one-point paths: k = 1 with anything
    ys[5] = ys[5][:1]
    X, lx = synth.pack(xs)
    Y, ly = synth.pack(ys)
    ix, iy = incs(X, lx), incs(Y, ly)
    ref = orc.series_pairs(ix, iy, N=28)
    kxx = orc.series_pairs(ix, ix, N=28)
    kyy = orc.series_pairs(iy, iy, N=28)
    k = S.pairs(*to_dev(X, lx), *to_dev(Y, ly), opts=S.Opts(order=10, rings=5)).cpu().numpy()
    assert k[3] == 1.0 and k[5] == 1.0
    e = rel_err(k, ref, kxx, kyy)
    assert e.max() < 1e-5, e
    # cross Gram X vs Y: its diagonal is the pairwise result
    Gxy = S.gram(*to_dev(X, lx), *to_dev(Y, ly), opts=S.Opts(order=10, rings=5)).cpu().numpy()
    np.testing.assert_allclose(np.diag(Gxy), k, rtol=1e-6)


def test_increments_mode(S, orc):
    from paper_2502_20392_gb300 import synth
    inc, segs, u, tot = synth.collinear_increments(5000, 8, seed=3002, n_paths=2)
    X = torch.from_numpy(inc).to(dev())
    L = torch.from_numpy(segs).to(dev())
    o = S.Opts(order=4, rings=2, flags=S.FLAG_INCREMENTS, max_len=5000)
    k = S.pairs(X[:5000], L[:1], X[5000:], L[1:], opts=o).cpu().numpy()[0]
    s = float(u @ u) * tot[0] * tot[1]
    ref = i0(2 * math.sqrt(s))
    assert abs(k - ref) / ref < 1e-5, (k, ref)


def test_mmd_small(S, orc):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.workload_mmd_2048(seed=5001, n_paths=5, n_seg=150, d=8)
    ref = orc.mmd2(incs(X, lx), incs(Y, ly), N=24)
    v = S.mmd(*to_dev(X, lx), *to_dev(Y, ly), opts=S.Opts(order=8, rings=4)).cpu().numpy()[0]
    Kxx = orc.series_gram(incs(X, lx))
    scale = np.abs(Kxx).max()
    assert abs(v - ref) <= 1e-5 * max(abs(ref), scale * 1e-2), (v, ref)


@pytest.mark.parametrize("sigma", [1.0, 3.0])
def test_plan_meets_tolerance(S, orc, sigma):
    # sigk_plan picks (order, rings) from device statistics of the increments;
    # the planned launch must meet the requested tolerance against the oracle
    from paper_2502_20392_gb300 import synth
    segs = np.array([300, 211, 257, 180, 299, 64])
    pts, lens = synth.brownian(len(segs), segs, 8, sigma * np.sqrt(segs / 300), seed=123)
    X, L = to_dev(pts, lens)
    tols = (1e-4, 1e-6)
    plans = [S.plan(S.OP_GRAM, X, L, tol=t) for t in tols]
    assert plans[1].order >= plans[0].order and plans[1].rings >= plans[0].rings
    ref = orc.series_gram(incs(pts, lens), N=28)
    dg = np.diag(ref)
    for t, o in zip(tols, plans):
        G = S.gram(X, L, opts=o).cpu().numpy()
        e = rel_err(G, ref, dg[:, None], dg[None, :])
        assert e.max() < max(t, 2e-6), (t, o, e.max())


def test_plan_reports_unreachable_tolerance(S):
    # a tolerance below what order 16 can certify even at the finest
    # refinement: SIGK_ERR_ACCURACY, with the finest plan still returned
    import warnings
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(2, [12, 9], 3, 3.0, seed=31)
    X, L = to_dev(pts, lens)
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        o = S.plan(S.OP_GRAM, X, L, tol=1e-300)
    assert any(issubclass(x.category, RuntimeWarning) for x in w)
    assert o.order == 16 and 0.0 < o.refine_c < 1.0
    assert b"a-priori" in S.load().sigk_last_error()
    # a reachable tolerance on the same paths plans without the warning
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        S.plan(S.OP_GRAM, X, L, tol=1e-4)
    assert not any("sigk.plan" in str(x.message) for x in w)


def test_cuda_graph_capture_and_replay(S, orc):
    # the C-ABI launches no host synchronisation, allocation or copy, so a call
    # with a preallocated workspace can be captured and replayed on new inputs
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(6, 200, 8, 1.0, seed=9)
    X, L = to_dev(pts, lens)
    o = S.Opts(order=8, rings=4, max_len=200)
    ws = S.Workspace()
    ws.get(S.workspace_size(S.OP_GRAM, 6, 0, 8, o), X.device)
    G = torch.empty((6, 6), dtype=torch.float64, device=X.device)
    S.gram(X, L, opts=o, out=G, ws=ws)  # warm-up outside capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            S.gram(X, L, opts=o, out=G, ws=ws, check=False)
    torch.cuda.current_stream().wait_stream(s)
    pts2, _ = synth.brownian(6, 200, 8, 1.0, seed=10)
    X.copy_(torch.from_numpy(pts2))
    G.zero_()
    g.replay()
    torch.cuda.synchronize()
    S.sync_status(ws)
    eager = S.gram(X, L, opts=o).cpu().numpy()
    np.testing.assert_array_equal(G.cpu().numpy(), eager)
    ref = orc.series_gram(incs(pts2, lens))
    np.testing.assert_allclose(G.cpu().numpy(), ref, rtol=1e-5)


def test_refinement_resolves_large_tiles(S, orc):
    # a one-segment path in R^16 with unit increments gives tiles with
    # |c| ~ 16 that orders <= 16 and rings <= 8 cannot resolve; refinement
    # (every segment split into s equal collinear pieces, which leaves k
    # unchanged) brings every tile below |c| = refine_c
    from paper_2502_20392_gb300 import synth
    segs = [300, 129, 1, 257, 64, 200]
    pts, lens = synth.brownian(len(segs), segs, 16, 1.0, seed=78)
    ref = orc.series_gram(incs(pts, lens), N=30)
    X, L = to_dev(pts, lens)
    o = S.Opts(order=12, rings=6, refine_c=1.0, max_len=20000)
    G = S.gram(X, L, opts=o).cpu().numpy()
    dg = np.diag(ref)
    e = rel_err(G, ref, dg[:, None], dg[None, :])
    assert e.max() < 1e-5, e.max()
    # the planner turns refinement on by itself for this input
    op = S.plan(S.OP_GRAM, X, L, tol=1e-5)
    assert op.refine_c > 0
    G2 = S.gram(X, L, opts=op).cpu().numpy()
    assert rel_err(G2, ref, dg[:, None], dg[None, :]).max() < 1e-5


def test_large_dimension_ragged_pairs(S, orc):
    # d = 256 (the two-phase kernel): ragged pairs, per-path scales
    # sigma_p ~ U(0.5, 4) as in the ragged d=256 workload, with refinement for
    # the rough short paths
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(6, 20, 300, 256, 0.5, 4.0, seed=4001)
    ix, iy = incs(X, lx), incs(Y, ly)
    ref = orc.series_pairs(ix, iy, N=28)
    kxx = orc.series_pairs(ix, ix, N=28)
    kyy = orc.series_pairs(iy, iy, N=28)
    o = S.plan(S.OP_PAIRS, *to_dev(X, lx), *to_dev(Y, ly), tol=1e-6, opts=S.Opts(max_len=20000))
    k = S.pairs(*to_dev(X, lx), *to_dev(Y, ly), opts=o).cpu().numpy()
    e = rel_err(k, ref, kxx, kyy)
    assert e.max() < 1e-5, (o, e)


def test_large_dimension_kernel_matches_register_kernel(S):
    # appending a zero coordinate leaves every tile coefficient unchanged, so
    # the d=17 (two-phase) kernel must reproduce the d=16 (register) kernel
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(5, [100, 37, 260, 64, 129], 16, 1.0, seed=44)
    pts17 = np.concatenate([pts, np.zeros((pts.shape[0], 1), np.float32)], 1)
    o = S.Opts(order=8, rings=4, max_len=300)
    G16 = S.gram(*to_dev(pts, lens), opts=o).cpu().numpy()
    G17 = S.gram(*to_dev(np.ascontiguousarray(pts17), lens), opts=o).cpu().numpy()
    np.testing.assert_allclose(G17, G16, rtol=2e-6)


@pytest.mark.parametrize("d", [4, 256])
def test_fp64_solver_matches_oracle(S, orc, d):
    # FLAG_FP64: point differences, contraction, refinement scaling and tile
    # map in double.  Against the FP64 oracle the gap is double rounding plus
    # the truncation the plan allows (tol 1e-11), on ragged pairs
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(6, 20, 300, d, 0.5, 2.0, seed=4101 + d)
    ix, iy = incs(X, lx), incs(Y, ly)
    ref = orc.series_pairs(ix, iy, N=30)
    kxx = orc.series_pairs(ix, ix, N=30)
    kyy = orc.series_pairs(iy, iy, N=30)
    o = S.plan(S.OP_PAIRS, *to_dev(X, lx), *to_dev(Y, ly), tol=1e-11,
               opts=S.Opts(max_len=20000, flags=S.FLAG_FP64))
    assert o.flags & S.FLAG_FP64
    k = S.pairs(*to_dev(X, lx), *to_dev(Y, ly), opts=o).cpu().numpy()
    e = rel_err(k, ref, kxx, kyy)
    assert e.max() < 1e-9, (o, e)
    # refinement factors up to 4 (the largest increment / sqrt(refine_c) is
    # 2.5, rounded up to a power of two)
    mx = max(np.linalg.norm(v, axis=1).max() for v in ix + iy)
    o3 = S.Opts(order=16, rings=8, refine_c=float((mx / 2.5) ** 2), max_len=20000,
                flags=S.FLAG_FP64)
    k3 = S.pairs(*to_dev(X, lx), *to_dev(Y, ly), opts=o3).cpu().numpy()
    e3 = rel_err(k3, ref, kxx, kyy)
    assert e3.max() < 1e-9, (o3, e3)


def test_fp64_rejected_by_backward(S):
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(2, [8, 9], 4, 1.0, seed=3)
    Xd, ld = to_dev(pts, lens)
    with pytest.raises(S.SigkError):
        S.backward(S.OP_GRAM, Xd, ld, None, None, torch.ones((2, 2), dtype=torch.float64),
                   S.Opts(flags=S.FLAG_FP64, max_len=16))


def test_schedules_agree_bitwise(S):
    # strip-major (default) and pair-major schedules run the same arithmetic
    # per tile: the results must be identical, on ragged lengths with a
    # one-point path, long row paths (many strips) and refinement
    from paper_2502_20392_gb300 import synth
    segs = [700, 1, 33, 257, 1200, 64, 5, 400]
    pts, lens = synth.brownian(len(segs), segs, 8, 1.5, seed=90)
    X, L = to_dev(pts, lens)
    for o in (S.Opts(order=8, rings=4, max_len=1300), S.Opts(order=12, rings=6, refine_c=0.5, max_len=8000)):
        G1 = S.gram(X, L, opts=o).cpu().numpy()
        o2 = S.Opts(order=o.order, rings=o.rings, refine_c=o.refine_c, max_len=o.max_len,
                    flags=S.FLAG_PAIR_MAJOR)
        G2 = S.gram(X, L, opts=o2).cpu().numpy()
        assert np.array_equal(G1, G2)
    # even strip counts (the strip-major schedule) against pair-major
    pts, lens = synth.brownian(12, 300, 8, 1.5, seed=92)
    X, L = to_dev(pts, lens)
    o = S.Opts(order=8, rings=4, max_len=320)
    G1 = S.gram(X, L, opts=o).cpu().numpy()
    G2 = S.gram(X, L, opts=S.Opts(order=8, rings=4, max_len=320, flags=S.FLAG_PAIR_MAJOR)).cpu().numpy()
    assert np.array_equal(G1, G2)
    (Xp, lxp), (Yp, lyp) = synth.ragged_pairs(9, 1, 600, 40, 0.5, 2.0, seed=91)
    o = S.Opts(order=10, rings=5, max_len=700)
    k1 = S.pairs(*to_dev(Xp, lxp), *to_dev(Yp, lyp), opts=o).cpu().numpy()
    o2 = S.Opts(order=10, rings=5, max_len=700, flags=S.FLAG_PAIR_MAJOR)
    k2 = S.pairs(*to_dev(Xp, lxp), *to_dev(Yp, lyp), opts=o2).cpu().numpy()
    assert np.array_equal(k1, k2)
