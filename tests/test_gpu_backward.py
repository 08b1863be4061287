"""GPU parity of the adjoint (sigk_backward through the C-ABI, and the
torch.autograd wrappers) against FP64 central finite differences of the oracle
and the single-tile closed form.  Gradients are with respect to the points
(or the increments); each checked coordinate must agree to 1e-4 relative (the
differentiation workload's tolerance) up to the FP32 rounding of the
contributions that cancel in it (tests/gradcheck.py)."""
import math

import numpy as np
import pytest
from gradcheck import assert_grad_close, increment_gradient_terms, point_gradient_terms
from scipy.special import i1, j1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OPTS = dict(order=12, rings=6)


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


def incs(paths):
    return [np.diff(p.astype(np.float64), axis=0) for p in paths]


def test_single_segment_gradient_closed_form(S):
    from paper_2502_20392_gb300 import synth
    cs = [0.3, 1.7, -0.9]
    (X, lx), (Y, ly) = synth.single_segment_pairs(cs)
    Xd, Yd = torch.from_numpy(X).to(dev()), torch.from_numpy(Y).to(dev())
    lxd, lyd = torch.from_numpy(lx).to(dev()), torch.from_numpy(ly).to(dev())
    g = torch.ones(len(cs), dtype=torch.float64)
    gX, gY, val = S.backward(S.OP_PAIRS, Xd, lxd, Yd, lyd, g, S.Opts(order=16, rings=8))
    gX = gX.cpu().numpy().reshape(len(cs), 2, 4)
    for p, c in enumerate(cs):
        # d/dc of I0(2 sqrt c) (c > 0) or J0(2 sqrt(-c)) (c < 0)
        dk = i1(2 * math.sqrt(c)) / math.sqrt(c) if c > 0 else j1(2 * math.sqrt(-c)) / math.sqrt(-c)
        # dk/d(dx) = dk/dc * dy, dy = e_0; point 1 gets +, point 0 gets -
        assert gX[p, 1, 0] == pytest.approx(dk, rel=2e-5)
        assert gX[p, 0, 0] == pytest.approx(-dk, rel=2e-5)
        assert np.abs(gX[p, :, 1:]).max() == 0.0


@pytest.mark.parametrize("d", [4, 8])
def test_pairs_gradient_vs_fd(S, orc, d):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(3, 20, 90, d, 0.7, 1.5, seed=60 + d)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    xs[1] = np.concatenate([xs[1], xs[1][-1:] + 0.05 * np.random.default_rng(1).standard_normal(
        (200, d)).cumsum(0).astype(np.float32)])  # one path over several 32-row strips
    X, lx = synth.pack(xs)
    rng = np.random.default_rng(7)
    w = rng.standard_normal(3)
    gX, gY, val = S.backward(S.OP_PAIRS, torch.from_numpy(X).to(dev()),
                             torch.from_numpy(lx).to(dev()), torch.from_numpy(Y).to(dev()),
                             torch.from_numpy(ly).to(dev()), torch.from_numpy(w),
                             S.Opts(**OPTS, max_len=400))
    gX = synth.split(gX.cpu().numpy(), lx)
    gY = synth.split(gY.cpu().numpy(), ly)
    for p in range(3):
        ix, iy = incs([xs[p], ys[p]])
        for which, g in ((0, gX[p]), (1, gY[p])):
            coords = rng.choice(g.size, size=min(12, g.size), replace=False)
            if which == 0:
                terms, inc = [(w[p], lambda z: orc.series_pair(z, iy))], ix
            else:
                terms, inc = [(w[p], lambda z: orc.series_pair(ix, z))], iy
            # the upstream weight w[p] is part of the computed gradient
            ref, scale = point_gradient_terms(terms, inc, coords)
            assert_grad_close(g.reshape(-1)[coords], ref, scale)


@pytest.mark.parametrize("order,rings", [(12, 6), (6, 6), (10, 6), (10, 5), (14, 7)])
def test_gram_self_gradient_vs_fd(S, orc, order, rings):
    # orders 6 and 10: the adjoint's per-lane record is wider than a seam
    # entry.  Order 6 with 6 rings keeps every coefficient of the 7 x 7 tile
    # matrices, the truncation N = 6 of the oracle, so the two compute the same
    # truncated function (the exact gradient differs from it by 1e-4 here).
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(4, [40, 70, 33, 100], 8, 1.0, seed=91)
    paths = synth.split(pts, lens)
    N = 6 if (order, rings) == (6, 6) else 24
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 4))  # not symmetric: both triangles weigh in
    gX, _, G = S.backward(S.OP_GRAM, torch.from_numpy(pts).to(dev()),
                          torch.from_numpy(lens).to(dev()), None, None, torch.from_numpy(W),
                          S.Opts(order=order, rings=rings, max_len=128))
    gX = synth.split(gX.cpu().numpy(), lens)
    zs = incs(paths)
    ref_G = orc.series_gram(zs, N=N)
    np.testing.assert_allclose(G.cpu().numpy(), ref_G, rtol=1e-5)
    for a in (0, 3):
        # f = sum_ab W_ab k(x_a, x_b) as a function of path a's increments
        terms = [(W[a, b] + W[b, a], (lambda z, b=b: orc.series_pair(z, zs[b], N=N)))
                 for b in range(4) if b != a]
        terms.append((W[a, a], lambda z: orc.series_pair(z, z, N=N)))
        coords = rng.choice(gX[a].size, size=10, replace=False)
        ref, scale = point_gradient_terms(terms, zs[a], coords)
        assert_grad_close(gX[a].reshape(-1)[coords], ref, scale)


def test_mmd_gradient_vs_fd(S, orc):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.workload_mmd_2048(seed=5001, n_paths=4, n_seg=120, d=8)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    gX, gY, v = S.backward(S.OP_MMD, torch.from_numpy(X).to(dev()), torch.from_numpy(lx).to(dev()),
                           torch.from_numpy(Y).to(dev()), torch.from_numpy(ly).to(dev()),
                           torch.ones(1, dtype=torch.float64), S.Opts(**OPTS, max_len=128))
    zx, zy = incs(xs), incs(ys)
    ref_v = orc.mmd2(zx, zy)
    assert v.item() == pytest.approx(ref_v, rel=1e-5, abs=1e-7)
    gX = synth.split(gX.cpu().numpy(), lx)
    rng = np.random.default_rng(11)
    m = n = 4
    for a in (0, 2):
        # U-statistic: k(x_a, x_b) appears twice among the m(m-1) ordered pairs
        terms = [(2.0 / (m * (m - 1)), (lambda z, b=b: orc.series_pair(z, zx[b]))) for b in range(m) if b != a]
        terms += [(-2.0 / (m * n), (lambda z, b=b: orc.series_pair(z, zy[b]))) for b in range(n)]
        coords = rng.choice(gX[a].size, size=10, replace=False)
        ref, scale = point_gradient_terms(terms, zx[a], coords)
        assert_grad_close(gX[a].reshape(-1)[coords], ref, scale)


def test_autograd_matches_backward(S):
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.workload_mmd_2048(seed=7, n_paths=3, n_seg=64, d=4)
    Xd = torch.from_numpy(X).to(dev()).requires_grad_(True)
    Yd = torch.from_numpy(Y).to(dev()).requires_grad_(True)
    lxd, lyd = torch.from_numpy(lx).to(dev()), torch.from_numpy(ly).to(dev())
    o = S.Opts(**OPTS, max_len=64)
    m = S.sig_kernel_mmd(Xd, lxd, Yd, lyd, o)
    gX, gY = torch.autograd.grad(m.sum(), (Xd, Yd))
    rX, rY, v = S.backward(S.OP_MMD, Xd.detach(), lxd, Yd.detach(), lyd,
                           torch.ones(1, dtype=torch.float64), o)
    torch.testing.assert_close(gX, rX)
    torch.testing.assert_close(gY, rY)
    assert m.item() == pytest.approx(v.item(), rel=1e-6)
    Gm = S.sig_kernel_gram(Xd, lxd, None, None, o)
    (gG,) = torch.autograd.grad(Gm.sum(), (Xd,))
    assert torch.isfinite(gG).all()


@pytest.mark.parametrize("op", ["pairs", "gram_xy", "gram_self", "mmd"])
def test_forward_train_then_adjoint(S, op):
    # the split entry points: sigk_forward_train leaves the seams and tile
    # records in the workspace, sigk_adjoint runs from them (twice here, with
    # different upstream gradients: no accumulation across calls)
    from paper_2502_20392_gb300 import synth
    px, lxp = synth.brownian(4, [70, 33, 1, 120], 8, 1.0, seed=101)
    py, lyp = synth.brownian(4, [90, 12, 64, 40], 8, 1.0, seed=102)
    X, lx = torch.from_numpy(px).to(dev()), torch.from_numpy(lxp).to(dev())
    Y, ly = torch.from_numpy(py).to(dev()), torch.from_numpy(lyp).to(dev())
    o = S.Opts(order=8, rings=4, max_len=160)
    rng = np.random.default_rng(103)
    code, args, gshape = {
        "pairs": (S.OP_PAIRS, (X, lx, Y, ly), (4,)),
        "gram_xy": (S.OP_GRAM, (X, lx, Y, ly), (4, 4)),
        "gram_self": (S.OP_GRAM, (X, lx, None, None), (4, 4)),
        "mmd": (S.OP_MMD, (X, lx, Y, ly), (1,)),
    }[op]
    g1 = torch.from_numpy(rng.standard_normal(gshape))
    value, state = S.forward_train(code, *args, o)
    aX, aY = S.adjoint(state, g1)
    bX, bY = S.adjoint(state, 2.0 * g1)
    rX, rY, rv = S.backward(code, *args, g1, o)
    assert torch.equal(value, rv)
    torch.testing.assert_close(aX, rX, rtol=1e-5, atol=1e-6 * float(rX.abs().max()))
    torch.testing.assert_close(bX, 2.0 * aX, rtol=1e-5, atol=1e-6 * float(rX.abs().max()))
    if op == "gram_self":
        assert aY is None and rY is None
    else:
        torch.testing.assert_close(aY, rY, rtol=1e-5, atol=1e-6 * float(rY.abs().max()))


def test_adjoint_refuses_foreign_workspace(S):
    # sigk_adjoint checks, on the device, that the workspace holds a
    # successful training forward of the same op, sizes and options; if not
    # it reports SIGK_ERR_ARG and touches nothing
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(3, [40, 33, 50], 4, 1.0, seed=105)
    X, L = torch.from_numpy(pts).to(dev()), torch.from_numpy(lens).to(dev())
    o = S.Opts(order=8, rings=4, max_len=64)
    g = torch.from_numpy(np.random.default_rng(106).standard_normal((3, 3)))
    nbytes = S.backward_workspace_size(S.OP_GRAM, 3, 0, 4, o)
    # the workspace holds an inference Gram
    ws = S.Workspace()
    ws.get(nbytes, X.device)
    S.gram(X, L, opts=o, ws=ws)
    with pytest.raises(S.SigkError):
        S.adjoint(S.TrainState(S.OP_GRAM, X, L, None, None, 3, 0, 4, o, ws), g)
    # the workspace holds the training forward of the first two paths
    n2 = int(lens[0] + lens[1])
    S.forward_train(S.OP_GRAM, X[:n2], L[:2], None, None, o, ws=ws)
    with pytest.raises(S.SigkError):
        S.adjoint(S.TrainState(S.OP_GRAM, X, L, None, None, 3, 0, 4, o, ws), g)
    # the matching training forward on the same workspace
    value, state = S.forward_train(S.OP_GRAM, X, L, None, None, o, ws=ws)
    gX, _ = S.adjoint(state, g)
    rX, _, rv = S.backward(S.OP_GRAM, X, L, None, None, g, o)
    assert torch.equal(value, rv)
    torch.testing.assert_close(gX, rX, rtol=1e-5, atol=1e-6 * float(rX.abs().max()))


def test_gradient_with_refinement(S, orc):
    # gradients of refined virtual segments are folded back to the segments
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(2, [3, 5], 4, 1.0, seed=17)  # rough: |c| up to ~2
    xs = synth.split(pts, lens)
    o = S.Opts(order=12, rings=6, refine_c=0.25, max_len=400)
    Xd = torch.from_numpy(xs[0]).to(dev())
    Yd = torch.from_numpy(xs[1]).to(dev())
    l0 = torch.tensor([4], device=dev())
    l1 = torch.tensor([6], device=dev())
    gX, gY, val = S.backward(S.OP_PAIRS, Xd, l0, Yd, l1, torch.ones(1, dtype=torch.float64), o)
    ref = orc.series_pair(*incs(xs), N=30)
    assert val.item() == pytest.approx(ref, rel=1e-5)

    ix, iy = incs(xs)
    gx_ref, sx = point_gradient_terms([(1.0, lambda z: orc.series_pair(z, iy, N=30))], ix,
                                      range(xs[0].size))
    gy_ref, sy = point_gradient_terms([(1.0, lambda z: orc.series_pair(ix, z, N=30))], iy,
                                      range(xs[1].size))
    assert_grad_close(gX.cpu().numpy().ravel(), gx_ref, sx)
    assert_grad_close(gY.cpu().numpy().ravel(), gy_ref, sy)


def test_backward_schedules_agree_bitwise(S):
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(5, [300, 1, 90, 500, 47], 8, 1.0, seed=93)
    Xd, ld = torch.from_numpy(pts).to(dev()), torch.from_numpy(lens).to(dev())
    W = torch.from_numpy(np.random.default_rng(5).standard_normal((5, 5)))
    o1 = S.Opts(order=8, rings=4, max_len=512)
    o2 = S.Opts(order=8, rings=4, max_len=512, flags=S.FLAG_PAIR_MAJOR)
    g1, _, G1 = S.backward(S.OP_GRAM, Xd, ld, None, None, W, o1)
    g2, _, G2 = S.backward(S.OP_GRAM, Xd, ld, None, None, W, o2)
    assert torch.equal(G1, G2)
    # gradients accumulate with float atomics: equal up to summation order
    torch.testing.assert_close(g1, g2, rtol=1e-5, atol=1e-6 * float(g1.abs().max()))


@pytest.mark.parametrize("d,order,rings,sigma", [(16, 8, 4, 2.0), (4, 12, 6, 1.0)])
def test_stored_records_match_replay(S, d, order, rings, sigma):
    # the training forward (one row per lane) stores every tile's record and
    # the adjoint skips its replay; with SIGK_FLAG_REPLAY it replays each
    # strip instead.  sigma = 2 drives the self-kernels past 2^64 (to 2.5e26,
    # gradients still inside the FP32 range), so the records carry exponent
    # alignments and renormalisations.
    from paper_2502_20392_gb300 import synth
    pts, lens = synth.brownian(6, [420, 1, 77, 300, 33, 129], d, sigma, seed=97)
    Xd, ld = torch.from_numpy(pts).to(dev()), torch.from_numpy(lens).to(dev())
    W = torch.from_numpy(np.random.default_rng(11).standard_normal((6, 6)))
    out = {}
    for flags in (0, S.FLAG_REPLAY):
        ws = S.Workspace()
        o = S.Opts(order=order, rings=rings, max_len=512, flags=flags)
        g, _, G = S.backward(S.OP_GRAM, Xd, ld, None, None, W, o, ws=ws)
        out[flags] = (g, G, S.counters(ws))
    (g0, G0, c0), (g1, G1, c1) = out[0], out[S.FLAG_REPLAY]
    tiles = sum((a - 1) * (b - 1) for i, a in enumerate(lens) for b in lens[i:])
    assert c0[2] == c1[2] == tiles
    assert c0[3] == 0 and c1[3] == tiles
    assert torch.isfinite(G0).all()
    if sigma > 2:
        assert float(G0.abs().max()) > 2.0 ** 64
    torch.testing.assert_close(G0, G1, rtol=1e-6, atol=0)
    torch.testing.assert_close(g0, g1, rtol=1e-5, atol=1e-6 * float(g1.abs().max()))


def test_increments_mode_gradient_and_gram_xy(S, orc):
    # FLAG_INCREMENTS: gradients are with respect to the increments; a Gram of
    # X against a different Y also returns grad_Y
    from paper_2502_20392_gb300 import synth
    px, lxp = synth.brownian(3, [30, 55, 41], 4, 1.0, seed=95)
    py, lyp = synth.brownian(2, [47, 36], 4, 1.0, seed=96)
    xs, ys = synth.split(px, lxp), synth.split(py, lyp)
    ix = [np.diff(p, axis=0).astype(np.float32) for p in xs]
    iy = [np.diff(p, axis=0).astype(np.float32) for p in ys]
    IX, lix = synth.pack(ix)  # increments mode: one row per segment, len counts rows
    IY, liy = synth.pack(iy)
    W = np.random.default_rng(9).standard_normal((3, 2))
    o = S.Opts(order=12, rings=6, max_len=128, flags=S.FLAG_INCREMENTS)
    gX, gY, G = S.backward(S.OP_GRAM, torch.from_numpy(IX).to(dev()), torch.from_numpy(lix).to(dev()),
                           torch.from_numpy(IY).to(dev()), torch.from_numpy(liy).to(dev()),
                           torch.from_numpy(W), o)
    ref_G = np.array([[orc.series_pair(a.astype(np.float64), b.astype(np.float64)) for b in iy]
                      for a in ix])
    np.testing.assert_allclose(G.cpu().numpy(), ref_G, rtol=1e-5)
    gX = synth.split(gX.cpu().numpy(), lix)
    gY = synth.split(gY.cpu().numpy(), liy)
    rng = np.random.default_rng(10)
    a64 = [v.astype(np.float64) for v in ix]
    b64 = [v.astype(np.float64) for v in iy]
    # f = sum_ab W_ab k(x_a, y_b): x path 1 enters the pairs (1, b), y path 0
    # the pairs (a, 0)
    for which, grads, p in ((0, gX, 1), (1, gY, 0)):
        if which == 0:
            terms = [(W[p, b], (lambda z, b=b: orc.series_pair(z, b64[b]))) for b in range(2)]
            inc = a64[p]
        else:
            terms = [(W[a, p], (lambda z, a=a: orc.series_pair(a64[a], z))) for a in range(3)]
            inc = b64[p]
        coords = rng.choice(grads[p].size, size=8, replace=False)
        ref, scale = increment_gradient_terms(terms, inc, coords)
        assert_grad_close(grads[p].reshape(-1)[coords], ref, scale)


@pytest.mark.parametrize("d,seed", [(64, 121), (256, 122)])
def test_large_dimension_gradient_vs_fd(S, orc, d, seed):
    # d > 16: the training forward is the two-phase kernel (FMA increment
    # Gram, seams kept), the adjoint replays each strip and chains to the
    # increments with the contraction; gradients w.r.t. the increments of a
    # Gram of X against Y
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(3, 30, 110, d, 0.5, 1.0, seed=seed)
    ix = [np.diff(p, axis=0).astype(np.float32) for p in synth.split(X, lx)]
    iy = [np.diff(p, axis=0).astype(np.float32) for p in synth.split(Y, ly)][:2]
    IX, lix = synth.pack(ix)
    IY, liy = synth.pack(iy)
    W = np.random.default_rng(seed).standard_normal((3, 2))
    o = S.Opts(order=12, rings=6, max_len=128, flags=S.FLAG_INCREMENTS)
    gX, gY, G = S.backward(S.OP_GRAM, torch.from_numpy(IX).to(dev()), torch.from_numpy(lix).to(dev()),
                           torch.from_numpy(IY).to(dev()), torch.from_numpy(liy).to(dev()),
                           torch.from_numpy(W), o)
    a64 = [v.astype(np.float64) for v in ix]
    b64 = [v.astype(np.float64) for v in iy]
    ref_G = np.array([[orc.series_pair(a, b) for b in b64] for a in a64])
    np.testing.assert_allclose(G.cpu().numpy(), ref_G, rtol=1e-5)
    gX = synth.split(gX.cpu().numpy(), lix)
    gY = synth.split(gY.cpu().numpy(), liy)
    rng = np.random.default_rng(seed + 1)
    for which, grads, p in ((0, gX, 2), (1, gY, 1)):
        if which == 0:
            terms = [(W[p, b], (lambda z, b=b: orc.series_pair(z, b64[b]))) for b in range(2)]
            inc = a64[p]
        else:
            terms = [(W[a, p], (lambda z, a=a: orc.series_pair(a64[a], z))) for a in range(3)]
            inc = b64[p]
        coords = rng.choice(grads[p].size, size=10, replace=False)
        ref, scale = increment_gradient_terms(terms, inc, coords)
        assert_grad_close(grads[p].reshape(-1)[coords], ref, scale)


def test_large_dimension_points_gradient(S, orc):
    # d = 40, points input, a pair whose row path spans several strips and a
    # refined rough pair: point gradients against the oracle
    from paper_2502_20392_gb300 import synth
    (X, lx), (Y, ly) = synth.ragged_pairs(2, 40, 100, 40, 0.5, 1.0, seed=123)
    xs, ys = synth.split(X, lx), synth.split(Y, ly)
    xs[0] = synth.brownian(1, 140, 40, 1.0, seed=124)[0]
    X, lx = synth.pack(xs)
    w = np.array([0.7, -1.3])
    gX, gY, val = S.backward(S.OP_PAIRS, torch.from_numpy(X).to(dev()), torch.from_numpy(lx).to(dev()),
                             torch.from_numpy(Y).to(dev()), torch.from_numpy(ly).to(dev()),
                             torch.from_numpy(w), S.Opts(order=12, rings=6, max_len=256))
    gX = synth.split(gX.cpu().numpy(), lx)
    rng = np.random.default_rng(125)
    for p in range(2):
        ix, iy = incs([xs[p], ys[p]])
        assert val.cpu().numpy()[p] == pytest.approx(orc.series_pair(ix, iy), rel=1e-5)
        coords = rng.choice(gX[p].size, size=10, replace=False)
        ref, scale = point_gradient_terms([(w[p], lambda z: orc.series_pair(z, iy))], ix, coords)
        assert_grad_close(gX[p].reshape(-1)[coords], ref, scale)
