"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own formulas (CPU only).

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
transposed operand, a wrong factorial or sign) fails at least one of them:

* single-tile Bessel closed form (Lemma "single-tile solution", Sec. 2.2.1),
* straight-path closed form I0(2 sqrt(<X,Y>)) (signature of a straight path is
  exp(X); with the corrected worked example of Sec. 2.2.2),
* the operator-power lemma of App. A.4 for one tile with monomial boundary data,
* brute force three ways on tiny inputs (series vs Chen signature vs FD PDE),
* second-order convergence of the FD scheme,
* invariants (symmetry, time reversal, zero/collinear insertion, constant path),
* Gram PSD and the Gram truncation bound of App. A.7.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import i0, i1, j0, j1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bessel_k(c):
    return i0(2 * math.sqrt(c)) if c >= 0 else j0(2 * math.sqrt(-c))


def bessel_dk(c):
    """d/dc of bessel_k."""
    if c > 0:
        return i1(2 * math.sqrt(c)) / math.sqrt(c)
    if c < 0:
        return j1(2 * math.sqrt(-c)) / math.sqrt(-c)
    return 1.0


@pytest.mark.parametrize("c", [-4.0, -0.5, 0.01, 0.5, 4.0])
def test_single_tile_bessel(orc, c):
    dx = np.array([[c, 0.0, 0.0, 0.0]])
    dy = np.array([[1.0, 0.0, 0.0, 0.0]])
    ref = bessel_k(c)
    assert orc.series_pair(dx, dy, N=30) == pytest.approx(ref, rel=1e-14, abs=1e-15)
    assert orc.chen_pair([[c]], [[1.0]], 40) == pytest.approx(ref, rel=1e-14, abs=1e-15)
    fd = orc.fd_richardson(dx, dy, 4)
    assert fd[3] == pytest.approx(ref, rel=1e-8, abs=1e-10)


def test_single_tile_series_truncation_is_bessel_partial_sum(orc):
    # With N-truncated tile matrices the single-tile result is the Bessel
    # partial sum sum_{i<=N} c^i/(i!)^2 (Lemma "single-tile solution").
    c = 1.7
    for N in range(1, 8):
        ref = sum(c**i / math.factorial(i) ** 2 for i in range(N + 1))
        assert orc.series_pair([[c]], [[1.0]], N=N) == pytest.approx(ref, rel=1e-15)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_straight_path_closed_form(orc, sign):
    rng = np.random.default_rng(7)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    r = rng.uniform(-0.3, 0.6, size=5)
    dx = r[:, None] * u[None, :]                   # straight x, 5 segments
    dy = sign * rng.standard_normal((6, 3)) * 0.5  # arbitrary y, 6 segments
    s = float(dx.sum(0) @ dy.sum(0))
    ref = bessel_k(s)
    assert orc.series_pair(dx, dy) == pytest.approx(ref, rel=1e-13)
    assert orc.series_pair(dy, dx) == pytest.approx(ref, rel=1e-13)
    assert orc.chen_pair(dx, dy, 13) == pytest.approx(ref, rel=1e-11)


def test_worked_example_corrected(orc):
    # Worked example of Sec. 2.2.2 on a 1x2 grid (and 2x1): with the j! that
    # the printed formula omits (Lemma of App. A.4 gives i! j! (i+j)!),
    # K(1,1) = sum_{i,j} c1^i c2^j / (i! j! (i+j)!) = I0(2 sqrt(c1 + c2)).
    c1, c2 = 0.37, -0.81
    ex = sum(c1**i * c2**j / (math.factorial(i) * math.factorial(j) * math.factorial(i + j))
             for i in range(30) for j in range(30))
    assert ex == pytest.approx(bessel_k(c1 + c2), rel=1e-14)
    assert orc.series_pair([[1.0]], [[c1], [c2]]) == pytest.approx(ex, rel=1e-14)
    assert orc.series_pair([[c1], [c2]], [[1.0]]) == pytest.approx(ex, rel=1e-14)
    # the uncorrected printed coefficient (no j!) gives a different value
    printed = sum(c1**i * c2**j / (math.factorial(i + j) * math.factorial(i))
                  for i in range(30) for j in range(30))
    assert abs(printed - ex) > 1e-2


@pytest.mark.parametrize("r", [0, 1, 2, 3])
@pytest.mark.parametrize("edge", ["bottom", "left"])
def test_operator_power_lemma_one_tile(orc, r, edge):
    # Lemma (operator powers), App. A.4: T^n (s-sigma)^r = rho^n/((r+1)^(n) n!)
    # (s-sigma)^{r+n} (t-tau)^n.  With bottom edge u^r (r >= 1) and left edge 0
    # (or the mirror), the tile solution is sum_n of those terms, so the top
    # edge has coefficient rho^n/((r+1)^(n) n!) at u^{r+n} and the right edge
    # the same at v^n.  r = 0 is the constant boundary (K = 1 on both edges).
    N, rho = 12, 0.83
    alpha = np.zeros(N + 1)
    beta = np.zeros(N + 1)
    if r == 0:
        alpha[0] = beta[0] = 1.0
    elif edge == "bottom":
        alpha[r] = 1.0
    else:
        beta[r] = 1.0

    def rising(x, n):
        return math.prod(x + k for k in range(n))

    exp_far = np.zeros(N + 1)   # edge that carries u^{r+n} (or v^{r+n})
    exp_near = np.zeros(N + 1)  # edge that carries v^n (or u^n)
    for n in range(N + 1):
        coef = rho**n / (rising(r + 1, n) * math.factorial(n))
        if r + n <= N:
            exp_far[r + n] += coef
        exp_near[n] += coef
    ao, bo = orc.tile_map(rho, alpha, beta, N)
    if r == 0:
        # both edges are sum_n rho^n/(n!)^2 (.)^n
        ref = np.array([rho**n / math.factorial(n) ** 2 for n in range(N + 1)])
        np.testing.assert_allclose(ao, ref, rtol=1e-14, atol=1e-17)
        np.testing.assert_allclose(bo, ref, rtol=1e-14, atol=1e-17)
        return
    # truncation: entries with both indices <= N; the near edge sums every n
    # whose far index r+n also fits.
    exp_near_tr = np.zeros(N + 1)
    for n in range(N + 1 - r):
        exp_near_tr[n] = rho**n / (rising(r + 1, n) * math.factorial(n))
    if edge == "bottom":
        np.testing.assert_allclose(ao, exp_far, rtol=1e-14, atol=1e-17)
        np.testing.assert_allclose(bo, exp_near_tr, rtol=1e-14, atol=1e-17)
    else:
        np.testing.assert_allclose(bo, exp_far, rtol=1e-14, atol=1e-17)
        np.testing.assert_allclose(ao, exp_near_tr, rtol=1e-14, atol=1e-17)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_three_ways(orc, seed):
    rng = np.random.default_rng(100 + seed)
    d = 2 + seed % 2
    L1, L2 = 1 + seed % 4, 1 + (seed * 3) % 4
    dx = rng.standard_normal((L1, d)) * 0.5
    dy = rng.standard_normal((L2, d)) * 0.5
    ks = orc.series_pair(dx, dy)
    kc, levels = orc.chen_pair(dx, dy, 16 if d == 2 else 13, levels=True)
    assert abs(levels[-1]) < 1e-13 * max(1.0, abs(kc))  # Chen tail converged
    kf = orc.fd_richardson(dx, dy, 3)[3]
    assert ks == pytest.approx(kc, rel=1e-12, abs=1e-13)
    assert ks == pytest.approx(kf, rel=1e-8, abs=1e-9)


def test_golden_chen_values(orc):
    # Values recorded in the golden fixture (written by tests/golden/make_golden.py
    # from the Chen brute force, which shares nothing with the series code).
    with open(os.path.join(GOLDEN, "chen_tiny.json")) as f:
        cases = json.load(f)
    for case in cases:
        dx = np.array(case["dx"])
        dy = np.array(case["dy"])
        assert orc.series_pair(dx, dy) == pytest.approx(case["k"], rel=1e-12), case["name"]


def test_fd_second_order(orc):
    rng = np.random.default_rng(11)
    dx = rng.standard_normal((3, 2)) * 0.7
    dy = rng.standard_normal((2, 2)) * 0.7
    k = [orc.fd_pair(dx, dy, lam) for lam in range(2, 7)]
    exact = orc.series_pair(dx, dy)
    errs = [abs(v - exact) for v in k]
    ratios = [errs[t] / errs[t + 1] for t in range(len(errs) - 1)]
    for q in ratios:
        assert 3.7 < q < 4.3  # error ~ h^2: halving h divides it by 4


def test_invariants(orc):
    rng = np.random.default_rng(21)
    dx = rng.standard_normal((7, 3)) * 0.4
    dy = rng.standard_normal((5, 3)) * 0.4
    k = orc.series_pair(dx, dy)
    # symmetry: transposes the grid
    assert orc.series_pair(dy, dx) == pytest.approx(k, rel=1e-13)
    # time reversal: reversed, negated increments (grid rotated by 180 degrees)
    assert orc.series_pair(-dx[::-1], -dy[::-1]) == pytest.approx(k, rel=1e-13)
    # constant path
    assert orc.series_pair(dx, np.zeros((4, 3))) == pytest.approx(1.0, abs=1e-15)
    assert orc.series_pair(dx, np.zeros((0, 3))) == 1.0
    # zero-increment insertion (padding by repeating a point, Sec. 2.1)
    dx_pad = np.concatenate([dx[:3], np.zeros((2, 3)), dx[3:], np.zeros((3, 3))])
    assert orc.series_pair(dx_pad, dy) == pytest.approx(k, rel=1e-13)
    # splitting a segment into collinear pieces
    dx_split = np.concatenate([dx[:2], dx[2:3] * 0.25, dx[2:3] * 0.75, dx[3:]])
    assert orc.series_pair(dx_split, dy) == pytest.approx(k, rel=1e-13)
    # orthogonal map, scaling, negation leave every c_ij unchanged
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert orc.series_pair(dx @ Q.T, dy @ Q.T) == pytest.approx(k, rel=1e-13)
    assert orc.series_pair(2.5 * dx, dy) == pytest.approx(orc.series_pair(dx, 2.5 * dy), rel=1e-13)
    assert orc.series_pair(-dx, -dy) == pytest.approx(k, rel=1e-13)


def test_gram_symmetric_psd(orc):
    rng = np.random.default_rng(31)
    paths = [rng.standard_normal((12 + p, 3)) / math.sqrt(12) for p in range(8)]
    G = orc.series_gram(paths)
    np.testing.assert_allclose(G, G.T, rtol=1e-13)
    w = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert w.min() > -1e-10 * np.abs(w).max()


def _gram_bound(paths, N, density):
    # Proposition of App. A.7: ||G - G_N||_F <= gamma X^{N+1} zeta_N / ((N+1)!)^2
    # with gamma = m/2 prod_{nu=0}^{2l-2} I0(2 sqrt(nu X)/(l-1)) and
    # zeta_N = [1 + (2l-2)/(N+2)] (2/(l-1))^{N+1}, common length l (points).
    m, ell = len(paths), paths[0].shape[0] + 1
    allinc = np.concatenate(paths)
    X = np.abs(allinc @ allinc.T).max()
    if density:
        X *= (ell - 1) ** 2  # the PDE coefficient on [0,1]^2 (Sec. 2.1)
    gamma = m / 2 * math.prod(i0(2 * math.sqrt(nu * X) / (ell - 1)) for nu in range(2 * ell - 1))
    zeta = (1 + (2 * ell - 2) / (N + 2)) * (2 / (ell - 1)) ** (N + 1)
    return gamma * X ** (N + 1) * zeta / math.factorial(N + 1) ** 2


FAMILIES = [(41, 0.8, 6, 4), (42, 0.3, 9, 3), (43, 1.5, 4, 5), (44, 0.1, 12, 3)]


@pytest.mark.parametrize("fam", FAMILIES)
def test_gram_truncation_bound(orc, fam):
    # The bound holds when X is read as the PDE density (l-1)^2 max|<dx,dy>|;
    # the truncation error also decreases monotonically in N.
    seed, scale, ell, m = fam
    rng = np.random.default_rng(seed)
    paths = [rng.standard_normal((ell - 1, 2)) * scale for _ in range(m)]
    G = orc.series_gram(paths, N=28)
    prev = None
    for N in range(1, 10):
        err = np.linalg.norm(G - orc.series_gram(paths, N=N))
        assert err <= _gram_bound(paths, N, density=True), (N, err)
        if seed in (41, 42) and prev is not None and prev > 1e-13 * np.abs(G).max():
            assert err < prev  # moderate |c|: truncation error falls with N
        prev = err


def test_gram_bound_unscaled_reading_is_rejected(orc):
    # Read with the unscaled max|<dx,dy>| the same bound fails (N = 2 here):
    # the truncation error decays like C^{N+1}/((N+1)!)^2 with C the row sum
    # of c over a whole edge, not 2 max|c|/(l-1).
    rng = np.random.default_rng(41)
    paths = [rng.standard_normal((5, 2)) * 0.8 for _ in range(4)]
    G = orc.series_gram(paths, N=28)
    err = np.linalg.norm(G - orc.series_gram(paths, N=2))
    assert err > _gram_bound(paths, 2, density=False)


def test_gradient_single_tile_closed_form(orc):
    for c in (-1.3, 0.4, 2.0):
        dy = np.array([[0.6, -0.8]])
        dx = np.array([[c * 0.6, -c * 0.8]])  # <dx, dy> = c
        g = orc.grad_fd(lambda z: orc.series_pair(z, dy), dx, [0, 1])
        ref = bessel_dk(c) * dy[0]
        np.testing.assert_allclose(g, ref, rtol=1e-8)


def test_mmd_properties(orc):
    rng = np.random.default_rng(51)
    xs = [rng.standard_normal((9, 2)) * 0.4 for _ in range(5)]
    ys = [rng.standard_normal((9, 2)) * 0.4 + 0.05 for _ in range(6)]
    assert orc.mmd2(xs, xs, unbiased=False) == pytest.approx(0.0, abs=1e-12)
    assert orc.mmd2(xs, ys, unbiased=False) >= 0.0
    Kxx = orc.series_gram(xs)
    Kyy = orc.series_gram(ys)
    Kxy = orc.series_gram(xs, ys)
    m, n = 5, 6
    u = ((Kxx.sum() - np.trace(Kxx)) / (m * (m - 1)) + (Kyy.sum() - np.trace(Kyy)) / (n * (n - 1))
         - 2 * Kxy.mean())
    assert orc.mmd2(xs, ys) == pytest.approx(u, rel=1e-12)


def _literal_statement_tile(rho, N, alpha, beta):
    # The proposition's statement read literally (alpha on the j >= i side):
    # kept here only to show that the pins reject that reading.
    f = [math.factorial(k) for k in range(N + 1)]
    C = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            mn, mx = min(i, j), max(i, j)
            b = alpha[j - i] if j >= i else beta[i - j]
            C[i, j] = rho**mn * b * f[mx - mn] / (f[mx] * f[mn])
    return C.sum(1), C.sum(0)


def test_statement_orientation_is_rejected(orc):
    # Planted mistake (in a Python copy, never in the product): the literal
    # alpha/beta orientation of the statement disagrees with the Chen brute
    # force, while the proof's orientation used by the oracle agrees.
    rng = np.random.default_rng(0)
    dx = rng.standard_normal((3, 2)) * 0.6
    dy = rng.standard_normal((4, 2)) * 0.6
    N = 20
    A = [np.eye(N + 1)[0] for _ in range(3)]
    B = [np.eye(N + 1)[0] for _ in range(4)]
    for dg in range(3 + 4 - 1):
        for i in range(max(0, dg - 3), min(dg, 2) + 1):
            j = dg - i
            A[i], B[j] = _literal_statement_tile(float(dx[i] @ dy[j]), N, A[i], B[j])
    k_literal = B[3].sum()
    k_chen = orc.chen_pair(dx, dy, 16)
    assert orc.series_pair(dx, dy) == pytest.approx(k_chen, rel=1e-12)
    assert abs(k_literal - k_chen) > 1e-2


def _straight_batch(rng, n, d, lens_x, lens_y, scale=0.5):
    """Ragged batch whose x_p are straight (collinear segments of varying
    length along a fixed direction) and whose y_p are arbitrary: k(x_p, y_p) =
    I0/J0 of <X_p, Y_p> with X_p, Y_p the total increments (straight-path
    closed form), so every pair's value depends on which rows are its own."""
    xs, ys = [], []
    for p in range(n):
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        r = rng.uniform(-0.2, 0.5, size=lens_x[p])
        xs.append(r[:, None] * u[None, :])
        ys.append(rng.standard_normal((lens_y[p], d)) * scale)
    return xs, ys


def test_series_pairs_ragged_packed_closed_form(orc):
    # The batched pair routine on packed ragged inputs (one path of the batch
    # has no segment): every value must be the straight-path closed form of
    # its own pair.  A slip in the prefix offsets of either side would pair a
    # path with a neighbour's rows and miss the closed form.
    rng = np.random.default_rng(23)
    lx = [3, 1, 7, 0, 5, 2]
    ly = [4, 6, 1, 3, 0, 8]
    xs, ys = _straight_batch(rng, 6, 3, lx, ly)
    got = orc.series_pairs(xs, ys)
    for p in range(6):
        s = float(xs[p].sum(0) @ ys[p].sum(0)) if lx[p] and ly[p] else 0.0
        assert got[p] == pytest.approx(bessel_k(s), rel=1e-13), p
        assert got[p] == orc.series_pair(xs[p], ys[p])  # the same arithmetic per pair


def test_series_gram_ragged_closed_form(orc):
    # Gram of straight x_a (ragged) against arbitrary y_b (ragged): entry
    # (a, b) is the closed form of <X_a, Y_b>; rows and columns may not mix.
    rng = np.random.default_rng(29)
    xs, _ = _straight_batch(rng, 4, 2, [2, 5, 1, 4], [1, 1, 1, 1])
    ys = [rng.standard_normal((n, 2)) * 0.6 for n in (3, 1, 6)]
    G = orc.series_gram(xs, ys)
    for a in range(4):
        for b in range(3):
            s = float(xs[a].sum(0) @ ys[b].sum(0))
            assert G[a, b] == pytest.approx(bessel_k(s), rel=1e-13), (a, b)


def test_mmd_u_statistic_hand_expanded(orc):
    # Two samples of two single-segment paths each: every kernel value is a
    # Bessel closed form, and the unbiased MMD^2 with m = n = 2 expands by hand
    # to k(x1,x2) + k(y1,y2) - (k(x1,y1) + k(x1,y2) + k(x2,y1) + k(x2,y2)) / 2
    # (the diagonal terms drop out; each off-diagonal pair appears twice over
    # m(m-1) = 2).  The biased form keeps the diagonals with weight 1/m^2.
    x1, x2 = np.array([[0.7, -0.2]]), np.array([[0.1, 0.9]])
    y1, y2 = np.array([[-0.4, 0.3]]), np.array([[1.1, 0.5]])

    def k(a, b):
        return bessel_k(float(a[0] @ b[0]))

    cross = k(x1, y1) + k(x1, y2) + k(x2, y1) + k(x2, y2)
    u = k(x1, x2) + k(y1, y2) - cross / 2
    v = ((k(x1, x1) + 2 * k(x1, x2) + k(x2, x2)) / 4 + (k(y1, y1) + 2 * k(y1, y2) + k(y2, y2)) / 4
         - cross / 2)
    assert orc.mmd2([x1, x2], [y1, y2]) == pytest.approx(u, rel=1e-13)
    assert orc.mmd2([x1, x2], [y1, y2], unbiased=False) == pytest.approx(v, rel=1e-13)


def test_mmd_u_statistic_is_unbiased(orc):
    # The U-statistic is an unbiased estimator of MMD^2, which is 0 when both
    # samples come from one distribution: its mean over independent draws
    # (single-segment paths, so each draw is cheap) is 0 within a few standard
    # errors, while the V-statistic is biased upwards by the mean diagonal.
    rng = np.random.default_rng(31)
    us, vs = [], []
    for _ in range(400):
        xs = [rng.standard_normal((1, 2)) * 0.8 for _ in range(3)]
        ys = [rng.standard_normal((1, 2)) * 0.8 for _ in range(3)]
        us.append(orc.mmd2(xs, ys, N=16))
        vs.append(orc.mmd2(xs, ys, N=16, unbiased=False))
    us, vs = np.array(us), np.array(vs)
    se = us.std(ddof=1) / math.sqrt(len(us))
    assert abs(us.mean()) < 4 * se, (us.mean(), se)
    assert vs.mean() > 10 * se
