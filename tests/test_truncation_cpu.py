"""CPU pins of the truncation the FP32 solvers use (the tile-matrix entries of
ring m <= n, edge degree k with m + k <= P and 2m + k <= 2n + 1).

The tile map of the tile-centred expansion (Sec. 2.3; orientation of the
proof in App. A.6) is restated here in FP64 in its factorial-scaled form,
with an arbitrary set of kept entries, and swept over the grid anti-diagonal
by anti-diagonal (App. C.1).  It is compared with the FP64 oracle's exact
kernel (truncation order 24).  Nothing here calls the CUDA library: these
tests pin the reading of the truncation, the kernels' own parity tests pin
the kernels.
"""
import math

import numpy as np
import pytest

from paper_2502_20392_gb300 import synth


def sweep(C, P, keep):
    """k(x, y) from the tile coefficients C (L1 x L2) with the entries
    keep(m, k) of every tile's matrix, edge polynomials of degree P.

    Scaled coefficients ah_p = p! a_p (bottom edge), bh_q = q! b_q (left
    edge), corner h:
      ah'_p = ah_p + sum_m c^m/m! ah_{p-m} + c^p sum_k bh_k / (p+k)!   (bh_0 = h)
      bh'_q  likewise with a and b exchanged,   h' = h + sum_p ah_p / p!
    """
    L1, L2 = C.shape
    inv = np.array([1.0 / math.factorial(i) for i in range(2 * P + 2)])
    A = np.zeros((L1, P + 1))
    bh_prev, b_prev = np.ones(L1), np.zeros((L1, P + 1))
    for t in range(L1 + L2 - 1):
        i = np.arange(max(0, t - L2 + 1), min(t, L1 - 1) + 1)
        c = C[i, t - i]
        h = np.where(i == 0, 1.0, bh_prev[np.maximum(i - 1, 0)])
        b = np.where((i == 0)[:, None], 0.0, b_prev[np.maximum(i - 1, 0)])
        a = A[i]
        a2, b2 = a.copy(), b.copy()
        for m in range(1, P + 1):
            cm = c ** m
            for k in range(0, P - m + 1):
                if not keep(m, k):
                    continue
                if k == 0:  # diagonal entry c^m h / (m!)^2, into both edges
                    a2[:, m] += cm * h * inv[m]
                    b2[:, m] += cm * h * inv[m]
                    continue
                # below the diagonal (bottom-edge data) and above it (left edge)
                a2[:, m + k] += cm * inv[m] * a[:, k]
                b2[:, m] += cm * a[:, k] * inv[m + k]
                b2[:, m + k] += cm * inv[m] * b[:, k]
                a2[:, m] += cm * b[:, k] * inv[m + k]
        S = sum(a[:, p] * inv[p] for p in range(1, P + 1))
        A[i] = a2
        nh, nb = bh_prev.copy(), b_prev.copy()
        nh[i] = h + S
        nb[i] = b2
        bh_prev, b_prev = nh, nb
    b = b_prev[L1 - 1]
    return bh_prev[L1 - 1] + sum(b[q] * inv[q] for q in range(1, P + 1))


def weighted(P, n):
    return lambda m, k: m <= n and m + k <= P and 2 * m + k <= 2 * n + 1


def square(P, n):
    return lambda m, k: m <= n and m + k <= P


def pair(n_seg, d, sigma, seed):
    pts, lens = synth.brownian(2, n_seg, d, sigma, seed=seed)
    x, y = (np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens))
    return x, y


def test_sweep_matches_oracle_when_nothing_is_dropped(orc):
    # every entry up to degree 12 on a weakly coupled pair: the exact kernel
    x, y = pair(24, 3, 1.0, seed=301)
    ref = orc.series_pair(x, y, N=24)
    k = sweep(x @ y.T, 12, square(12, 12))
    assert abs(k - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("sigma", [0.35, 0.7, 1.0, 2.0])
def test_weighted_truncation_within_the_ring_rule(orc, sigma):
    # Brownian pairs of 64 segments in R^4 (a cross and a self pair), rings
    # n = 3..6 at order 2n: the error of the weighted-degree truncation
    # against the exact kernel stays below the plan's a-priori quantity for
    # the first dropped ring, sum |c|^(n+1) / ((n+1)!)^2 over the tiles (the
    # rule sigk_plan applies), and within a factor of the square
    # truncation's error (every entry of ring <= n up to degree P)
    x, y = pair(64, 4, sigma, seed=int(310 + 10 * sigma))
    for u, v in ((x, y), (x, x)):
        ref = orc.series_pair(u, v, N=24)
        C = u @ v.T
        for n in (3, 4, 5, 6):
            P = 2 * n
            e_w = abs(sweep(C, P, weighted(P, n)) - ref) / abs(ref)
            e_s = abs(sweep(C, P, square(P, n)) - ref) / abs(ref)
            rule = float((np.abs(C) ** (n + 1)).sum()) / math.factorial(n + 1) ** 2
            assert e_w <= rule + 1e-13, (n, e_w, rule)
            assert e_w <= 20 * e_s + 1e-9, (n, e_w, e_s)


def test_order_above_twice_the_rings_changes_nothing():
    # no kept entry reaches a degree above 2n: the coefficients of degree
    # 2n + 1 .. P stay zero, so order P and order 2n give the same sweep
    # (the solvers launch with the order clamped to 2n)
    x, y = pair(40, 4, 2.0, seed=331)
    C = x @ y.T
    for n in (3, 4, 6):
        k_small = sweep(C, 2 * n, weighted(2 * n, n))
        k_large = sweep(C, 16, weighted(16, n))
        assert k_small == k_large, (n, k_small, k_large)


def test_weighted_keeps_fewer_entries_than_the_square():
    def count(keep, P):
        return sum((1 if k == 0 else 2) for m in range(1, P + 1) for k in range(P + 1)
                   if m + k <= P and keep(m, k))
    # ring m contributes 2 (2n + 1 - 2m) + 1 entries when that is within the order
    assert count(weighted(8, 4), 8) == 15 + 11 + 7 + 3
    assert count(square(8, 4), 8) == 15 + 13 + 11 + 9
    assert count(weighted(12, 6), 12) == 23 + 19 + 15 + 11 + 7 + 3
