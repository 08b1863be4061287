"""Seeded synthetic inputs for the signature-kernel workloads.

This module holds no arithmetic of the method: it only draws random paths.
Both the CUDA path (tests, bench) and the FP64 oracle consume its outputs;
neither imports the other.

Recipe (stand-ins for the paper's Brownian / fractional-Brownian workloads,
Sec. 3; no dataset is used):

* increments are drawn in FP64 from numpy's PCG64 (``default_rng(seed)``),
  points are the cumulative sums starting at 0, and the points are rounded to
  FP32 ONCE.  Consumers that need FP64 increments take differences of the
  FP32 points (the rounded inputs are the truth; input quantisation is not an
  error of the method).
* ``brownian``: increments iid N(0, sigma^2 / n_seg) per coordinate, optional
  constant drift added to every coordinate of every increment.
* ``collinear_increments``: every increment is ``u * r_i`` with a fixed unit
  direction u and r_i ~ U(0, 2/n_seg); u's entries carry 8 significant bits
  and r_i 16, so every FP32 product is exact and the path is exactly straight
  (the closed form I0(2 sqrt(<X,Y>)) then holds for the rounded inputs).
* ``ragged_pairs``: independent pairs with lengths U{lo..hi} segments and a
  per-path scale sigma_p ~ U(s_lo, s_hi), increments N(0, sigma_p^2 / L_p).
* ``fbm``: fractional Brownian motion on [0, 1] with Hurst index H, every
  coordinate independent, sampled exactly on the grid by circulant embedding
  of the fractional Gaussian noise covariance (the Davies-Harte method):
  gamma(k) = (|k+1|^{2H} - 2|k|^{2H} + |k-1|^{2H}) / 2 embedded in a
  circulant of size 2n, whose FFT gives non-negative eigenvalues for every
  H in (0, 1); increments are scaled by n^{-H}.

Layout: a batch of paths is a packed row-major FP32 array of shape
``(sum(lengths), d)`` plus an int64 ``lengths`` vector counting POINTS per path
(segments + 1); path p occupies rows ``[off_p, off_p + lengths[p])`` with
``off`` the exclusive prefix sum.
"""
from __future__ import annotations

import numpy as np


def _points_from_increments(inc: np.ndarray) -> np.ndarray:
    pts = np.zeros((inc.shape[0] + 1, inc.shape[1]), dtype=np.float64)
    np.cumsum(inc, axis=0, out=pts[1:])
    return pts


def brownian(n_paths: int, n_seg, d: int, sigma=1.0, seed: int = 0, drift: float = 0.0):
    """Packed FP32 points and int64 point counts for Brownian-type paths.

    ``n_seg`` may be an int or a per-path sequence; ``sigma`` likewise."""
    rng = np.random.default_rng(seed)
    segs = np.broadcast_to(np.asarray(n_seg, dtype=np.int64), (n_paths,))
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n_paths,))
    out = []
    for p in range(n_paths):
        L = int(segs[p])
        inc = rng.standard_normal((L, d)) * (sig[p] / np.sqrt(max(L, 1))) + drift
        out.append(_points_from_increments(inc).astype(np.float32))
    pts = np.ascontiguousarray(np.concatenate(out, 0)) if out else np.zeros((0, d), np.float32)
    lengths = segs.astype(np.int64) + 1
    return pts, np.ascontiguousarray(lengths)


def split(points: np.ndarray, lengths: np.ndarray):
    """List of per-path point arrays from the packed layout."""
    off = np.concatenate([[0], np.cumsum(lengths)])
    return [points[off[p]:off[p + 1]] for p in range(len(lengths))]


def pack(paths):
    """Inverse of ``split``."""
    lengths = np.array([len(p) for p in paths], dtype=np.int64)
    return np.ascontiguousarray(np.concatenate(paths, 0)), lengths


def _round_sig_bits(v: np.ndarray, bits: int) -> np.ndarray:
    m, e = np.frexp(v)
    return np.ldexp(np.round(m * (1 << bits)) / (1 << bits), e)


def collinear_increments(n_seg: int, d: int, seed: int, n_paths: int = 2):
    """FP32 increments (packed, rows = segments) of ``n_paths`` paths that all
    run along one fixed direction u; returns (increments, segment counts, u,
    per-path totals R_p = sum_i r_i) so that <X_a, X_b> = |u|^2 R_a R_b."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(d)
    u = _round_sig_bits(u / np.linalg.norm(u), 8)
    incs, totals = [], []
    for _ in range(n_paths):
        r = _round_sig_bits(rng.uniform(0.0, 2.0 / n_seg, size=n_seg), 16)
        incs.append((r[:, None] * u[None, :]).astype(np.float32))
        totals.append(float(np.sum(r.astype(np.float64))))
    segs = np.full(n_paths, n_seg, dtype=np.int64)
    return np.ascontiguousarray(np.concatenate(incs, 0)), segs, u, np.array(totals)


def ragged_pairs(n_pairs: int, lo: int, hi: int, d: int, s_lo: float, s_hi: float, seed: int):
    """Independent pairs (x_p, y_p) with their own lengths and scales.
    Returns ((X points, X lengths), (Y points, Y lengths))."""
    rng = np.random.default_rng(seed)
    lx = rng.integers(lo, hi + 1, size=n_pairs)
    ly = rng.integers(lo, hi + 1, size=n_pairs)
    sx = rng.uniform(s_lo, s_hi, size=n_pairs)
    sy = rng.uniform(s_lo, s_hi, size=n_pairs)
    seeds = rng.integers(0, 2**63 - 1, size=2)
    X = brownian(n_pairs, lx, d, sx, int(seeds[0]))
    Y = brownian(n_pairs, ly, d, sy, int(seeds[1]))
    return X, Y


def single_segment_pairs(cs, d: int = 4):
    """Pairs of one-segment paths with <dx, dy> = c exactly: dx = c e_0,
    dy = e_0.  Returns ((X points, lengths), (Y points, lengths))."""
    xs, ys = [], []
    for c in cs:
        x = np.zeros((2, d), np.float32); x[1, 0] = np.float32(c)
        y = np.zeros((2, d), np.float32); y[1, 0] = 1.0
        xs.append(x); ys.append(y)
    return pack(xs), pack(ys)


# The five workloads (sizes and seeds).  Each returns the arrays the C-ABI
# consumes.

def workload_pair_256(seed: int = 1001):
    """One pair in R^4, 256 segments each, increments N(0, 1/256)."""
    pts, lens = brownian(2, 256, 4, 1.0, seed)
    return pts, lens


def workload_gram_1024(sigma: float = 1.0, seed: int | None = None, n_paths: int = 64,
                       n_seg: int = 1024, d: int = 16):
    """B=64 paths, 1024 segments, d=16, N(0, sigma^2/1024); seed 2001 (sigma 1)
    or 2004 (sigma 4)."""
    if seed is None:
        seed = 2001 if sigma == 1.0 else 2004
    return brownian(n_paths, n_seg, d, sigma, seed)


def workload_mmd_2048(seed: int = 5001, n_paths: int = 32, n_seg: int = 2048, d: int = 8):
    """X: 32 Brownian paths, 2048 segments, d=8, N(0,1/2048); Y: the same law
    plus a drift of 0.5/2048 on every coordinate of every increment."""
    X = brownian(n_paths, n_seg, d, 1.0, seed)
    Y = brownian(n_paths, n_seg, d, 1.0, seed + 1, drift=0.5 / n_seg)
    return X, Y


def workload_ragged_512(seed: int = 4001, n_pairs: int = 512, lo: int = 64, hi: int = 8192,
                        d: int = 256):
    """512 independent pairs, lengths U{64..8192} segments, d=256,
    sigma_p ~ U(0.5, 4), increments N(0, sigma_p^2 / L_p)."""
    return ragged_pairs(n_pairs, lo, hi, d, 0.5, 4.0, seed)


def workload_long_pair(n_seg: int = 1_000_000, d: int = 8, seed: int = 3001):
    """One Brownian pair of n_seg-segment paths in R^8 as FP32 increments
    (rows = segments), N(0, 1/n_seg)."""
    rng = np.random.default_rng(seed)
    inc = (rng.standard_normal((2 * n_seg, d)) / np.sqrt(n_seg)).astype(np.float32)
    return np.ascontiguousarray(inc), np.array([n_seg, n_seg], dtype=np.int64)


def fgn_autocov(n: int, hurst: float) -> np.ndarray:
    """Autocovariance gamma(0..n-1) of unit fractional Gaussian noise."""
    k = np.arange(n, dtype=np.float64)
    h2 = 2.0 * hurst
    return 0.5 * (np.abs(k + 1) ** h2 - 2.0 * np.abs(k) ** h2 + np.abs(k - 1) ** h2)


def fbm(n_paths: int, n_seg: int, d: int, hurst: float, seed: int = 0):
    """Packed FP32 points and int64 point counts of fBM paths (Davies-Harte).

    Each path has n_seg segments on [0, 1]; each coordinate is an independent
    fBM with Hurst index ``hurst`` (increment variance n_seg^(-2H))."""
    if not 0.0 < hurst < 1.0:
        raise ValueError("hurst must be in (0, 1)")
    rng = np.random.default_rng(seed)
    n = int(n_seg)
    g = fgn_autocov(n + 1, hurst)
    circ = np.concatenate([g[:n + 1], g[n - 1:0:-1]])  # first row of the 2n circulant
    lam = np.fft.fft(circ).real
    lam = np.maximum(lam, 0.0)  # round-off only: exact eigenvalues are >= 0
    m = circ.size
    paths = []
    for _ in range(n_paths):
        inc = np.empty((n, d))
        for e in range(d):
            z = rng.standard_normal(m) + 1j * rng.standard_normal(m)
            w = np.fft.fft(np.sqrt(lam / m) * z)
            inc[:, e] = w.real[:n]
        paths.append(_points_from_increments(inc * float(n) ** (-hurst)).astype(np.float32))
    return pack(paths)
