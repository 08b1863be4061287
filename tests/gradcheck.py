"""Gradient comparison used by the GPU gradient tests.

The GPU gradient is the exact adjoint of the FP32 scheme; the reference is a
central finite difference (FP64) of the oracle.  A gradient coordinate is often
a small difference of large contributions -- of the two segments that share a
point (a point moves the end of one increment and the start of the next), and
of the many pairs a path enters in a Gram or an MMD -- and each contribution
carries the FP32 scheme's own relative rounding, about 1e-6 on the path
lengths of these tests (the forward parity tests measure 1e-7 .. 3e-6).  So a
coordinate is held to

    |got - ref| <= RTOL * |ref| + EPS32 * S,

with RTOL = 1e-4 (the differentiation workload's tolerance), S the sum of the
magnitudes of the contributions that cancel in that coordinate (from the same
finite differences), and EPS32 = 4e-6.  Where no contribution scale is
available, coordinates below 1e-3 of the largest are held to RTOL * 1e-3 of
the largest instead.  The relative error of the whole gradient vector over
the checked coordinates must also stay below RTOL.
"""
import numpy as np

RTOL = 1e-4
EPS32 = 4e-6


def assert_grad_close(got, ref, scale=None, rtol=RTOL, eps=EPS32, small=1e-3):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    big = np.abs(ref).max()
    if scale is None:
        bound = np.maximum(rtol * np.abs(ref), rtol * small * big)
    else:
        bound = rtol * np.abs(ref) + eps * np.asarray(scale, dtype=np.float64)
    err = np.abs(got - ref)
    assert (err <= bound).all(), [(g, r, e / max(abs(r), 1e-300), b)
                                  for g, r, e, b in zip(got, ref, err, bound) if e > b]
    assert np.linalg.norm(got - ref) <= rtol * np.linalg.norm(ref), (
        np.linalg.norm(got - ref) / np.linalg.norm(ref))


def _central(f, z, idx, h, richardson):
    """d f / d z[idx] by a central difference (one Richardson step: error
    O(h^4))."""
    vals = []
    for hh in ((h, h / 2) if richardson else (h,)):
        zp = z.copy(); zp.reshape(-1)[idx] += hh
        zm = z.copy(); zm.reshape(-1)[idx] -= hh
        vals.append((f(zp) - f(zm)) / (2 * hh))
    return (4 * vals[1] - vals[0]) / 3 if richardson else vals[0]


def point_gradient_terms(terms, inc, coords, h=1e-3, richardson=True):
    """Reference gradient of sum_t w_t f_t(inc) with respect to POINT
    coordinates of the path whose increments are `inc` (L x d), and the
    contribution scale S of each coordinate.

    terms: list of (w_t, f_t), f_t a function of this path's increments (one
    pair's kernel value, say).  Point (q, e) is the end of increment q-1 and the
    start of increment q, so its derivative is D_{q-1,e} - D_{q,e}; S sums
    |w_t| (|D_{q-1,e} f_t| + |D_{q,e} f_t|) over the terms."""
    L, d = inc.shape
    ref, S = [], []
    for c in coords:
        q, e = divmod(int(c), d)
        r = s = 0.0
        for w, f in terms:
            lo = _central(f, inc, (q - 1) * d + e, h, richardson) if q >= 1 else 0.0
            hi = _central(f, inc, q * d + e, h, richardson) if q < L else 0.0
            r += w * (lo - hi)
            s += abs(w) * (abs(lo) + abs(hi))
        ref.append(r)
        S.append(s)
    return np.array(ref), np.array(S)


def increment_gradient_terms(terms, inc, coords, h=1e-3, richardson=True):
    """As point_gradient_terms, with respect to the increments themselves."""
    ref, S = [], []
    for c in coords:
        r = s = 0.0
        for w, f in terms:
            g = _central(f, inc, int(c), h, richardson)
            r += w * g
            s += abs(w * g)
        ref.append(r)
        S.append(s)
    return np.array(ref), np.array(S)
