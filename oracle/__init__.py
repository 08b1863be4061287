"""FP64 CPU oracle for the signature kernel -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path never does: it has no CPU fallback.

The oracle is plain C (``sigk_oracle.c``), compiled with gcc into
``oracle/_build/liboracle.so`` and called through ctypes.  It shares no code
with the CUDA path.  Inputs are FP64 increment arrays (``L x d``, one row per
segment); a path with one point has ``L = 0`` segments.

Functions (each cites the passage it follows; see the C file for details):

* ``series_pair``  -- tile-centred local power series (Sec. 2.3), truncation
  order ``N`` (App. A.7); ``N = 24`` is exact to FP64 for the inputs used here.
* ``fd_pair`` / ``fd_richardson`` -- finite-difference Goursat scheme derived
  from the Volterra form (Sec. 2.1) with dyadic refinement and Richardson
  extrapolation.
* ``chen_pair``    -- truncated signature inner product via Chen's identity.
* ``tile_map``     -- one tile of the tile-centred expansion (for unit pins).
* ``series_gram`` / ``series_pairs`` / ``mmd2`` -- batched forms.
* ``grad_fd``      -- central finite differences of ``series_pair`` with one
  Richardson step (FP64), the gradient reference.

Parity is pinned by ``tests/test_oracle.py`` against closed forms (Bessel
I0/J0 for straight paths, the corrected worked example of Sec. 2.2.2, the
operator-power lemma of App. A.4), brute force (Chen vs FD vs series),
invariants, and the Gram error bound of App. A.7.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sigk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_N = 24


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP across pairs)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build()
        lib = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.POINTER(ctypes.c_int64)
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_tile_map.argtypes = [f64, i32, D, D, D, D]
        lib.orc_tile_map.restype = None
        lib.orc_series_pair.argtypes = [D, i64, D, i64, i32, i32, D]
        lib.orc_fd_pair.argtypes = [D, i64, D, i64, i32, i32, D]
        lib.orc_fd_richardson.argtypes = [D, i64, D, i64, i32, i32, D]
        lib.orc_chen_pair.argtypes = [D, i64, D, i64, i32, i32, D, D]
        lib.orc_series_gram.argtypes = [D, I64, i64, D, I64, i64, i32, i32, i32, D]
        lib.orc_series_pairs.argtypes = [D, I64, D, I64, i64, i32, i32, i32, D]
        lib.orc_mmd2_from_grams.argtypes = [D, i64, D, i64, D, i32]
        lib.orc_mmd2_from_grams.restype = f64
        lib.orc_num_threads.restype = i32
        for name in ("orc_series_pair", "orc_fd_pair", "orc_fd_richardson", "orc_chen_pair",
                     "orc_series_gram", "orc_series_pairs"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _as_inc(z, d=None) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
    if z.ndim == 1:
        z = z.reshape(-1, 1 if d is None else d)
    return z


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} failed with code {rc}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def tile_map(rho: float, alpha, beta, N: int | None = None):
    """One tile of the tile-centred expansion: returns (alpha_out, beta_out)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if N is None:
        N = len(alpha) - 1
    assert len(alpha) == N + 1 and len(beta) == N + 1
    ao = np.zeros(N + 1)
    bo = np.zeros(N + 1)
    _load().orc_tile_map(float(rho), int(N), _dptr(alpha), _dptr(beta), _dptr(ao), _dptr(bo))
    return ao, bo


def series_pair(dx, dy, N: int = DEFAULT_N) -> float:
    dx = _as_inc(dx)
    dy = _as_inc(dy, dx.shape[1])
    assert dx.shape[1] == dy.shape[1]
    out = ctypes.c_double()
    rc = _load().orc_series_pair(_dptr(dx), dx.shape[0], _dptr(dy), dy.shape[0], dx.shape[1],
                                 int(N), ctypes.byref(out))
    _check(rc, "series_pair")
    return out.value


def fd_pair(dx, dy, lam: int) -> float:
    dx = _as_inc(dx)
    dy = _as_inc(dy, dx.shape[1])
    out = ctypes.c_double()
    rc = _load().orc_fd_pair(_dptr(dx), dx.shape[0], _dptr(dy), dy.shape[0], dx.shape[1],
                             int(lam), ctypes.byref(out))
    _check(rc, "fd_pair")
    return out.value


def fd_richardson(dx, dy, lam0: int):
    """Returns (k_lam0, k_lam0+1, k_lam0+2, extrapolated)."""
    dx = _as_inc(dx)
    dy = _as_inc(dy, dx.shape[1])
    out = np.zeros(4)
    rc = _load().orc_fd_richardson(_dptr(dx), dx.shape[0], _dptr(dy), dy.shape[0], dx.shape[1],
                                   int(lam0), _dptr(out))
    _check(rc, "fd_richardson")
    return tuple(out)


def chen_pair(dx, dy, M: int, levels: bool = False):
    dx = _as_inc(dx)
    dy = _as_inc(dy, dx.shape[1])
    out = ctypes.c_double()
    lv = np.zeros(M + 1)
    rc = _load().orc_chen_pair(_dptr(dx), dx.shape[0], _dptr(dy), dy.shape[0], dx.shape[1],
                               int(M), ctypes.byref(out), _dptr(lv))
    _check(rc, "chen_pair")
    return (out.value, lv) if levels else out.value


def _pack(paths, d=None):
    paths = [_as_inc(p, d) for p in paths]
    d = paths[0].shape[1] if paths else (d or 1)
    lens = np.array([p.shape[0] for p in paths], dtype=np.int64)
    packed = np.ascontiguousarray(
        np.concatenate([p.reshape(-1, d) for p in paths], 0) if paths else np.zeros((0, d)))
    return packed, lens, d


def series_gram(xs, ys=None, N: int = DEFAULT_N, threads: int = 0) -> np.ndarray:
    """Gram matrix G[a, b] = k(x_a, y_b) (ys=None: ys = xs)."""
    X, lx, d = _pack(xs)
    if ys is None:
        Y, ly = X, lx
    else:
        Y, ly, _ = _pack(ys, d)
    G = np.zeros((len(lx), len(ly)))
    rc = _load().orc_series_gram(_dptr(X), _iptr(lx), len(lx), _dptr(Y), _iptr(ly), len(ly), d,
                                 int(N), int(threads), _dptr(G))
    _check(rc, "series_gram")
    return G


def series_pairs(xs, ys, N: int = DEFAULT_N, threads: int = 0) -> np.ndarray:
    """k(x_p, y_p) for independent pairs p."""
    X, lx, d = _pack(xs)
    Y, ly, _ = _pack(ys, d)
    assert len(lx) == len(ly)
    out = np.zeros(len(lx))
    rc = _load().orc_series_pairs(_dptr(X), _iptr(lx), _dptr(Y), _iptr(ly), len(lx), d, int(N),
                                  int(threads), _dptr(out))
    _check(rc, "series_pairs")
    return out


def mmd2_from_grams(Kxx, Kyy, Kxy, unbiased: bool = True) -> float:
    Kxx = np.ascontiguousarray(Kxx, dtype=np.float64)
    Kyy = np.ascontiguousarray(Kyy, dtype=np.float64)
    Kxy = np.ascontiguousarray(Kxy, dtype=np.float64)
    return float(_load().orc_mmd2_from_grams(_dptr(Kxx), Kxx.shape[0], _dptr(Kyy), Kyy.shape[0],
                                             _dptr(Kxy), int(bool(unbiased))))


def mmd2(xs, ys, N: int = DEFAULT_N, unbiased: bool = True, threads: int = 0) -> float:
    """Signature-kernel MMD^2 between two samples of paths (U- or V-statistic)."""
    Kxx = series_gram(xs, None, N, threads)
    Kyy = series_gram(ys, None, N, threads)
    Kxy = series_gram(xs, ys, N, threads)
    return mmd2_from_grams(Kxx, Kyy, Kxy, unbiased)


def grad_fd(f, z: np.ndarray, coords, rel_step: float = 1e-4):
    """Central differences of scalar f at increments z for the given flat
    coordinates, with one Richardson step (h and h/2): error O(h^4)."""
    z = np.array(z, dtype=np.float64)
    flat = z.reshape(-1)
    scale = max(np.abs(flat).max(), 1e-300)
    out = []
    for c in coords:
        h = rel_step * scale
        vals = []
        for hh in (h, h / 2):
            zp = flat.copy(); zp[c] += hh
            zm = flat.copy(); zm[c] -= hh
            vals.append((f(zp.reshape(z.shape)) - f(zm.reshape(z.shape))) / (2 * hh))
        out.append((4 * vals[1] - vals[0]) / 3)
    return np.array(out)
