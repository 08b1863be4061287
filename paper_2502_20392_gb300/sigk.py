"""Thin ctypes binding of libsigk.so (include/sigk.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no CPU fallback -- if the library or a GPU is missing, every
call raises.  PyTorch supplies device memory and the current stream.

Conventions (see include/sigk.h): a batch of paths is a packed FP32 CUDA
tensor of shape ``(sum(lengths), d)`` plus an int64 CUDA tensor ``lengths``
(points per path, or segments per path with ``increments=True``).
"""
from __future__ import annotations

import ctypes
import os
import re
import warnings
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsigk.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sigk.h")

OP_PAIRS, OP_GRAM, OP_MMD = 0, 1, 2
FLAG_INCREMENTS, FLAG_GRAM_FULL, FLAG_MMD_BIASED, FLAG_FP64, FLAG_PAIR_MAJOR, FLAG_REPLAY = 1, 2, 4, 8, 16, 32
FLAG_TEST_WITHHOLD_SEAM = 64
FLAG_NO_TENSOR = 128
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_LENGTH", -3: "ERR_NONFINITE", -4: "ERR_WORKSPACE",
          -5: "ERR_CUDA", -6: "ERR_TIMEOUT", -7: "ERR_ACCURACY", -8: "ERR_UNSUPPORTED",
          -9: "ERR_BOUNDS"}
ERR_ACCURACY = -7


class SigkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sigk {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("rings", ctypes.c_int), ("flags", ctypes.c_int),
                ("grid_ctas", ctypes.c_int), ("max_len", ctypes.c_int64),
                ("refine_c", ctypes.c_float), ("wait_ms", ctypes.c_int), ("ring_tol", ctypes.c_float)]


@dataclass
class Opts:
    order: int = 8
    rings: int = 4
    flags: int = 0
    grid_ctas: int = 0
    max_len: int = 8193
    refine_c: float = 0.0
    wait_ms: int = 0
    ring_tol: float = 0.0

    def c(self) -> _Opts:
        return _Opts(self.order, self.rings, self.flags, self.grid_ctas, self.max_len,
                     self.refine_c, self.wait_ms, self.ring_tol)


_lib = None


def exported_functions() -> list[str]:
    """Function names declared in include/sigk.h."""
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sigk_[a-z_0-9]+)\s*\(", src)))


def load(path: str | None = None):
    """Load libsigk.so (built by paper_2502_20392_gb300.build); `path`, else
    the SIGK_LIB environment variable, selects another build of it (e.g. the
    bounds-checked one of build(debug=True))."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("SIGK_LIB") or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libsigk.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    op = ctypes.POINTER(_Opts)
    lib.sigk_workspace_size.argtypes = [i32, i64, i64, i32, op]
    lib.sigk_workspace_size.restype = sz
    lib.sigk_pairs.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp, sz, vp, op]
    lib.sigk_gram.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, vp, sz, vp, op]
    lib.sigk_mmd.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, vp, vp, sz, vp, op]
    lib.sigk_plan.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, ctypes.c_double, vp, sz, vp, op, op]
    lib.sigk_backward_workspace_size.argtypes = [i32, i64, i64, i32, op]
    lib.sigk_backward_workspace_size.restype = sz
    lib.sigk_backward.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, vp, vp, vp, vp, vp, sz, vp, op]
    lib.sigk_forward_train.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, vp, vp, sz, vp, op]
    lib.sigk_adjoint.argtypes = [i32, i64, i64, i32, vp, vp, vp, vp, sz, vp, op]
    lib.sigk_sync_status.argtypes = [vp, sz, vp]
    lib.sigk_counters.argtypes = [vp, sz, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sigk_autotune.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, vp, vp, sz, vp, op, i32, op,
                                  ctypes.POINTER(ctypes.c_double)]
    lib.sigk_tune_key.argtypes = [i32, i64, i64, i32, op, ctypes.c_char_p, sz]
    lib.sigk_tune_cache_put.argtypes = [ctypes.c_char_p, i32, i32, ctypes.c_double]
    lib.sigk_tune_cache_get.argtypes = [ctypes.c_char_p, op, ctypes.POINTER(ctypes.c_double)]
    lib.sigk_tune_cache_save.argtypes = [ctypes.c_char_p]
    lib.sigk_tune_cache_load.argtypes = [ctypes.c_char_p]
    lib.sigk_tune_cache_size.restype = i64
    lib.sigk_tune_cache_clear.restype = None
    for name in ("sigk_autotune", "sigk_tune_key", "sigk_tune_cache_put", "sigk_tune_cache_get",
                 "sigk_tune_cache_save", "sigk_tune_cache_load"):
        getattr(lib, name).restype = i32
    lib.sigk_ring_histogram.argtypes = [vp, sz, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sigk_launch_info.argtypes = [i32, i64, i64, i32, op, i32, ctypes.POINTER(ctypes.c_int)]
    lib.sigk_launch_info.restype = i32
    lib.sigk_profile_events.argtypes = [vp, vp]
    lib.sigk_profile_events.restype = None
    lib.sigk_last_error.restype = ctypes.c_char_p
    lib.sigk_version.restype = ctypes.c_char_p
    for name in ("sigk_pairs", "sigk_gram", "sigk_mmd", "sigk_plan", "sigk_sync_status",
                 "sigk_counters", "sigk_ring_histogram", "sigk_backward"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(st: int):
    if st != 0:
        raise SigkError(st, load().sigk_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _paths(pts, lens):
    if not (pts.is_cuda and lens.is_cuda):
        raise ValueError("paths and lengths must be CUDA tensors")
    if pts.dtype != torch.float32 or lens.dtype != torch.int64:
        raise TypeError("paths must be float32 and lengths int64")
    if pts.dim() != 2:
        raise ValueError("paths must be a 2-D (rows, d) tensor")
    return pts.contiguous(), lens.contiguous()


class Workspace:
    """Caller-owned device scratch, grown on demand (torch allocates it)."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        return self.buf


_default_ws = {}


def _ws(ws, device):
    if ws is None:
        ws = _default_ws.setdefault(device, Workspace())
    return ws


def workspace_size(op: int, n_x: int, n_y: int, d: int, opts: Opts) -> int:
    o = opts.c()
    n = load().sigk_workspace_size(op, n_x, n_y, d, ctypes.byref(o))
    if n == 0:
        raise SigkError(-1, "workspace_size rejected the arguments")
    return int(n)


def sync_status(ws: Workspace):
    """Wait for the stream and raise if a device-side error was recorded."""
    if ws.buf is None:
        torch.cuda.current_stream().synchronize()
        return
    lib = load()
    _check(lib.sigk_sync_status(_ptr(ws.buf), ws.buf.numel(), _stream()))


def profile_events(start=None, stop=None):
    """Record torch.cuda.Event pair around every later solver launch (None: off)."""
    h = (lambda e: ctypes.c_void_p(e.cuda_event) if e is not None else ctypes.c_void_p(0))
    load().sigk_profile_events(h(start), h(stop))


def counters(ws: Workspace):
    out = (ctypes.c_double * 4)()
    _check(load().sigk_counters(_ptr(ws.buf), ws.buf.numel(), _stream(), out))
    return list(out)


def ring_histogram(ws: Workspace):
    """Tiles of the last forward on ws solved with <= 2, 3-4, 5-6, 7-8 rings (adaptive
    ring counts only)."""
    out = (ctypes.c_double * 4)()
    _check(load().sigk_ring_histogram(_ptr(ws.buf), ws.buf.numel(), _stream(), out))
    return list(out)


def pairs(X, len_x, Y, len_y, opts: Opts | None = None, out=None, ws: Workspace | None = None,
          check: bool = True):
    """k(x_p, y_p) for independent pairs -> FP64 CUDA tensor [n_pairs]."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    Y, len_y = _paths(Y, len_y)
    n, d = len_x.numel(), X.shape[1]
    if len_y.numel() != n or Y.shape[1] != d:
        raise ValueError("x and y batches must match in count and dimension")
    out = out if out is not None else torch.empty(n, dtype=torch.float64, device=X.device)
    ws = _ws(ws, X.device)
    buf = ws.get(workspace_size(OP_PAIRS, n, n, d, opts), X.device)
    o = opts.c()
    _check(load().sigk_pairs(_ptr(X), _ptr(len_x), _ptr(Y), _ptr(len_y), n, d, _ptr(out),
                             _ptr(buf), buf.numel(), _stream(), ctypes.byref(o)))
    if check:
        sync_status(ws)
    return out


def gram(X, len_x, Y=None, len_y=None, opts: Opts | None = None, out=None,
         ws: Workspace | None = None, check: bool = True):
    """Gram matrix k(x_a, y_b) -> FP64 CUDA tensor [n_x, n_y] (Y=None: Y = X)."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    n_x, d = len_x.numel(), X.shape[1]
    if Y is not None:
        Y, len_y = _paths(Y, len_y)
        n_y = len_y.numel()
    else:
        n_y = 0
    out = out if out is not None else torch.empty((n_x, n_y or n_x), dtype=torch.float64,
                                                  device=X.device)
    ws = _ws(ws, X.device)
    buf = ws.get(workspace_size(OP_GRAM, n_x, n_y, d, opts), X.device)
    o = opts.c()
    _check(load().sigk_gram(_ptr(X), _ptr(len_x), n_x, _ptr(Y), _ptr(len_y), n_y, d, _ptr(out),
                            _ptr(buf), buf.numel(), _stream(), ctypes.byref(o)))
    if check:
        sync_status(ws)
    return out


def mmd(X, len_x, Y, len_y, opts: Opts | None = None, gram_out=None,
        ws: Workspace | None = None, check: bool = True):
    """Signature-kernel MMD^2 -> FP64 CUDA tensor [1]."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    Y, len_y = _paths(Y, len_y)
    m, n, d = len_x.numel(), len_y.numel(), X.shape[1]
    out = torch.empty(1, dtype=torch.float64, device=X.device)
    ws = _ws(ws, X.device)
    buf = ws.get(workspace_size(OP_MMD, m, n, d, opts), X.device)
    o = opts.c()
    _check(load().sigk_mmd(_ptr(X), _ptr(len_x), m, _ptr(Y), _ptr(len_y), n, d, _ptr(out),
                           _ptr(gram_out), _ptr(buf), buf.numel(), _stream(), ctypes.byref(o)))
    if check:
        sync_status(ws)
    return out


def backward_workspace_size(op: int, n_x: int, n_y: int, d: int, opts: Opts) -> int:
    o = opts.c()
    n = load().sigk_backward_workspace_size(op, n_x, n_y, d, ctypes.byref(o))
    if n == 0:
        raise SigkError(-1, "backward_workspace_size rejected the arguments")
    return int(n)


def backward(op: int, X, len_x, Y, len_y, grad_out, opts: Opts | None = None,
             need_x: bool = True, need_y: bool = True, ws: Workspace | None = None,
             check: bool = True):
    """Adjoint of pairs / gram / mmd.  Returns (grad_X, grad_Y, value):
    gradients w.r.t. the points (increments with FLAG_INCREMENTS) as FP32
    tensors shaped like X and Y (None where not requested; for a Gram of X with
    itself grad_Y is None), and the forward output recomputed by the call."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    n_x, d = len_x.numel(), X.shape[1]
    self_gram = op == OP_GRAM and Y is None
    if Y is not None:
        Y, len_y = _paths(Y, len_y)
        n_y = len_y.numel()
    else:
        n_y = 0 if self_gram else n_x
    if op == OP_PAIRS:
        n_y = n_x
        vshape = (n_x,)
    elif op == OP_GRAM:
        vshape = (n_x, n_y or n_x)
    else:
        vshape = (1,)
    value = torch.empty(vshape, dtype=torch.float64, device=X.device)
    gout = grad_out.to(device=X.device, dtype=torch.float64).contiguous()
    gX = torch.empty_like(X) if need_x else None
    gY = torch.empty_like(Y) if (need_y and Y is not None and not self_gram) else None
    ws = _ws(ws, X.device)
    buf = ws.get(backward_workspace_size(op, n_x, n_y, d, opts), X.device)
    o = opts.c()
    _check(load().sigk_backward(op, _ptr(X), _ptr(len_x), n_x, _ptr(Y), _ptr(len_y), n_y, d,
                                _ptr(gout), _ptr(gX), _ptr(gY), _ptr(value), _ptr(buf),
                                buf.numel(), _stream(), ctypes.byref(o)))
    if check:
        sync_status(ws)
    return gX, gY, value


class TrainState:
    """What forward_train leaves for adjoint: the workspace (seams and tile
    records of the training forward) and the inputs it refers to, which must
    stay unchanged until the adjoint has run."""

    def __init__(self, op, X, len_x, Y, len_y, n_x, n_y, d, opts, ws):
        self.op, self.X, self.len_x, self.Y, self.len_y = op, X, len_x, Y, len_y
        self.n_x, self.n_y, self.d, self.opts, self.ws = n_x, n_y, d, opts, ws


def _train_shapes(op, X, len_x, Y, len_y):
    X, len_x = _paths(X, len_x)
    n_x, d = len_x.numel(), X.shape[1]
    self_gram = op == OP_GRAM and Y is None
    if Y is not None:
        Y, len_y = _paths(Y, len_y)
        n_y = len_y.numel()
    else:
        n_y = 0 if self_gram else n_x
    if op == OP_PAIRS:
        n_y = n_x
        vshape = (n_x,)
    elif op == OP_GRAM:
        vshape = (n_x, n_y or n_x)
    else:
        vshape = (1,)
    return X, len_x, Y, len_y, n_x, n_y, d, vshape


def forward_train(op: int, X, len_x, Y, len_y, opts: Opts | None = None,
                  ws: Workspace | None = None, out=None, check: bool = True):
    """Training forward of pairs / gram / mmd: returns (value, state); the
    state feeds adjoint() once the upstream gradient is known.  The state owns
    its workspace (a fresh one unless `ws` is given)."""
    opts = opts or Opts()
    X, len_x, Y, len_y, n_x, n_y, d, vshape = _train_shapes(op, X, len_x, Y, len_y)
    value = out if out is not None else torch.empty(vshape, dtype=torch.float64, device=X.device)
    ws = ws if ws is not None else Workspace()
    buf = ws.get(backward_workspace_size(op, n_x, n_y, d, opts), X.device)
    o = opts.c()
    _check(load().sigk_forward_train(op, _ptr(X), _ptr(len_x), n_x, _ptr(Y), _ptr(len_y), n_y, d,
                                     _ptr(value), _ptr(buf), buf.numel(), _stream(),
                                     ctypes.byref(o)))
    if check:
        sync_status(ws)
    return value, TrainState(op, X, len_x, Y, len_y, n_x, n_y, d, opts, ws)


def adjoint(state: TrainState, grad_out, need_x: bool = True, need_y: bool = True,
            check: bool = True):
    """Adjoint from a forward_train state: (grad_X, grad_Y) as in backward()."""
    X, Y = state.X, state.Y
    gout = grad_out.to(device=X.device, dtype=torch.float64).contiguous()
    gX = torch.empty_like(X) if need_x else None
    gY = torch.empty_like(Y) if (need_y and Y is not None and state.n_y > 0) else None
    buf = state.ws.buf
    o = state.opts.c()
    _check(load().sigk_adjoint(state.op, state.n_x, state.n_y, state.d, _ptr(gout), _ptr(gX),
                               _ptr(gY), _ptr(buf), buf.numel(), _stream(), ctypes.byref(o)))
    if check:
        sync_status(state.ws)
    return gX, gY


# The autograd functions run the training forward when an input needs a
# gradient and keep its state (seams, tile records: the workspace) on the
# context until backward, which then runs only the adjoint.

class _PairsFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, len_x, len_y, opts):
        ctx.opts = opts
        if not (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            return pairs(X.detach(), len_x, Y.detach(), len_y, opts=opts)
        value, ctx.state = forward_train(OP_PAIRS, X.detach(), len_x, Y.detach(), len_y, opts)
        return value

    @staticmethod
    def backward(ctx, g):
        gX, gY = adjoint(ctx.state, g, need_x=ctx.needs_input_grad[0],
                         need_y=ctx.needs_input_grad[1])
        return gX, gY, None, None, None


class _GramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, len_x, len_y, opts):
        ctx.self_gram = Y is None
        ctx.opts = opts
        Yd = None if Y is None else Y.detach()
        if not (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            return gram(X.detach(), len_x, Yd, len_y, opts=opts)
        value, ctx.state = forward_train(OP_GRAM, X.detach(), len_x, Yd, len_y, opts)
        return value

    @staticmethod
    def backward(ctx, g):
        gX, gY = adjoint(ctx.state, g, need_x=ctx.needs_input_grad[0],
                         need_y=(not ctx.self_gram) and ctx.needs_input_grad[1])
        return gX, (None if ctx.self_gram else gY), None, None, None


class _MMDFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, len_x, len_y, opts):
        ctx.opts = opts
        if not (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            return mmd(X.detach(), len_x, Y.detach(), len_y, opts=opts)
        value, ctx.state = forward_train(OP_MMD, X.detach(), len_x, Y.detach(), len_y, opts)
        return value

    @staticmethod
    def backward(ctx, g):
        gX, gY = adjoint(ctx.state, g, need_x=ctx.needs_input_grad[0],
                         need_y=ctx.needs_input_grad[1])
        return gX, gY, None, None, None


def sig_kernel_pairs(X, len_x, Y, len_y, opts: Opts | None = None):
    """Differentiable k(x_p, y_p) (torch.autograd)."""
    return _PairsFn.apply(X, Y, len_x, len_y, opts or Opts())


def sig_kernel_gram(X, len_x, Y=None, len_y=None, opts: Opts | None = None):
    """Differentiable Gram matrix (torch.autograd); Y=None: Gram of X with itself."""
    return _GramFn.apply(X, Y, len_x, len_y, opts or Opts())


def sig_kernel_mmd(X, len_x, Y, len_y, opts: Opts | None = None):
    """Differentiable signature-kernel MMD^2 (torch.autograd)."""
    return _MMDFn.apply(X, Y, len_x, len_y, opts or Opts())


def plan(op: int, X, len_x, Y=None, len_y=None, tol: float = 1e-5, opts: Opts | None = None,
         ws: Workspace | None = None) -> Opts:
    """A-priori (order, rings) for relative tolerance `tol` from device
    statistics of the increments (synchronises the stream)."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    n_x, d = len_x.numel(), X.shape[1]
    if Y is not None:
        Y, len_y = _paths(Y, len_y)
        n_y = len_y.numel()
    else:
        n_y = 0 if op == OP_GRAM else n_x
    big = Opts(order=16, rings=8, flags=opts.flags, grid_ctas=opts.grid_ctas, max_len=opts.max_len,
               refine_c=opts.refine_c, wait_ms=opts.wait_ms)
    nb = workspace_size(op, n_x, n_y if op != OP_PAIRS else n_x, d, big)
    npairs = n_x if op == OP_PAIRS else (n_x * (n_x + 1) // 2 if n_y == 0 else
                                         (n_x * n_y if op == OP_GRAM else (n_x + n_y) ** 2))
    nb += 8 * (12 * npairs + (n_x + n_y) ** 2 + n_x * max(n_y, n_x)) + 4096
    ws = _ws(ws, X.device)
    buf = ws.get(nb, X.device)
    o_in = opts.c()
    o_out = _Opts()
    st = load().sigk_plan(op, _ptr(X), _ptr(len_x), n_x, _ptr(Y), _ptr(len_y), n_y, d,
                          float(tol), _ptr(buf), buf.numel(), _stream(), ctypes.byref(o_in),
                          ctypes.byref(o_out))
    if st == ERR_ACCURACY:  # the finest plan is still returned
        warnings.warn(f"sigk.plan: tolerance {tol:g} not certified by the a-priori rule "
                      f"({load().sigk_last_error().decode()})", RuntimeWarning)
    else:
        _check(st)
    return _from_c(o_out)


def _from_c(o: "_Opts") -> Opts:
    return Opts(o.order, o.rings, o.flags, o.grid_ctas, o.max_len, o.refine_c, o.wait_ms, o.ring_tol)


def autotune(op: int, X, len_x, Y=None, len_y=None, opts: Opts | None = None,
             allow_fma_gram: bool = False, ws: Workspace | None = None):
    """Times the op under each candidate launch layout on these inputs and
    returns (the fastest Opts, its milliseconds per call); the choice is cached
    in the library under the call's shape class and merged by later plans."""
    opts = opts or Opts()
    X, len_x = _paths(X, len_x)
    n_x, d = len_x.numel(), X.shape[1]
    if Y is not None:
        Y, len_y = _paths(Y, len_y)
        n_y = len_y.numel()
    else:
        n_y = 0 if op == OP_GRAM else n_x
    nn = n_y if op != OP_PAIRS else n_x
    sizes = [workspace_size(op, n_x, nn, d, opts)]
    out = torch.empty(max(1, n_x if op == OP_PAIRS else (n_x * (n_y or n_x))), dtype=torch.float64,
                      device=X.device)
    ws = _ws(ws, X.device)
    buf = ws.get(max(sizes), X.device)
    o_in, o_out, ms = opts.c(), _Opts(), ctypes.c_double()
    _check(load().sigk_autotune(op, _ptr(X), _ptr(len_x), n_x, _ptr(Y), _ptr(len_y), n_y, d, _ptr(out),
                                _ptr(buf), buf.numel(), _stream(), ctypes.byref(o_in),
                                int(allow_fma_gram), ctypes.byref(o_out), ctypes.byref(ms)))
    return _from_c(o_out), ms.value


def tune_key(op: int, n_x: int, n_y: int, d: int, opts: Opts) -> str:
    buf = ctypes.create_string_buffer(256)
    o = opts.c()
    _check(load().sigk_tune_key(op, n_x, n_y, d, ctypes.byref(o), buf, 256))
    return buf.value.decode()


def tune_cache_put(key: str, grid_ctas: int, flags: int, ms: float):
    _check(load().sigk_tune_cache_put(key.encode(), grid_ctas, flags, ms))


def tune_cache_get(key: str, opts: Opts):
    """opts with the cached layout of `key` merged in, or None if absent."""
    o, ms = opts.c(), ctypes.c_double()
    if load().sigk_tune_cache_get(key.encode(), ctypes.byref(o), ctypes.byref(ms)) != 0:
        return None
    return _from_c(o), ms.value


def tune_cache_save(path: str):
    _check(load().sigk_tune_cache_save(path.encode()))


def tune_cache_load(path: str):
    _check(load().sigk_tune_cache_load(path.encode()))


def tune_cache_size() -> int:
    return int(load().sigk_tune_cache_size())


def tune_cache_clear():
    load().sigk_tune_cache_clear()


def launch_info(op: int, n_x: int, n_y: int, d: int, opts: Opts, train: bool = False) -> dict:
    """The launch configuration the library would use (no launch)."""
    out = (ctypes.c_int * 6)()
    o = opts.c()
    _check(load().sigk_launch_info(op, n_x, n_y, d, ctypes.byref(o), int(train), out))
    return {"grid": out[0], "ctas_per_sm": out[1], "threads": out[2], "smem_bytes": out[3],
            "rows_per_lane": out[4], "kernel": ("register", "fma-two-phase", "tensor-core")[out[5]]}
