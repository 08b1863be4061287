"""GPU test of sigk_pairs_static, the entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
It must give the same k values as sigk_pairs with a caller workspace, on two
calls in a row (the second call reuses the static scratch the first left
behind).  Collected last so that a failing run has already run every other
test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_scratch_matches_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20392_gb300 import build, sigk, synth
    build.build()
    lib = sigk.load()
    lib.sigk_pairs_static.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(sigk._Opts)]
    lib.sigk_pairs_static.restype = ctypes.c_int
    lib.sigk_static_sync_status.argtypes = [ctypes.c_void_p]
    lib.sigk_static_sync_status.restype = ctypes.c_int
    dev = torch.device("cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((31, 32)):
        (X, lx), (Y, ly) = synth.ragged_pairs(24, 1, 600, 8, 0.5, 2.0, seed=seed)
        Xd, lxd = torch.from_numpy(X).to(dev), torch.from_numpy(lx).to(dev)
        Yd, lyd = torch.from_numpy(Y).to(dev), torch.from_numpy(ly).to(dev)
        opts = sigk.Opts(order=10, rings=5, max_len=600)
        ref = sigk.pairs(Xd, lxd, Yd, lyd, opts=opts).cpu().numpy()
        out = torch.full((24,), float("nan"), dtype=torch.float64, device=dev)
        o = opts.c()
        st = lib.sigk_pairs_static(Xd.data_ptr(), lxd.data_ptr(), Yd.data_ptr(), lyd.data_ptr(),
                                   24, 8, out.data_ptr(), stream, ctypes.byref(o))
        assert st == 0, lib.sigk_last_error()
        assert lib.sigk_static_sync_status(stream) == 0, lib.sigk_last_error()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-6, err_msg=f"call {call}")
    # a problem that cannot fit in the static scratch is refused before launch
    big = sigk.Opts(order=16, rings=6, max_len=4_000_000)
    o = big.c()
    st = lib.sigk_pairs_static(Xd.data_ptr(), lxd.data_ptr(), Yd.data_ptr(), lyd.data_ptr(),
                               24, 8, out.data_ptr(), stream, ctypes.byref(o))
    assert st == -4 and b"static scratch" in lib.sigk_last_error()
