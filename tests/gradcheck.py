"""Gradient comparison used by the GPU gradient tests."""
import numpy as np


def assert_grad_close(got, ref, rtol=1e-4, small=1e-3):
    """Per-coordinate relative error <= rtol; coordinates whose reference is
    below `small` of the largest one are held to rtol * small * max|ref| in
    absolute terms instead (a relative error of a near-zero difference of
    large contributions is not meaningful)."""
    got, ref = np.asarray(got), np.asarray(ref)
    big = np.abs(ref).max()
    bound = np.maximum(rtol * np.abs(ref), rtol * small * big)
    err = np.abs(got - ref)
    assert (err <= bound).all(), list(zip(got[err > bound], ref[err > bound]))
