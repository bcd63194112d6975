"""The prior-art context library (the paper's Thrust / CUB variants, used
only by `bench.py --workload prior-art`) builds, loads, exports its two
entry points and rejects bad arguments on the host (no GPU needed)."""
import ctypes

import pytest

from paper_2303_10581_gb300 import build as build_mod


@pytest.fixture(scope="module")
def lib():
    l = ctypes.CDLL(build_mod.build_prior_art())
    l.pa_workspace_size.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    l.pa_filter.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    return l


def test_workspace_size(lib):
    out = ctypes.c_size_t()
    assert lib.pa_workspace_size(1000, ctypes.byref(out)) == 0
    assert out.value >= 1000 * 5            # flags and scan positions
    big = ctypes.c_size_t()
    assert lib.pa_workspace_size(10**8, ctypes.byref(big)) == 0 and big.value > out.value
    assert lib.pa_workspace_size(0, ctypes.byref(out)) == 1
    assert lib.pa_workspace_size(10, None) == 1


def test_bad_arguments_are_rejected_on_the_host(lib):
    one = ctypes.c_void_p(16)   # never dereferenced: the checks fail first
    assert lib.pa_filter(None, 10, 0, one, one, one, 1 << 30, None) == 1
    assert lib.pa_filter(one, 0, 0, one, one, one, 1 << 30, None) == 1
    assert lib.pa_filter(one, 10, 3, one, one, one, 1 << 30, None) == 1
    assert lib.pa_filter(one, 10, 0, one, one, one, 16, None) == 1     # workspace too small
