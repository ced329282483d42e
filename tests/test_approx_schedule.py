"""The library's Alg. 2 schedule (bucket upper ends and the round cap per bucket, computed on the
host by nh_approx_thresholds / nh_approx_round_cap, which both approximate peels use) equals the
oracle's, which is pinned to exact rational arithmetic in test_oracle.py.  Host-only calls: no GPU
is needed."""
import ctypes
import os
import shutil

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08623_gb300 import build
    L = ctypes.CDLL(build.build())
    L.nh_approx_thresholds.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
    L.nh_approx_round_cap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)]
    return L


def lib_thresholds(L, C, delta, max_cnt, cap=1 << 16):
    out = np.zeros(cap, dtype=np.uint32)
    n = ctypes.c_int()
    assert L.nh_approx_thresholds(C, delta, max_cnt, out.ctypes.data, cap, ctypes.byref(n)) == 0
    return out[:n.value]


@pytest.mark.parametrize("C", [1, 2, 3, 4, 5, 6, 10, 15, 20, 21, 35])
def test_thresholds_and_round_cap_equal_the_oracle(lib, C):
    for delta in (0.001, 0.01, 0.1, 0.25, 0.5, 1.0, 2.0, 7.5):
        for max_cnt in (0, 1, 3, 7, 100, 12345, 10 ** 6, 2 ** 31, 2 ** 32 - 1):
            want = oracle.approx_thresholds(C, delta, max_cnt)
            got = lib_thresholds(lib, C, delta, max_cnt)
            assert np.array_equal(got, want), (C, delta, max_cnt)
        for n_r in (0, 1, 2, 3, 10, 1000, 82666190, 423560870, 2 ** 31 - 1):
            T = ctypes.c_uint32()
            assert lib.nh_approx_round_cap(C, delta, n_r, ctypes.byref(T)) == 0
            assert T.value == oracle.approx_round_cap(C, delta, n_r), (C, delta, n_r)


def test_short_output_buffer_and_bad_arguments(lib):
    full = lib_thresholds(lib, 3, 0.1, 10 ** 6)
    part = lib_thresholds(lib, 3, 0.1, 10 ** 6, cap=5)
    assert len(part) == 5 and np.array_equal(part, full[:5])
    out = np.zeros(4, dtype=np.uint32)
    n = ctypes.c_int()
    T = ctypes.c_uint32()
    assert lib.nh_approx_thresholds(0, 0.1, 10, out.ctypes.data, 4, ctypes.byref(n)) == 1
    assert lib.nh_approx_thresholds(3, 0.0, 10, out.ctypes.data, 4, ctypes.byref(n)) == 1
    assert lib.nh_approx_thresholds(3, 0.1, 10, out.ctypes.data, 0, ctypes.byref(n)) == 1
    assert lib.nh_approx_round_cap(3, -1.0, 10, ctypes.byref(T)) == 1
    assert lib.nh_approx_round_cap(3, 0.1, -1, ctypes.byref(T)) == 1
