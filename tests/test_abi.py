"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every entry point
that include/nucleus.h declares (no compute call: there may be no GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(nh_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["nh_build_orientation", "nh_index_r_cliques", "nh_count_s_cliques", "nh_peel_and_link",
                 "nh_construct_tree", "nh_approx_nucleus", "nh_oriented_free", "nh_rindex_free", "nh_batch_run"]:
        assert want in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_loads_and_exports_every_symbol():
    from paper_2306_08623_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.nh_status_string.restype = ctypes.c_char_p
    assert lib.nh_status_string(0) == b"ok"
    assert lib.nh_version() >= 100


def test_oracle_shares_no_code_with_the_cuda_path():
    """The oracle directory neither includes nor imports the CUDA library, and vice versa."""
    csrc = os.path.join(ROOT, "paper_2306_08623_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        p = os.path.join(ROOT, "oracle", f)
        if os.path.isfile(p) and f.endswith((".c", ".py")):
            txt = open(p).read()
            assert "paper_2306_08623_gb300" not in txt.replace("paper_2306_08623_gb300/", "") or f == "__init__.py"
            assert "nucleus.h" not in txt and "libnucleus" not in txt


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_debug_injection_validates_its_arguments():
    """nucleus_debug.h: host-side settings only (no GPU needed to set them)."""
    from paper_2306_08623_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.nh_debug_inject.argtypes = [ctypes.c_int, ctypes.c_int64]
    assert lib.nh_debug_inject(1, 1000) == 0
    assert lib.nh_debug_inject(1, 0) == 0
    assert lib.nh_debug_inject(2, 64) == 0
    assert lib.nh_debug_inject(2, 0) == 0
    assert lib.nh_debug_inject(2, 48) == 1   # not a power of two
    assert lib.nh_debug_inject(1, -5) == 1
    assert lib.nh_debug_inject(9, 1) == 1
    assert lib.nh_debug_inject(3, (1 << 32) - 3) == 0
    assert lib.nh_debug_inject(3, 1 << 32) == 1  # beyond uint32
    assert lib.nh_debug_inject(3, 0) == 0
    lib.nh_status_string.restype = ctypes.c_char_p
    assert b"2^32" in lib.nh_status_string(9)
