"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports every entry point that include/jiffy.h declares. No compute call is
made here (there is no GPU on this machine)."""
import ctypes
import os
import re

import pytest

from paper_2209_08196_gb300 import build as jbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(jiffy_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(jbuild.build())


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert "jiffy_encode" in names and "jiffy_decode" in names and "jiffy_stream_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_size_bound(lib):
    lib.jiffy_status_string.restype = ctypes.c_char_p
    assert lib.jiffy_status_string(0) == b"ok"
    assert lib.jiffy_status_string(2) == b"output capacity too small"
    from paper_2209_08196_gb300 import jiffy as J
    import oracle
    for H, W, attrs in [(1, 8, [(4, 10)]), (64, 1024, [(4, 10)]), (128, 2048, [(4, 10), (4, 10), (2, 1), (1, 1), (2, 1)])]:
        bound = J.jiffy_max_encoded_size(H, W, attrs, 1)
        assert bound == oracle.Codec(H, W, attrs).bound()


def test_library_has_no_host_fallback_symbols(lib):
    # the product path has no CPU codec: nothing from the oracle is linked in
    for n in ("jo_encode", "jo_decode", "jo_quantize"):
        assert not hasattr(lib, n)
