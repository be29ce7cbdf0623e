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


def test_binding_structs_match_the_c_layout(tmp_path):
    # the ctypes mirrors of the ABI's structs have the C compiler's sizes and
    # field offsets (a field added on one side only would shift the rest)
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    from paper_2209_08196_gb300 import jiffy as J
    structs = {
        "jiffy_attr_desc": (J._AttrDesc, ["dtype_bytes", "precision"]),
        "jiffy_options": (J._Options, ["test_lines", "force_mode", "stages"]),
        "jiffy_sensor_desc": (J._SensorDesc, ["H", "W", "beam_altitude", "azimuth0", "clockwise", "units_per_m",
                                              "range_bytes", "min_range", "max_range"]),
        "jiffy_point_attr": (J._PointAttr, ["values", "out", "scale", "dtype_bytes"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "jiffy.h"', "int main(void) {"]
    for name, (_, fields) in structs.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % name)
        for f in fields:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = iter(int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    for name, (cls, fields) in structs.items():
        assert next(got) == ctypes.sizeof(cls), name
        for f in fields:
            assert next(got) == getattr(cls, f).offset, (name, f)
    # the stage switch constants agree with the header's
    text = open(os.path.join(ROOT, "include", "jiffy.h")).read()
    for cname, val in (("JIFFY_STAGE_NO_MASK", J.STAGE_NO_MASK), ("JIFFY_STAGE_NO_DELTA", J.STAGE_NO_DELTA),
                       ("JIFFY_STAGE_NO_ZIGZAG", J.STAGE_NO_ZIGZAG)):
        assert re.search(r"#define %s %du\b" % (cname, val), text), cname
