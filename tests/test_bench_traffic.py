"""CPU check of bench.py's DRAM-traffic report: the figure captured with ncu
is reported only for the kernel sources it was taken on (a hash of them) and
the default workload; any change to those sources reports null."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path):
    b = load_bench()
    for k in ("k_encode", "k_decode"):
        assert b.traffic(k, 100) == b.TRAFFIC[k][0]
        assert b.traffic(k, 48) is None  # another workload
    assert b.traffic("k_trial", 100) is None
    # a copy of the sources with one byte changed in the encoder
    csrc = tmp_path / "paper_2209_08196_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2209_08196_gb300", "csrc"), csrc)
    with open(csrc / "jiffy_encode.cu", "a") as f:
        f.write("\n")
    b.ROOT = str(tmp_path)
    assert b.traffic("k_encode", 100) is None
    assert b.traffic("k_decode", 100) == b.TRAFFIC["k_decode"][0]
