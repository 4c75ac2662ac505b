"""The committed ncu records that bench.py reads are keyed by a hash of the
kernel sources; this checks that they were taken on the sources as they are
now, so that the benchmark line's `roofline.traffic` and the 16-bit issue
roofline are not silently dropped (bench.py reports null for a stale record).
CPU only: it reads the files."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_records_match_the_kernel_sources():
    b = _bench()
    for prec in ("fp32", "fp16", "bf16"):
        t = b.recorded_traffic(f"k_stream_collide_vec_d3q19_{prec}_jet384x256x256")
        assert t is not None, prec
        # every population read and written once, less what stays in L2
        algorithmic = (152 if prec == "fp32" else 76) * 384 * 256 * 256
        assert 0.9 * algorithmic < t <= 1.05 * algorithmic, (prec, t)


def test_issue_and_fp64_records_match_the_kernel_sources():
    b = _bench()
    for prec in ("fp16", "bf16"):
        assert b.recorded_issue(f"k_stream_collide_vec_d3q19_{prec}_jet", "384x256x256") is not None, prec
    assert b.recorded_fp64_inst("k_stream_collide_d3q19_fp64_jet") is not None
