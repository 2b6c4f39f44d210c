"""Host-side rules of bench.py's roofline object (no GPU): the committed
DRAM record of the FB kernels is used only while their source is unchanged
and the factor has the recorded size; otherwise `traffic` is null."""
import json
import os
import runpy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    return runpy.run_path(os.path.join(ROOT, "bench.py"), run_name="bench_host_test")


def test_fb_traffic_record_matches_the_current_kernels():
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "fb_solve_traffic.json")))
    assert rec["fb_kernels_sha256"] == b["fb_source_hash"]()
    assert b["fb_traffic"](rec["nnz_L"]) == rec["dram_bytes_per_solve"]
    # bytes per solve within the five captured solves, and above the
    # algorithmic bytes of the stored factor (each panel read once per sweep)
    each = rec["dram_bytes_per_solve_each"]
    assert min(each) <= rec["dram_bytes_per_solve"] <= max(each)
    assert rec["dram_bytes_per_solve"] >= rec["algorithmic_bytes_stored_per_solve"]


def test_fb_traffic_is_null_for_another_factor():
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "fb_solve_traffic.json")))
    assert b["fb_traffic"](rec["nnz_L"] + 1) is None
