"""Host logic of bench.py that needs no GPU: the DRAM traffic recorded from
an ncu capture is reported only while the captured kernel's sources are
unchanged (hash of the forward part of the compositor source and the common
header), and a change anywhere in that part makes it unavailable; the
summary of the clock samples taken during the timed region."""

import hashlib
import importlib.util
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(root=None):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    if root is not None:
        b.ROOT = root
    return b


def test_source_hash_covers_the_part_before_the_marker():
    b = _bench()
    comp = os.path.join(ROOT, "paper_2506_02741_gb300", "csrc", "vt_composite.cu")
    data = open(comp, "rb").read()
    cut = data.index(b.FWD_END.encode())
    assert 0 < cut < len(data)
    want = hashlib.sha256(data[:cut]).hexdigest()[:16]
    got = b.source_hash([("paper_2506_02741_gb300/csrc/vt_composite.cu", b.FWD_END)])
    assert got == want


def _copy_tree(tmp_path):
    for rel in ("paper_2506_02741_gb300/csrc/vt_composite.cu",
                "paper_2506_02741_gb300/csrc/vt_common.cuh", "profiles/traffic.json"):
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    return tmp_path


def test_traffic_follows_the_forward_source(tmp_path):
    root = _copy_tree(tmp_path)
    b = _bench(str(root))
    entry = json.load(open(root / "profiles" / "traffic.json"))[b.WORKLOAD]["k_composite_fwd"]
    # a stored entry whose hash matches the sources is reported
    entry_sha = b.source_hash(b.KERNEL_SRC["k_composite_fwd"])
    t = {b.WORKLOAD: {"k_composite_fwd": dict(entry, source_sha=entry_sha)}}
    json.dump(t, open(root / "profiles" / "traffic.json", "w"))
    assert b.traffic_for("k_composite_fwd") == float(entry["dram_bytes_per_launch"])
    assert b.capture_for("k_composite_fwd", "warp_instructions_per_launch") == float(
        entry["warp_instructions_per_launch"])
    comp = root / "paper_2506_02741_gb300" / "csrc" / "vt_composite.cu"
    text = comp.read_text()
    # an edit after the forward part (the backward) keeps it
    comp.write_text(text + "\n// trailing comment\n")
    assert b.traffic_for("k_composite_fwd") == float(entry["dram_bytes_per_launch"])
    # an edit inside the forward part drops it
    comp.write_text("// leading comment\n" + text)
    assert b.traffic_for("k_composite_fwd") is None
    assert b.capture_for("k_composite_fwd", "warp_instructions_per_launch") is None
    # so does an edit of the common header
    comp.write_text(text)
    hdr = root / "paper_2506_02741_gb300" / "csrc" / "vt_common.cuh"
    hdr.write_text(hdr.read_text() + "\n")
    assert b.traffic_for("k_composite_fwd") is None


def test_clock_summary_median_and_throttle_reasons():
    """The clock record of the timed region: median SM clock over the
    samples, the maximum clock, and every throttle reason seen active in any
    sample; an empty record says it was not sampled."""
    b = _bench()
    s = b.ClockSampler(0)
    idle = "Not Active"
    s.lines = [
        f"2070, 2070, 812.4, 0x0000000000000000, {idle}, {idle}, {idle}, {idle}",
        f"1980, 2070, 1391.0, 0x0000000000000004, {idle}, {idle}, {idle}, Active",
        f"2070, 2070, 1200.0, 0x0000000000000000, {idle}, {idle}, {idle}, {idle}",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",   # unreadable: skipped
        "2070, 2070",                                                # short: skipped
    ]
    got = s.summary()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    s.lines.append(f"1400, 2070, 900.0, 0x0000000000000048, {idle}, Active, {idle}, {idle}")
    got = s.summary()
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 2025.0 and got["samples"] == 4
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                           "samples": 0}
