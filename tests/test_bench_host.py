"""Host logic of bench.py that needs no GPU: the DRAM traffic recorded from
an ncu capture is reported only while the captured kernel's sources are
unchanged (hash of the forward part of the compositor source and the common
header), and a change anywhere in that part makes it unavailable."""

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
