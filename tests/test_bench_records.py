"""Host-side logic of bench.py's roofline record: the kernel-source hash that ties a committed
ncu record to the code it measured ignores comments and blank lines but not code, and the
recorded DRAM bytes of a step are spread over the closest-hit launches the run issues."""
import os

import pytest

import bench


def _write(root, rel, text):
    path = os.path.join(root, rel)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(text)


SOURCES = ("paper_2407_19977_gb300/csrc/pt_device.cuh", "paper_2407_19977_gb300/csrc/pt_render.cu",
           "paper_2407_19977_gb300/csrc/pt_bvh.cu")


def _tree(tmp_path, body):
    for rel in SOURCES:
        _write(str(tmp_path), rel, body)
    return str(tmp_path)


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    code = "int f(int x) {\n    return x + 1;\n}\n"
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", code))
    h0 = bench._source_hash()
    commented = "// a note\nint f(int x) {  /* inline\n   block */\n\n    return x + 1;   // trailing\n}\n"
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", commented))
    assert bench._source_hash() == h0
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "c", code.replace("x + 1", "x + 2")))
    assert bench._source_hash() != h0


def test_recorded_traffic_and_issue_follow_the_record(tmp_path, monkeypatch):
    root = _tree(tmp_path, "int g;\n")
    monkeypatch.setattr(bench, "ROOT", root)
    rec = ("# comment: with a colon\n"
           f"source_hash: {bench._source_hash()}\n"
           "workload: pushbutton\nspp_per_step: 4\ndram_bytes_per_step: 1000\n"
           "issue_slots_busy_pct: 75.0\nactive_threads_per_inst: 8.0\nissue_source: test\n")
    _write(root, "profiles/trace_traffic.txt", rec)
    assert bench._recorded_traffic("trace", "pushbutton", 4, 4) == pytest.approx(250.0)
    assert bench._recorded_traffic("trace", "pushbutton", 4, 5) == pytest.approx(200.0)
    iv = bench._recorded_issue("trace", "pushbutton", 4)
    assert iv["issue_slots_busy"] == pytest.approx(0.75) and iv["lane_fraction"] == pytest.approx(0.25)
    # another launch shape or another source: no figures
    assert bench._recorded_traffic("trace", "pushbutton", 1, 4) is None
    assert bench._recorded_traffic("trace", "heavy", 4, 4) is None
    _write(root, SOURCES[0], "int g2;\n")
    assert bench._recorded_traffic("trace", "pushbutton", 4, 4) is None
    assert bench._recorded_issue("trace", "pushbutton", 4) is None
