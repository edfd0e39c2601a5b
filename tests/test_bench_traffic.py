"""Host logic of the benchmark's roofline `traffic` field: DRAM bytes per launch
come from the ncu figures in profiles/traffic.json only while they were taken
on the current kernel source; a capture of the very workload wins over a
smaller workload's bytes per row scaled by rows."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _use(tmp_path, monkeypatch, h):
    """Profiles under tmp_path; the source hash is the repository's (h)."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)


def _write_profiles(tmp_path, h, medium=True):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entries = [
        {"kernel": "aprod1", "workload": "small", "bytes_per_row": 240.5, "kernel_source_hash": h},
        {"kernel": "aprod2", "workload": "small", "bytes_per_row": 250.0, "kernel_source_hash": h},
    ]
    if medium:
        entries += [
            {"kernel": "aprod1", "workload": "medium", "n_rows": 1000, "bytes_per_launch": 262000,
             "kernel_source_hash": h},
            {"kernel": "aprod2", "workload": "medium", "n_rows": 1000, "bytes_per_launch": 251000,
             "kernel_source_hash": h},
        ]
    (prof / "traffic.json").write_text(json.dumps({"entries": entries}))


def test_direct_capture_wins_for_its_workload(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    _write_profiles(tmp_path, h)
    _use(tmp_path, monkeypatch, h)
    assert bench.profiled_traffic("aprod1", 1000) == 262000.0
    assert bench.profiled_traffic("aprod2", 1000) == 251000.0


def test_other_workloads_scale_the_small_counters(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    _write_profiles(tmp_path, h)
    _use(tmp_path, monkeypatch, h)
    assert bench.profiled_traffic("aprod1", 2000) == 240.5 * 2000
    assert bench.profiled_traffic("aprod2", 3) == 250.0 * 3


def test_no_direct_capture(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    _write_profiles(tmp_path, h, medium=False)
    _use(tmp_path, monkeypatch, h)
    assert bench.profiled_traffic("aprod1", 1000) == 240.5 * 1000


def test_stale_summaries_give_none(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert h != "0123456789abcdef"
    _write_profiles(tmp_path, "0123456789abcdef")
    _use(tmp_path, monkeypatch, h)
    assert bench.profiled_traffic("aprod1", 1000) is None
    assert bench.profiled_traffic("aprod2", 5) is None


def test_stale_capture_of_the_workload_is_not_replaced_by_scaling(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    _write_profiles(tmp_path, h)
    entries = json.loads((tmp_path / "profiles" / "traffic.json").read_text())
    entries["entries"].append({"kernel": "aprod1", "workload": "large", "n_rows": 5000,
                               "bytes_per_launch": 9e6, "kernel_source_hash": "0123456789abcdef"})
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entries))
    _use(tmp_path, monkeypatch, h)
    assert bench.profiled_traffic("aprod1", 5000) is None
    assert bench.profiled_traffic("aprod2", 5000) == 250.0 * 5000
