"""Host-side logic of bench.py that needs no GPU: which committed ncu
summary a roofline may quote."""
import os

import pytest

import bench


def _write(tmp_path, prec, source_hash, shape):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / f"force_{prec}_n16384.md").write_text(
        f"source_hash: {source_hash}  (x)\n"
        f"launch_shape: {shape}  (x)\n"
        "traffic_bytes_per_launch: 12345\n"
        "thread_instructions_per_interaction: 70.5\n")


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    return tmp_path


def test_profile_used_only_for_matching_source_and_kernel_shape(fake_root):
    _write(fake_root, "hybrid", "abc123", "2,1,3")
    assert bench.profiled_metric("hybrid") == 12345.0
    assert bench.profiled_metric("hybrid", shape=(2, 1, 3)) == 12345.0
    # the CTAs per SM may differ: same kernel, another grid
    assert bench.profiled_metric("hybrid", shape=(2, 1, 4)) == 12345.0
    assert bench.profiled_metric("hybrid", "thread_instructions_per_interaction",
                                 (2, 1, 3)) == 70.5
    # another i-tile or j split is another kernel
    assert bench.profiled_metric("hybrid", shape=(1, 1, 3)) is None
    assert bench.profiled_metric("hybrid", shape=(2, 4, 3)) is None


def test_profile_ignored_after_a_kernel_change_or_when_missing(fake_root):
    _write(fake_root, "ds", "old999", "1,1,4")
    assert bench.profiled_metric("ds", shape=(1, 1, 4)) is None
    assert bench.profiled_metric("mixed") is None


def test_committed_profiles_record_a_shape():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for prec in ("hybrid", "ds", "mixed"):
        text = open(os.path.join(root, "profiles", f"force_{prec}_n16384.md")).read()
        assert "launch_shape:" in text and "source_hash:" in text
