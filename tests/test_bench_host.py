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


def test_error_stats_and_algorithmic_bytes():
    import numpy as np
    a0 = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    j0 = np.array([[0.0, 0.0, 4.0], [1.0, 1.0, 0.0]])
    p0 = np.array([-1.0, -2.0])
    st = bench.error_stats((a0 * (1 + 1e-7), j0, p0 * (1 - 3e-6)), (a0, j0, p0))
    assert abs(st["acc_rel_max"] - 1e-7) < 1e-12 and st["jerk_rel_max"] == 0.0
    assert abs(st["max_rel"] - 3e-6) < 1e-12 and st["n_above_1e-6"] == 2
    # j layout once plus per-i reads and writes: hybrid reads its state a, j,
    # dt and noise estimate on top of the DS record
    assert bench.algorithmic_bytes("ds", 1000, 10) == 64000 + 10 * 124
    assert bench.algorithmic_bytes("hybrid", 1000, 10) == 64000 + 10 * 196
    assert bench.algorithmic_bytes("mixed", 1000, 0) == 40000


def test_cpu_baseline_leg_references(orc):
    """The oracle references every gate of the bench line reads (no timing)."""
    import numpy as np
    from paper_1104_2700_gb300 import ics
    wl = ics.FORCE_SWEEP_N16K
    m, r, v = wl.particles()
    leg = bench.cpu_baseline_leg(m, r, v, wl.eps, 1.0, timed=False, extra=True)
    a, j, p = leg["refs"]["sweep"]
    assert a.shape == (wl.n, 3) and np.all(np.isfinite(a)) and np.all(p < 0)
    for key, w in (("n65536", ics.MIXED_N64K), ("n262144", ics.SALPETER_N256K)):
        sidx, (sa, sj, sp) = leg["refs"][key]
        assert 256 <= len(sidx) <= 320 and sa.shape == (len(sidx), 3)
        assert np.all(np.diff(sidx) > 0) and sidx[-1] < w.n
    pick, off, *_rest, t_end, rows = leg["refs"]["ensemble16"]
    assert len(pick) == 16 and len(rows) == 16 and t_end == 1.0 / 16
    assert all(0.0 < x["de"] < 1e-6 for x in rows)
    assert "cpu" not in leg
