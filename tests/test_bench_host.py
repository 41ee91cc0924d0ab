"""Host-side logic of the benchmark's JSON line, on CPU: the committed DRAM traffic is
reported only for the kernel sources it was measured on, the clock record flags the
throttle reasons that invalidate a timing, and the algorithmic bytes behind the roofline
are the per-point figures of the three step-loop kernels."""
import json
import os
import shutil

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_1802_07625_gb300", "csrc")


def test_traffic_is_reported_for_the_profiled_sources_only(tmp_path, monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for k in ("inverse_rows", "inverse_cols_velocity", "heun_step"):
        assert bench._traffic(k) == d[k]
    assert bench._traffic("no_such_kernel") is None
    # a copy of the tree whose kernel sources differ by one byte reports no traffic
    root = tmp_path / "tree"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), root / "profiles" / "traffic.json")
    shutil.copytree(CSRC, root / "paper_1802_07625_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("heun_step") == d["heun_step"]
    f = root / "paper_1802_07625_gb300" / "csrc" / d["sources"][0]
    f.write_bytes(f.read_bytes() + b"\n")
    assert bench._traffic("heun_step") is None


def _summary(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return s.summary()


def test_clock_record_flags_throttle_reasons(tmp_path):
    idle = "Not Active"
    row = lambda sm, hw, thermal, swcap: ", ".join(
        ["0", str(sm), "2070", "900.5", "0x0", hw, thermal, idle, swcap])
    ok = _summary(tmp_path, [row(2070, idle, idle, idle), row(2055, idle, idle, idle), row(2070, idle, idle, idle)])
    assert ok == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    bad = _summary(tmp_path, [row(1500, "Active", idle, idle), row(2070, idle, "Active", "Active")])
    assert bad["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert bad["sm_mhz"] == pytest.approx(1785.0)
    assert _summary(tmp_path, [])["reasons"] == ["unavailable"]


def test_roofline_bytes_and_single_rank_throughput():
    # pass 1: spectrum in, (A, B) out; pass 2: (A, B) in, v out; step: displacement in and
    # out plus one gather of v(t) and of v(t + h) per point
    assert bench.bytes_per_point(4) == {"inverse_rows": 12, "inverse_cols_velocity": 16, "heun_step": 32}
    assert bench.bytes_per_point(8) == {"inverse_rows": 24, "inverse_cols_velocity": 32, "heun_step": 64}
    assert bench.replica_throughput(1, 3.0e9, 1.5) == pytest.approx(2.0e9)
    # the launch count grows by three kernels per attempted step
    assert bench.launches_per_cartogram(34, 2827) - bench.launches_per_cartogram(34, 2826) == 3
