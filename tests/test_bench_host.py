"""Host-side logic of bench.py that needs no GPU: the clock summary taken from
nvidia-smi samples and the rule that a DRAM-traffic figure is reported only while the
profiled kernel source is unchanged."""

import json
import os
import shutil

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s


def test_clock_summary_median_max_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _sampler(lines).summary()
    assert s["sm_mhz"] == 2070.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_clock_summary_flags_thermal_slowdown():
    lines = ["0, 1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["reasons"] == ["hw_thermal_slowdown"]
    assert _sampler([]).summary()["sm_mhz"] is None


def _tree(tmp_path, src_text, rec):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "k.cu").write_text(src_text)
    rec = dict(rec, sources=["k.cu"])
    (root / "profiles" / "k_rays_layered_single.json").write_text(json.dumps(rec))
    return root


def test_traffic_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    root = _tree(tmp_path, src, {"dram_bytes_per_launch": 123})
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = json.loads((root / "profiles" / "k_rays_layered_single.json").read_text())
    rec["source_hash"] = bench.source_hash(["k.cu"])
    (root / "profiles" / "k_rays_layered_single.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic() == 123
    # the kernel changes after the capture: the figure no longer describes it
    (root / "k.cu").write_text(src + "// changed\n")
    assert bench.ncu_traffic() is None
    # no summary at all
    os.remove(root / "profiles" / "k_rays_layered_single.json")
    assert bench.ncu_traffic() is None


def test_committed_traffic_record_is_well_formed():
    path = os.path.join(bench.ROOT, "profiles", "k_rays_layered_single.json")
    rec = json.load(open(path))
    for f in rec["sources"]:
        assert os.path.exists(os.path.join(bench.ROOT, f))
    full = rec["full_launch"]
    assert full["passes"] == 1
    assert rec["dram_bytes_per_launch"] == full["dram_bytes_read"] + full["dram_bytes_write"]
    assert "--clock-control none" in full["command"]


def test_flop_count_per_ray_step_adds_up():
    # four right-hand sides and seven fused multiply-adds per integrated value per step
    assert bench.FLOPS_PER_RAY_STEP_2D == 4 * 280 + 22 * 7 * 2
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9
