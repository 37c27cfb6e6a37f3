"""Host-side helpers of bench.py, on the CPU: the clock record taken from
nvidia-smi samples (median and maximum SM clock, the slowdown reasons seen
active), the emit kernel's DRAM bytes per row read from its ncu summary only
while the kernel source is the one captured, and the roofline peak with its
fallback."""
import hashlib
import json

import bench

SAMPLE = "0, {sm}, 2070, 900.5, {act}, {hw}, {hwt}, {swt}, {cap}"


def _line(sm, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active", act="0x0"):
    return SAMPLE.format(sm=sm, act=act, hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_clock_record_median_max_and_reasons():
    lines = [_line(2070), _line(1965), _line(2070, cap="Active"), _line(1800),
             _line(2070, hwt="Active")]
    r = bench.ClockSampler.summarize(lines)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 5
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_record_skips_partial_and_unparsable_lines():
    lines = ["", "0, 2070", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1500, [N/A], 1, 0x0, Active, Not Active, Not Active, Not Active",
             _line(1950), _line(2010)]
    r = bench.ClockSampler.summarize(lines)
    # neither unparsable sample counts, nor does the reason on one of them
    assert r["samples"] == 2 and r["sm_mhz"] == 2010.0 and r["reasons"] == []


def test_clock_record_without_samples():
    r = bench.ClockSampler.summarize([])
    assert r["sm_mhz"] is None and r["samples"] == 0 and r["reasons"] == []


def test_emit_traffic_follows_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "gj_emit.cu"
    src.write_bytes(b"// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "k_emit.md"
    prof.write_text("# summary\n\n- kernel_source_sha256: `%s`\n- dram_bytes_per_row: 69.070\n" % sha)
    monkeypatch.setattr(bench, "EMIT_PROFILE", str(prof))
    monkeypatch.setattr(bench, "EMIT_SOURCE", str(src))
    v, note = bench.emit_traffic_per_row()
    assert v == 69.07 and "ncu" in note
    src.write_bytes(b"// kernel v2\n")
    v, note = bench.emit_traffic_per_row()
    assert v is None and "changed" in note
    monkeypatch.setattr(bench, "EMIT_PROFILE", str(tmp_path / "missing.md"))
    assert bench.emit_traffic_per_row()[0] is None


def test_committed_emit_summary_has_both_fields():
    text = open(bench.EMIT_PROFILE).read()
    assert "- kernel_source_sha256: `" in text and "- dram_bytes_per_row: " in text


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6775.9}))
    assert bench.measured_peaks() == (6775.9, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{}")
    assert bench.measured_peaks() == (6800.0, "fallback")
