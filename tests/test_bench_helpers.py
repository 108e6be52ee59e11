"""Host helpers of bench.py: the listing-code hash that decides whether the
recorded ncu DRAM counters still describe the kernels, and the peak lookup."""
import json

import bench


def test_code_only_ignores_comments_and_blank_lines():
    a = "int f(int x) {  // add one\n  return x + 1;\n}\n"
    b = "/* header\n   text */\nint f(int x) {\n\n  return x + 1;   \n}\n"
    assert bench.code_only(a) == bench.code_only(b) == "int f(int x) {\n  return x + 1;\n}"
    assert bench.code_only(a) != bench.code_only(a.replace("x + 1", "x + 2"))


def test_recorded_traffic_only_for_the_current_kernels(monkeypatch):
    with open(bench.os.path.join(bench.ROOT, "profiles", "list_rmat20_traffic.json")) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "list_source_hash", lambda: rec["list_source_sha256_16"])
    assert bench.recorded_traffic() == rec["dram_bytes_per_step"] > 0
    monkeypatch.setattr(bench, "list_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic() is None


def test_peaks_measured_or_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    assert bench.read_peaks() == (1234.5, "measured")
