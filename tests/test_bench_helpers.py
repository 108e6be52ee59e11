"""Host helpers of bench.py: the listing-code hash that decides whether the
recorded ncu DRAM counters still describe the kernels, and the peak lookup."""
import json

import bench


def test_code_only_ignores_comments_and_blank_lines():
    a = "int f(int x) {  // add one\n  return x + 1;\n}\n"
    b = "/* header\n   text */\nint f(int x) {\n\n  return x + 1;   \n}\n"
    assert bench.code_only(a) == bench.code_only(b) == "int f(int x) {\n  return x + 1;\n}"
    assert bench.code_only(a) != bench.code_only(a.replace("x + 1", "x + 2"))


def test_recorded_traffic_only_for_the_current_kernels(monkeypatch, tmp_path):
    with open(bench.os.path.join(bench.ROOT, "profiles", "list_rmat20_traffic.json")) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "list_source_hash", lambda: rec["list_source_sha256_16"])
    assert bench.recorded_traffic("rmat20") == rec["dram_bytes_per_step"] > 0
    # counters belong to the workload they were taken on
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("chunglu1e8") is None
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "list_chunglu1e8_traffic.json").write_text(json.dumps(
        {"list_source_sha256_16": rec["list_source_sha256_16"], "dram_bytes_per_step": 100,
         "scale_to_workload": 12.5}))
    assert bench.recorded_traffic("chunglu1e8") == 1250
    monkeypatch.setattr(bench, "list_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("chunglu1e8") is None


def test_peaks_measured_or_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    assert bench.read_peaks() == (1234.5, "measured")


def test_oracle_sample_ranges():
    r = bench.sample_ranges(100_000_000, 2048)
    assert len(r) == 16 and r[0] == (0, 3051) and r[15][0] == 15 * 6_250_000
    assert all(b - a == 3051 for a, b in r)
    assert bench.sample_ranges(10, 64) == [(0, 1)] * 16  # tiny graphs: one vertex each


def test_h2d_bytes_per_step():
    assert bench.h2d_bytes("chunglu1e8", 100_000_000) == 2_000_000_000 * 8 + 400_000_000
    assert bench.h2d_bytes("rmat20", 1 << 20) == (16 << 20) * 8 + (4 << 20)


def test_oracle_sample_threads_split_the_same_work():
    """The threaded sample lists the same seed ranges as the one-thread one
    (each range cut into parts), so both count the same triangles."""
    import oracle
    from paper_2203_04774_gb300 import synth
    n = 3000
    e = synth.chung_lu(n, 12, 2.3, 7)
    g = oracle.Graph(n, e)
    g.order_apply(synth.order_degree_from_degrees(g.degrees()))
    assert bench.oracle_sample(g, n, 4, 1) == bench.oracle_sample(g, n, 4, 5) > 0
    assert bench.oracle_threads("rmat20") == 1
    assert bench.oracle_threads("chunglu1e8") == (__import__("os").cpu_count() or 1)
