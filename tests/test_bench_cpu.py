"""Host-side rules of bench.py (CPU only): when a committed ncu summary may be
quoted as the kernel's DRAM traffic, and the peak the roofline divides by."""
import json

import bench


def _summary(tmp_path, digest, shape, dram=123456789):
    p = tmp_path / "summary.txt"
    p.write_text("kernel: test\n"
                 f"stream-collide sources sha256 prefix: {digest}\n"
                 f"launch shape: {shape}\n"
                 f"dram bytes per launch: {dram}\n")
    return str(p)


def test_traffic_needs_current_sources_storage_and_variant(tmp_path, monkeypatch):
    current = bench.source_digest(bench.SC_SOURCES)
    monkeypatch.setattr(bench, "TRAFFIC_FILES", {"fp32": _summary(tmp_path, current, "0,64,2,2,8")})
    assert bench.ncu_traffic("fp32", "0,64,2,2,8") == 123456789.0
    # another block size of the same kernel: same traffic
    assert bench.ncu_traffic("fp32", "0,256,2,2,8") == 123456789.0
    # another kernel variant, another storage form: nothing to quote
    assert bench.ncu_traffic("fp32", "2,64,2,2,8") is None
    assert bench.ncu_traffic("fp16", "0,64,2,2,8") is None
    assert bench.ncu_traffic("fp64", "0,64,2,2,8") is None


def test_traffic_is_dropped_once_the_kernel_sources_change(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILES",
                        {"fp32": _summary(tmp_path, "0000000000000000", "0,64,2,2,8")})
    assert bench.ncu_traffic("fp32", "0,64,2,2,8") is None


def test_committed_summaries_parse():
    for storage, path in bench.TRAFFIC_FILES.items():
        vals = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        assert int(vals["dram bytes per launch"]) > 0, storage
        assert len(vals["stream-collide sources sha256 prefix"]) == 16, storage
        assert vals["launch shape"].count(",") == 4, storage


def test_peak_comes_from_the_measured_file(tmp_path, monkeypatch):
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(p))
    assert bench.hbm_peak() == (1234.5, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
