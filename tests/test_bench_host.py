"""Host-side arithmetic of bench.py's roofline entry (no GPU): the dominant
kernel's achieved FP32 rate, its fraction of the measured (else derived)
peak, and its
algorithmic HBM bytes per second."""
import bench


class P0:
    N, M = 65536, 65340


def test_roofline_entry_arithmetic():
    prof = {"nnz_per_image": 15149028.0,
            "project": {"launches": 60, "total_ms": 138.0, "mean_ms": 2.3, "images_per_launch": 256.0},
            "backproject": {"launches": 60, "total_ms": 120.0, "mean_ms": 2.0, "images_per_launch": 256.0}}
    r = bench.roofline_entry(prof, P0, 256)
    assert r["kernel"] == "k_project" and r["bound"] == "alu"
    flops = 2 * 15149028.0 * 256 / 2.3e-3
    assert abs(r["achieved"] - flops / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    gbs = 256 * (65536 + 65340) * 4 / 2.3e-3 / 1e9          # s (N + M)
    assert abs(r["algorithmic_gbs"] - gbs) < 1e-6
    assert 0.0 < r["hbm_frac_of_measured"] < 0.1


def test_roofline_uses_the_measured_peak_when_given():
    prof = {"nnz_per_image": 15149028.0, "fp32_fma_tflops_measured": 75.0,
            "project": {"launches": 60, "total_ms": 138.0, "mean_ms": 2.3, "images_per_launch": 256.0},
            "backproject": {"launches": 60, "total_ms": 120.0, "mean_ms": 2.0, "images_per_launch": 256.0}}
    r = bench.roofline_entry(prof, P0, 256)
    assert r["peak"] == 75.0 and abs(r["frac"] - r["achieved"] / 75.0) < 1e-12
    assert "peak measured" in r["note"]


def test_roofline_counts_the_2h_projections_in_the_choice_not_the_rate():
    base = {"nnz_per_image": 15149028.0,
            "project": {"launches": 28, "total_ms": 45.0, "mean_ms": 1.6, "images_per_launch": 256.0},
            "backproject": {"launches": 57, "total_ms": 55.0, "mean_ms": 0.96, "images_per_launch": 230.0}}
    r = bench.roofline_entry(base, P0, 256)
    assert r["kernel"] == "k_backproject"
    prof = dict(base, project_2h={"launches": 28, "total_ms": 24.0, "mean_ms": 0.86, "images_per_launch": 203.0})
    r = bench.roofline_entry(prof, P0, 256)
    assert r["kernel"] == "k_project"
    assert abs(r["achieved"] - 2 * 15149028.0 * 256 / 1.6e-3 / 1e12) < 1e-9      # W's grid launches only
    assert "28 launches on the 2h grid" in r["note"]


def test_whole_job_value():
    assert bench.whole_job_value(256, 2, 5, 2.0) == 256 * 2 * 5 / 2.0


def test_study_helpers():
    from paper_1310_0956_gb300 import study
    ks = study.log_ks(3000, 6)
    assert ks[0] == 1 and ks[-1] == 3000 and all(b > a for a, b in zip(ks, ks[1:]))
    assert len(ks) < 30
    curve = [(1, 1, 0.9, 1.0), (2, 2, 0.5, 0.7), (4, 4, 0.3, 0.6), (8, 8, 0.35, 0.5)]
    k, row = study.k_opt(curve)
    assert k == 4 and row[2] == 0.3


def test_traffic_is_reported_only_for_the_measured_source(monkeypatch, tmp_path):
    import hashlib
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"// kernel source\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "project",
                        {"source": "kernel.cu", "sha256_16": h, "bytes_per_image": 1000.0})
    assert bench._kernel_traffic("project", 256) == 256000.0
    src.write_bytes(b"// kernel source, changed\n")
    assert bench._kernel_traffic("project", 256) is None
    src.unlink()
    assert bench._kernel_traffic("project", 256) is None
