"""Host-side arithmetic of bench.py that needs no GPU."""
import bench

PEAKS = {"fp32": {"tflops": 80.0, "fma_warp_inst_per_s": 1.25e12},
         "fp32x2": {"tflops": 79.0, "fma_warp_inst_per_s": 0.62e12},
         "fp64": {"tflops": 1.2, "fma_warp_inst_per_s": 1.8e10}}


def test_roofline_names_the_roof_with_the_largest_fraction(monkeypatch):
    monkeypatch.setattr(bench, "counters_current", lambda: True)
    cells = 6_795_264
    r = bench.roofline(cells, "rz", 1.0, 1, 6680.5, PEAKS)
    fr = {k: v["frac"] for k, v in r["roofs"].items()}
    assert r["binding_roof"] == max(fr, key=fr.get)
    assert r["frac"] == fr[r["binding_roof"]]
    # compulsory bytes: 64 B per cell and step
    comp = r["roofs"]["hbm_compulsory"]
    assert abs(comp["achieved"] - 64 * cells / 1.0e-3 / 1e9) < 1e-6
    assert r["roofs"]["hbm_stage_by_stage"]["frac"] > comp["frac"]
    # an issue-bound kernel: the issue roof binds and the bound is "alu"
    assert r["binding_roof"] == "issue" and r["bound"] == "alu"
    # traffic per launch: a whole step in one launch, a third of it per stage launch
    assert r["traffic"] == bench.COUNTERS["dram_bytes_per_cell_step"]["rz"] * cells
    r3 = bench.roofline(cells, "rz", 1.0, 3, 6680.5, PEAKS)
    assert abs(r3["traffic"] - r["traffic"] / 3) < 1e-6 and r3["avg_launch_ms"] == 1.0 / 3
    assert r3["frac"] == r["frac"]


def test_stale_counters_are_not_reported(monkeypatch):
    monkeypatch.setattr(bench, "counters_current", lambda: False)
    r = bench.roofline(1_000_000, "xy", 0.15, 3, 6680.5, PEAKS)
    assert r["traffic"] is None and not r["counters_current"]
    assert r["roofs"]["issue"]["achieved"] is None and r["roofs"]["fp32"]["frac"] is None
    assert r["binding_roof"].startswith("hbm_")     # only the byte roofs remain


def test_kernel_hash_covers_the_stage_kernel_sources():
    h = bench.kernel_sources_sha256()
    assert len(h) == 64 and bench.counters_current() == (h == bench.COUNTERS["sources_sha256"])
