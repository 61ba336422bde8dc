"""bench.py's roofline arithmetic and its guard on committed profile figures (host logic, no GPU)."""
import hashlib
import os

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_alu_roofline_counts_the_stated_operations(bench):
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}
    ex, acc, ms, mhz = 4.0e10, 5.0e9, 40.0, 2000.0
    prof = {"source": "profiles/x.md", "traffic": 1.2e10, "warp_inst_per_examined": 0.8}
    blk = bench.roofline_block(0, ex, acc, ms, mhz, peaks, "measured", prof, 16 * ex)
    ops = 8 * ex + 13 * acc  # the window gather's accounting
    peak = 152 * 128 * mhz * 1e6 / 1e12
    assert blk["bound"] == "alu" and blk["unit"] == "TFLOP/s"
    assert blk["achieved"] == pytest.approx(ops / (ms / 1e3) / 1e12)
    assert blk["peak"] == pytest.approx(peak) and blk["frac"] == pytest.approx(blk["achieved"] / peak)
    assert blk["traffic"] == 1.2e10
    assert blk["hbm"]["frac"] == pytest.approx(1.2e10 / (ms / 1e3) / 1e9 / 6000.0)
    assert blk["issue"]["frac"] == pytest.approx(0.8 * ex / (152 * 4 * mhz * 1e6 * ms / 1e3))
    assert blk["touched_bytes"]["frac_of_hbm"] == pytest.approx(16 * ex / (ms / 1e3) / 1e9 / 6000.0)
    # without profile figures there is no traffic, HBM or issue entry
    bare = bench.roofline_block(1, ex, acc, ms, mhz, peaks, "measured", {}, 16 * ex)
    assert bare["traffic"] is None and "hbm" not in bare and "issue" not in bare
    assert bare["achieved"] == pytest.approx((17 * ex + 14 * acc) / (ms / 1e3) / 1e12)  # the aperture's


def test_profile_figures_only_for_the_profiled_source_and_launch(bench, tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2102_03011_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "ssvp_gather.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    name, _ = bench.PROFILE_SUMMARIES["fhd"]
    (tmp_path / "profiles" / name).write_text(
        "# summary\n\nMachine-readable:\n\n"
        f"    source_sha256: {sha}\n    workload: fhd\n    colour: fp32\n    out_frames: 8\n"
        "    dram_bytes_per_launch: 1000\n    warp_inst_per_examined: 0.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench._profile_figures("fhd", "fp32", 8)
    assert got["traffic"] == 1000 and got["warp_inst_per_examined"] == 0.5
    assert "traffic" not in bench._profile_figures("fhd", "fp32", 1)  # bytes scale with the launch
    assert bench._profile_figures("fhd", "fp16", 8) == {}
    assert bench._profile_figures("hd", "fp32", 8) == {}
    src.write_text("// kernel source, changed\n")
    assert bench._profile_figures("fhd", "fp32", 8) == {}  # stale: the source changed since


def test_committed_counters_summary_names_the_benchmark_launch(bench):
    name, src_name = bench.PROFILE_SUMMARIES["fhd"]
    text = open(os.path.join(bench.ROOT, "profiles", name)).read()
    assert f"source: paper_2102_03011_gb300/csrc/{src_name}" in text
    for key in ("source_sha256:", "workload: fhd", "colour: fp32", "out_frames: 8", "dram_bytes_per_launch:",
                "warp_inst_per_examined:"):
        assert key in text


def test_clock_summary_reads_the_sampled_lines(bench):
    """The clock record of a timed region: median and minimum SM clock, the maximum clock, the
    median power and every throttle reason that was active in any sample."""
    cs = bench.ClockSampler(0)
    cs.out = "\n".join([
        "2070, 2070, 450.5, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 460.0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, [N/A], Not Active, Not Active, Not Active, Not Active",
    ])
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_mhz_min"] == 1980.0
    assert s["sm_max_mhz"] == 2070.0 and s["power_w_median"] == pytest.approx(460.0)
    assert s["reasons"] == ["sw_power_cap"]
    empty = bench.ClockSampler(0)
    empty.out = ""
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
