"""Host logic of bench.py that needs no GPU: the clock-sample summary that
decides whether a run is kept, and the algorithmic byte count of a step."""
import tempfile

import bench


def _summary(lines):
    s = bench.ClockSampler(0)
    s.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.file.write("\n".join(lines) + "\n")
    return s.summary()


def test_clock_summary_median_max_and_reasons():
    out = _summary([
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1320.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_thermal_slowdown_and_empty_runs():
    out = _summary(["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"])
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and out["sm_mhz"] == 1500.0
    assert _summary([])["reasons"] == ["no nvidia-smi samples"]


def test_algorithmic_bytes_of_the_single_view_step():
    # 1M SH-degree-3 Gaussians (236 B raw record), one 1237x822 view at 32x16 tiles
    n, slots, inst, pix, tiles = 1_000_000, 1_000_000, 3_561_880, 1237 * 822, 39 * 52
    got = bench.algorithmic_bytes(n, 3, slots, inst, pix, tiles)
    assert got == 3 * n * 236 + 132 * slots + 108 * inst + 36 * pix + 8 * tiles == 1_261_304_568
    assert bench.algorithmic_bytes(10, 0, 10, 0, 0, 0) == 3 * 10 * 56 + 132 * 10


def test_stage_bytes_partition_the_step():
    """The per-stage algorithmic bytes cover the step's total: the stages sum
    to the total except 4 B per instance (the step total counts 108 B per
    instance, the three instance-touching stages 24 + 40 + 40)."""
    n, slots, inst, pix, tiles = 1_000_000, 1_000_000, 3_561_880, 1237 * 822, 39 * 52
    sb = bench.stage_bytes(n, 3, slots, inst, pix, tiles)
    assert set(sb) == {"gs_project", "gs_bin_sort", "gs_render_fwd", "gs_rasterize_bwd", "gs_project_bwd"}
    assert sum(sb.values()) + 4 * inst == bench.algorithmic_bytes(n, 3, slots, inst, pix, tiles)
