"""Host-side pieces of bench.py that need no GPU: the algorithmic byte count behind the
roofline, the peak lookup with its fallback, and the parsing of the nvidia-smi clock samples
that decide whether a measurement is kept."""
import json

import pytest

import bench


def test_paqif_algorithmic_bytes():
    # band (2 beta + 1 doubles per row) and rhs read, x written: 369.1 MB for the standalone batch
    assert bench.paqif_bytes(4096, 1024, 4) == 4096 * (1024 * 9 * 8 + 2 * 1024 * 8) == 369_098_752
    assert bench.paqif_bytes(1, 7, 1) == 7 * 3 * 8 + 2 * 7 * 8


def test_peaks_measured_then_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6651.4}))
    assert bench.peaks() == (6651.4, "measured")


def _summary(lines):
    s = bench.ClockSampler(0)  # not entered: no nvidia-smi process
    s.out.write("".join(line + "\n" for line in lines))
    return s.summary()


def test_clock_summary_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1301.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    got = _summary(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]}


def test_clock_summary_flags_thermal_slowdown():
    got = _summary(["0, 1500, 2070, 1400, 0x20, Not Active, Active, Not Active, Not Active"])
    assert got["reasons"] == ["hw_thermal_slowdown"] and got["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    assert _summary([])["reasons"] == ["unsampled"]


@pytest.mark.parametrize("world,units,ms,rate", [(1, 512, 122.4, 512 / 0.1224), (4, 512, 130.0, 2048 / 0.13)])
def test_job_rate(world, units, ms, rate):
    assert bench.job_rate(world, units, ms) == pytest.approx(rate)


def test_cpu_baseline_runs_on_a_spawned_pool():
    """The oracle leg of the bench: one single-threaded worker per core, whole instances each;
    a short budget still runs one round of each leg and reports the workers as its cores."""
    import os

    from paper_2008_03276_gb300 import inputs

    band, rhs = inputs.dd_band_systems(2 * (os.cpu_count() or 1), 1024, 4, seed=0)
    out = bench.cpu_baseline(band, rhs, budget_s=0.5)
    assert out["kind"] == "oracle" and out["cores"] == (os.cpu_count() or 1)
    assert out["value"] > 0 and "single-threaded worker processes" in out["sample"]


def test_issue_fraction_of_the_paqif_launch():
    # the capture's 852.5 M warp instructions in 0.964 ms at 2070 MHz fill 70 % of 608 schedulers' slots
    assert bench.issue_fraction(852_480_330, 0.964224, 2070.0) == pytest.approx(0.7025, abs=1e-4)
    assert bench.issue_fraction(None, 1.0, 2070.0) is None
    assert bench.issue_fraction(1, 1.0, None) is None
    assert bench.SCHEDULERS == 608


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle, no GPU) prints one JSON line with the keys the
    bench contract asks of the reference arm."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
