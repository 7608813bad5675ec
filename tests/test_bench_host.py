"""Host logic of bench.py that needs no GPU: the clock record, the gather's HBM roofline arithmetic, and the
reference arm's JSON line (the oracle timed on a few sources of the 32^3 workload)."""
import json

import pytest

import bench


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 1965, 2070, 1210.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2070, 1301.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1500, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",      # unreadable sample
        "garbage",
    ]
    got = s.summary()
    assert got == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines.append("0, 2000, 2070, 1000.0, 0x8, Active, Not Active, Active, Not Active")
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_gather_roofline_counts_the_cache_once_and_the_field():
    """192^3, R = 8, BF16 cache with FP32 accumulation: each of the N (2R+1)^3 stored values is read once
    (2 B), plus the FP32 scaled field (4 B) and the FP64 output (8 B) per cell."""
    N, R = 192 ** 3, 8
    nbytes = N * 17 ** 3 * 2 + N * 4 + N * 8
    r = bench.gather_roofline("bf16", "fp32", N, R, 10.0)
    peak = bench._peaks()[0]["hbm_gbs"]
    assert r["achieved"] == pytest.approx(nbytes / 10e-3 / 1e9, rel=1e-15)
    assert r["peak"] == peak and r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-15)
    assert r["traffic"] == pytest.approx(bench.GATHER_FP32_BF16_DRAM_PER_ALGORITHMIC_BYTE * nbytes, rel=1e-15)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    ff = bench.gather_roofline("fp32", "ff", N, R, 10.0)            # float-float field: 8 B pairs
    assert ff["achieved"] * 10e-3 * 1e9 == pytest.approx(N * 17 ** 3 * 4 + N * 8 + N * 8, rel=1e-15)
    assert ff["traffic"] is None                                     # no capture of that kernel is scaled
    assert 0.99 <= bench.GATHER_FP32_BF16_DRAM_PER_ALGORITHMIC_BYTE < 1.01      # DRAM bytes match the algorithmic ones


def test_job_rate_is_all_units_over_the_slowest_rank():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(4, 20, 500.0) == pytest.approx(160.0)


def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.main(["--impl", "reference", "--workload", "fdirw-32c-r3", "--steps", "2", "--warmup", "1",
                       "--ref-sample", "64", "--ref-sample-1t", "16"]) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == bench.UNIT and d["metric"] == bench.METRIC
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1000.0 / d["value"], rel=1e-12)
    assert d["config"]["workload"] == "fdirw-32c-r3"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "64 seeded random sources" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the line says that it extrapolates a timed sample, and gives the single-thread rate and the CPU model
    assert d["timing"]["kind"] == "sample-extrapolated" and d["timing"]["sources_per_step"] == 64
    assert d["timing"]["timed_ms_per_step"] == pytest.approx(d["ms_per_step"] * 64 / 32 ** 3, rel=1e-9)
    st = d["cpu_baseline"]["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "16 seeded random sources" in st["sample"]
    assert isinstance(d["cpu_baseline"]["cpu_model"], str) and d["cpu_baseline"]["cpu_model"]


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--workload", "fdirw-32c-r3", "--steps", "1", "--warmup", "0",
                       "--ref-sample", "8"]) == 0
    assert capsys.readouterr().out.strip() == ""


def test_batch_reference_arm_line(capsys, monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.main(["--impl", "reference", "--workload", "fdirw-batch2x48c-r3to10", "--steps", "1", "--warmup",
                       "0", "--ref-sample", "8"]) == 0
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["config"]["workload"] == "fdirw-batch2x48c-r3to10"
    assert d["config"]["structures"] == 2 and d["config"]["cells"] == 2 * 48 ** 3
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert "32 seeded random sources" in d["cpu_baseline"]["sample"]


def test_our_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without CUDA the CUDA arm stops with an error instead of timing anything else."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(SystemExit) as e:
        bench.main(["--steps", "1", "--warmup", "3"])
    assert "needs a CUDA GPU" in str(e.value.code)
