"""The CPU legs of bench.py (the oracle timed on a host core): the headline workload's
projected solve and the Bratu cycle sample, on small stand-ins, and the reference arm's
JSON line."""
import json

import pytest

import workloads as W


def test_cpu_baseline_fields():
    import bench
    cb = bench.cpu_baseline(W.workload1(), budget_steps=3)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == bench.UNIT
    assert cb["value"] > 0 and cb["s_per_step"] > 0
    assert cb["projected_solve_s"] == pytest.approx(cb["setup_s"] + cb["s_per_step"] *
                                                    bench.PROJECT_ITERS, rel=1e-12)


def test_bratu_cpu_sample_fields():
    import bench
    r = bench.bratu_cpu_sample(n=3, steps=4)
    assert r["n"] == 3 and r["dof"] == 7 ** 3 and r["kind"] == "oracle"
    assert r["us_per_step"] > 0


def test_reference_arm_prints_one_line(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class Args:
        gpus, steps, warmup, ref_sample_steps = 1, 1, 3, 2

    # the reference arm samples the headline workload; a small stand-in keeps this quick
    monkeypatch.setattr(W, "workload2", lambda n=1024: W.workload1())
    bench.run_reference(Args())
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["higher_is_better"] is True


def test_clock_summary():
    import bench
    rows = [["1965", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Active"],
            ["2010", "2070", "910.0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["[N/A]", "2070", "0", "Not Active", "Active", "Not Active", "Not Active"],
            ["1980", "2070", "905.5", "Not Active", "Not Active", "Not Active", "Not Active"]]
    c = bench.summarise_clocks(rows)
    # the unparsable row is skipped whole, its reasons included
    assert c == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert bench.summarise_clocks([])["sm_mhz"] is None


def test_job_rate_counts_every_rank():
    import bench
    assert bench.job_rate(1, 10, 1000.0) == 10.0
    assert bench.job_rate(4, 10, 2000.0) == 20.0
