"""Host-side pieces of the benchmark (no GPU): the ncu summary lookup and the clock
record."""
import os

import bench


def summary(hash16: str, traffic: str) -> str:
    return ("# scan kernel, genome-scale\n\n"
            f"- kernel_source_sha256_16: `{hash16}`\n"
            f"- dram_bytes_per_launch_full_size: `{traffic}`\n")


def test_traffic_is_reported_only_for_the_profiled_kernel_source(tmp_path):
    p = tmp_path / "s.md"
    p.write_text(summary(bench.kernel_source_hash(), "908681216"))
    assert bench.profiled_traffic(str(p)) == 908681216.0
    p.write_text(summary("0123456789abcdef", "908681216"))
    assert bench.profiled_traffic(str(p)) is None          # the kernel changed since
    p.write_text(summary(bench.kernel_source_hash(), "n/a"))
    assert bench.profiled_traffic(str(p)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md")) is None


def test_committed_summary_states_its_source_and_traffic():
    path = os.path.join(bench.ROOT, "profiles", "scan_kernel_genome_scan.md")
    vals = bench.profile_fields(open(path).read())
    h = vals["kernel_source_sha256_16"]
    assert len(h) == 16 and int(h, 16) >= 0
    assert int(vals["dram_bytes_per_launch_full_size"]) > 0


def test_clock_summary_counts_samples_under_load_only():
    s = bench.ClockSampler(0)
    s.lines = list(enumerate([
        # index, sm, max sm, power, util, active, hw, hw thermal, sw thermal, sw power cap
        "0, 1965, 2070, 300.0, 0, 0x0, Not Active, Not Active, Active, Not Active",   # idle
        "0, 2032, 2070, 900.0, 100, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 950.0, 98, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1995, 2070, 980.0, 99, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "0, N/A, 2070, 0, 50, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]))
    got = s.summary()
    assert got["samples_under_load"] == 3
    assert got["sm_mhz"] == 2010 and got["sm_max_mhz"] == 2070
    # a thermal reason seen while idle is not the timed region's
    assert got["reasons"] == ["sw_power_cap"]
    # a window of host times keeps only the samples taken inside it
    win = s.summary(2.5, 3.5)
    assert win["samples_under_load"] == 1 and win["sm_mhz"] == 1995 and win["reasons"] == []


def test_clock_summary_without_samples():
    got = bench.ClockSampler(0).summary()
    assert got == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples_under_load": 0}


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle alone) prints one JSON line with the
    fields of the benchmark contract, its CPU baseline and an end-to-end object with no
    host-device traffic."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--n-bases", str(1 << 20), "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["unit"] == bench.UNIT and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n_bases"] == 1 << 20 and len(d["config"]["inputs"]["text_sha256"]) == 64
