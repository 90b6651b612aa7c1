"""CPU check of bench.py's reference arm: it runs the oracle with no GPU and prints one JSON
line with the keys that the measurement contract asks for.  It also stays within its time
budget by sampling fewer instances."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, check=True, cwd=ROOT, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = _run("--workload", "cavity64", "--steps", "3", "--warmup", "3")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    import bench
    assert d["config"]["workload"] == bench._workload_desc("cavity64")   # our arm's config


def test_reference_arm_sampling_follows_the_budget():
    """On the batched sweep the sample is one instance of each kind (three); a tiny budget keeps
    only the cheapest one."""
    wide = _run("--workload", "sweep", "--steps", "1", "--warmup", "3", "--ref-budget", "1e9")
    assert "3 instances" in wide["cpu_baseline"]["sample"]
    tight = _run("--workload", "sweep", "--steps", "1", "--warmup", "3", "--ref-budget", "1e-9")
    assert "1 instances" in tight["cpu_baseline"]["sample"]
    assert tight["config"]["sample_cells"] < wide["config"]["sample_cells"]


def test_fp64_roofline_reads_the_committed_counts(monkeypatch):
    """The FP64 line's achieved rate is the committed per-cell and per-SST-cell FP64 flop counts
    times the units over the step time; counts taken on other kernel sources are not used."""
    import re
    import bench

    class Peak:
        @staticmethod
        def fvlbm_fp64_peak(dev):
            return 2.0

    with open(os.path.join(ROOT, "profiles", "k_flux_stage_fp64_sweep.md")) as fh:
        m = re.search(r"kernel_source_sha256=([0-9a-f]{64}) fp64_flops_per_cell=([0-9.]+) "
                      r"fp64_flops_per_sst_cell=([0-9.]+)", fh.read())
    assert m, "the profile records no FP64 flop counts"
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda: m.group(1))
    r = bench._fp64_roofline(Peak, 0, 1000, 400, 0.5, "sweep", "twopass")
    flops = 1000 * float(m.group(2)) + 400 * float(m.group(3))
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 2.0
    assert abs(r["achieved"] - flops / 0.5e-3 / 1e12) <= 1e-12 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 2.0) <= 1e-15
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda: "0" * 64)
    stale = bench._fp64_roofline(Peak, 0, 1000, 400, 0.5, "sweep", "twopass")
    assert stale["achieved"] is None and "other kernel sources" in stale["source"]
    assert bench._fp64_roofline(Peak, 0, 1000, 400, 0.5, "sweep", "fused")["achieved"] is None
