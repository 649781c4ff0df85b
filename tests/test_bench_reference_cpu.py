"""The reference arm of the benchmark (the CPU oracle timed on the host cores) prints one JSON
line with the keys the measurement contract asks for; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "o10v30", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "CCSD iteration time (s)" and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["steps"] == 1 and d["warmup"] >= 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "ccsd_fp64_o10_v30_naux120"


def test_triples_cpu_baseline_helper():
    """The triples CPU baseline times the oracle's per-pair form on a bounded sample."""
    import bench
    est, sample = bench.oracle_triples_time(dict(bench.WORKLOADS["o10v30"]))
    assert est > 0.0 and "extrapolated" in sample


def test_split_ladder_fraction_counts_packed_digit_pair_flops(monkeypatch):
    """The e4m3 fraction of a split ladder launch: s(s+1)/2 digit pairs x 8 P(o) P(v)^2 flops over
    the launch time, against twice the measured bf16 burst rate."""
    import bench
    monkeypatch.setattr(bench, "load_peaks", lambda: ({"bf16_tflops": 1000.0}, "measured"))
    o, v, s, ms = 20, 120, 8, 2.0
    flops = 36 * 8.0 * (20 * 19 // 2) * (120 * 119 // 2) ** 2
    assert abs(bench.split_ladder_frac(ms, o, v, s) - flops / 2e-3 / 1e12 / 2000.0) < 1e-12
    assert bench.split_ladder_frac(None, o, v, s) is None
