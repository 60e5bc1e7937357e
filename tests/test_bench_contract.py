"""bench.py's host-side contract, on CPU: the reference arm's JSON line (the
FP64 oracle timed on the host), its silence on ranks other than 0, and the
committed DRAM-traffic figure being tied to the current hopping-kernel
source."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config")


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--workload", "dwf_4x4x4x4_ls8", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in REQUIRED:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "dwf_4x4x4x4_ls8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks():
    r = _run(["--impl", "reference", "--workload", "dwf_4x4x4x4_ls8", "--steps", "1", "--warmup", "1"],
             env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_committed_traffic_matches_the_hopping_kernel_source():
    """The DRAM traffic the benchmark line reports is read from
    profiles/traffic.json only while the hash of the kernel sources matches the
    one recorded with the ncu capture; the committed figure must belong to the
    committed source."""
    shash = bench.source_hash("paper_2103_05034_gb300/csrc/dhop_impl.cuh",
                              "paper_2103_05034_gb300/csrc/dhop_pair.cuh")
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert d, "no traffic record"
    for key, rec in d.items():
        assert rec["source_hash"] == shash, key
        assert bench.profile_traffic(key, shash) == rec["dram_bytes_per_launch"]
    assert bench.profile_traffic(next(iter(d)), "0" * 16) is None


def test_measured_peaks_are_read_from_the_driver_file():
    peaks, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peaks["hbm_gbs"] > 1000
    else:
        assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
