"""The reference arm of bench.py (the oracle on the host cores) prints one
JSON line with the fields the benchmark contract needs; runs without a GPU
on a small per-step sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-sample", "64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "Mrays/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["warmup"] >= 3 and line["n_gpus"] == 1 and line["vs_baseline"] is None
    assert line["config"]["workload"] == bench.WORKLOAD and line["config"]["rays_per_step"] == 64
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_committed_fused_profile_matches_the_kernel_sources():
    """The roofline's DRAM traffic, L2 sectors per gathered point and tensor
    activity come from the committed ncu summary of the fused kernel, tied to
    a hash of its sources; a change to those sources must come with a new
    capture (the bench reports null for them otherwise)."""
    sys.path.insert(0, ROOT)
    import bench
    for key in ("dram_bytes_per_launch", "l2_sectors_per_gathered_point", "tensor_pipe_active_pct"):
        v = bench.recorded_profile(key)
        assert v is not None and v > 0, key
