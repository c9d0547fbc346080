"""Host-side pieces of bench.py that need no GPU (the drift fit of its sweeps
is tested in test_drift_fit.py)."""


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the keys of the benchmark contract; its config names the lattices
    it ran (256 x 256, FP64, one per host core) and the GPU arm's workload they
    sample."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    cfg = line["config"]
    assert cfg["Lx"] == 256 and cfg["precision"] == "fp64" and "4096x4096" in cfg["sample_of"]
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == cfg["replicas"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
