"""Host-side pieces of bench.py that need no GPU: the drift fit of the u_x0
sweeps (the paper fits l u + q u^2 over -0.25 <= u_x0 <= 0.25; the diagonal
variances are even in u_x0, so the runs at u >= 0 stand for their mirror
images)."""
import numpy as np

import bench


def test_fit_drift_is_the_symmetric_least_squares_fit():
    rng = np.random.Generator(np.random.PCG64(1))
    us = np.array([0.0, 0.05, 0.1, 0.2, 0.3])
    D = rng.normal(size=(5, 9)) * 1e-3 + np.outer(us ** 2, np.linspace(0.5, 2.0, 9))
    q = bench.fit_drift(us, D)
    # the paper's fit written out: l u + q u^2 by least squares over the mirrored
    # points with |u| <= 0.25 (u = 0 once)
    keep = us <= 0.25
    u_all = np.concatenate([us[keep], -us[keep][1:]])
    D_all = np.concatenate([D[keep], D[keep][1:]])
    A = np.stack([u_all, u_all ** 2], axis=1)
    (l_ref, q_ref), *_ = np.linalg.lstsq(A, D_all, rcond=None)
    np.testing.assert_allclose(q, q_ref, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(l_ref, 0.0, atol=1e-12)


def test_fit_drift_recovers_a_pure_quadratic():
    us = [0.0, 0.05, 0.1, 0.2, 0.3]
    D = np.array([[1.7 * u * u, 0.5 * u * u] for u in us])
    np.testing.assert_allclose(bench.fit_drift(us, D), [1.7, 0.5], rtol=1e-12)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the keys of the benchmark contract and the GPU arm's config."""
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
    assert line["config"]["Lx"] == 4096 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
