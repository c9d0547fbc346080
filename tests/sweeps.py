"""The u_x0 sweep of the paper's 21 x 21 lattice shared by the drift-fit tests:
kT = 1e-4, shear 1.0, bulk 0.8, ghost 1.0, u_x0 in US, seed 40 + k, 6500 steps
sampled every step after 500, each run measured in its own basis at u0."""
import numpy as np

from paper_1204_6734_gb300 import drift, inputs

KT = 1e-4
OMEGA = inputs.omega_groups(1.0, 0.8, 1.0)
US = np.array([0.05, 0.1, 0.15, 0.2, 0.25])
STEPS, WARMUP = 6500, 500


def sweep_params(basis, precision):
    return [inputs.LatticeParams(21, 21, 1.0, u, 0.0, KT, OMEGA, basis, precision, seed=40 + k)
            for k, u in enumerate(US)]


def oracle_sweep(oracle, basis):
    """Normalised moment correlators (len(US) x 9 x 9) of the oracle's runs."""
    D = []
    for p in sweep_params(basis, "fp64"):
        run = oracle.Run(p, warmup=WARMUP, every=1).step(STEPS)
        C, _ = run.covariance()
        D.append(drift.normalised(oracle.moment_covariance(C, basis, p.ux0, 0.0), KT, 1.0))
    return np.array(D)
