"""The paper's Section 4 experiment on the GPU path: the drift of the moment
variances with the background velocity, <dM^a dM^a>/(kT rho0) - 1 = l u + q u^2
fitted over -0.25 <= u_x0 <= 0.25, in the Hermite norm and in the f-norm.
The diagonal variances are even in u_x0 (the lattice's x reflection), so the
points u_x0 >= 0 stand for their mirror images, l = 0 and
q = sum D u^2 / sum u^4.

The paper prints q for rho, Pi_xx-yy and j_y on 21x21 lattices (Hermite
1.9 / 1.6 / 1.14, f-norm look-up-table variant 0.47 / 0.54 / 0.75); its
relaxation rates are not stated. Here (512^2, shear 1.0, bulk 0.8, ghost 1.0)
both sets must land within 20 % of the printed ones and the f-norm must cut
the density and stress drift at least twofold: the qualitative and
quantitative claim of Figs. 7 and 18. Statistical error of q at this size:
about 0.02.
"""
import json
import os

import numpy as np
import pytest

import sweeps
from paper_1204_6734_gb300 import drift, flb, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_q_coefficients.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def sweep(basis, side=512, steps=3000, warm=300):
    us = [u for u in inputs.SWEEP_UX0 if u <= 0.25]
    D = []
    for u in us:
        p = inputs.single_lattice(u, basis, side=side)
        with flb.Lattice(p) as lat:
            lat.set_sampling(warm, 1)
            lat.step(steps)
            _, CMM, _, _ = lat.correlations(basis)
        D.append(np.diag(CMM) / (p.kT * p.rho0) - 1.0)
    return drift.fit_diagonal_q(us, np.array(D))


def test_drift_coefficients():
    gold = json.load(open(GOLD))
    idx = gold["moments"]
    qh = sweep("standard")
    qf = sweep("local")
    for name, a in idx.items():
        assert qh[a] == pytest.approx(gold["q_hermite"][name], rel=0.2)
        assert qf[a] == pytest.approx(gold["q_fnorm"][name], rel=0.2)
    for name in ("rho", "Pi_xx-yy"):
        a = idx[name]
        assert qf[a] < 0.5 * qh[a]
    assert qf[idx["j_y"]] < qh[idx["j_y"]]


def test_gpu_fit_equals_oracle_fit(oracle):
    """The paper's fit of all 45 correlators (paper_1204_6734_gb300.drift) applied
    to FP32 runs on the GPU agrees with the same fit applied to the oracle's FP64
    runs of the same 21 x 21 lattices (same seeds, so the same noise draws):
    every correlator within 1 % of kT (the FP32 tolerance on <dM dM>) carries
    into l and q through the fit's weights."""
    us = sweeps.US
    tol_l = 0.01 * np.abs(us).sum() / (us ** 2).sum()
    tol_q = 0.01 * (us ** 2).sum() / (us ** 4).sum()
    fits = {}
    for basis in ("standard", "local"):
        D = []
        for p in sweeps.sweep_params(basis, "fp32"):
            with flb.Lattice(p) as lat:
                lat.set_sampling(sweeps.WARMUP, 1)
                lat.step(sweeps.STEPS)
                _, CMM, _, _ = lat.correlations(basis)
            D.append(drift.normalised(CMM, sweeps.KT, 1.0))
        l, q = drift.fit_lq(us, np.array(D))
        lr, qr = drift.fit_lq(us, sweeps.oracle_sweep(oracle, basis))
        assert np.abs(l - lr).max() <= tol_l, np.abs(l - lr).max()
        assert np.abs(q - qr).max() <= tol_q, np.abs(q - qr).max()
        fits[basis] = (l, q)
    # and the GPU fit carries the paper's finding on its own
    assert np.abs(fits["standard"][0]).max() > 10 * np.abs(fits["local"][0]).max()
