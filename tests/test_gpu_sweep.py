"""The paper's Section 4 experiment on the GPU path: the drift of the moment
variances with the background velocity, <dM^a dM^a>/(kT rho0) - 1 = l u + q u^2
fitted over |u_x0| <= 0.25, in the Hermite norm and in the f-norm.

The paper prints q for rho, Pi_xx-yy and j_y on 21x21 lattices (Hermite
1.9 / 1.6 / 1.14, f-norm look-up-table variant 0.47 / 0.54 / 0.75); its
relaxation rates are not stated. Here (512^2, shear 1.0, bulk 0.8, ghost 1.0)
the Hermite coefficients must land within 20 % of the printed ones and the
f-norm must cut the density and stress drift at least twofold, with the
linear terms small (|l| < 0.1): the qualitative and quantitative claim of
Figs. 7 and 18. Statistical error of q at this size: about 0.02.
"""
import json
import os

import numpy as np
import pytest

from paper_1204_6734_gb300 import flb, inputs

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
    us = np.array(us)
    A = np.stack([us, us ** 2], axis=1)
    (l, q), *_ = np.linalg.lstsq(A, np.array(D), rcond=None)
    return l, q


def test_drift_coefficients():
    gold = json.load(open(GOLD))
    idx = gold["moments"]
    lh, qh = sweep("standard")
    lf, qf = sweep("local")
    for name, a in idx.items():
        assert qh[a] == pytest.approx(gold["q_hermite"][name], rel=0.2)
        assert abs(lh[a]) < 0.1 and abs(lf[a]) < 0.1
    for name in ("rho", "Pi_xx-yy"):
        a = idx[name]
        assert qf[a] < 0.5 * qh[a]
    assert qf[idx["j_y"]] < qh[idx["j_y"]]
