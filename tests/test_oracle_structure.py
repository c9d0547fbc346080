"""Pins of the oracle's static structure factors (Eqs. sfactorr, sfactoru,
rcorrelator): drho(k) = sum_x [rho(x) - rho0] exp(-i k.x) and the same for
j - rho0 u0.

* the transform is the definition, written out as a double sum on a small
  lattice (sign of the exponent, no normalisation, index order [m_y, m_x]);
* Parseval: sum_k |a(k)|^2 = N sum_x |a(x)|^2;
* the k = 0 components vanish: total mass and momentum are conserved;
* for the ideal gas at rest the structure factors are flat in k (the isotropy
  the paper tests against): S_k(rho) = N kT and S_k(j_x) = N kT / 3 at every
  k != 0 for a lattice of N sites (per-site <drho^2> = kT rho0 and
  <dj_x^2> = kT rho0 / 3 from <dM dM> = kT rho delta), and R_k(j_x, j_y) = 0.
"""
import numpy as np
import pytest

from paper_1204_6734_gb300 import inputs


def test_dft_is_the_definition(oracle):
    rng = np.random.Generator(np.random.PCG64(4))
    Lx, Ly = 5, 3
    a = rng.standard_normal((Ly, Lx))
    want = np.zeros((Ly, Lx), dtype=complex)
    for my in range(Ly):
        for mx in range(Lx):
            for y in range(Ly):
                for x in range(Lx):
                    want[my, mx] += a[y, x] * np.exp(-2j * np.pi * (mx * x / Lx + my * y / Ly))
    np.testing.assert_allclose(oracle.dft2(a), want, atol=1e-12)


def test_parseval_and_conserved_zero_mode(oracle):
    p = inputs.LatticeParams(12, 7, 1.0, 0.1, 0.0, 1e-3, inputs.omega_groups(1.2, 0.8, 1.1),
                             "local", "fp64", seed=2)
    run = oracle.Run(p).step(30)
    dr, djx, djy = oracle.hydro_fields(run.f, p)
    a, b, c = oracle.structure_sample(run.f, p)
    N = p.Lx * p.Ly
    assert a.sum() == pytest.approx(N * (dr ** 2).sum(), rel=1e-12)
    assert b.sum() == pytest.approx(N * (djx ** 2).sum(), rel=1e-12)
    assert c.sum().real == pytest.approx(N * (djx * djy).sum(), rel=1e-10, abs=1e-20)
    assert a[0, 0] < 1e-24 and b[0, 0] < 1e-24


@pytest.mark.parametrize("basis", ["standard", "local"])
def test_ideal_gas_at_rest_is_flat_in_k(oracle, basis):
    kT = 1e-4
    p = inputs.LatticeParams(21, 21, 1.0, 0.0, 0.0, kT, inputs.omega_groups(1.0, 1.0, 1.0), basis,
                             "fp64", seed=6)
    sr = oracle.StructureRun(p, warmup=200, every=5).step(200 + 5 * 800)
    Sr, Sx, R = sr.factors()
    N = p.Lx * p.Ly
    mask = np.ones_like(Sr, dtype=bool)
    mask[0, 0] = False
    # 800 correlated samples per k: each k within 20 %, the mean over k within 2 %
    assert np.abs(Sr[mask] / (N * kT) - 1).max() < 0.2
    assert abs(Sr[mask].mean() / (N * kT) - 1) < 0.02
    assert abs(Sx[mask].mean() / (N * kT / 3) - 1) < 0.02
    assert np.abs(R[mask]).mean() < 0.05 * N * kT / 3
