"""Pins of the oracle's collision (Eq. LBEMRT with the Hermite basis of the
appendix or the f-norm basis of Section 4).

* exact per-node conservation of rho and j with the noise on (Eq. LBE1 text);
* zero noise and one common rate: both bases reduce to BGK (Eq. LBE1 with
  Lambda = -omega I), and at omega = 1 to the local equilibrium;
* the noise has the covariance the FDT prescribes (Eqs. FDT, noiseamp):
  kT rho omega_a (2 - omega_a) per non-conserved moment of the colliding node.
"""
import numpy as np
import pytest

from paper_1204_6734_gb300 import inputs

BASES = ["standard", "local"]


def params(basis, omega=(1.0, 1.0, 1.0), kT=1e-4, seed=3, ux0=0.0):
    return inputs.LatticeParams(1, 1, 1.0, ux0, 0.0, kT, inputs.omega_groups(*omega), basis,
                                "fp64", seed=seed)


def random_state(oracle, k, amp=0.05):
    """Populations of a node near equilibrium at a random velocity."""
    ux, uy = inputs.random_velocities(1, seed=100 + k, umax=0.25)[0]
    rho = 0.8 + 0.05 * k
    g = oracle.feq(rho, ux, uy) * (1 + amp * inputs.perturbation(9, seed=200 + k))
    return g


@pytest.mark.parametrize("basis", BASES)
@pytest.mark.parametrize("k", range(6))
def test_conserves_mass_and_momentum(oracle, basis, k):
    vx, vy, *_ = oracle.tables()
    g = random_state(oracle, k)
    p = params(basis, omega=(1.3, 0.7, 1.6), kT=1e-3)
    fs = oracle.collide_node(p, g, node=k, step=7)
    assert fs.sum() == pytest.approx(g.sum(), rel=1e-14)
    assert fs @ vx == pytest.approx(g @ vx, abs=1e-14)
    assert fs @ vy == pytest.approx(g @ vy, abs=1e-14)
    assert np.abs(fs - g).max() > 1e-4          # something did happen


@pytest.mark.parametrize("basis", BASES)
@pytest.mark.parametrize("omega", [0.6, 1.0, 1.7])
def test_single_rate_without_noise_is_bgk(oracle, basis, omega):
    vx, vy, *_ = oracle.tables()
    for k in range(5):
        g = random_state(oracle, k)
        rho = g.sum()
        ux, uy = g @ vx / rho, g @ vy / rho
        f0 = oracle.feq(rho, ux, uy)
        fs = oracle.collide_node(params(basis, (omega,) * 3, kT=0.0), g, k, 0)
        np.testing.assert_allclose(fs, f0 + (1 - omega) * (g - f0), atol=2e-15)


@pytest.mark.parametrize("basis", BASES)
def test_noise_covariance_matches_fdt_amplitude(oracle, basis):
    """Over many independent draws at a fixed pre-collision state, the moments of
    f* in the basis used by the collision have covariance
    diag(kT rho omega_a (2 - omega_a)) on a = 3..8 and zero on a = 0..2."""
    vx, vy, w, m, _ = oracle.tables()
    g = 1.7 * random_state(oracle, 3)      # local rho far from rho0 = 1
    rho = g.sum()
    ux, uy = g @ vx / rho, g @ vy / rho
    om = (1.3, 0.7, 1.6)
    kT = 1e-3
    p = params(basis, om, kT=kT)
    basis_rows = m if basis == "standard" else oracle.local_basis(ux, uy)
    n = 20000
    M = np.array([basis_rows @ oracle.collide_node(p, g, 0, s) for s in range(n)])
    cov = np.cov(M.T)
    omega = np.array(inputs.omega_groups(*om))
    expect = np.zeros(9)
    expect[3:] = kT * rho * omega[3:] * (2 - omega[3:])
    np.testing.assert_allclose(np.diag(cov)[:3], 0.0, atol=1e-20)
    for a in range(3, 9):
        assert cov[a, a] == pytest.approx(expect[a], rel=5 * np.sqrt(2 / n)), a
    off = cov[3:, 3:] - np.diag(np.diag(cov[3:, 3:]))
    assert np.abs(off).max() < 5 * kT * rho / np.sqrt(n)


@pytest.mark.parametrize("basis", BASES)
def test_invalid_velocity_is_an_error(oracle, basis):
    """A node whose velocity leaves the region f_i^0(1,u) > 0 (Fig. 11): the
    f-norm has no basis and the oracle reports it; the Hermite basis does not
    need one."""
    g = np.array([0.1, 0.9, 0.1, 0.0, 0.1, 0.3, 0.0, 0.0, 0.3])   # u_x ~ 0.8
    p = params(basis, kT=0.0)
    if basis == "local":
        with pytest.raises(oracle.OracleError) as e:
            oracle.collide_node(p, g, 0, 0)
        assert e.value.code == -3
    else:
        oracle.collide_node(p, g, 0, 0)


@pytest.mark.parametrize("basis", BASES)
def test_total_mass_and_momentum_do_not_drift(oracle, basis):
    """Eq. LBEMRT adds sum_a n^a_i dM^a with dM^a = 0 for the conserved moments,
    so the totals change only by rounding of random sign: after 4000 steps of a
    noisy 6x5 lattice they agree with the start to 1e-13 (a systematic bias of
    one ulp per step would give ~1e-12)."""
    vx, vy, *_ = oracle.tables()
    p = inputs.LatticeParams(6, 5, 1.0, 0.1, -0.05, 1e-3, inputs.omega_groups(1.3, 0.7, 1.6),
                             basis, "fp64", seed=8)
    run = oracle.Run(p)
    tot0 = [run.f.sum(), np.einsum("i,iyx->", vx, run.f), np.einsum("i,iyx->", vy, run.f)]
    run.step(4000)
    tot1 = [run.f.sum(), np.einsum("i,iyx->", vx, run.f), np.einsum("i,iyx->", vy, run.f)]
    assert abs(tot1[0] - tot0[0]) < 1e-13 * tot0[0]
    assert abs(tot1[1] - tot0[1]) < 1e-13 * tot0[0]
    assert abs(tot1[2] - tot0[2]) < 1e-13 * tot0[0]
