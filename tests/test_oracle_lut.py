"""Pins of the oracle's look-up-table f-norm (Section 4, the practical variant
the paper's f-norm figures use): the basis at the nearest velocity u_g of a
51 x 51 table (spacing 0.02, |u_g| <= 0.5) instead of the node's own u.

* the table velocity is the nearest grid velocity (brute force over the grid),
  and velocities off the table or at table points where some f_i^0(1, u_g) <= 0
  are errors (Fig. 11: the paper's run fails there);
* mass and momentum are conserved exactly with the noise on, for any u;
* one common rate without noise is BGK exactly, whatever u_g is (the projected
  equilibrium moments make the conserved part cancel);
* on a table velocity the variant is the fully local f-norm collision;
* off the table velocities it differs from it, by an amount of the order of
  the grid spacing times the non-equilibrium part;
* on a 1x1 lattice (u frozen at an off-grid u0) the moments in the table basis
  have the FDT variance kT rho0 and lag-1 autocorrelation 1 - omega_a.
"""
import numpy as np
import pytest

from paper_1204_6734_gb300 import inputs


def params(omega=(1.3, 0.7, 1.6), kT=1e-3, ux0=0.0, uy0=0.0, seed=5, Lx=1, Ly=1):
    return inputs.LatticeParams(Lx, Ly, 1.0, ux0, uy0, kT, inputs.omega_groups(*omega), "lut",
                                "fp64", seed=seed)


def state(oracle, ux, uy, rho=0.9, amp=0.04, seed=1):
    return oracle.feq(rho, ux, uy) * (1 + amp * inputs.perturbation(9, seed=seed))


def velocity(oracle, g):
    vx, vy, *_ = oracle.tables()
    rho = g.sum()
    return g @ vx / rho, g @ vy / rho


def test_table_velocity_is_the_nearest_grid_point(oracle):
    grid = np.arange(-25, 26) / 50.0
    rng = np.random.Generator(np.random.PCG64(8))
    for ux, uy in rng.uniform(-0.509, 0.509, size=(2000, 2)):
        gx, gy = oracle.lut_velocity(ux, uy)
        assert gx == grid[np.argmin(np.abs(grid - ux))]
        assert gy == grid[np.argmin(np.abs(grid - uy))]
    # ties round up; the edge of the table
    assert oracle.lut_velocity(0.01, -0.01) == (0.02, 0.0)
    assert oracle.lut_velocity(0.5099, -0.5099)[0] == 0.5
    for u in ((0.511, 0.0), (0.0, -0.511), (np.nan, 0.0)):
        with pytest.raises(oracle.OracleError):
            oracle.lut_velocity(*u)


@pytest.mark.parametrize("k", range(6))
def test_conserves_mass_and_momentum(oracle, k):
    vx, vy, *_ = oracle.tables()
    u = inputs.random_velocities(1, seed=300 + k, umax=0.3)[0]
    g = state(oracle, *u, seed=k)
    fs = oracle.collide_node(params(), g, node=k, step=3)
    assert fs.sum() == pytest.approx(g.sum(), rel=1e-14)
    assert fs @ vx == pytest.approx(g @ vx, abs=1e-14)
    assert fs @ vy == pytest.approx(g @ vy, abs=1e-14)
    assert np.abs(fs - g).max() > 1e-4


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.7])
def test_single_rate_without_noise_is_bgk(oracle, omega):
    for k in range(6):
        u = inputs.random_velocities(1, seed=400 + k, umax=0.3)[0]
        g = state(oracle, *u, seed=10 + k)
        rho = g.sum()
        f0 = oracle.feq(rho, *velocity(oracle, g))
        fs = oracle.collide_node(params((omega,) * 3, kT=0.0), g, k, 0)
        np.testing.assert_allclose(fs, f0 + (1 - omega) * (g - f0), atol=3e-15)


def on_grid_state(oracle, ugx, ugy, seed):
    """Populations with velocity u_g (to rounding): f^0(rho, u_g) plus a
    perturbation without mass or momentum."""
    vx, vy, w, *_ = oracle.tables()
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal(9) * 0.01
    # remove the components along 1, v_x, v_y (least squares, exact to rounding)
    A = np.stack([np.ones(9), vx, vy], axis=1).astype(float)
    d -= A @ np.linalg.lstsq(A, d, rcond=None)[0]
    return oracle.feq(0.95, ugx, ugy) + d


@pytest.mark.parametrize("ug", [(0.0, 0.0), (0.1, 0.0), (0.2, -0.14), (-0.3, 0.26)])
def test_on_a_table_velocity_it_is_the_local_f_norm(oracle, ug):
    g = on_grid_state(oracle, *ug, seed=int(1000 * (ug[0] + 1)))
    assert oracle.lut_velocity(*velocity(oracle, g)) == ug
    pl = params(seed=9)
    pl.basis = "local"
    for step in range(3):
        a = oracle.collide_node(params(seed=9), g, 17, step)
        b = oracle.collide_node(pl, g, 17, step)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_off_the_table_velocities_it_differs_from_the_local_f_norm(oracle):
    pl = params(kT=0.0)
    pl.basis = "local"
    for du in (0.004, 0.009):
        g = state(oracle, 0.2 + du, -0.1, seed=3)
        a = oracle.collide_node(params(kT=0.0), g, 0, 0)
        b = oracle.collide_node(pl, g, 0, 0)
        diff = np.abs(a - b).max()
        noneq = np.abs(g - oracle.feq(g.sum(), *velocity(oracle, g))).max()
        assert 1e-9 < diff < 3 * 0.02 * noneq


def test_invalid_table_velocity_is_an_error(oracle):
    # u = (0.48, 0.48): on the table, but f_3^0(1, u_g) < 0 there (Fig. 11)
    g = oracle.feq(1.0, 0.48, 0.48)
    assert oracle.lut_velocity(0.48, 0.48) == (0.48, 0.48)
    with pytest.raises(oracle.OracleError):
        oracle.collide_node(params(kT=0.0), g, 0, 0)


@pytest.mark.parametrize("u0", [(0.105, 0.0), (0.213, -0.071)])
def test_single_node_fdt_in_the_table_basis(oracle, u0):
    kT, rho0 = 1e-3, 1.0
    om = np.array(inputs.omega_groups(1.4, 0.6, 1.2))
    p = params(tuple(om[[3, 5, 6]]), kT=kT, ux0=u0[0], uy0=u0[1], seed=21)
    run = oracle.Run(p)
    run.step(200)
    n = 40000
    F = np.empty((n, 9))
    for t in range(n):
        run.step(1)
        F[t] = run.f[:, 0, 0]
    rows = oracle.local_basis(*oracle.lut_velocity(*u0))
    M = F @ rows.T
    nb = 40
    var_b = M[:, 3:].reshape(nb, n // nb, 6).var(axis=1)
    var, err = var_b.mean(axis=0), var_b.std(axis=0) / np.sqrt(nb)
    assert np.all(np.abs(var - kT * rho0) < 5 * err + 1e-3 * kT), var / (kT * rho0)
    Mc = M[:, 3:] - M[:, 3:].mean(0)
    ac = (Mc[1:] * Mc[:-1]).mean(0) / Mc.var(0)
    np.testing.assert_allclose(ac, 1 - om[3:], atol=5 / np.sqrt(n))
