"""Pins of the oracle's D2Q9 tables and equilibrium (appendix, Eqs. d2q9f0,
d2q9w, d2q93a, d2q93b, d2q94; Eqs. symmetry and fluctf5).

Each check compares two things the paper states independently (two printed
tables, a printed table and the orthogonality it must satisfy, a formula and
the moment constraints it is built to satisfy), so that a mistyped entry, a
wrong sign or a permuted velocity fails one of them.
"""
import itertools

import numpy as np
import pytest

THETA = 1.0 / 3.0


def test_hermite_rows_orthonormal_in_w(oracle):
    """Eq. fluctf5: sum_i m^a_i m^b_i w_i = delta^ab for the printed m."""
    _, _, w, m, _ = oracle.tables()
    np.testing.assert_allclose(m @ np.diag(w) @ m.T, np.eye(9), atol=1e-15)


def test_back_transform_is_m_times_w(oracle):
    """Below Eq. d2q93b: n^a_i = m^a_i w_i -- two printed tables agree."""
    _, _, w, m, n = oracle.tables()
    np.testing.assert_allclose(n, (m * w[None, :]).T, atol=1e-16)


def test_biorthogonality(oracle):
    """Eq. symmetry: sum_i m^a_i n^b_i = delta^ab and sum_a m^a_i n^a_j = delta_ij."""
    _, _, _, m, n = oracle.tables()
    np.testing.assert_allclose(m @ n, np.eye(9), atol=1e-15)
    np.testing.assert_allclose(n @ m, np.eye(9), atol=1e-15)


def test_weights_and_lattice_isotropy(oracle):
    """Eq. d2q9w: the weights sum to one and give the isotropic second moment
    theta = 1/3 and fourth moment theta^2 (the lattice symmetry f^0 relies on)."""
    vx, vy, w, _, _ = oracle.tables()
    assert w.sum() == pytest.approx(1.0, abs=1e-16)
    v = np.stack([vx, vy], 1).astype(float)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, v, v), THETA * np.eye(2), atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, v, v, v, v)
    d = np.eye(2)
    iso = THETA ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(four, iso, atol=1e-16)
    # odd moments vanish
    assert np.abs(w @ v).max() == 0.0


def test_velocity_order_matches_hermite_rows(oracle):
    """The velocity order (Fig. 1 is not available) is the one the j rows of
    Eq. d2q93a imply, and the named moments of Eq. d2q93a are the stress and
    ghost polynomials of those velocities."""
    vx, vy, w, m, _ = oracle.tables()
    s3 = np.sqrt(3.0)
    np.testing.assert_allclose(m[0], 1.0)
    np.testing.assert_allclose(m[1], s3 * vx, atol=1e-15)
    np.testing.assert_allclose(m[2], s3 * vy, atol=1e-15)
    # the velocity set is the full D2Q9 set, each vector once
    assert sorted(zip(vx, vy)) == sorted(itertools.product((-1, 0, 1), repeat=2))
    # Pi_xx-yy is proportional to vx^2 - vy^2, Pi_xy to vx vy
    c = m[3] / np.where(vx ** 2 - vy ** 2 != 0, vx ** 2 - vy ** 2, np.inf)
    assert np.allclose(m[3][vx ** 2 == vy ** 2], 0)
    assert np.allclose(c[vx ** 2 != vy ** 2], c[vx ** 2 != vy ** 2][0])
    assert np.allclose(m[4][vx * vy == 0], 0)
    assert np.allclose(m[4][vx * vy != 0] / (vx * vy)[vx * vy != 0], 3.0)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.3, 0.1, -0.05), (0.7, -0.2, 0.25),
                                       (2.0, 0.3, 0.0)])
def test_equilibrium_moment_constraints(oracle, rho, ux, uy):
    """Eq. d2q9f0 reproduces density, momentum and the isothermal momentum flux
    rho (theta I + u u) exactly (Qian's construction)."""
    vx, vy, _, _, _ = oracle.tables()
    f0 = oracle.feq(rho, ux, uy)
    v = np.stack([vx, vy], 1).astype(float)
    u = np.array([ux, uy])
    assert f0.sum() == pytest.approx(rho, rel=1e-15)
    np.testing.assert_allclose(f0 @ v, rho * u, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f0, v, v),
                               rho * (THETA * np.eye(2) + np.outer(u, u)), atol=1e-15)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.3, 0.1, -0.05), (0.7, -0.2, 0.25)])
def test_hermite_equilibrium_moments(oracle, rho, ux, uy):
    """Eq. d2q94 equals the forward transform (Eq. d2q93a) of Eq. d2q9f0,
    including exactly vanishing ghost moments."""
    _, _, _, m, _ = oracle.tables()
    np.testing.assert_allclose(m @ oracle.feq(rho, ux, uy), oracle.hermite_meq(rho, ux, uy),
                               atol=2e-15)


def test_equilibrium_positivity_region(oracle):
    """Section 4 / Fig. 11: the f-norm basis exists exactly where every
    f_i^0(1,u) > 0; outside it the oracle reports an invalid velocity. The region
    contains |u| < 0.3 and excludes the corners of the 51x51 table (|u_x| = |u_y| = 0.5)."""
    vx, vy, w, _, _ = oracle.tables()
    for ux in np.linspace(-0.8, 0.8, 33):
        for uy in np.linspace(-0.8, 0.8, 33):
            f0 = oracle.feq(1.0, ux, uy)
            ok = bool(np.all(f0 > 0))
            try:
                oracle.local_basis(ux, uy)
                got = True
            except oracle.OracleError as e:
                assert e.code == -3
                got = False
            assert got == ok, (ux, uy)
    for phi in np.linspace(0, 2 * np.pi, 24, endpoint=False):
        assert np.all(oracle.feq(1.0, 0.3 * np.cos(phi), 0.3 * np.sin(phi)) > 0)
    assert np.any(oracle.feq(1.0, 0.5, 0.5) <= 0)
