"""Pins of the oracle's f-norm basis (Section 4, Eqs. fnorm, gramschmidt,
gsortho, Mtilde, fnormmeq).

The oracle builds the basis with a literal Gram-Schmidt loop. Here it is checked
against what the paper fixes (orthonormality, vanishing equilibrium moments,
the u = 0 limit), against closed forms derived from the equilibrium's moment
constraints, against a different algorithm (a LAPACK Cholesky of the Gram
matrix), and against the lattice's mirror symmetry.
"""
import numpy as np
import pytest

from paper_1204_6734_gb300 import inputs

VELS = inputs.random_velocities(40, seed=11, umax=0.35)


@pytest.mark.parametrize("k", range(0, 40, 3))
def test_orthonormal_in_f_norm(oracle, k):
    """Eq. fnorm: sum_i mt^a mt^b f_i^0(1,u) = delta^ab at the node's own u."""
    ux, uy = VELS[k]
    mt = oracle.local_basis(ux, uy)
    W = oracle.feq(1.0, ux, uy)
    np.testing.assert_allclose(mt @ np.diag(W) @ mt.T, np.eye(9), atol=2e-14)


@pytest.mark.parametrize("k", range(1, 40, 3))
def test_equilibrium_moments_vanish(oracle, k):
    """Eq. fnormmeq: Mt^{a,0} = rho delta^{a0} for the equilibrium at the same u."""
    ux, uy = VELS[k]
    rho = 0.5 + k / 20.0
    mt = oracle.local_basis(ux, uy)
    Meq = mt @ oracle.feq(rho, ux, uy)
    expect = np.zeros(9)
    expect[0] = rho
    np.testing.assert_allclose(Meq, expect, atol=5e-15 * rho)


def test_rest_limit_is_hermite(oracle):
    """Eq. u=0: at u = 0 the f-norm is the Hermite norm, and the Gram-Schmidt of
    the Hermite rows returns them unchanged."""
    _, _, _, m, _ = oracle.tables()
    np.testing.assert_allclose(oracle.local_basis(0.0, 0.0), m, atol=1e-15)


@pytest.mark.parametrize("k", range(2, 40, 4))
def test_conserved_rows_closed_form(oracle, k):
    """mt^0 = 1 and mt^{1,2} = sqrt(3)(v - u): with sum_i W_i v_a v_b = theta d_ab
    + u_a u_b (Eq. d2q9f0) these are the normalised projections of rho, j."""
    vx, vy, _, _, _ = oracle.tables()
    ux, uy = VELS[k]
    mt = oracle.local_basis(ux, uy)
    np.testing.assert_allclose(mt[0], 1.0, atol=1e-15)
    np.testing.assert_allclose(mt[1], np.sqrt(3) * (vx - ux), atol=1e-14)
    np.testing.assert_allclose(mt[2], np.sqrt(3) * (vy - uy), atol=1e-14)


@pytest.mark.parametrize("k", range(3, 40, 4))
def test_equals_cholesky_construction(oracle, k):
    """Gram-Schmidt in a fixed order equals L^{-1} P with L the lower Cholesky
    factor (positive diagonal) of the Gram matrix G = P diag(W) P^T, computed
    here by LAPACK. This fixes the order of the start vectors, the square-root
    normalisation and the sign convention."""
    _, _, _, P, _ = oracle.tables()
    ux, uy = VELS[k]
    W = oracle.feq(1.0, ux, uy)
    G = P @ np.diag(W) @ P.T
    L = np.linalg.cholesky(G)
    ref = np.linalg.solve(L, P)
    np.testing.assert_allclose(oracle.local_basis(ux, uy), ref, atol=5e-14)


@pytest.mark.parametrize("k", range(0, 40, 5))
def test_triangular_in_start_vectors(oracle, k):
    """Each mt^a lies in span(p^0..p^a) with a positive coefficient on p^a."""
    _, _, w, P, n = oracle.tables()
    ux, uy = VELS[k]
    mt = oracle.local_basis(ux, uy)
    T = mt @ n          # coefficients in the Hermite rows (P n = I)
    assert np.abs(np.triu(T, 1)).max() < 1e-13
    assert np.all(np.diag(T) > 0)


def test_mirror_symmetry(oracle):
    """Reflecting y -> -y permutes the velocities (2<->4, 5<->8, 6<->7) and flips
    the sign of the y-odd moments (j_y, Pi_xy, q_y); the basis must follow."""
    perm = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5])
    sign = np.array([1, 1, -1, 1, -1, 1, 1, -1, 1], dtype=float)
    for ux, uy in VELS[:10]:
        a = oracle.local_basis(ux, uy)
        b = oracle.local_basis(ux, -uy)
        np.testing.assert_allclose(b[:, perm], sign[:, None] * a, atol=1e-14)


def test_x_y_exchange_symmetry(oracle):
    """Exchanging x and y permutes the velocities (1<->2, 3<->4, 6<->8); the
    density row is invariant and the two momentum rows map onto each other."""
    perm = np.array([0, 2, 1, 4, 3, 5, 8, 7, 6])
    for ux, uy in VELS[10:16]:
        a = oracle.local_basis(ux, uy)
        b = oracle.local_basis(uy, ux)
        np.testing.assert_allclose(b[0][perm], a[0], atol=1e-14)
        # j_x(u) maps to j_y(u') and vice versa for the first three rows
        np.testing.assert_allclose(b[1][perm], a[2], atol=1e-14)
        np.testing.assert_allclose(b[2][perm], a[1], atol=1e-14)
