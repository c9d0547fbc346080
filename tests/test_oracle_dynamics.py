"""Pins of the oracle's lattice dynamics (Eqs. LBE1, LBEft5, LBEft8, FDT,
fluctf2-fluctf4, dfdf).

* Linear modes at kT = 0: a small plane-wave perturbation along an eigenvector
  of the linearised one-step operator Gamma(k)(1 + J) evolves as lambda^t
  (Eqs. LBEft5, LBEft8). The operator is built here with NumPy from the
  printed tables, the equilibrium formula and a LAPACK Cholesky basis -- not
  from the oracle's Gram-Schmidt.
* The shear wave decays at the rate nu k^2, nu = (1/omega_s - 1/2)/3.
* On a 1x1 periodic lattice streaming is the identity and rho, u are frozen, so
  every non-conserved moment is an AR(1) process: stationary variance kT rho0
  (Eq. FDT with Eq. fluctf4) and lag-1 autocorrelation 1 - omega_a. The
  stationary <df_i df_j> then has a closed form: f^0-based for the f-norm,
  w-based for the Hermite norm.
"""
import numpy as np
import pytest

from paper_1204_6734_gb300 import inputs

THETA = 1.0 / 3.0


# --------------------------------------------------------------------------
# independent NumPy linearisation
# --------------------------------------------------------------------------

def _feq_np(vx, vy, w, rho, u):
    uv = u[0] * vx + u[1] * vy
    return rho * w * (1 + uv / THETA + uv ** 2 / (2 * THETA ** 2) - (u @ u) / (2 * THETA))


def _jacobian_feq(vx, vy, w, rho, u):
    """d f^0_i(rho(g), u(g)) / d g_j at a state with density rho and velocity u."""
    uv = u[0] * vx + u[1] * vy
    dfdrho = _feq_np(vx, vy, w, 1.0, u)
    dfdu = np.stack([rho * w * (vx / THETA + uv * vx / THETA ** 2 - u[0] / THETA),
                     rho * w * (vy / THETA + uv * vy / THETA ** 2 - u[1] / THETA)], 1)
    dudg = np.stack([(vx - u[0]) / rho, (vy - u[1]) / rho], 0)       # (2, 9)
    return np.outer(dfdrho, np.ones(9)) + dfdu @ dudg


def linear_operator(oracle, basis, rho0, u0, omega, k):
    vx, vy, w, P, _ = oracle.tables()
    u0 = np.asarray(u0, float)
    if basis == "standard":
        rows, Wt = P, w
    else:
        Wt = _feq_np(vx, vy, w, 1.0, u0)
        L = np.linalg.cholesky(P @ np.diag(Wt) @ P.T)
        rows = np.linalg.solve(L, P)
    relax = (Wt[:, None] * rows.T) @ np.diag(omega) @ rows      # sum_a omega_a n^a m^a
    J = np.eye(9) - relax @ (np.eye(9) - _jacobian_feq(vx, vy, w, rho0, u0))
    E = np.diag(np.exp(-1j * (k[0] * vx + k[1] * vy)))
    return E @ J


CASES = [("standard", (0.0, 0.0), (1, 12), (0, 1)),
         ("local", (0.0, 0.0), (1, 12), (0, 1)),
         ("standard", (0.1, 0.0), (1, 12), (0, 1)),
         ("local", (0.1, 0.0), (1, 12), (0, 1)),
         ("local", (0.15, -0.1), (8, 8), (1, 1)),
         ("standard", (0.15, -0.1), (8, 8), (1, 1)),
         ("local", (0.2, 0.05), (10, 1), (1, 0))]


@pytest.mark.parametrize("basis,u0,shape,mode", CASES)
def test_linear_eigenmodes(oracle, basis, u0, shape, mode):
    Lx, Ly = shape
    om = inputs.omega_groups(1.3, 0.8, 1.6)
    k = (2 * np.pi * mode[0] / Lx, 2 * np.pi * mode[1] / Ly)
    A = linear_operator(oracle, basis, 1.0, u0, np.array(om), k)
    lam, V = np.linalg.eig(A)
    x = np.arange(Lx)[None, :]
    y = np.arange(Ly)[:, None]
    phase = np.exp(1j * (k[0] * x + k[1] * y))
    eps = 1e-6
    f0 = oracle.feq(1.0, *u0)
    nsteps = 6
    for q in range(9):
        v = V[:, q] / np.abs(V[:, q]).max()
        init = f0[:, None, None] + eps * np.real(v[:, None, None] * phase[None])
        p = inputs.LatticeParams(Lx, Ly, 1.0, u0[0], u0[1], 0.0, om, basis, "fp64", seed=1)
        run = oracle.Run(p, f=init).step(nsteps)
        expect = f0[:, None, None] + eps * np.real(lam[q] ** nsteps * v[:, None, None] * phase[None])
        err = np.abs(run.f - expect).max()
        assert err < 200 * eps ** 2 + 1e-14, (q, lam[q], err)


@pytest.mark.parametrize("basis", ["standard", "local"])
@pytest.mark.parametrize("omega_s", [0.7, 1.0, 1.6])
def test_shear_wave_viscosity(oracle, basis, omega_s):
    """u_x = A sin(2 pi y / L) at rest: the amplitude decays as exp(-nu k^2 t),
    nu = (1/omega_s - 1/2) theta, to O(k^2) relative."""
    L = 96
    k = 2 * np.pi / L
    nu = (1 / omega_s - 0.5) * THETA
    A = 1e-5
    y = np.arange(L)
    f = np.stack([oracle.feq(1.0, A * np.sin(k * yy), 0.0) for yy in y], 1)[:, :, None]
    p = inputs.LatticeParams(1, L, 1.0, 0.0, 0.0, 0.0, inputs.omega_groups(omega_s, 1.0, 1.0),
                             basis, "fp64", seed=1)
    vx, *_ = oracle.tables()
    run = oracle.Run(p, f=f)
    amps = []
    t_points = [20, 120]
    t = 0
    for tp in t_points:
        run.step(tp - t)
        t = tp
        jx = np.einsum("i,iyx->y", vx.astype(float), run.f)
        amps.append(2 / L * np.sum(jx * np.sin(k * y)))
    rate = -np.log(amps[1] / amps[0]) / (t_points[1] - t_points[0])
    assert rate / k ** 2 == pytest.approx(nu, rel=0.01)


# --------------------------------------------------------------------------
# 1x1 lattice: fluctuation-dissipation closed form
# --------------------------------------------------------------------------

def _series(oracle, p, nsteps, warmup):
    run = oracle.Run(p)
    run.step(warmup)
    out = np.empty((nsteps, 9))
    for t in range(nsteps):
        run.step(1)
        out[t] = run.f[:, 0, 0]
    return out


@pytest.mark.parametrize("basis,u0", [("standard", (0.0, 0.0)), ("local", (0.0, 0.0)),
                                      ("standard", (0.2, 0.0)), ("local", (0.2, 0.0)),
                                      ("local", (0.1, -0.15))])
def test_single_node_fdt(oracle, basis, u0):
    vx, vy, w, P, _ = oracle.tables()
    kT, rho0 = 1e-3, 1.0
    om = np.array(inputs.omega_groups(1.4, 0.6, 1.2))
    p = inputs.LatticeParams(1, 1, rho0, u0[0], u0[1], kT, tuple(om), basis, "fp64", seed=21)
    n = 40000
    F = _series(oracle, p, n, warmup=200)
    rows = P if basis == "standard" else oracle.local_basis(*u0)
    M = F @ rows.T
    # conserved moments are frozen up to a few ulp of rounding per step
    assert np.abs(M[:, :3] - M[0, :3]).max() < n * 4 * np.finfo(float).eps
    nb = 40
    Mb = M[:, 3:].reshape(nb, n // nb, 6)
    var_b = Mb.var(axis=1)
    var = var_b.mean(axis=0)
    err = var_b.std(axis=0) / np.sqrt(nb)
    assert np.all(np.abs(var - kT * rho0) < 5 * err + 1e-3 * kT), (var / (kT * rho0))
    # lag-1 autocorrelation 1 - omega_a
    Mc = M[:, 3:] - M[:, 3:].mean(0)
    ac = (Mc[1:] * Mc[:-1]).mean(0) / Mc.var(0)
    np.testing.assert_allclose(ac, 1 - om[3:], atol=5 / np.sqrt(n))
    # equal-time <df df>: kT rho0 [diag(W) - sum_{a<3} n^a n^a^T], W = f^0(1,u0)
    # for the f-norm, W = w for the Hermite norm (closed form of the
    # conserved rows, no Gram-Schmidt)
    if basis == "local":
        Wt = _feq_np(vx, vy, w, 1.0, np.array(u0))
        cons = [Wt, Wt * np.sqrt(3) * (vx - u0[0]), Wt * np.sqrt(3) * (vy - u0[1])]
    else:
        Wt = w
        cons = [w * P[0], w * P[1], w * P[2]]
    expect = kT * rho0 * (np.diag(Wt) - sum(np.outer(c, c) for c in cons))
    Cf = np.cov(F.T)
    scale = kT * rho0 * np.sqrt(np.outer(Wt, Wt))
    assert np.abs(Cf - expect).max() / scale.max() < 0.03
