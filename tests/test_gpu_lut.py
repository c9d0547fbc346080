"""The look-up-table f-norm (Section 4, the paper's practical variant) on the
GPU against the FP64 oracle.

The table cell is an integer the floating-point velocity decides
(k = floor(50 u + 25.5)). In FP64 both sides take it in FP64, so they agree
except when u lies within a few ulp of a cell edge (never in these tests; the
single-node cases keep u at least 1e-6 from an edge). In FP32 the kernel
decides in FP32: single-node checks keep u at least 1e-3 of a cell from an
edge, and full FP32 runs are compared with the FP32 generic kernel, which
takes the same decisions on the same FP32 state.

Tolerances: FP64 single collisions 1e-14 and trajectories 1e-12 relative to
the largest population (the two sides build the basis by independent exact
algorithms); FP32 single collisions 2e-6 absolute (FP32 rounding of the
table and the arithmetic at rho ~ 1).
"""
import numpy as np
import pytest

import oracle
from tolerances import assert_sums_close, staged_corr_bounds
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def states(n, seed, umax=0.3, margin=1e-3):
    """Near-equilibrium node states whose velocity is at least `margin` (in
    table cells) away from a cell edge."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vx, vy, *_ = oracle.tables()
    out = []
    while len(out) < n:
        ux, uy = rng.uniform(-umax, umax, 2)
        rho = rng.uniform(0.6, 1.4)
        g = oracle.feq(rho, ux, uy) * (1 + 0.05 * rng.standard_normal(9))
        u = np.array([g @ vx, g @ vy]) / g.sum()
        x = 50 * u + 25.5
        if np.all(np.abs(x - np.round(x)) > margin):
            out.append(g)
    return np.array(out)


def params(precision, kT=1e-3, seed=99):
    return inputs.LatticeParams(1, 1, 1.0, 0.0, 0.0, kT, inputs.omega_groups(1.3, 0.7, 1.6), "lut",
                                precision, seed=seed)


@pytest.mark.parametrize("precision,tol,margin", [("fp64", 1e-14, 1e-6), ("fp32", 2e-6, 1e-3)])
def test_collide_nodes(precision, tol, margin):
    p = params(precision)
    g = states(400, seed=5, margin=margin)
    ids = np.arange(len(g), dtype=np.uint32) * 7919
    out, st = flb.flb_collide_nodes(p, g, ids, 42)
    assert np.all(st == 0)
    ref = np.array([oracle.collide_node(p, g[k], int(ids[k]), 42) for k in range(len(g))])
    assert np.abs(out - ref).max() < tol * np.abs(ref).max()


def test_table_velocity_gives_the_local_f_norm():
    """Nodes whose velocity is a table velocity: the table variant equals the
    fully local f-norm, on the GPU as in the oracle."""
    vx, vy, *_ = oracle.tables()
    gs = []
    for k, (ugx, ugy) in enumerate([(0.0, 0.0), (0.1, 0.0), (0.2, -0.14), (-0.3, 0.26)]):
        rng = np.random.Generator(np.random.PCG64(k))
        d = rng.standard_normal(9) * 0.01
        A = np.stack([np.ones(9), vx, vy], axis=1).astype(float)
        d -= A @ np.linalg.lstsq(A, d, rcond=None)[0]
        gs.append(oracle.feq(0.95, ugx, ugy) + d)
    g = np.array(gs)
    ids = np.arange(len(g), dtype=np.uint32)
    a, sa = flb.flb_collide_nodes(params("fp64"), g, ids, 3)
    pl = params("fp64")
    pl.basis = "local"
    b, sb = flb.flb_collide_nodes(pl, g, ids, 3)
    assert np.all(sa == 0) and np.all(sb == 0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_off_table_and_invalid_table_velocities_are_reported():
    g = np.array([oracle.feq(1.0, 0.52, 0.0), oracle.feq(1.0, 0.48, 0.48)])
    _, st = flb.flb_collide_nodes(params("fp64"), g, np.arange(2, dtype=np.uint32), 0)
    assert np.all(st == flb.ERR_INVALID_VELOCITY)


@pytest.mark.parametrize("shape", [(21, 21), (37, 19), (130, 9)])
def test_fp64_trajectory(shape):
    Lx, Ly = shape
    p = inputs.LatticeParams(Lx, Ly, 1.0, 0.13, -0.07, 1e-3, inputs.omega_groups(1.3, 0.8, 1.6),
                             "lut", "fp64", seed=3 + Lx)
    f0 = oracle.init_equilibrium(p)
    f_init = f0 * (1 + 0.02 * inputs.perturbation(f0.shape, seed=Lx * 31 + Ly))
    run = oracle.Run(p, f=f_init, warmup=5, every=3).step(60)
    with flb.Lattice(p) as lat:
        lat.set_populations(f_init)
        lat.set_sampling(5, 3)
        lat.step(60)
        lat.sync()
        f = lat.populations()
        S1, S2, n = lat.raw_sums()
    assert np.abs(f - run.f).max() / np.abs(run.f).max() < 1e-12
    assert n == run.nsamp
    np.testing.assert_allclose(S2, run.S2, rtol=1e-9, atol=1e-12 * n * 1e-3)


def test_fp32_pipelined_equals_generic():
    p = inputs.LatticeParams(1000, 77, 1.0, 0.1, 0.02, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             "lut", "fp32", seed=9)
    out = {}
    for kernel in ("generic", "pipelined"):
        with flb.Lattice(p, kernel=kernel) as lat:
            lat.set_sampling(2, 1)
            lat.step(30)
            out[kernel] = (lat.populations(), lat.raw_sums())
    # the scalar generic kernel contracts multiply-adds the packed one keeps
    # apart: a few FP32 roundings per step, 30 steps
    assert np.abs(out["generic"][0] - out["pipelined"][0]).max() < 5e-6
    S2g, S2p, n = out["generic"][1][1], out["pipelined"][1][1], out["generic"][1][2]
    S1g, S1p = out["generic"][1][0], out["pipelined"][1][0]
    assert_sums_close(S1p, S2p, S1g, S2g, n, 1e-4, 3e-6 * n * np.sqrt(p.kT), 1e-6 * n * p.kT)


def test_fp32_correlations_against_oracle():
    """FP32 trajectory of the table variant: cell decisions may differ from the
    FP64 oracle's at a few nodes near cell edges, so the check is on the
    correlations (1 % of kT w_max, as for the other bases)."""
    p = inputs.LatticeParams(200, 48, 1.0, 0.2, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             "lut", "fp32", seed=12)
    run = oracle.Run(p, warmup=100, every=1).step(600)
    with flb.Lattice(p) as lat:
        lat.set_sampling(100, 1)
        lat.step(600)
        Cff, CMM, mean, n = lat.correlations("local")
    C_ref, _ = run.covariance()
    assert n == run.nsamp
    assert np.abs(Cff - C_ref).max() < 0.01 * p.kT * 4.0 / 9.0
    assert np.abs(CMM - run.moment_covariance("local")).max() < 0.01 * p.kT
