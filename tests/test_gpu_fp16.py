"""The FP16 deviation store: populations kept as h = (f - c) / sqrt(kT) in FP16
(c = f^0(rho0, u0) in FP32), collided in FP32.

Tolerances, from FP16's 11-bit significand: encoding h rounds to nearest, so a
stored population is off by at most half a unit in the last place of h times
sqrt(kT); thermal deviations keep |h| below 8 (ulp <= 2^-8), so one encoding
costs at most 2^-9 sqrt(kT) = 2e-5 at kT = 1e-4. These errors are independent
from node to node and step to step; over a trajectory they random-walk in the
conserved (slow) modes, which bounds the drift from the FP64 oracle after n
steps by about sqrt(n) 2^-11 sqrt(kT) per population.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu

BASES = [inputs.STANDARD, inputs.LOCAL]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def params(basis, Lx=200, Ly=48, kT=1e-4, precision="fp16dev", seed=12):
    return inputs.LatticeParams(Lx, Ly, 1.0, 0.2, 0.0, kT, inputs.omega_groups(1.0, 0.8, 1.0),
                                basis, precision, seed=seed)


def codec(p):
    ref = oracle.feq(p.rho0, p.ux0, p.uy0).astype(np.float32).astype(np.float64)
    return ref[:, None, None], float(np.float32(np.sqrt(p.kT)))


def encode(f, p):
    ref, s = codec(p)
    return np.float16((f - ref) / s)


def decode(h, p):
    ref, s = codec(p)
    return ref + s * h.astype(np.float64)


def test_kT_zero_is_rejected():
    with pytest.raises(flb.FlbError) as e:
        flb.Lattice(params(inputs.LOCAL, kT=0.0))
    assert e.value.code == flb.ERR_ARG


@pytest.mark.parametrize("shape", [(1, 1), (37, 19), (130, 9)])
def test_roundtrip_is_the_fp16_encoding(shape):
    p = params(inputs.LOCAL, *shape)
    f0 = oracle.init_equilibrium(p)
    f = f0 * (1 + 0.02 * inputs.perturbation(f0.shape, seed=3))
    with flb.Lattice(p) as lat:
        # the initial state is h = 0: f = c in FP32
        np.testing.assert_array_equal(lat.populations(), np.broadcast_to(codec(p)[0], f0.shape))
        lat.set_populations(f)
        back = lat.populations()
    np.testing.assert_allclose(back, decode(encode(f, p), p), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("basis", BASES + [inputs.LUT])
def test_one_step_is_fp32_then_rounded(basis):
    """From a state FP16 holds exactly, one FP16-store step equals the FP32 step
    up to the rounding of the encoded result."""
    p16 = params(basis, 130, 20)
    p32 = params(basis, 130, 20, precision="fp32")
    f0 = oracle.init_equilibrium(p16)
    f = decode(encode(f0 * (1 + 0.03 * inputs.perturbation(f0.shape, seed=5)), p16), p16)
    out = {}
    for p in (p16, p32):
        with flb.Lattice(p) as lat:
            lat.set_populations(f)
            lat.step(1)
            out[p.precision] = lat.populations()
    _, s = codec(p16)
    h32 = (out["fp32"] - codec(p16)[0]) / s
    bound = 0.5 * np.spacing(np.abs(np.float16(h32))).astype(np.float64) * s + 1e-7
    assert np.all(np.abs(out["fp16dev"] - out["fp32"]) <= bound)


@pytest.mark.parametrize("basis", BASES)
def test_trajectory_and_correlations_against_oracle(basis):
    p = params(basis)
    nsteps, warm = 300, 100
    run = oracle.Run(p, warmup=warm, every=1).step(nsteps)
    with flb.Lattice(p) as lat:
        lat.set_sampling(warm, 1)
        lat.step(nsteps)
        lat.sync()
        f = lat.populations()
        Cff, CMM, mean, n = lat.correlations(basis)
    assert n == run.nsamp
    assert np.abs(f - run.f).max() < 4 * np.sqrt(nsteps) * 2.0 ** -11 * np.sqrt(p.kT)
    C_ref, _ = run.covariance()
    assert np.abs(Cff - C_ref).max() < 0.01 * p.kT * 4.0 / 9.0
    assert np.abs(CMM - run.moment_covariance(basis)).max() < 0.01 * p.kT


def test_table_basis_correlations_against_oracle():
    """The look-up-table f-norm on the FP16 store: its table cell is an FP32
    decision on the decoded state, which may differ from the FP64 oracle's at
    a node near a cell edge, so the check is on the correlations (1 %)."""
    p = params(inputs.LUT)
    nsteps, warm = 300, 100
    run = oracle.Run(p, warmup=warm, every=1).step(nsteps)
    with flb.Lattice(p) as lat:
        lat.set_sampling(warm, 1)
        lat.step(nsteps)
        Cff, CMM, mean, n = lat.correlations("local")
    assert n == run.nsamp
    C_ref, _ = run.covariance()
    assert np.abs(Cff - C_ref).max() < 0.01 * p.kT * 4.0 / 9.0
    assert np.abs(CMM - run.moment_covariance("local")).max() < 0.01 * p.kT


def test_mass_and_momentum_drift_is_rounding_only():
    p = params(inputs.LOCAL, 256, 256)
    with flb.Lattice(p) as lat:
        before = lat.conservation()
        lat.step(50)
        after = lat.conservation()
    N = p.Lx * p.Ly
    # 9 N independent roundings per step of at most 2^-9 sqrt(kT) each
    assert np.all(np.abs(after - before) <= 50 * 3 * np.sqrt(9 * N) * 2.0 ** -9 * np.sqrt(p.kT))


def test_state_difference_matches_host():
    p16, p64 = params(inputs.LOCAL, 64, 40), params(inputs.LOCAL, 64, 40, precision="fp64")
    with flb.Lattice(p16) as a, flb.Lattice(p64) as b:
        a.step(7)
        b.step(7)
        mx, rms, mb = flb.flb_state_difference(a.h, b.h)
        fa, fb = a.populations(), b.populations()
    d = fa - fb
    assert mx == pytest.approx(np.abs(d).max(), rel=1e-12, abs=1e-300)
    assert rms == pytest.approx(np.sqrt((d ** 2).mean()), rel=1e-12)
    assert mb == pytest.approx(np.abs(fb).max(), rel=1e-15)
