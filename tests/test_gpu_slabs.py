"""Slab decomposition on one GPU: a lattice split along y into slabs (lattice
handles marked with flb_set_slab) that exchange the populations crossing
their boundaries after every step (flb_halo_pack / flb_halo_unpack) gives the
whole lattice's populations bit for bit -- the noise is keyed by the global
node and every node collides the same inputs in the same arithmetic -- and its
sums add up to the lattice's (to the rounding of their summation order)."""
import numpy as np
import pytest

import oracle
from paper_1204_6734_gb300 import flb, inputs, slabs
from tolerances import assert_sums_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def _perturbed(p, seed):
    f0 = oracle.init_equilibrium(p)
    return f0 * (1 + 0.02 * inputs.perturbation(f0.shape, seed=seed))


def _run_whole(p, f, nsteps, warmup, every, kernel=None):
    with flb.Lattice(p, kernel=kernel) as lat:
        lat.set_populations(f)
        lat.set_sampling(warmup, every)
        lat.step(nsteps)
        lat.sync()
        return lat.populations(), lat.raw_sums()


@pytest.mark.parametrize("nslabs", [1, 2, 3])
@pytest.mark.parametrize("basis", [inputs.STANDARD, inputs.LOCAL])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_slabs_equal_the_whole_lattice(precision, basis, nslabs):
    p = inputs.LatticeParams(300, 37, 1.0, 0.12, -0.05, 1e-3, inputs.omega_groups(1.2, 0.8, 1.4),
                             basis, precision, seed=31)
    f = _perturbed(p, seed=5)
    n, w, e = 23, 3, 2
    ref, (R1, R2, rn) = _run_whole(p, f, n, w, e)
    with slabs.LocalSlabs(p, nslabs) as s:
        s.set_populations(f)
        s.set_sampling(w, e)
        s.step(n)
        s.sync()
        got = s.populations()
        S1, S2, ns = s.raw_sums()
    np.testing.assert_array_equal(got, ref)
    assert ns == rn
    if precision == "fp64":
        np.testing.assert_allclose(S2, R2, rtol=1e-12, atol=1e-12 * rn * p.kT)
        np.testing.assert_allclose(S1, R1, rtol=1e-12, atol=1e-12 * rn * np.sqrt(p.kT))
    else:
        # the same staged values summed in other groupings
        assert_sums_close(S1, S2, R1, R2, rn, 1e-4, 1e-6 * rn * np.sqrt(p.kT), 1e-6 * rn * p.kT)


def test_fp16_store_and_table_fnorm_slabs():
    for basis, prec in ((inputs.LOCAL, "fp16dev"), (inputs.LUT, "fp32")):
        p = inputs.LatticeParams(200, 24, 1.0, 0.1, 0.02, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                                 basis, prec, seed=8)
        f = oracle.init_equilibrium(p)
        ref, _ = _run_whole(p, f, 17, 0, 0)
        with slabs.LocalSlabs(p, 2) as s:
            s.set_populations(f)
            s.step(17)
            got = s.populations()
        np.testing.assert_array_equal(got, ref)


def test_slab_reports_global_error_locations():
    p = inputs.LatticeParams(16, 12, 1.0, 0.0, 0.0, 1e-4, inputs.omega_groups(1, 1, 1),
                             inputs.LOCAL, "fp64", seed=1)
    f = oracle.init_equilibrium(p)
    f[:, 9, 5] = [0.1, 0.9, 0.1, 0.0, 0.1, 0.3, 0.0, 0.0, 0.3]     # invalid velocity at (5, 9)
    with slabs.LocalSlabs(p, 2) as s:                                 # rows 0-5 and 6-11
        s.set_populations(f)
        s.step(1)
        with pytest.raises(flb.FlbError) as e:
            s.lats[1].sync()
        assert e.value.code == flb.ERR_INVALID_VELOCITY
        assert flb.flb_error_location(s.lats[1].h) == (5 + 16 * 9, 0)


def test_slab_arguments():
    p = inputs.LatticeParams(8, 8, precision="fp64")
    with flb.Lattice(p) as lat:
        buf = 1 << 20
        with pytest.raises(flb.FlbError):
            flb.flb_halo_pack(lat.h, buf, buf)             # not a slab
        for Ly_total, y0 in ((7, 0), (16, 9), (16, -1)):
            with pytest.raises(flb.FlbError):
                flb.flb_set_slab(lat.h, Ly_total, y0)
        flb.flb_set_slab(lat.h, 16, 8)
        assert flb.flb_halo_bytes(lat.h) == 3 * 8 * 8
        with pytest.raises(flb.FlbError):
            lat.set_structure_sampling(0, 1)              # whole-lattice quantity
