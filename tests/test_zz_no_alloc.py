"""The allocation-free entry point flb_step_noalloc, for callers that cannot call
cudaMalloc (code running during CUDA-graph capture, plugins whose host owns all
device memory, loops with pre-planned memory): its output is checked against
the regular lattice entry points (flb_create / flb_set_populations / flb_step /
flb_raw_sums) on two calls in a row. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("basis", [inputs.STANDARD, inputs.LOCAL])
def test_noalloc_matches_lattice_entry_points(basis):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = inputs.LatticeParams(37, 29, 1.0, 0.1, -0.05, 1e-3, inputs.omega_groups(1.3, 0.8, 1.6),
                             basis, "fp64", seed=17)
    n1, n2 = 7, 5
    with flb.Lattice(p) as lat:
        f_init = lat.populations() * (1 + 0.02 * inputs.perturbation((9, p.Ly, p.Lx), seed=3))
        lat.set_populations(f_init)
        lat.set_sampling(0, 1)
        lat.step(n1)
        ref1 = lat.populations()
        r1 = lat.raw_sums()
        flb.flb_reset_statistics(lat.h)
        lat.step(n2)
        ref2 = lat.populations()
        r2 = lat.raw_sums()

    dev_f = torch.tensor(f_init, dtype=torch.float64, device="cuda")
    dev_w = torch.empty_like(dev_f)
    for (t0, n, ref, (S1r, S2r, nr)) in ((0, n1, ref1, r1), (n1, n2, ref2, r2)):
        S1, S2 = flb.flb_step_noalloc(p, dev_f, dev_w, t0, n)
        torch.cuda.synchronize()
        got = dev_f.cpu().numpy()
        # same collision code and noise draws: equal to FP64 rounding
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
        # the sums are reduced in a different order
        np.testing.assert_allclose(S1, S1r, rtol=1e-9, atol=1e-13 * nr)
        np.testing.assert_allclose(S2, S2r, rtol=1e-9, atol=1e-16 * nr)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    p = inputs.LatticeParams(513, 512, precision="fp64")     # 262656 > 262144 nodes
    with pytest.raises(flb.FlbError) as e:
        flb.flb_step_noalloc(p, 1 << 20, 2 << 20, 0, 1)      # rejected before any device access
    assert e.value.code == flb.ERR_ARG
    q = inputs.LatticeParams(8, 8, precision="fp32")
    with pytest.raises(flb.FlbError):
        flb.flb_step_noalloc(q, 1 << 20, 2 << 20, 0, 1)
