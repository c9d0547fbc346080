"""The allocation-free entry point flb_step_noalloc, for callers that cannot call
cudaMalloc (plugins whose host application owns all device memory, loops with
pre-planned memory): its output is checked against the regular lattice entry
points (flb_create / flb_set_populations / flb_step / flb_raw_sums) on two calls
in a row, at the largest lattice its fixed scratch holds, on a stream of the
caller's, and with a node whose velocity leaves the valid region. This file is
collected last on purpose."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check_two_calls(p, n1, n2, stream=None, amp=0.02):
    torch = _cuda()
    with flb.Lattice(p) as lat:
        f_init = lat.populations() * (1 + amp * inputs.perturbation((9, p.Ly, p.Lx), seed=3))
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
    torch.cuda.synchronize()
    for (t0, n, ref, (S1r, S2r, nr)) in ((0, n1, ref1, r1), (n1, n2, ref2, r2)):
        S1, S2 = flb.flb_step_noalloc(p, dev_f, dev_w, t0, n, stream=stream)
        torch.cuda.synchronize()
        got = dev_f.cpu().numpy()
        # same collision code and noise draws: equal to FP64 rounding
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
        # the sums are reduced in a different order
        np.testing.assert_allclose(S1, S1r, rtol=1e-9, atol=1e-13 * nr)
        np.testing.assert_allclose(S2, S2r, rtol=1e-9, atol=1e-16 * nr)


@pytest.mark.parametrize("basis", [inputs.STANDARD, inputs.LOCAL])
def test_noalloc_matches_lattice_entry_points(basis):
    p = inputs.LatticeParams(37, 29, 1.0, 0.1, -0.05, 1e-3, inputs.omega_groups(1.3, 0.8, 1.6),
                             basis, "fp64", seed=17)
    _check_two_calls(p, 7, 5)


def test_noalloc_at_its_largest_lattice():
    """512 x 512 = 262144 nodes fill the 1024 partial-sum blocks of the scratch exactly."""
    p = inputs.LatticeParams(512, 512, 1.0, 0.1, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             inputs.LOCAL, "fp64", seed=23)
    _check_two_calls(p, 3, 2)


def test_noalloc_on_a_caller_stream():
    torch = _cuda()
    p = inputs.LatticeParams(64, 24, 1.0, 0.05, 0.02, 1e-4, inputs.omega_groups(1.2, 0.9, 1.1),
                             inputs.LOCAL, "fp64", seed=29)
    s = torch.cuda.Stream()
    _check_two_calls(p, 4, 3, stream=s)


def test_noalloc_reports_an_invalid_velocity():
    """A node whose velocity leaves the f^0 > 0 region (Fig. 11) is reported and
    left uncollided; every other node is stepped as usual."""
    torch = _cuda()
    p = inputs.LatticeParams(16, 8, 1.0, 0.0, 0.0, 1e-4, inputs.omega_groups(1, 1, 1),
                             inputs.LOCAL, "fp64", seed=1)
    f = oracle.init_equilibrium(p)
    f[:, 3, 5] = [0.1, 0.9, 0.1, 0.0, 0.1, 0.3, 0.0, 0.0, 0.3]   # u = (1.5/1.8, 0)
    dev_f = torch.tensor(f, dtype=torch.float64, device="cuda")
    dev_w = torch.empty_like(dev_f)
    with pytest.raises(flb.FlbError) as e:
        flb.flb_step_noalloc(p, dev_f, dev_w, 0, 1)
    assert e.value.code == flb.ERR_INVALID_VELOCITY
    # the next call starts from a clean error record
    dev_f.copy_(torch.tensor(oracle.init_equilibrium(p), dtype=torch.float64))
    flb.flb_step_noalloc(p, dev_f, dev_w, 0, 2)


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises, so it cannot be captured: it is refused before
    anything is queued and the caller's capture stays valid."""
    torch = _cuda()
    p = inputs.LatticeParams(8, 8, precision="fp64")
    dev_f = torch.tensor(oracle.init_equilibrium(p), dtype=torch.float64, device="cuda")
    dev_w = torch.empty_like(dev_f)
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        with pytest.raises(flb.FlbError) as e:
            flb.flb_step_noalloc(p, dev_f, dev_w, 0, 1, stream=s)
    assert e.value.code == flb.ERR_ARG
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0


def _raw_call(s):
    """flb_step_noalloc with a hand-made flb_params and invalid device pointers:
    every case below must be rejected before any device access."""
    S1, S2 = np.zeros(9), np.zeros(81)
    return flb.load().flb_step_noalloc(C.byref(s), 1 << 20, 2 << 20, 0, 1,
                                       S1.ctypes.data_as(C.POINTER(C.c_double)),
                                       S2.ctypes.data_as(C.POINTER(C.c_double)), None)


def test_noalloc_rejects_bad_arguments():
    base = inputs.LatticeParams(16, 16, 1.0, 0.1, 0.0, 1e-4, precision="fp64")
    assert _raw_call(flb.make_params(inputs.LatticeParams(513, 512, precision="fp64"))) == flb.ERR_ARG
    assert _raw_call(flb.make_params(inputs.LatticeParams(8, 8, precision="fp32"))) == flb.ERR_ARG
    assert _raw_call(flb.make_params(inputs.LatticeParams(8, 8, basis=inputs.LUT,
                                                          precision="fp64"))) == flb.ERR_ARG
    for field, value in (("rho0", 0.0), ("rho0", math.nan), ("ux0", math.nan), ("uy0", math.inf),
                         ("kT", math.inf), ("kT", -1.0), ("reserved", 1), ("ux0", 0.9)):
        s = flb.make_params(base)
        setattr(s, field, value)
        assert _raw_call(s) == flb.ERR_ARG, (field, value)
    s = flb.make_params(base)
    s.omega[4] = 2.0
    assert _raw_call(s) == flb.ERR_ARG
