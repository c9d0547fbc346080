"""Failure detection without a GPU fault: the bounded waits of the pipelined
kernels give up after their limit, record a timeout the host reads as
FLB_ERR_TIMEOUT, and leave the context usable. The probe waits on a barrier
that nothing completes (a flag that nothing sets), for about 1 ms."""
import time

import pytest

from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def test_bounded_wait_times_out_and_the_context_survives():
    flb.flb_wait_probe(0)   # first launch of the module, not timed
    t0 = time.perf_counter()
    rc = flb.flb_wait_probe(2_000_000)
    assert rc == flb.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert flb.flb_wait_probe(-1) == flb.ERR_ARG
    p = inputs.LatticeParams(64, 16, 1.0, 0.1, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0), "local", "fp32",
                             seed=1)
    with flb.Lattice(p) as lat:
        lat.set_sampling(0, 1)
        lat.step(5)
        lat.sync()
        assert lat.t == 5
        assert lat.raw_sums()[2] == 5 * 64 * 16
