"""The continuous-batching request server: every request's result is the
same whether it runs alone or in a mix that joins and leaves around it, in
either serving mode, and the same as a lattice handle stepped alone.

Tolerance: a request computes exactly what a lattice handle with the same
parameters computes (same draws, same FP32 algebra); only the order in which
its sampled terms are summed depends on the mix (FP32 per warp and tile run,
FP64 across). Sums agree to 1e-4 relative, and to 1e-6 n kT absolute for the
second moments (3e-6 n sqrt(kT) for the first) where they are near zero;
sample counts exactly.
"""
import numpy as np
import pytest

from tolerances import assert_sums_close, staged_corr_bounds
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def mix(basis=inputs.LOCAL, n=10, seed=21):
    """Small requests of uneven sizes, step counts and sampling schedules."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(n):
        Lx, Ly = int(g.integers(8, 220)), int(g.integers(3, 160))
        p = inputs.LatticeParams(Lx, Ly, 1.0, float(g.uniform(0, 0.3)), 0.0,
                                 float(np.exp(g.uniform(np.log(1e-5), np.log(1e-3)))),
                                 inputs.omega_groups(float(g.uniform(0.6, 1.8)), 1.0, 1.0),
                                 basis, "fp32", seed=500 + r, replica=r)
        steps = int(g.integers(9, 70))
        out.append((p, steps, int(g.integers(0, 5)), int(g.integers(1, 4))))
    return out


def close(a, b, n, kT):
    assert a["status"] == b["status"] == flb.OK
    assert a["n_samples"] == b["n_samples"] == n
    # per-lattice requests take their sums from the tensor cores (FP16-staged
    # deviations), batched ones from FP32 products
    assert_sums_close(a["S1"], a["S2"], b["S1"], b["S2"], n, 1e-4, 3e-6 * n * np.sqrt(kT), 1e-6 * n * kT)


def expected_samples(p, steps, warmup, every):
    return len(range(warmup, steps, every)) * p.Lx * p.Ly if every > 0 else 0


def serve(reqs, mode="batched", pool=None, slots=4, chunk=8):
    pool = pool or sum(flb.flb_batch_replica_bytes(p) for p, *_ in reqs) * 2 + (64 << 20)
    with flb.Server(reqs[0][0].basis, pool, slots, chunk, mode=mode) as s:
        ids = [s.submit(p, n, w, e) for p, n, w, e in reqs]
        res = {r["id"]: r for r in s.drain()}
        st = s.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
    assert st["finishing"] == 0
    return [res[i] for i in ids], st


@pytest.mark.parametrize("mode", ["batched", "per_lattice"])
def test_result_same_alone_and_in_the_mix(mode):
    reqs = mix()
    together, st = serve(reqs, mode=mode)
    assert st["replica_steps"] == sum(n for _, n, _, _ in reqs)
    for (p, n, w, e), got in zip(reqs, together):
        alone, _ = serve([(p, n, w, e)], mode=mode)
        ns = expected_samples(p, n, w, e)
        close(got, alone[0], ns, p.kT)
        assert got["steps"] == n
        assert got["t_submit"] <= got["t_admit"] <= got["t_done"]
        with flb.Lattice(p, kernel="pipelined") as lat:
            lat.set_sampling(w, e)
            lat.step(n)
            S1, S2, nh = lat.raw_sums()
        close(got, {"status": flb.OK, "n_samples": nh, "S1": S1, "S2": S2}, ns, p.kT)


@pytest.mark.parametrize("basis", [inputs.LOCAL, inputs.LUT])
def test_modes_agree(basis):
    reqs = mix(basis=basis, n=6, seed=3)
    a, _ = serve(reqs, mode="batched", slots=3)
    b, _ = serve(reqs, mode="per_lattice", slots=3)
    for (p, n, w, e), x, y in zip(reqs, a, b):
        close(x, y, expected_samples(p, n, w, e), p.kT)


def test_admission_respects_the_pool():
    """A pool that holds two of the requests at a time: never more than two
    run, everything completes, in submission order of admission."""
    reqs = [(inputs.LatticeParams(150, 100, 1.0, 0.1, 0.0, 1e-4, seed=k, replica=k), 30, 0, 1)
            for k in range(5)]
    one = flb.flb_batch_replica_bytes(reqs[0][0])
    with flb.Server(inputs.LOCAL, 2 * one, 8, 4) as s:
        for p, n, w, e in reqs:
            s.submit(p, n, w, e)
        seen, out = 0, []
        while len(out) < len(reqs):
            out += s.poll(wait=True)
            st = s.stats()
            seen = max(seen, st["running"])
            assert st["pool_used"] <= st["pool_size"]
    assert seen <= 2
    admits = sorted(out, key=lambda r: r["id"])
    assert all(a["t_admit"] <= b["t_admit"] for a, b in zip(admits, admits[1:]))
    for r in out:
        assert r["status"] == flb.OK and r["n_samples"] == 30 * 150 * 100


def test_submit_rejects_what_can_never_run():
    with flb.Server(inputs.LOCAL, 64 << 20, 4, 4) as s:
        with pytest.raises(flb.FlbError) as e:
            s.submit(inputs.LatticeParams(2048, 2048), 10)       # larger than the pool
        assert e.value.code == flb.ERR_OOM
        for bad in (inputs.LatticeParams(8, 8, basis=inputs.STANDARD),
                    inputs.LatticeParams(8, 8, precision="fp64"),
                    inputs.LatticeParams(8, 8, ux0=0.9)):
            with pytest.raises(flb.FlbError) as e:
                s.submit(bad, 10)
            assert e.value.code == flb.ERR_ARG
        with pytest.raises(flb.FlbError):
            s.submit(inputs.LatticeParams(8, 8), 0)


def test_failed_request_reports_its_status_only():
    """A request whose lattice goes invalid mid-run (flow too fast: some
    f_i^0(1,u) <= 0) is reported with that status; the others are unaffected."""
    reqs = mix(n=4, seed=8)
    # a large uniform kick along +x: u_x0 = 0.78 is valid at the start, and the
    # noise at kT = 0.05 soon drives some node past u^2 = 2/3
    bad = inputs.LatticeParams(40, 40, 1.0, 0.78, 0.0, 5e-2, seed=77, replica=99)
    with flb.Server(inputs.LOCAL, 256 << 20, 8, 8) as s:
        ids = [s.submit(p, n, w, e) for p, n, w, e in reqs]
        bid = s.submit(bad, 200, 0, 1)
        res = {r["id"]: r for r in s.drain()}
    assert res[bid]["status"] in (flb.ERR_INVALID_VELOCITY, flb.ERR_NONFINITE)
    ok, _ = serve(reqs)
    for (p, n, w, e), i, o in zip(reqs, ids, ok):
        close(res[i], o, expected_samples(p, n, w, e), p.kT)
