"""Batches of uneven FP32 lattices in one launch per step, against lattice
handles stepped alone (same parameters, seeds and replica ids) and against the
FP64 oracle.

Tolerances: every replica is the same computation as a lattice handle with the
same parameters -- the same draws and the same algebra on the same FP32 state.
The 2-nodes-per-thread tile shapes run the identical packed FP32x2 arithmetic,
so their populations are expected bit-identical to the one-lattice pipelined
kernel; the scalar 1-node-per-thread shape may round differently in the last
bit (scalar FMA contraction), so it is held to 1e-6 absolute at rho0 = 1 over a
few dozen steps. Sums are FP32 per warp and FP64 across warps in a different
order than the one-lattice kernel: 1e-4 relative, and absolute 1e-6 n kT for
the second moments (3e-6 n sqrt(kT) for the first), about 20 FP32 roundings
of the sum of |terms| (|df| ~ sqrt(kT)), for entries that are near zero.
"""
import numpy as np
import pytest

import oracle
from tolerances import assert_sums_close, staged_corr_bounds
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu

BASES = [inputs.STANDARD, inputs.LOCAL]
# the look-up-table f-norm: its table cell is an FP32 decision, so it is held
# to the lattice handles (same decisions), not to the FP64 oracle
ALL_BASES = BASES + [inputs.LUT]
TILES = list(flb.TILE)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


def uneven(basis, n=8, seed=11):
    """Small replicas of ragged sizes (partial tiles in x and y, one-node
    lattices, more than one tile column; for the mixed tiling, every kind of
    column band: 32, 64, 64 + 32 and a 128-wide last column) with their own u0,
    kT, rates, seeds."""
    shapes = [(37, 29), (64, 64), (130, 17), (1, 1), (200, 131), (5, 3), (129, 9), (110, 7)][:n]
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r, (Lx, Ly) in enumerate(shapes):
        out.append(inputs.LatticeParams(
            Lx, Ly, 1.0, float(g.uniform(0, 0.25)), float(g.uniform(-0.05, 0.05)),
            float((1e-5, 1e-4, 1e-3)[r % 3]), inputs.omega_groups(float(g.uniform(0.6, 1.8)), 0.8, 1.2),
            basis, "fp32", seed=1000 + 17 * r, replica=r))
    return out


def alone(p, nsteps, warmup=0, every=0, f_init=None):
    with flb.Lattice(p, kernel="pipelined") as lat:
        if f_init is not None:
            lat.set_populations(f_init)
        lat.set_sampling(warmup, every)
        lat.step(nsteps)
        lat.sync()
        return lat.populations(), lat.raw_sums()


def check_pop(tile, got, ref):
    if flb.TILE[tile] == flb.TILE["128x2"]:
        assert np.abs(got - ref).max() < 1e-6
    else:
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("basis", ALL_BASES)
def test_batch_equals_lattices_alone(basis, tile):
    ps = uneven(basis)
    nsteps = 23
    with flb.Batch(ps, tile=tile) as b:
        b.step(nsteps)
        b.sync()
        got = [b.populations(k) for k in range(len(ps))]
        assert b.t == nsteps
        assert all(b.replica_time(k) == nsteps for k in range(len(ps)))
    for k, p in enumerate(ps):
        ref, _ = alone(p, nsteps)
        check_pop(tile, got[k], ref)


@pytest.mark.parametrize("basis", BASES)
def test_mixed_tiling_band_boundaries(basis):
    """The mixed tiling at every width where its column bands change (the
    remainder w of the width past the 128-wide columns: 0, 1-32 one 32-wide
    band, 33-64 one 64-wide, 65-96 one of each, 97-127 one more 128-wide
    column), with heights around the band kinds' 6, 12 and 24 rows, sampled
    every step: populations bit-identical to the lattices stepped alone, sums
    within the FP32 tolerances."""
    widths = [1, 31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128, 129, 160, 193, 255, 256, 289]
    heights = [5, 6, 7, 12, 13, 24, 25, 49]
    g = np.random.Generator(np.random.PCG64(21))
    ps = []
    for r, Lx in enumerate(widths):
        Ly = heights[r % len(heights)]
        ps.append(inputs.LatticeParams(
            Lx, Ly, 1.0, float(g.uniform(0, 0.2)), float(g.uniform(-0.05, 0.05)), 1e-4,
            inputs.omega_groups(float(g.uniform(0.7, 1.6)), 0.9, 1.1), basis, "fp32",
            seed=3000 + 7 * r, replica=r))
    nsteps = 9
    with flb.Batch(ps, tile="mixed") as b:
        b.set_sampling(0, 1)
        b.step(nsteps)
        b.sync()
        got = [b.populations(k) for k in range(len(ps))]
        sums = [b.raw_sums(k) for k in range(len(ps))]
    for k, p in enumerate(ps):
        ref, ref_sums = alone(p, nsteps, warmup=0, every=1)
        np.testing.assert_array_equal(got[k], ref)
        n = sums[k][2]
        assert n == ref_sums[2]
        assert_sums_close(sums[k][0], sums[k][1], ref_sums[0], ref_sums[1], n, 1e-4,
                          3e-6 * n * np.sqrt(p.kT), 1e-6 * n * p.kT)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("basis", BASES)
def test_batch_against_oracle_with_sampling(basis, tile):
    """Perturbed initial states, sampled on every step: each replica against the
    FP64 oracle (FP32 tolerances of the one-lattice tests)."""
    ps = uneven(basis, n=5)
    f_inits = [oracle.init_equilibrium(p) * (1 + 0.02 * inputs.perturbation((9, p.Ly, p.Lx), seed=k))
               for k, p in enumerate(ps)]
    with flb.Batch(ps, tile=tile) as b:
        for k, f in enumerate(f_inits):
            b.set_populations(k, f)
        b.set_sampling(0, 1)
        b.step(5)
        b.sync()
        res = [(b.populations(k), b.raw_sums(k)) for k in range(len(ps))]
    for k, p in enumerate(ps):
        run = oracle.Run(p, f=f_inits[k], warmup=0, every=1).step(5)
        f, (S1, S2, n) = res[k]
        assert np.abs(f - run.f).max() < 2e-6
        assert n == run.nsamp
        # the 12-warp shapes take their sums on the tensor cores (FP16-staged deviations)
        assert_sums_close(S1, S2, run.S1, run.S2, n, 2e-4, 1e-7 * n, 1e-9 * n)


@pytest.mark.parametrize("basis", ALL_BASES)
def test_batch_sampling_schedule_matches_lattice(basis):
    ps = uneven(basis)
    with flb.Batch(ps) as b:
        b.set_sampling(4, 3)
        b.step(31)
        b.sync()
        sums = [b.raw_sums(k) for k in range(len(ps))]
    for k, p in enumerate(ps):
        _, (S1, S2, n) = alone(p, 31, warmup=4, every=3)
        assert sums[k][2] == n
        # the lattice's sums come from the tensor cores (FP16-staged deviations)
        assert_sums_close(sums[k][0], sums[k][1], S1, S2, n, 1e-4, 3e-6 * n * np.sqrt(p.kT),
                          1e-6 * n * p.kT)


@pytest.mark.parametrize("basis", BASES)
def test_graph_replay_equals_direct_launches(basis):
    ps = uneven(basis, n=4)
    out = []
    for graph in (0, 4):
        with flb.Batch(ps, graph_steps=graph) as b:
            b.set_sampling(1, 2)
            b.step(11)          # 2 replays of 4 launches + 3 direct launches
            b.step(5)           # 1 replay + 1 direct
            b.sync()
            assert b.t == 16
            out.append([(b.populations(k), b.raw_sums(k)) for k in range(len(ps))])
    for (fa, sa), (fb, sb) in zip(*out):
        np.testing.assert_array_equal(fa, fb)
        assert sa[2] == sb[2]
        np.testing.assert_allclose(sa[1], sb[1], rtol=1e-12, atol=0)


@pytest.mark.parametrize("basis", BASES)
def test_membership_changes(basis):
    """Replicas join at different batch steps, stop at their step limit and
    leave; a freed slot and its pool range are reused. Each replica ends where
    a lattice stepped alone for its own number of steps ends."""
    A, B, C = uneven(basis, n=3)
    pool = 3 * max(flb.flb_batch_replica_bytes(p) for p in (A, B, C))
    with flb.Batch.open(basis, 2, pool, graph_steps=3) as b:
        sa = b.add(A, nsteps=10)
        b.set_sampling(2, 1, slot=sa)
        b.step(4)
        sb = b.add(B)
        b.step(8)                       # A stops at 10 after 6 of these
        assert b.replica_time(sa) == 10 and b.replica_time(sb) == 8
        fa, suma = b.populations(sa), b.raw_sums(sa)
        with pytest.raises(flb.FlbError) as e:
            b.add(C)                    # both slots taken
        assert e.value.code == flb.ERR_OOM
        b.remove(sa)
        sc = b.add(C, nsteps=7)
        assert sc == sa
        b.step(9)                       # B to 17, C stops at 7
        b.sync()
        assert b.replica_time(sb) == 17 and b.replica_time(sc) == 7
        fb, fc = b.populations(sb), b.populations(sc)
        n, tiles, used, size = b.info()
        assert n == 2 and used <= size == pool
    ref_a, ref_suma = alone(A, 10, warmup=2, every=1)
    np.testing.assert_array_equal(fa, ref_a)
    assert suma[2] == ref_suma[2] == 8 * A.Lx * A.Ly
    assert_sums_close(suma[0], suma[1], ref_suma[0], ref_suma[1], suma[2], 1e-4,
                      3e-6 * suma[2] * np.sqrt(A.kT), 1e-6 * suma[2] * A.kT)
    np.testing.assert_array_equal(fb, alone(B, 17)[0])
    np.testing.assert_array_equal(fc, alone(C, 7)[0])


def test_autotune_reports_every_shape_and_keeps_results():
    ps = uneven(inputs.LOCAL)
    with flb.Batch(ps) as b:
        tile, ms = b.autotune(trial_steps=5)
        assert 0 <= tile < flb.TILE_COUNT and b.tile == tile
        assert np.all(ms > 0)
        assert b.t == flb.TILE_COUNT * (2 + 5)
        b.step(3)
        b.sync()
        got = [b.populations(k) for k in range(len(ps))]
    for k, p in enumerate(ps):
        ref, _ = alone(p, flb.TILE_COUNT * 7 + 3)
        assert np.abs(got[k] - ref).max() < 1e-6


def test_bad_arguments_are_rejected():
    ps = uneven(inputs.LOCAL, n=2)
    with flb.Batch(ps) as b:
        for bad in (lambda: b.raw_sums(5), lambda: b.remove(7), lambda: b.set_tile(9),
                    lambda: b.add(inputs.LatticeParams(8, 8, basis=inputs.STANDARD)),
                    lambda: b.add(inputs.LatticeParams(8, 8, precision="fp64")),
                    lambda: b.add(inputs.LatticeParams(9000, 8))):
            with pytest.raises(flb.FlbError) as e:
                bad()
            assert e.value.code == flb.ERR_ARG
        b.remove(1)
        with pytest.raises(flb.FlbError):
            b.remove(1)
        with pytest.raises(flb.FlbError) as e:
            b.add(inputs.LatticeParams(4000, 4000))    # larger than the pool
        assert e.value.code == flb.ERR_OOM


def test_invalid_replica_does_not_disturb_the_others():
    """A replica driven to an invalid velocity (some f_i^0(1,u) <= 0) reports it
    in its own status; the other replicas run on unchanged."""
    ps = uneven(inputs.LOCAL, n=3)
    with flb.Batch(ps) as b:
        bad = oracle.init_equilibrium(ps[1]).copy()
        bad[1] *= 40.0            # strong +x flow at every node: u_x > 1
        b.set_populations(1, bad)
        b.step(6)
        assert b.status(1) == flb.ERR_INVALID_VELOCITY
        assert b.status(0) == flb.OK and b.status(2) == flb.OK
        f0, f2 = b.populations(0), b.populations(2)
    np.testing.assert_array_equal(f0, alone(ps[0], 6)[0])
    np.testing.assert_array_equal(f2, alone(ps[2], 6)[0])


@pytest.mark.slow
def test_full_ensemble_sampled_replicas():
    """The 256-replica ensemble (sides log-uniform in [64, 1024]) in one batch
    with CUDA graphs: a few steps, then replicas at the smallest, median and
    largest sizes against the same lattices stepped alone."""
    ps = inputs.replica_ensemble()
    with flb.Batch(ps, graph_steps=2) as b:
        b.set_sampling(0, 1)
        b.step(5)
        b.sync()
        sizes = np.array([p.nodes for p in ps])
        pick = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(ps) // 2]), int(np.argmax(sizes))]
        got = {k: (b.populations(k), b.raw_sums(k)) for k in pick}
    for k in pick:
        f, (S1, S2, n) = got[k]
        ref, (R1, R2, rn) = alone(ps[k], 5, warmup=0, every=1)
        np.testing.assert_array_equal(f, ref)
        assert n == rn
        assert_sums_close(S1, S2, R1, R2, n, 1e-4, 3e-6 * n * np.sqrt(ps[k].kT),
                          1e-6 * n * ps[k].kT)


@pytest.mark.parametrize("tile", ["64x12", "mixed"])
def test_many_runs_per_cta(tile):
    """1216 one-tile replicas (8 per SM): every CTA meets eight runs of sampled
    tiles, more than the four it keeps in shared memory, so the later runs add
    their sums straight to the replicas' FP64 sums. Every replica has its
    sample count, and the replicas checked have their populations and sums
    as the lattices stepped alone."""
    nrep = 1216
    ps = [inputs.LatticeParams(16 + r % 5, 9 + r % 3, 1.0, 0.05 * (r % 4), 0.0, 1e-4,
                               inputs.omega_groups(1.0 + 0.1 * (r % 3), 0.8, 1.0), inputs.LOCAL,
                               "fp32", seed=5000 + r, replica=r) for r in range(nrep)]
    nsteps = 4
    with flb.Batch(ps, tile=tile) as b:
        b.set_sampling(0, 1)
        b.step(nsteps)
        b.sync()
        counts = [b.raw_sums(k)[2] for k in range(nrep)]
        pick = list(range(0, nrep, 97)) + [nrep - 1]
        got = {k: (b.populations(k), b.raw_sums(k)) for k in pick}
    assert counts == [nsteps * p.nodes for p in ps]
    for k in pick:
        f, (S1, S2, n) = got[k]
        ref, (R1, R2, rn) = alone(ps[k], nsteps, warmup=0, every=1)
        np.testing.assert_array_equal(f, ref)
        assert n == rn
        assert_sums_close(S1, S2, R1, R2, n, 1e-4, 3e-6 * n * np.sqrt(ps[k].kT),
                          1e-6 * n * ps[k].kT)


@pytest.mark.parametrize("basis", ALL_BASES)
def test_pooled_correlations(basis):
    """flb_batch_correlations over copies with one rho0, u0 (different seeds
    and sizes): the covariance of the pooled raw sums (the definition, Eqs.
    dfdef and efif0, evaluated here from the per-replica sums), and the moment
    covariance m C m^T with the oracle's measurement basis at u0
    (Eq. dfidfj2dmadmb). One slot alone equals flb_correlations of the same
    lattice stepped alone."""
    shapes = [(21, 21), (37, 8), (64, 16)]
    ps = [inputs.LatticeParams(Lx, Ly, 1.0, 0.1, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0), basis, "fp32",
                               seed=77 + r, replica=r) for r, (Lx, Ly) in enumerate(shapes)]
    with flb.Batch(ps) as b:
        b.set_sampling(10, 2)
        b.step(60)
        b.sync()
        mb = "standard" if basis == inputs.STANDARD else "local"
        Cff, CMM, mean, n = b.correlations([0, 1, 2], mb)
        sums = [b.raw_sums(r) for r in range(3)]
        one = b.correlations([1], mb)
        with pytest.raises(flb.FlbError):
            b.correlations([0, 7], mb)
    S1 = sum(s[0] for s in sums)
    S2 = sum(s[1] for s in sums)
    ns = sum(s[2] for s in sums)
    assert n == ns == sum(p.Lx * p.Ly for p in ps) * 25
    mu = S1 / ns
    C = S2 / ns - np.outer(mu, mu)
    np.testing.assert_allclose(mean, mu, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(Cff, C, rtol=1e-9, atol=1e-9 * ps[0].kT)
    m = oracle.tables()[3] if basis == inputs.STANDARD else oracle.local_basis(0.1, 0.0)
    np.testing.assert_allclose(CMM, m @ C @ m.T, rtol=1e-7, atol=1e-9 * ps[0].kT)
    with flb.Lattice(ps[1], kernel="pipelined") as lat:
        lat.set_sampling(10, 2)
        lat.step(60)
        ref = lat.correlations(mb)
        rS1, rS2, rn = lat.raw_sums()
    assert one[3] == ref[3] == rn
    # the lattice's sums come from the tensor cores (FP16-staged deviations)
    dC, dmu, dCM = staged_corr_bounds(rS1, rS2, rn, m)
    for a, c, d in zip(one[:3], ref[:3], (dC, dCM, dmu)):
        assert np.all(np.abs(a - c) <= 1e-4 * np.abs(c) + 1e-6 * ps[0].kT + d)
    # pooling needs one reference state f^0(rho0, u0)
    q = [ps[0], inputs.LatticeParams(21, 21, 1.0, 0.2, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0), basis,
                                     "fp32", seed=5)]
    with flb.Batch(q) as b:
        b.set_sampling(0, 1)
        b.step(3)
        with pytest.raises(flb.FlbError) as e:
            b.correlations([0, 1], mb)
        assert e.value.code == flb.ERR_ARG
