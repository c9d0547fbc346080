"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Tolerances (written here, derived from the arithmetic):
* integer noise fields: bit-exact;
* FP64 normals: 1e-14 relative (log/sincos differ by an ulp or two);
* FP32 normals: per draw, 2.2e-7/(2r) + 6.4e-7 r + 1e-7 (SFU log2 absolute
  error 2^-22.6 near u1 = 1, SFU sine/cosine 2^-21.4, radius r);
* FP64 populations: 1e-12 relative to the largest population, after up to
  10^4 steps (the collisions follow different but exact algebra: Cholesky of
  the Gram matrix versus Gram-Schmidt; differences of a few ulp per step
  random-walk in the conserved modes);
* FP32 populations: 1e-5 absolute at rho0 = 1 (FP32 rounding of the state,
  ~3e-8 per step, diffusing over the run) and correlations within 1% of
  kT w_max.
"""
import numpy as np
import pytest

import oracle
from tolerances import assert_sums_close, staged_corr_bounds
from paper_1204_6734_gb300 import flb, inputs

pytestmark = pytest.mark.gpu

BASES = [inputs.STANDARD, inputs.LOCAL]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flb.load()


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noise_draws(precision):
    g = np.random.Generator(np.random.PCG64(1))
    nodes = np.concatenate([np.arange(64), g.integers(0, 2 ** 32, 2000, dtype=np.uint64)])
    nodes = nodes.astype(np.uint32)
    for seed, rep, step in [(1, 0, 0), (0xDEADBEEFCAFEF00D, 7, 123456), (2 ** 64 - 1, 2 ** 32 - 1, 2 ** 32 - 1)]:
        fields, normals = flb.flb_noise_draws(seed, rep, step, nodes, precision)
        ref_f = np.array([oracle.draw_fields(seed, rep, int(n), step) for n in nodes])
        np.testing.assert_array_equal(fields, ref_f)
        ref_n = np.array([oracle.normals(seed, rep, int(n), step) for n in nodes])
        if precision == "fp64":
            np.testing.assert_allclose(normals, ref_n, rtol=1e-14, atol=1e-14)
        else:
            # SFU log2 has absolute error 2^-22.6 on [0.5, 1] (2 ulp below), so
            # r^2 = -2 ln u1 is off by <= 2.2e-7 absolute and r by d(r^2)/(2r);
            # the SFU sine/cosine add 2^-21.4 times r
            r = np.sqrt(ref_n[:, 0::2] ** 2 + ref_n[:, 1::2] ** 2).repeat(2, axis=1)
            bound = 2.2e-7 / (2 * r) + 4e-7 * r + 2.4e-7 * r + 1e-7
            assert np.all(np.abs(normals - ref_n) <= bound)


# ---------------------------------------------------------------------------
# single-node collision
# ---------------------------------------------------------------------------

def _states(n, seed, amp=0.05, umax=0.3):
    vel = inputs.random_velocities(n, seed=seed, umax=umax)
    pert = inputs.perturbation((n, 9), seed=seed + 1)
    rho = 0.5 + 1.5 * np.random.Generator(np.random.PCG64(seed + 2)).uniform(size=n)
    return np.array([oracle.feq(rho[k], *vel[k]) * (1 + amp * pert[k]) for k in range(n)])


@pytest.mark.parametrize("basis", BASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_collide_nodes(basis, precision):
    om = inputs.omega_groups(1.3, 0.7, 1.6)
    p = inputs.LatticeParams(1, 1, 1.0, 0.0, 0.0, 1e-3, om, basis, precision, seed=99)
    g = _states(500, seed=5)
    ids = np.arange(500, dtype=np.uint32) * 7919
    out, st = flb.flb_collide_nodes(p, g, ids, 42)
    assert np.all(st == 0)
    ref = np.array([oracle.collide_node(p, g[k], int(ids[k]), 42) for k in range(500)])
    if precision == "fp64":
        np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-15)
    else:
        assert np.abs(out - ref).max() < 2e-6 * g.sum(1).max()


def test_fp32_noise_at_the_smallest_radius():
    """Box-Muller at u1 = 1 (the 21-bit field 2^21 - 1): the radius, and the two
    normals of the pair, are exactly 0; the FP32 collision forms the radius from
    log2(u1), exact there, so the node collides as the FP64 oracle's does to
    FP32 rounding even with a large noise amplitude."""
    import philox_np
    om = inputs.omega_groups(1.3, 0.7, 1.6)
    for basis in BASES:
        p = inputs.LatticeParams(1, 1, 1.0, 0.0, 0.0, 1e-2, om, basis, "fp32", seed=99)
        cand = np.arange(1 << 23, dtype=np.uint64)
        k = philox_np.fields(p.seed, 0, cand, 42)
        hit = cand[np.any(k[:, 0::2] == (1 << 21) - 1, axis=1)][:8].astype(np.uint32)
        assert len(hit) >= 4
        for n in hit:
            assert (1 << 21) - 1 in oracle.draw_fields(p.seed, 0, int(n), 42)[0::2]
        g = _states(len(hit), seed=11)
        out, st = flb.flb_collide_nodes(p, g, hit, 42)
        assert np.all(st == 0)
        ref = np.array([oracle.collide_node(p, g[j], int(hit[j]), 42) for j in range(len(hit))])
        assert np.abs(out - ref).max() < 2e-6 * g.sum(1).max()


def test_collide_nodes_invalid_velocity_status():
    p = inputs.LatticeParams(1, 1, kT=0.0, basis=inputs.LOCAL, precision="fp64")
    g = np.array([[0.1, 0.9, 0.1, 0.0, 0.1, 0.3, 0.0, 0.0, 0.3],
                  list(oracle.feq(1.0, 0.1, 0.0))])
    out, st = flb.flb_collide_nodes(p, g, [0, 1], 0)
    assert st[0] == flb.ERR_INVALID_VELOCITY and st[1] == 0
    np.testing.assert_array_equal(out[0], g[0])      # invalid node left uncollided


# ---------------------------------------------------------------------------
# lattice trajectories
# ---------------------------------------------------------------------------

def _perturbed_state(p, seed, amp=0.02):
    f0 = oracle.init_equilibrium(p)
    return f0 * (1 + amp * inputs.perturbation(f0.shape, seed=seed))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (37, 19), (130, 64)])
def test_set_get_populations_roundtrip(precision, shape):
    Lx, Ly = shape
    p = inputs.LatticeParams(Lx, Ly, precision=precision)
    f = 0.1 + inputs.perturbation((9, Ly, Lx), seed=Lx + Ly) ** 2
    with flb.Lattice(p) as lat:
        np.testing.assert_allclose(lat.populations(), oracle.init_equilibrium(p),
                                   rtol=1e-15 if precision == "fp64" else 1e-7)
        lat.set_populations(f)
        back = lat.populations()
    if precision == "fp64":
        np.testing.assert_array_equal(back, f)
    else:
        np.testing.assert_array_equal(back, f.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("shape", inputs.small_lattices())
@pytest.mark.parametrize("basis", BASES)
def test_fp64_trajectory_small_lattices(shape, basis):
    Lx, Ly = shape
    p = inputs.LatticeParams(Lx, Ly, 1.0, 0.12, -0.07, 1e-3, inputs.omega_groups(1.3, 0.8, 1.6),
                             basis, "fp64", seed=3 + Lx)
    nsteps = 40 if Lx * Ly > 5000 else 100
    f_init = _perturbed_state(p, seed=Lx * 1000 + Ly)
    run = oracle.Run(p, f=f_init, warmup=5, every=3).step(nsteps)
    with flb.Lattice(p) as lat:
        lat.set_populations(f_init)
        lat.set_sampling(5, 3)
        lat.step(nsteps)
        lat.sync()
        f = lat.populations()
        S1, S2, n = lat.raw_sums()
        assert lat.t == nsteps
    scale = np.abs(run.f).max()
    assert np.abs(f - run.f).max() / scale < 1e-12
    assert n == run.nsamp
    np.testing.assert_allclose(S1, run.S1, rtol=1e-9, atol=1e-12 * n * 1e-3)
    np.testing.assert_allclose(S2, run.S2, rtol=1e-9, atol=1e-12 * n * 1e-6)


@pytest.fixture(scope="module")
def parity_run():
    """The oracle's run of the 32x32 parity workload (u0 = (0.1, 0), all rates 1,
    f-norm, seed 1): 10^4 steps sampled every step after 10^3, computed once for
    the FP64 and FP32 checks below (the oracle is FP64 whatever the precision
    the GPU runs in, and draws the same noise)."""
    p = inputs.fp64_parity_lattice()
    T, W = inputs.FP64_PARITY_STEPS, inputs.FP64_PARITY_WARMUP
    run = oracle.Run(p, warmup=W, every=1).step(T)
    C_ref, mean_ref = run.covariance()
    return p, T, W, run, C_ref, mean_ref, run.moment_covariance("local")


@pytest.mark.slow
def test_fp64_parity_lattice_full_run(parity_run):
    """32x32 FP64 f-norm lattice, u0 = (0.1, 0), 10^4 steps, sampled every step
    after 10^3: populations within 1e-12 relative, correlations to 1e-9."""
    p, T, W, run, C_ref, mean_ref, CM_ref = parity_run
    with flb.Lattice(p) as lat:
        lat.set_sampling(W, 1)
        lat.step(T)
        lat.sync()
        f = lat.populations()
        Cff, CMM, mean, n = lat.correlations("local")
    assert np.abs(f - run.f).max() / np.abs(run.f).max() < 1e-12
    assert n == run.nsamp == (T - W) * 32 * 32
    assert np.abs(Cff - C_ref).max() < 1e-9 * np.abs(C_ref).max()
    assert np.abs(CMM - CM_ref).max() < 1e-9 * np.abs(CM_ref).max()
    np.testing.assert_allclose(mean, mean_ref, atol=1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["generic", "pipelined", "pipelined-samplers", "pipelined16"])
def test_fp32_parity_lattice_full_run(parity_run, kernel):
    """The same workload with FP32 populations and arithmetic, over the full 10^4
    steps: every population within 1e-5 of the oracle's FP64 trajectory (same
    draws) and the correlations within 1% (of kT w_max for <df_i df_j>, of kT for
    <dM^a dM^b>), for the generic kernel and the pipelined one with each way of
    accumulating the sums."""
    p64, T, W, run, C_ref, mean_ref, CM_ref = parity_run
    p = inputs.LatticeParams(p64.Lx, p64.Ly, p64.rho0, p64.ux0, p64.uy0, p64.kT, p64.omega,
                             p64.basis, "fp32", seed=p64.seed)
    with lattice(p, kernel) as lat:
        lat.set_sampling(W, 1)
        lat.step(T)
        lat.sync()
        f = lat.populations()
        Cff, CMM, mean, n = lat.correlations("local")
    assert n == run.nsamp
    assert np.abs(f - run.f).max() < 1e-5
    assert np.abs(Cff - C_ref).max() < 0.01 * p.kT * 4.0 / 9.0
    assert np.abs(CMM - CM_ref).max() < 0.01 * p.kT


KERNELS = ["generic", "pipelined", "pipelined-samplers", "pipelined-fused", "pipelined16",
           "pipelined12", "pipelined8"]


def lattice(p, kernel):
    """A lattice with the given FP32 step kernel: the generic one, or the
    pipelined one -- by default the sums on the tensor cores, 16 colliding
    warps in the f-norm bases and 12 in the Hermite norm; sampler warps with 8
    colliding warps; sums fused into the colliding warps; 16, 12 or 8 colliding
    warps with the tensor-core sums."""
    if kernel == "pipelined16":
        return flb.Lattice(p, kernel="pipelined", pipeline_warps=16)
    if kernel == "pipelined12":
        return flb.Lattice(p, kernel="pipelined", pipeline_warps=12)
    if kernel == "pipelined8":
        return flb.Lattice(p, kernel="pipelined", pipeline_warps=8)
    if kernel == "pipelined-samplers":
        return flb.Lattice(p, kernel="pipelined", pipeline_sampling=1, pipeline_warps=8)
    if kernel == "pipelined-fused":
        return flb.Lattice(p, kernel="pipelined", pipeline_sampling=2)
    return flb.Lattice(p, kernel=kernel)


@pytest.mark.parametrize("basis", BASES)
def test_warp_counts_give_identical_states(basis):
    """8, 12 and 16 colliding warps pair the same nodes (x, x + 64) in the same
    packed arithmetic: identical populations, with and without sampling."""
    p = inputs.LatticeParams(300, 37, 1.0, 0.15, 0.05, 1e-3, inputs.omega_groups(1.2, 0.8, 1.3), basis,
                             "fp32", seed=8)
    out = []
    for kernel in ("pipelined", "pipelined8", "pipelined12", "pipelined16", "pipelined-samplers"):
        with lattice(p, kernel) as lat:
            lat.set_sampling(10, 3)
            lat.step(40)
            out.append(lat.populations())
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("basis", BASES)
def test_fp32_trajectory(basis, kernel):
    """FP32 state and arithmetic against the FP64 oracle, same noise draws."""
    p = inputs.LatticeParams(200, 48, 1.0, 0.2, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             basis, "fp32", seed=12)
    nsteps = 600
    run = oracle.Run(p, warmup=100, every=1).step(nsteps)
    with lattice(p, kernel) as lat:
        lat.set_sampling(100, 1)
        lat.step(nsteps)
        lat.sync()
        f = lat.populations()
        Cff, CMM, mean, n = lat.correlations(basis)
    assert np.abs(f - run.f).max() < 1e-5
    C_ref, _ = run.covariance()
    w_max = 4.0 / 9.0
    assert np.abs(Cff - C_ref).max() < 0.01 * p.kT * w_max
    CM_ref = run.moment_covariance(basis)
    assert np.abs(CMM - CM_ref).max() < 0.01 * p.kT


@pytest.mark.parametrize("basis", BASES)
def test_correlation_api_matches_oracle_reduction(basis):
    p = inputs.LatticeParams(21, 21, 1.0, 0.15, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             basis, "fp64", seed=77)
    run = oracle.Run(p, warmup=50, every=2).step(300)
    with flb.Lattice(p) as lat:
        lat.set_sampling(50, 2)
        lat.step(300)
        for mb in BASES:
            Cff, CMM, mean, n = lat.correlations(mb)
            C_ref, mean_ref = run.covariance()
            np.testing.assert_allclose(Cff, C_ref, rtol=1e-8, atol=1e-16)
            np.testing.assert_allclose(CMM, run.moment_covariance(mb), rtol=1e-8, atol=1e-15)
            np.testing.assert_allclose(mean, mean_ref, rtol=1e-8, atol=1e-15)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", [(1, 1), (5, 3), (37, 19), (128, 4), (129, 5), (300, 9)])
@pytest.mark.parametrize("basis", BASES)
def test_fp32_kernels_agree_with_oracle_step_by_step(shape, basis, kernel):
    """Ragged and tiny lattices (partial tiles, ghost frame on every side): a few
    steps of either FP32 kernel against the oracle from a perturbed state, with
    sampling on every step."""
    Lx, Ly = shape
    p = inputs.LatticeParams(Lx, Ly, 1.0, 0.15, -0.1, 1e-3, inputs.omega_groups(1.3, 0.8, 1.6),
                             basis, "fp32", seed=40 + Lx)
    f_init = _perturbed_state(p, seed=Lx + 7 * Ly)
    run = oracle.Run(p, f=f_init, warmup=0, every=1).step(5)
    with lattice(p, kernel) as lat:
        lat.set_populations(f_init)
        lat.set_sampling(0, 1)
        lat.step(5)
        lat.sync()
        f = lat.populations()
        S1, S2, n = lat.raw_sums()
    assert np.abs(f - run.f).max() < 2e-6
    assert n == run.nsamp
    assert_sums_close(S1, S2, run.S1, run.S2, n, 2e-4, 1e-7 * n, 1e-9 * n)


@pytest.mark.parametrize("basis", BASES)
def test_pipelined_equals_generic_fp32(basis):
    """Both FP32 kernels compute the same thing (same draws, same algebra) on a
    lattice of many tiles with a ragged edge: populations agree to FP32 rounding."""
    p = inputs.LatticeParams(1000, 77, 1.0, 0.1, 0.02, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             basis, "fp32", seed=9)
    out = {}
    for kernel in KERNELS:
        with lattice(p, kernel) as lat:
            lat.set_sampling(2, 1)
            lat.step(30)
            out[kernel] = (lat.populations(), lat.raw_sums())
    for k in KERNELS[1:]:
        assert np.abs(out["generic"][0] - out[k][0]).max() < 1e-6
        g1, g2, gn = out["generic"][1]
        assert_sums_close(out[k][1][0], out[k][1][1], g1, g2, gn, 1e-4, 3e-6 * gn * np.sqrt(p.kT),
                          1e-6 * gn * p.kT)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_conservation_sums(precision):
    p = inputs.LatticeParams(37, 19, 1.0, 0.1, 0.05, 1e-3, inputs.omega_groups(1.1, 0.9, 1.3),
                             inputs.LOCAL, precision, seed=5)
    f_init = _perturbed_state(p, seed=9, amp=0.05)
    vx, vy, *_ = oracle.tables()
    tot = np.array([f_init.sum(), np.einsum("i,iyx->", vx, f_init), np.einsum("i,iyx->", vy, f_init)])
    with flb.Lattice(p) as lat:
        lat.set_populations(f_init)
        s0 = lat.conservation()
        lat.step(200)
        s1 = lat.conservation()
    tol = 1e-12 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(s0, tot, rtol=0, atol=tol * tot[0])
    np.testing.assert_allclose(s1, tot, rtol=0, atol=tol * tot[0])


def test_invalid_velocity_reported_not_hung():
    """A node whose velocity leaves the f^0 > 0 region (Fig. 11): the step kernel
    records it, leaves the node uncollided, and the host gets an error code; the
    handle refuses further steps until the state is replaced."""
    p = inputs.LatticeParams(16, 8, 1.0, 0.0, 0.0, 1e-4, inputs.omega_groups(1, 1, 1),
                             inputs.LOCAL, "fp32", seed=1)
    f = oracle.init_equilibrium(p)
    bad = np.array([0.1, 0.9, 0.1, 0.0, 0.1, 0.3, 0.0, 0.0, 0.3])
    f[:, 3, 5] = bad                    # node x=5, y=3
    with flb.Lattice(p) as lat:
        lat.set_populations(f)
        lat.step(1)
        with pytest.raises(flb.FlbError) as e:
            lat.sync()
        assert e.value.code == flb.ERR_INVALID_VELOCITY
        assert flb.flb_error_location(lat.h) == (5 + 16 * 3, 0)
        with pytest.raises(flb.FlbError):
            lat.step(1)
        lat.set_populations(oracle.init_equilibrium(p))
        lat.step(3)
        lat.sync()


def test_run_host_matches_handle_path():
    p = inputs.LatticeParams(33, 17, 1.0, 0.05, 0.0, 1e-4, inputs.omega_groups(1.0, 0.8, 1.0),
                             inputs.LOCAL, "fp64", seed=4)
    f_init = _perturbed_state(p, seed=2)
    f_out = np.empty_like(f_init)
    S1, S2, n = flb.flb_run_host(p, f_init, 30, warmup=10, every=1, f_out=f_out)
    run = oracle.Run(p, f=f_init, warmup=10, every=1).step(30)
    assert np.abs(f_out - run.f).max() < 1e-13
    assert n == run.nsamp
    np.testing.assert_allclose(S2, run.S2, rtol=1e-9, atol=1e-20)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("basis", BASES)
def test_full_size_sampled_nodes(basis, kernel):
    """4096^2 FP32, the benchmark's configuration and launch: after 20 steps one
    more step is checked at sampled nodes against the oracle's collision of the
    same pre-collision populations (pull streaming checked by position)."""
    p = inputs.single_lattice(0.1, basis)
    Lx, Ly = p.Lx, p.Ly
    with lattice(p, kernel) as lat:
        lat.step(20)
        F0 = lat.populations()
        lat.step(1)
        F1 = lat.populations()
    vx, vy, *_ = oracle.tables()
    g = np.random.Generator(np.random.PCG64(3))
    xs = np.concatenate([[0, Lx - 1, 5, Lx - 1], g.integers(0, Lx, 300)])
    ys = np.concatenate([[0, Ly - 1, Ly - 1, 0], g.integers(0, Ly, 300)])
    err = 0.0
    for x, y in zip(xs, ys):
        for i in range(9):
            xs_, ys_ = (x - vx[i]) % Lx, (y - vy[i]) % Ly     # origin of f_i(x, t+1)
            fs = oracle.collide_node(p, F0[:, ys_, xs_], int(xs_ + Lx * ys_), 20)
            err = max(err, abs(F1[i, y, x] - fs[i]))
    assert err < 2e-6


@pytest.mark.parametrize("precision,basis", [("fp32", inputs.LOCAL), ("fp32", inputs.STANDARD),
                                             ("fp64", inputs.LOCAL), ("fp16dev", inputs.LUT)])
def test_checkpoint_resume_continues_exactly(precision, basis):
    """A run checkpointed at t = 23 (state, time, raw sums) and resumed on a new
    handle ends in the same state as the uninterrupted run (the noise counter
    is the step), with the same sums up to FP64 summation order."""
    p = inputs.LatticeParams(150, 41, 1.0, 0.1, -0.02, 1e-4, inputs.omega_groups(1.1, 0.8, 1.2), basis,
                             precision, seed=77)
    with flb.Lattice(p) as lat:
        lat.set_sampling(5, 2)
        lat.step(50)
        f_ref, (S1r, S2r, nr) = lat.populations(), lat.raw_sums()
    with flb.Lattice(p) as lat:
        lat.set_sampling(5, 2)
        lat.step(23)
        state = lat.checkpoint()
    with flb.Lattice(p) as lat:
        lat.resume(state, 5, 2)
        assert lat.t == 23
        lat.step(27)
        f, (S1, S2, n) = lat.populations(), lat.raw_sums()
    np.testing.assert_array_equal(f, f_ref)
    assert n == nr
    np.testing.assert_allclose(S2, S2r, rtol=1e-12, atol=1e-12 * n * p.kT)
    np.testing.assert_allclose(S1, S1r, rtol=1e-12, atol=1e-12 * n * np.sqrt(p.kT))
