"""Pins of the oracle's noise source: Philox4x32-10 (Salmon et al., SC'11)
against the CUDA toolkit's own implementation, the 21-bit field cut against
big-integer arithmetic, and the Box-Muller normals against their distribution."""
import numpy as np
import pytest
from scipy import stats

from paper_1204_6734_gb300 import inputs


def _ref(curand_ref, ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    n = ctr.shape[0]
    out = np.zeros((n, 4), dtype=np.uint32)
    curand_ref.ref_philox4x32_10(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n)
    return out


def test_philox_matches_curand(oracle, curand_ref):
    g = np.random.Generator(np.random.PCG64(7))
    ctr = g.integers(0, 2 ** 32, size=(300, 4), dtype=np.uint64).astype(np.uint32)
    key = g.integers(0, 2 ** 32, size=(300, 2), dtype=np.uint64).astype(np.uint32)
    # edge counters and keys
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ref = _ref(curand_ref, ctr, key)
    for k in range(ctr.shape[0]):
        np.testing.assert_array_equal(oracle.philox(ctr[k], key[k]), ref[k])


def test_draw_uses_node_step_replica_counter_and_seed_key(oracle, curand_ref):
    """Counter (node, step, replica, 0) and key (seed lo, seed hi)."""
    seed, rep, node, step = 0x1234_5678_9ABC_DEF0, 5, 4097, 123456
    ref = _ref(curand_ref, [[node, step, rep, 0]], [[seed & 0xFFFFFFFF, seed >> 32]])[0]
    X = sum(int(ref[q]) << (32 * q) for q in range(4))
    expect = [(X >> (21 * q)) & ((1 << 21) - 1) for q in range(6)]
    np.testing.assert_array_equal(oracle.draw_fields(seed, rep, node, step), expect)


def test_fields_are_bit_cuts_of_the_block(oracle):
    for (node, step) in [(0, 0), (1, 0), (0, 1), (12345, 999), (2 ** 32 - 1, 2 ** 31)]:
        out = oracle.philox([node, step, 3, 0], [17, 0])
        X = sum(int(out[q]) << (32 * q) for q in range(4))
        f = oracle.draw_fields(17, 3, node, step)
        assert [int(v) for v in f] == [(X >> (21 * q)) & 0x1FFFFF for q in range(6)]


def test_distinct_streams(oracle):
    """Different nodes, steps, replicas and seeds give different blocks."""
    seen = set()
    for args in [(1, 0, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1), (1, 1, 0, 0), (2, 0, 0, 0)]:
        seen.add(tuple(oracle.draw_fields(*args)))
    assert len(seen) == 5


def _sample_normals(oracle, n_nodes, seed=99):
    return np.array([oracle.normals(seed, 0, k, 7) for k in range(n_nodes)])


def test_normals_are_standard_gaussian(oracle):
    z = _sample_normals(oracle, 30000)           # 180000 draws
    flat = z.ravel()
    n = flat.size
    assert abs(flat.mean()) < 4 / np.sqrt(n)
    assert abs(flat.var() - 1) < 4 * np.sqrt(2 / n)
    kurt = stats.kurtosis(flat, fisher=False)
    assert abs(kurt - 3) < 4 * np.sqrt(24 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # each of the six slots separately is standard normal and the slots are
    # uncorrelated (independent moments a = 3..8)
    for q in range(6):
        assert stats.kstest(z[:, q], "norm").pvalue > 1e-4
    cc = np.corrcoef(z.T)
    assert np.abs(cc - np.eye(6)).max() < 5 / np.sqrt(z.shape[0])


def test_box_muller_pairs(oracle):
    """N_{2p}^2 + N_{2p+1}^2 = -2 ln u1 with u1 = (k_{2p} + 1) 2^-21, and the
    angle is 2 pi k_{2p+1} 2^-21."""
    for node in range(50):
        k = oracle.draw_fields(5, 2, node, 11).astype(np.float64)
        z = oracle.normals(5, 2, node, 11)
        for p in range(3):
            r2 = z[2 * p] ** 2 + z[2 * p + 1] ** 2
            u1 = (k[2 * p] + 1) / 2 ** 21
            assert r2 == pytest.approx(-2 * np.log(u1), rel=1e-12, abs=1e-14)
            if r2 > 1e-20:
                ang = np.arctan2(z[2 * p + 1], z[2 * p]) % (2 * np.pi)
                assert ang == pytest.approx(2 * np.pi * k[2 * p + 1] / 2 ** 21, abs=1e-9)


def test_numpy_philox_helper_matches_the_oracle(oracle):
    """tests/philox_np.py (used to search for draws with given fields) gives the
    oracle's fields."""
    import philox_np
    nodes = np.concatenate([np.arange(40), np.array([2 ** 32 - 1, 123456789, 2 ** 31])])
    for seed, rep, step in [(1, 0, 0), (0xDEADBEEFCAFEF00D, 7, 123456), (99, 3, 42)]:
        got = philox_np.fields(seed, rep, nodes, step)
        ref = np.array([oracle.draw_fields(seed, rep, int(n), step) for n in nodes])
        np.testing.assert_array_equal(got, ref)
