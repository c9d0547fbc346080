"""Philox4x32-10 (Salmon et al., SC'11) over arrays of counters, in NumPy, for the
tests that need to find nodes whose draw has a given property (e.g. the
Box-Muller field that makes u1 = 1). Counter (node, step, replica, 0), key the
64-bit seed, six 21-bit fields per draw; checked against the oracle's
draw_fields in test_oracle_rng.py."""
import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def fields(seed, replica, nodes, step):
    """(len(nodes), 6) array of the 21-bit fields of the draws of `nodes`."""
    c0 = np.asarray(nodes, dtype=np.uint64) & MASK32
    c1 = np.full_like(c0, np.uint64(step) & MASK32)
    c2 = np.full_like(c0, np.uint64(replica) & MASK32)
    c3 = np.zeros_like(c0)
    k0, k1 = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    for _ in range(10):
        p0, p1 = M0 * c0, M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & MASK32,
                          (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & MASK32)
        k0, k1 = (k0 + W0) & 0xFFFFFFFF, (k1 + W1) & 0xFFFFFFFF
    x = c0 | (c1 << np.uint64(32))          # bits 0..63
    y = c2 | (c3 << np.uint64(32))          # bits 64..127
    m = np.uint64(0x1FFFFF)
    return np.stack([x & m, (x >> np.uint64(21)) & m, (x >> np.uint64(42)) & m,
                     ((x >> np.uint64(63)) | (y << np.uint64(1))) & m,
                     (y >> np.uint64(20)) & m, (y >> np.uint64(41)) & m], axis=1)
