"""Tolerances of correlation sums formed on the tensor cores.

The pipelined FP32 step accumulates S1_i = sum d_i and S2_ij = sum d_i d_j of the
centred populations d = f - f^0(rho0, u0) from deviations staged in FP16 (round
to nearest: each staged value is off by at most 2^-11 of itself), in FP32
partials of at most 1024 products (relative error below 2^-14 of the sum of
absolute terms) that are added up in FP64. Bounds on the error of a sum, by the
Cauchy-Schwarz inequality (sum |d_i d_j| <= sqrt(S2_ii S2_jj),
sum |d_i| <= sqrt(n S2_ii)):

    |dS2_ij| <= (2^-10 + 2^-14) sqrt(S2_ii S2_jj),
    |dS1_i|  <= (2^-11 + 2^-14) sqrt(n S2_ii).

These are worst cases; the rounding errors are unbiased and independent, so the
actual errors are of order 2^-12 / sqrt(n) of the sums. A wrong index, sign or
scale in the sums is an error of the order of the sums themselves.
"""
import numpy as np

S2_REL = 2.0 ** -10 + 2.0 ** -14
S1_REL = 2.0 ** -11 + 2.0 ** -14


def staged_s2_bound(S2):
    d = np.sqrt(np.abs(np.diag(np.asarray(S2, dtype=float))))
    return S2_REL * np.outer(d, d)


def staged_s1_bound(S2, n):
    return S1_REL * np.sqrt(max(int(n), 1) * np.abs(np.diag(np.asarray(S2, dtype=float))))


def assert_sums_close(S1, S2, S1_ref, S2_ref, n, rtol, atol1, atol2):
    """|S - S_ref| within the given FP32-trajectory tolerances (rtol relative,
    atol1 / atol2 absolute for S1 / S2) plus the FP16-staging bound above."""
    S1, S2, S1_ref, S2_ref = (np.asarray(x, dtype=float) for x in (S1, S2, S1_ref, S2_ref))
    b2 = rtol * np.abs(S2_ref) + atol2 + staged_s2_bound(S2_ref)
    b1 = rtol * np.abs(S1_ref) + atol1 + staged_s1_bound(S2_ref, n)
    bad2 = np.abs(S2 - S2_ref) > b2
    bad1 = np.abs(S1 - S1_ref) > b1
    assert not bad2.any(), (np.argwhere(bad2)[:5], S2[bad2][:5], S2_ref[bad2][:5], b2[bad2][:5])
    assert not bad1.any(), (np.argwhere(bad1)[:5], S1[bad1][:5], S1_ref[bad1][:5], b1[bad1][:5])


def staged_corr_bounds(S1, S2, n, m):
    """Bounds on the error of the centred covariance C = S2/n - mu mu^T
    (mu = S1/n), of mu and of m C m^T implied by the bounds on the sums."""
    S1 = np.asarray(S1, dtype=float)
    mu = S1 / n
    dmu = staged_s1_bound(S2, n) / n
    dC = staged_s2_bound(S2) / n + np.outer(dmu, np.abs(mu)) + np.outer(np.abs(mu), dmu)
    am = np.abs(np.asarray(m, dtype=float))
    return dC, dmu, am @ dC @ am.T
