"""The drift of the moment correlators with the background velocity (Section 3
Fig. 7 and Section 4 Fig. 18): <dM^a dM^b> / (kT rho0) - delta^{ab} fitted by
l u_x0 + q u_x0^2 over -0.25 <= u_x0 <= 0.25, for all 45 unique pairs (a, b).

Analysis only: the correlators come from runs of the step (the library or the
oracle); nothing here takes part in a step.

The lattice and the D2Q9 velocities are symmetric under the x reflection
v_x -> -v_x. A Hermite row (Eq. d2q93a) has parity s_a = -1 when it is odd in
v_x (j_x, Pi_xy, q_x) and +1 otherwise, and the f-norm rows at -u0 are those at
u0 reflected with the same signs (the Gram-Schmidt of Eq. gramschmidt keeps
parity), so in both norms <dM^a dM^b>(-u0) = s_a s_b <dM^a dM^b>(u0). Runs at
u0 >= 0 therefore stand for their mirror images: for a pair with s_a s_b = -1
the correlator is odd in u_x0 and the least-squares fit over the mirrored
points gives q = 0, l = sum u D / sum u^2; for s_a s_b = +1 it is even, l = 0,
q = sum u^2 D / sum u^4 (the paper reads l on the odd pairs and q on the even
ones). fit_lq_points fits l and q by plain least squares over any given
points, mirrored or not.
"""
from __future__ import annotations

import numpy as np

MOMENTS = ("rho", "j_x", "j_y", "Pi_xx-yy", "Pi_xy", "Pi_xx+yy", "q_x", "q_y", "eps")
# parity of each Hermite row under v_x -> -v_x (-1: odd in v_x)
X_PARITY = np.array([1, -1, 1, 1, -1, 1, -1, 1, 1])
FIT_RANGE = 0.25


def normalised(CMM, kT, rho0):
    """<dM^a dM^b> / (kT rho0) - delta^{ab} of one run (9 x 9)."""
    return np.asarray(CMM, dtype=float) / (kT * rho0) - np.eye(9)


def odd_pairs():
    """Boolean 9 x 9 mask of the pairs whose correlator is odd in u_x0."""
    return np.outer(X_PARITY, X_PARITY) < 0


def mirror(us, D):
    """The points u >= 0 and their mirror images -u (u = 0 once), with the
    correlators of the mirrored runs s_a s_b D(u)."""
    us = np.asarray(us, dtype=float)
    D = np.asarray(D, dtype=float)
    sgn = np.outer(X_PARITY, X_PARITY)
    neg = us > 0
    return (np.concatenate([us, -us[neg]]),
            np.concatenate([D, D[neg] * sgn[None, :, :]], axis=0))


def fit_lq_points(us, D):
    """Least-squares l, q (each 9 x 9) of D[k] ~ l u_k + q u_k^2 over the given
    points u_k (any signs), element by element, using |u_k| <= 0.25."""
    us = np.asarray(us, dtype=float)
    D = np.asarray(D, dtype=float)
    use = np.abs(us) <= FIT_RANGE + 1e-12
    A = np.stack([us[use], us[use] ** 2], axis=1)
    coef, *_ = np.linalg.lstsq(A, D[use].reshape(int(use.sum()), -1), rcond=None)
    return coef[0].reshape(9, 9), coef[1].reshape(9, 9)


def fit_lq(us, D):
    """l and q (each 9 x 9, symmetric) of the paper's fit from runs at
    0 <= u_x0 (points beyond 0.25 are ignored), using the x-reflection symmetry
    (module docstring): closed forms on the odd and even pairs."""
    us = np.asarray(us, dtype=float)
    D = np.asarray(D, dtype=float)
    if np.any(us < 0):
        raise ValueError("fit_lq takes runs at u_x0 >= 0 (use fit_lq_points for signed points)")
    use = us <= FIT_RANGE + 1e-12
    u, d = us[use], D[use]
    odd = odd_pairs()
    l = (d * u[:, None, None]).sum(axis=0) / (u ** 2).sum()
    q = (d * u[:, None, None] ** 2).sum(axis=0) / (u ** 4).sum()
    l = np.where(odd, l, 0.0)
    q = np.where(odd, 0.0, q)
    return l, q


def fit_diagonal_q(us, D):
    """q of the diagonal variances (the numbers the paper prints for rho, j_y and
    Pi_xx-yy): the even special case of fit_lq, D[point, a] = diagonal."""
    us = np.asarray(us, dtype=float)
    D = np.asarray(D, dtype=float)
    use = us <= FIT_RANGE + 1e-12
    return (D[use] * us[use, None] ** 2).sum(axis=0) / (us[use] ** 4).sum()


def unique_pairs():
    """The 45 pairs (a, b), a <= b, in row order."""
    return [(a, b) for a in range(9) for b in range(a, 9)]


def as_table(l, q):
    """{"a,b": {"l": .., "q": ..}} with the moments' names, for JSON output."""
    return {f"{MOMENTS[a]},{MOMENTS[b]}": {"l": float(l[a, b]), "q": float(q[a, b])}
            for a, b in unique_pairs()}
