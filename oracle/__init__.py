"""FP64 CPU oracle of the fluctuating D2Q9 lattice-Boltzmann step
(Kaehler & Wagner, arXiv:1204.6734) -- ctypes binding plus plain NumPy helpers.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product (``paper_1204_6734_gb300``) never imports it, and it never
imports the product: parameters are duck-typed objects with the attributes
``Lx, Ly, rho0, ux0, uy0, kT, omega (9), basis ('standard'|'local'|'lut'),
seed, replica``.

The C part (``flb_oracle.c``) holds the method; the NumPy helpers here reduce
the sampled sums to covariances (Eq. dfidfj2dmadmb) with the oracle's own
basis matrices, and form the static structure factors of Eqs. sfactorr,
sfactoru, rcorrelator from the oracle's state (NumPy's forward FFT as the
transform, pinned against the written-out double sum).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BASIS = {"standard": 0, "local": 1, "lut": 2}
ERRORS = {0: "ok", -1: "invalid argument", -3: "invalid velocity (some f_i^0(1,u) <= 0)",
          -4: "non-finite value"}


class OracleError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {where}".strip())
        self.code = code


class _Params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32),
                ("rho0", C.c_double), ("ux0", C.c_double), ("uy0", C.c_double),
                ("kT", C.c_double), ("omega", C.c_double * 9),
                ("basis", C.c_int32), ("replica", C.c_uint32), ("seed", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        u32p = C.POINTER(C.c_uint32)
        L.orc_tables.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), dp, dp, dp]
        L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_hermite_meq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_local_basis.argtypes = [C.c_double, C.c_double, dp]
        L.orc_local_basis.restype = C.c_int
        L.orc_lut_velocity.argtypes = [C.c_double, C.c_double, dp, dp]
        L.orc_lut_velocity.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_draw_fields.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u32p]
        L.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp]
        L.orc_collide_node.argtypes = [C.POINTER(_Params), dp, C.c_uint32, C.c_uint32, dp]
        L.orc_collide_node.restype = C.c_int
        L.orc_init_equilibrium.argtypes = [C.POINTER(_Params), dp]
        L.orc_run.argtypes = [C.POINTER(_Params), dp, C.c_int64, C.c_int64, C.c_int64,
                              C.c_int64, dp, dp, C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_run.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def to_struct(p) -> _Params:
    s = _Params()
    s.Lx, s.Ly = int(p.Lx), int(p.Ly)
    s.rho0, s.ux0, s.uy0, s.kT = float(p.rho0), float(p.ux0), float(p.uy0), float(p.kT)
    om = list(p.omega)
    if len(om) != 9:
        raise ValueError("omega must have 9 entries")
    for a in range(9):
        s.omega[a] = float(om[a])
    b = p.basis
    s.basis = BASIS[b] if isinstance(b, str) else int(b)
    s.replica = int(getattr(p, "replica", 0))
    s.seed = int(p.seed) & 0xFFFFFFFFFFFFFFFF
    return s


# --------------------------------------------------------------------------
# Tables and single-node pieces
# --------------------------------------------------------------------------

def tables():
    """(vx, vy, w, m[a,i], n[i,a]) of the appendix (Eqs. d2q9w, d2q93a, d2q93b)."""
    vx = (C.c_int * 9)()
    vy = (C.c_int * 9)()
    w = np.zeros(9)
    m = np.zeros((9, 9))
    n = np.zeros((9, 9))
    lib().orc_tables(vx, vy, _dp(w), _dp(m), _dp(n))
    return np.array(vx[:]), np.array(vy[:]), w, m, n


def feq(rho, ux, uy):
    """Eq. d2q9f0."""
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _dp(out))
    return out


def hermite_meq(rho, ux, uy):
    """Eq. d2q94."""
    out = np.zeros(9)
    lib().orc_hermite_meq(rho, ux, uy, _dp(out))
    return out


def local_basis(ux, uy):
    """f-norm basis mt[a, i] at velocity u (Section 4, Gram-Schmidt)."""
    out = np.zeros((9, 9))
    rc = lib().orc_local_basis(ux, uy, _dp(out))
    if rc:
        raise OracleError(rc, f"at u=({ux},{uy})")
    return out


def lut_velocity(ux, uy):
    """Table velocity u_g of the look-up-table f-norm (Section 4) nearest to u."""
    gx, gy = C.c_double(), C.c_double()
    rc = lib().orc_lut_velocity(float(ux), float(uy), C.byref(gx), C.byref(gy))
    if rc != 0:
        raise OracleError(rc, "lut_velocity")
    return gx.value, gy.value


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def draw_fields(seed, replica, node, step):
    out = np.zeros(6, dtype=np.uint32)
    lib().orc_draw_fields(seed & 0xFFFFFFFFFFFFFFFF, replica, node, step, _u32p(out))
    return out


def normals(seed, replica, node, step):
    out = np.zeros(6)
    lib().orc_normals(seed & 0xFFFFFFFFFFFFFFFF, replica, node, step, _dp(out))
    return out


def collide_node(p, g, node, step):
    """Post-collision populations of one node (Eq. LBEMRT)."""
    s = to_struct(p)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(9)
    rc = lib().orc_collide_node(C.byref(s), _dp(gg), node, step, _dp(out))
    if rc:
        raise OracleError(rc, f"at node {node} step {step}")
    return out


# --------------------------------------------------------------------------
# Lattice runs
# --------------------------------------------------------------------------

def init_equilibrium(p):
    """Uniform state f_i = f_i^0(rho0, u0), shape (9, Ly, Lx)."""
    s = to_struct(p)
    f = np.zeros((9, s.Ly, s.Lx))
    lib().orc_init_equilibrium(C.byref(s), _dp(f))
    return f


class Run:
    """A lattice advanced by the oracle; keeps the sampled sums of Eq. dfidfj2dmadmb."""

    def __init__(self, p, f=None, warmup=0, every=0):
        self.p = p
        self.s = to_struct(p)
        self.f = init_equilibrium(p) if f is None else np.array(f, dtype=np.float64, copy=True)
        if self.f.shape != (9, self.s.Ly, self.s.Lx):
            raise ValueError("state must have shape (9, Ly, Lx)")
        self.t = 0
        self.warmup, self.every = int(warmup), int(every)
        self.S1 = np.zeros(9)
        self.S2 = np.zeros((9, 9))
        self.nsamp = 0

    def step(self, n):
        ns = C.c_int64(self.nsamp)
        en, es = C.c_int64(-1), C.c_int64(-1)
        rc = lib().orc_run(C.byref(self.s), _dp(self.f), self.t, int(n), self.warmup,
                           self.every, _dp(self.S1), _dp(self.S2), C.byref(ns),
                           C.byref(en), C.byref(es))
        if rc:
            raise OracleError(rc, f"at node {en.value} step {es.value}")
        self.nsamp = ns.value
        self.t += int(n)
        return self

    def covariance(self):
        return covariance(self.S1, self.S2, self.nsamp)

    def moment_covariance(self, measure_basis):
        return moment_covariance(self.covariance()[0], measure_basis, self.p.ux0, self.p.uy0)


def covariance(S1, S2, nsamp):
    """Centred equal-time covariance <df_i df_j> from the sums of f - f^0(rho0,u0)
    (Eqs. dfdef, efif0); returns (C, mean deviation)."""
    if nsamp <= 0:
        raise ValueError("no samples")
    mean = np.asarray(S1) / nsamp
    Cm = np.asarray(S2).reshape(9, 9) / nsamp - np.outer(mean, mean)
    return Cm, mean


def measure_matrix(measure_basis, ux0, uy0):
    """Rows of the basis the moments are measured in: the Hermite rows
    (Eq. d2q93a) or the f-norm at the mean velocity u0 (discussion after
    Eq. fidjx), both orthonormal under their own weights."""
    if measure_basis in ("standard", 0):
        return tables()[3]
    return local_basis(ux0, uy0)


def moment_covariance(Cff, measure_basis, ux0, uy0):
    """<dM^a dM^b> = sum_ij m^a_i m^b_j <df_i df_j> (Eq. dfidfj2dmadmb)."""
    m = measure_matrix(measure_basis, ux0, uy0)
    return m @ np.asarray(Cff) @ m.T


# --------------------------------------------------------------------------
# Static structure factors (Eqs. sfactorr, sfactoru, rcorrelator)
# --------------------------------------------------------------------------

def hydro_fields(f, p):
    """delta rho(x) = rho(x) - rho0 and delta j(x) = j(x) - rho0 u0 of a state
    f[i, y, x] (the fields the structure factors transform)."""
    vx, vy, *_ = tables()
    rho = f.sum(axis=0)
    jx = np.tensordot(vx, f, axes=1)
    jy = np.tensordot(vy, f, axes=1)
    return rho - p.rho0, jx - p.rho0 * p.ux0, jy - p.rho0 * p.uy0


def dft2(a):
    """a(k) = sum_x a(x) exp(-i k.x), k = 2 pi (m_x / Lx, m_y / Ly); array
    index [m_y, m_x] (numpy's forward FFT has this sign and no normalisation)."""
    return np.fft.fft2(a)


def structure_sample(f, p):
    """One sample's |drho(k)|^2, |dj_x(k)|^2 and dj_x(k) dj_y(-k) (complex),
    each of shape (Ly, Lx)."""
    dr, djx, djy = hydro_fields(f, p)
    R, X, Y = dft2(dr), dft2(djx), dft2(djy)
    return np.abs(R) ** 2, np.abs(X) ** 2, X * np.conj(Y)


class StructureRun:
    """An oracle run that also accumulates the structure factors of the
    pre-collision state at t = warmup, warmup + every, ...:
    S_k(rho) = <drho(k) drho(-k)> / rho0, S_k(j_x) = <dj_x(k) dj_x(-k)> / rho0,
    R_k(j_x, j_y) = <dj_x(k) dj_y(-k)> / rho0 (complex)."""

    def __init__(self, p, f=None, warmup=0, every=1):
        self.run = Run(p, f=f)
        self.p, self.warmup, self.every = p, int(warmup), int(every)
        shape = (p.Ly, p.Lx)
        self.srr, self.sxx = np.zeros(shape), np.zeros(shape)
        self.rxy = np.zeros(shape, dtype=complex)
        self.nsamp = 0

    def step(self, n):
        for _ in range(int(n)):
            t = self.run.t
            if self.every > 0 and t >= self.warmup and (t - self.warmup) % self.every == 0:
                a, b, c = structure_sample(self.run.f, self.p)
                self.srr += a
                self.sxx += b
                self.rxy += c
                self.nsamp += 1
            self.run.step(1)
        return self

    def factors(self):
        k = 1.0 / (self.nsamp * self.p.rho0)
        return self.srr * k, self.sxx * k, self.rxy * k
