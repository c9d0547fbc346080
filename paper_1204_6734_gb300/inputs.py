"""Seeded synthetic workloads for the fluctuating D2Q9 lattice-Boltzmann step.

This module only draws and names parameters; it holds none of the method's
arithmetic and imports nothing else from this package, so the tests can feed
the same inputs to the CUDA library and to the CPU oracle. The paper's own runs
(Section 3) are 21x21 periodic lattices at rest density rho0 = 10^6 with Poisson
statistics; since the update is invariant under f -> lambda f, kT -> lambda kT,
the workloads below use rho0 = 1 and a small k_B T instead.

Relaxation rates are given per moment a = 0..8 in the order of the Hermite
rows (rho, j_x, j_y, Pi_xx-yy, Pi_xy, Pi_xx+yy, q_x, q_y, epsilon); the
conserved entries 0..2 are ignored by both implementations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

STANDARD = "standard"
LOCAL = "local"
LUT = "lut"         # the f-norm from the paper's velocity table (Section 4)


def omega_groups(shear: float, bulk: float, ghost: float) -> tuple:
    """Rates per moment: shear on Pi_xx-yy and Pi_xy, bulk on Pi_xx+yy, ghost on
    q_x, q_y, epsilon."""
    return (0.0, 0.0, 0.0, shear, shear, bulk, ghost, ghost, ghost)


@dataclasses.dataclass
class LatticeParams:
    Lx: int
    Ly: int
    rho0: float = 1.0
    ux0: float = 0.0
    uy0: float = 0.0
    kT: float = 1e-4
    omega: Sequence[float] = omega_groups(1.0, 1.0, 1.0)
    basis: str = LOCAL
    precision: str = "fp32"     # "fp64" | "fp32" | "fp16dev"
    seed: int = 1
    replica: int = 0

    @property
    def nodes(self) -> int:
        return self.Lx * self.Ly


# ---------------------------------------------------------------------------
# The five workloads the hot path is measured and tested on
# ---------------------------------------------------------------------------

def fp64_parity_lattice() -> LatticeParams:
    """32x32, FP64, u0 = (0.1, 0), kT = 1e-4, all rates 1, f-norm basis, seed 1.
    Run for 10^4 steps with <df_i df_j> sampled every step after 10^3."""
    return LatticeParams(32, 32, 1.0, 0.1, 0.0, 1e-4, omega_groups(1.0, 1.0, 1.0),
                         LOCAL, "fp64", seed=1)


FP64_PARITY_STEPS = 10_000
FP64_PARITY_WARMUP = 1_000

SWEEP_UX0 = (0.0, 0.05, 0.1, 0.2, 0.3)


def single_lattice(ux0: float = 0.1, basis: str = LOCAL, side: int = 4096,
                   precision: str = "fp32") -> LatticeParams:
    """The 4096^2 FP32 lattice: kT = 1e-4, shear 1.0, bulk 0.8, ghost 1.0,
    seed 1000 + 10 i_u + (0 standard | 1 local | 2 look-up-table f-norm)."""
    iu = SWEEP_UX0.index(ux0) if ux0 in SWEEP_UX0 else 0
    seed = 1000 + 10 * iu + {STANDARD: 0, LOCAL: 1, LUT: 2}[basis]
    return LatticeParams(side, side, 1.0, ux0, 0.0, 1e-4, omega_groups(1.0, 0.8, 1.0),
                         basis, precision, seed=seed)


SINGLE_LATTICE_STEPS = 2000


def small_sweep_replicas(ux0: float, basis: str, n: int = 256, side: int = 21) -> List[LatticeParams]:
    """n independent copies of the paper's small lattice (side x side, the
    sweep's rates and kT as single_lattice) at one u_x0: seeds
    0x21000000 + 4096 i_u + 1024 b + r (b = 0 standard, 1 local, 2 table
    f-norm), so that every replica of every sweep point draws its own noise."""
    iu = SWEEP_UX0.index(ux0) if ux0 in SWEEP_UX0 else 0
    b = {STANDARD: 0, LOCAL: 1, LUT: 2}[basis]
    return [LatticeParams(side, side, 1.0, ux0, 0.0, 1e-4, omega_groups(1.0, 0.8, 1.0), basis, "fp32",
                          seed=0x21000000 + 4096 * iu + 1024 * b + r) for r in range(n)]


def replica_ensemble(n: int = 256, seed: int = 3, lo: int = 64, hi: int = 1024,
                     basis: str = LOCAL) -> List[LatticeParams]:
    """Uneven replicas: sides log-uniform integers in [lo, hi], u_x0 ~ U[0, 0.3],
    kT in {1e-5, 1e-4, 1e-3}, shear rate ~ U[0.6, 1.8], bulk = ghost = 1,
    replica seed 0x5EED0000 + r."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(n):
        Lx = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        Ly = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        ux0 = float(g.uniform(0.0, 0.3))
        kT = float((1e-5, 1e-4, 1e-3)[int(g.integers(0, 3))])
        ws = float(g.uniform(0.6, 1.8))
        out.append(LatticeParams(Lx, Ly, 1.0, ux0, 0.0, kT, omega_groups(ws, 1.0, 1.0),
                                 basis, "fp32", seed=0x5EED0000 + r, replica=r))
    return out


REPLICA_STEPS = 5000


def precision_lattice(precision: str, side: int = 8192) -> LatticeParams:
    """8192^2, u0 = (0.2, 0), kT = 1e-4, all rates 1, seed 4, 1000 steps."""
    return LatticeParams(side, side, 1.0, 0.2, 0.0, 1e-4, omega_groups(1.0, 1.0, 1.0),
                         LOCAL, precision, seed=4)


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    params: LatticeParams
    steps: int
    warmup: int = 0     # correlations sampled every `every` steps from `warmup` on
    every: int = 1


def serving_requests(n: int = 10_000, rate_hz: float = 200.0, seed: int = 5,
                     lo: int = 32, hi: int = 2048, basis: str = LOCAL) -> List[Request]:
    """Poisson arrivals; sides log-uniform in [lo, hi]; u_x0 ~ U[0, 0.3];
    kT log-uniform in [1e-5, 1e-3]; shear rate ~ U[0.6, 1.8]; steps uniform
    integers in [500, 20000]; seed = request id. Each request samples its
    correlations on every step after a warm-up of a tenth of its steps."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(n):
        t += float(g.exponential(1.0 / rate_hz))
        Lx = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        Ly = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        ux0 = float(g.uniform(0.0, 0.3))
        kT = float(math.exp(g.uniform(math.log(1e-5), math.log(1e-3))))
        ws = float(g.uniform(0.6, 1.8))
        steps = int(g.integers(500, 20001))
        p = LatticeParams(Lx, Ly, 1.0, ux0, 0.0, kT, omega_groups(ws, 1.0, 1.0), basis,
                          "fp32", seed=rid, replica=rid)
        out.append(Request(rid, t, p, steps, warmup=steps // 10, every=1))
    return out


# ---------------------------------------------------------------------------
# Generic seeded arrays
# ---------------------------------------------------------------------------

def perturbation(shape, seed: int) -> np.ndarray:
    """Standard-normal array (float64) for perturbed initial states."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def random_velocities(n: int, seed: int, umax: float = 0.3) -> np.ndarray:
    """n velocities (ux, uy) uniform in the disc |u| < umax."""
    g = np.random.Generator(np.random.PCG64(seed))
    r = umax * np.sqrt(g.uniform(0, 1, n))
    phi = g.uniform(0, 2 * np.pi, n)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def small_lattices() -> List[tuple]:
    """Lattice shapes (Lx, Ly) for parity: odd, tiny, ragged and several tiles."""
    return [(1, 1), (3, 3), (5, 7), (21, 21), (32, 32), (37, 19), (129, 67), (256, 130)]
