"""Slab decomposition of one periodic lattice along y.

The step is local plus streaming (Eq. LBE1), so a lattice of Lx x Ly nodes
splits into slabs of whole rows that exchange, after every step, only the
populations that cross their y boundaries: 3 of the 9 (v_y = +1 upwards,
v_y = -1 downwards) on each of the slab's two edge rows, 3 Lx values per
boundary and direction. Each slab is a lattice handle marked with
flb_set_slab, so its noise is keyed by the global node and a decomposed run
draws what the whole lattice draws.

Two ways to hold the slabs:
* LocalSlabs: all slabs in this process, on one device and one stream; the
  exchange is a device copy between the slabs' halo buffers.
* RankSlab: one slab per rank (one GPU each); the exchange is a periodic ring
  of sends and receives over torch.distributed (exchange_halos), NCCL between
  GPUs, gloo for CPU tests of the plumbing.
"""
from __future__ import annotations

import dataclasses

from . import flb


def slab_rows(Ly: int, nslabs: int, k: int):
    """(y0, rows) of slab k when Ly rows are split into nslabs slabs as evenly
    as possible (the first Ly mod nslabs slabs take one row more)."""
    if not 0 <= k < nslabs or nslabs > Ly:
        raise ValueError("need 0 <= k < nslabs <= Ly")
    base, extra = divmod(Ly, nslabs)
    y0 = k * base + min(k, extra)
    return y0, base + (1 if k < extra else 0)


def slab_params(p, nslabs: int, k: int):
    """The parameters of slab k: those of the whole lattice with its rows."""
    y0, rows = slab_rows(p.Ly, nslabs, k)
    return dataclasses.replace(p, Ly=rows)


def exchange_halos(send_lo, send_hi, recv_lo, recv_hi, dist=None, rank=0, world=1):
    """The halo exchange of one slab per rank, periodic in y: rank r receives
    rank r-1's hi (the populations moving up out of that slab) into recv_lo and
    rank r+1's lo (those moving down) into recv_hi. Tensors of equal size, on
    the device for NCCL or on the host for gloo."""
    if world == 1 or dist is None:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    below, above = (rank - 1) % world, (rank + 1) % world
    ops = [dist.P2POp(dist.isend, send_hi, above, tag=1),
           dist.P2POp(dist.irecv, recv_lo, below, tag=1),
           dist.P2POp(dist.isend, send_lo, below, tag=2),
           dist.P2POp(dist.irecv, recv_hi, above, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def _buffers(torch, lat, device):
    n = flb.flb_halo_bytes(lat.h)
    return [torch.empty(n, dtype=torch.uint8, device=device) for _ in range(4)]


class LocalSlabs:
    """The slabs of lattice p (nslabs of them), all on the current device and on
    one stream: step(n) steps every slab and exchanges the halos after each
    step. populations() / raw_sums() give the whole lattice's."""

    def __init__(self, p, nslabs: int, stream=None, **lattice_kw):
        import torch
        self.p, self.n = p, nslabs
        self.stream = stream
        self.lats = []
        for k in range(nslabs):
            y0, _ = slab_rows(p.Ly, nslabs, k)
            lat = flb.Lattice(slab_params(p, nslabs, k), stream=stream, **lattice_kw)
            flb.flb_set_slab(lat.h, p.Ly, y0)
            self.lats.append(lat)
        self.bufs = [_buffers(torch, lat, "cuda") for lat in self.lats]   # send lo, hi; recv lo, hi

    def exchange(self):
        import torch
        with torch.cuda.stream(self.stream) if self.stream is not None else _nullctx():
            for lat, (slo, shi, _, _) in zip(self.lats, self.bufs):
                flb.flb_halo_pack(lat.h, slo, shi)
            for k, (_, _, rlo, rhi) in enumerate(self.bufs):
                rlo.copy_(self.bufs[(k - 1) % self.n][1])
                rhi.copy_(self.bufs[(k + 1) % self.n][0])
            for lat, (_, _, rlo, rhi) in zip(self.lats, self.bufs):
                flb.flb_halo_unpack(lat.h, rlo, rhi)

    def step(self, n: int = 1):
        for _ in range(n):
            for lat in self.lats:
                flb.flb_step(lat.h, 1)
            self.exchange()

    def set_sampling(self, warmup, every):
        for lat in self.lats:
            lat.set_sampling(warmup, every)

    def set_populations(self, f):
        for k, lat in enumerate(self.lats):
            y0, rows = slab_rows(self.p.Ly, self.n, k)
            lat.set_populations(f[:, y0:y0 + rows, :].copy())

    def populations(self):
        import numpy as np
        return np.concatenate([lat.populations() for lat in self.lats], axis=1)

    def raw_sums(self):
        sums = [lat.raw_sums() for lat in self.lats]
        return sum(s[0] for s in sums), sum(s[1] for s in sums), sum(s[2] for s in sums)

    def sync(self):
        for lat in self.lats:
            lat.sync()

    def close(self):
        for lat in self.lats:
            lat.close()
        self.lats = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class RankSlab:
    """Slab `rank` of lattice p, one per rank of a torch.distributed group (the
    device of this rank current): step(n) steps it and exchanges its halos
    with the neighbouring ranks after each step."""

    def __init__(self, p, dist, rank: int, world: int, stream=None, **lattice_kw):
        import torch
        self.p, self.dist, self.rank, self.world = p, dist, rank, world
        self.stream = stream
        y0, _ = slab_rows(p.Ly, world, rank)
        self.lat = flb.Lattice(slab_params(p, world, rank), stream=stream, **lattice_kw)
        flb.flb_set_slab(self.lat.h, p.Ly, y0)
        self.slo, self.shi, self.rlo, self.rhi = _buffers(torch, self.lat, "cuda")

    def step(self, n: int = 1):
        import torch
        for _ in range(n):
            flb.flb_step(self.lat.h, 1)
            flb.flb_halo_pack(self.lat.h, self.slo, self.shi)
            with torch.cuda.stream(self.stream) if self.stream is not None else _nullctx():
                exchange_halos(self.slo, self.shi, self.rlo, self.rhi, self.dist, self.rank,
                               self.world)
            flb.flb_halo_unpack(self.lat.h, self.rlo, self.rhi)

    def close(self):
        self.lat.close()


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False
