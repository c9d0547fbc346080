"""Host logic of the slab decomposition (paper_1204_6734_gb300.slabs): the split
of the rows, and the halo exchange between ranks (one slab each) run as gloo
ranks on the CPU -- each rank receives its lower neighbour's upward halo and its
upper neighbour's downward halo, periodically in y."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1204_6734_gb300 import inputs, slabs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("Ly,n", [(37, 1), (37, 2), (37, 3), (4096, 8), (5, 5)])
def test_rows_cover_the_lattice(Ly, n):
    parts = [slabs.slab_rows(Ly, n, k) for k in range(n)]
    assert parts[0][0] == 0
    for (y0, r), (y1, _) in zip(parts, parts[1:]):
        assert y1 == y0 + r
    assert sum(r for _, r in parts) == Ly
    assert max(r for _, r in parts) - min(r for _, r in parts) <= 1
    p = inputs.LatticeParams(16, Ly)
    assert [slabs.slab_params(p, n, k).Ly for k in range(n)] == [r for _, r in parts]
    with pytest.raises(ValueError):
        slabs.slab_rows(Ly, n, n)


def _pattern(rank, which, n=12):
    return torch.arange(n, dtype=torch.float32) + 1000.0 * rank + 100.0 * which


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = _pattern(rank, 0), _pattern(rank, 1)
        rlo, rhi = torch.zeros_like(lo), torch.zeros_like(hi)
        for _ in range(3):      # repeated exchanges stay matched
            slabs.exchange_halos(lo, hi, rlo, rhi, dist, rank, world)
        out[rank] = (rlo.tolist(), rhi.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_their_edge_rows(world):
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rlo, rhi = res[r]
        assert rlo == _pattern((r - 1) % world, 1).tolist()    # below's upward halo
        assert rhi == _pattern((r + 1) % world, 0).tolist()    # above's downward halo


def test_single_slab_exchanges_with_itself():
    lo, hi = _pattern(0, 0), _pattern(0, 1)
    rlo, rhi = torch.zeros_like(lo), torch.zeros_like(hi)
    slabs.exchange_halos(lo, hi, rlo, rhi)
    assert torch.equal(rlo, hi) and torch.equal(rhi, lo)
