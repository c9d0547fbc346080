"""The multi-GPU form runs independent replicas: each rank its own lattice and
noise stream, ranks meeting only to take the slowest rank's time. The host
logic runs here as two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1204_6734_gb300 import inputs, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = replicas.rank_params(inputs.single_lattice(0.1, inputs.LOCAL, side=64), rank)
        # a rank's "time": made different per rank on purpose
        t = 1.0 + 0.5 * rank
        tmax = replicas.max_over_ranks(t, dist)
        out[rank] = (p.seed, p.replica, tmax,
                     replicas.whole_job_rate(64 * 64 * 10, world, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_distinct_streams_and_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    (s0, r0, t0, v0), (s1, r1, t1, v1) = res[0], res[1]
    assert (r0, r1) == (0, 1) and s1 - s0 == replicas.SEED_STRIDE
    assert t0 == t1 == 1.5
    assert v0 == v1 == pytest.approx(64 * 64 * 10 * 2 / 1.5)


def test_replica_streams_are_independent_draws():
    """Different ranks draw different noise for the same node and step (the
    oracle's Philox with the ranks' keys and counters)."""
    base = inputs.single_lattice(0.1, inputs.LOCAL, side=64)
    p0, p1 = replicas.rank_params(base, 0), replicas.rank_params(base, 1)
    a = np.array([oracle.draw_fields(p0.seed, p0.replica, n, 7) for n in range(64)])
    b = np.array([oracle.draw_fields(p1.seed, p1.replica, n, 7) for n in range(64)])
    assert not np.any(np.all(a == b, axis=1))


def test_single_rank_needs_no_process_group():
    assert replicas.max_over_ranks(3.25) == 3.25


def _worker_failing(rank, world, port, out):
    """Rank 1 fails before the end of the timed region (it returns without
    joining the max over ranks, as a crashed rank would); rank 0 must get an
    error from its collective within the group's timeout, not hang."""
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        return
    t0 = time.monotonic()
    try:
        replicas.max_over_ranks(1.0, dist)
        out[rank] = ("no error", time.monotonic() - t0)
    except Exception as e:   # the failure the surviving rank must see
        out[rank] = (type(e).__name__, time.monotonic() - t0)


@pytest.mark.timeout(120)
def test_a_failed_rank_is_reported_not_waited_for():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker_failing, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    kind, waited = res[0]
    assert kind != "no error"
    assert waited < 60
