"""The bench's multi-rank path on CPU ranks (gloo, world size 2): populations are
replicated per rank with disjoint seeds (no data-path collective), and the timing
reduction takes the maximum time and the summed work over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workloads.s_sweep()
        pops = bench.rank_populations(w["pops"], rank)
        seeds = torch.tensor([q["seed"] for q in pops], dtype=torch.int64)
        gathered = [torch.zeros_like(seeds) for _ in range(world)]
        dist.all_gather(gathered, seeds)
        t, units = bench.reduce_over_ranks(dist, "cpu", seconds=1.0 + rank, units=10 * (rank + 1))
        out[rank] = dict(t=t, units=units, seeds=[g.tolist() for g in gathered],
                         same_shape=all(q["L"] == p["L"] and q["n_clones"] == p["n_clones"]
                                        for q, p in zip(pops, w["pops"])))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r]["t"] == 2.0            # max over ranks
        assert res[r]["units"] == 30.0       # sum over ranks
        assert res[r]["same_shape"]
    seeds0, seeds1 = res[0]["seeds"]
    assert not set(seeds0) & set(seeds1)     # independent replicas


def test_seconds_to_se():
    # SE = sigma / sqrt(R) reaches the target after R = (sigma / target)^2 runs of
    # this cost: 16 runs of 2/64 s each
    assert bench.seconds_to_se(sigma=0.004, seconds_per_run=2.0 / 64, target=1e-3) == pytest.approx(0.5)
    # below one run's spread the time is a fraction of a run (the same SE from a run
    # that much shorter), not rounded up
    assert bench.seconds_to_se(sigma=5e-4, seconds_per_run=1.0, target=1e-3) == pytest.approx(0.25)
