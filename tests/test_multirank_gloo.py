"""Host-side logic of the multi-GPU path on CPU ranks (gloo, world size 2).

Slices are independent problems: a volume is split over ranks by
workloads.shard_slices with no exchange while solving; a benchmark step's
time is the maximum over ranks.  Two CPU processes check that the shards
partition the slices, that their costs are balanced, that per-rank results
(here the FP64 oracle's objective of each slice) reassemble in slice order,
and the max-reduction of the step time.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2202_08627_gb300 import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from tests.problems import small_problem
    slices = [(8, 6, 12), (12, 9, 16), (8, 6, 12), (16, 6, 20), (10, 7, 14)]
    parts = workloads.shard_slices(slices, world)
    mine = parts[rank]
    vals = torch.zeros(len(slices), dtype=torch.float64)
    for i in mine:
        n, nth, nd = slices[i]
        spec, geom, s_exp = small_problem(seed=i, n=n, n_theta=nth, n_det=nd, n_m=3)
        vals[i], _ = oracle.objective_grad(spec.truth, s_exp, geom, want_grad=False)
    dist.all_reduce(vals)                         # each slice filled by exactly one rank
    t = torch.tensor([0.25 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    owners = [torch.zeros(len(slices), dtype=torch.int64) for _ in range(world)]
    own = torch.zeros(len(slices), dtype=torch.int64)
    own[mine] = 1
    dist.all_gather(owners, own)
    if rank == 0:
        np.savez(out_path, vals=vals.numpy(), t=t.numpy(), owners=torch.stack(owners).numpy())
    dist.destroy_process_group()


def test_two_rank_sharding(tmp_path):
    world, port = 2, _free_port()
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    res = np.load(out)
    assert np.all(res["owners"].sum(axis=0) == 1)            # a partition
    assert res["t"][0] == 0.5                                 # max over ranks
    import oracle
    from tests.problems import small_problem
    slices = [(8, 6, 12), (12, 9, 16), (8, 6, 12), (16, 6, 20), (10, 7, 14)]
    for i, (n, nth, nd) in enumerate(slices):
        spec, geom, s_exp = small_problem(seed=i, n=n, n_theta=nth, n_det=nd, n_m=3)
        S, _ = oracle.objective_grad(spec.truth, s_exp, geom, want_grad=False)
        assert res["vals"][i] == pytest.approx(S, rel=1e-15)


def test_shards_are_balanced():
    wl = workloads.uneven1024()
    parts = workloads.shard_slices(wl.slices, 4)
    costs = [sum(wl.slices[i][0] ** 2 * wl.slices[i][1] + wl.slices[i][1] * wl.slices[i][2]
                 for i in p) for p in parts]
    assert sorted(i for p in parts for i in p) == list(range(wl.n_slices))
    assert max(costs) <= 1.02 * min(costs)
