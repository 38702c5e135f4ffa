"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
system shards are disjoint, cover every system, balance the work, and each
rank's oracle solves of its own shard need no collective; the job time is the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2408_05444_gb300.shard import max_over_ranks, my_systems, shard_systems


def test_shards_cover_and_balance():
    rng = np.random.default_rng(0)
    work = [int(x) for x in rng.integers(128, 513, 192) ** 2]
    for world in (1, 2, 3, 8):
        sh = shard_systems(work, world)
        flat = sorted(s for part in sh for s in part)
        assert flat == list(range(len(work)))
        loads = [sum(work[s] for s in part) for part in sh]
        assert max(loads) - min(loads) <= max(work)
    assert shard_systems([5, 5, 5], 2) == [[0, 2], [1]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import workloads
    sy = workloads.blur_systems(n_images=4, min_side=16, max_side=32, noise=0.0, mild=True, seed=3)
    work = [s["A"].shape[0] * s["B"].shape[1] for s in sy]
    mine = my_systems(work, rank, world)
    errs = {}
    for k in mine:
        s = sy[k]
        r = oracle.solve(s["A"], s["B"], s["C"], "grbk", seed=1, sys=k, maxit=100000, stop=oracle.STOP_RELRES,
                         tol=1e-10, trace=False, mode=oracle.MODE_FACTORED)
        errs[k] = float(np.linalg.norm(r["X"] - s["X"]) / np.linalg.norm(s["X"]))
    t_job = max_over_ranks(float(rank + 1))
    # gather only for the test's own check (not part of the solve)
    got = [None] * world
    dist.all_gather_object(got, errs)
    if rank == 0:
        np.save(os.path.join(out_dir, "result.npy"), np.array([t_job, len(sy)] + [max(e.values()) for e in got]))
    dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = np.load(tmp_path / "result.npy")
    assert res[0] == 2.0            # max over ranks
    assert np.all(res[2:] < 1e-6)   # every rank solved its own shard
