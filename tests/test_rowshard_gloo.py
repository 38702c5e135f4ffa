"""CPU-rank simulation of the row-sharded multi-GPU design (gloo backend).

The design for one system on several GPUs: each rank owns a contiguous block of
rows of R, C and A (and their a_i); B and X are replicated.  Per iteration
(Algorithm 3): local row norms s_i and r_i = s_i / a_i; an all-gather of the
per-rank (S, r_max, argmax); the threshold t; an all-gather of the per-rank
admitted sums S_J; the same Philox draw on every rank, which locates the owning
rank; the owner finds i_k and broadcasts it; the owner of row i_k broadcasts
R_{i_k} and A_{i_k}; every rank forms w = R_{i_k} B^T, v = w B and its own
u_i = A_i A_{i_k}^T, updates its rows of R and its copy of X.

The simulation runs that exchange on world_size gloo ranks in FP64 and must
reproduce the oracle's selected rows (one process, full R) while the residual is
above the rounding floor, and the oracle's X to 1e-9.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _uniform(seed, k, sys=0):
    """Word 0 of Philox4x64-10 with key (seed, 0) and counter (k, sys, 0, 0),
    top 53 bits scaled by 2^-53, via numpy's Philox (which steps its counter
    before each block)."""
    c = ((k | (sys << 64)) - 1) % (1 << 256)
    words = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=words)).random()


def _gather(x):
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, x)
    return out


def sharded_solve(A, B, C, variant, theta, alpha, seed, maxit):
    rank, world = dist.get_rank(), dist.get_world_size()
    m, p = A.shape
    r0, r1 = m * rank // world, m * (rank + 1) // world
    Al = A[r0:r1]
    R = C[r0:r1].copy()
    a = np.einsum("ij,ij->i", Al, Al)
    F = sum(_gather(float(a.sum())))
    X = np.zeros((p, B.shape[0]))
    rows, Ss = [], []
    for k in range(maxit):
        s = np.einsum("ij,ij->i", R, R)
        rr = np.where(a > 0, s / np.where(a > 0, a, 1.0), -np.inf)
        li = int(np.argmax(rr)) if len(rr) else 0
        parts = _gather((float(s.sum()), float(rr[li]) if len(rr) else -np.inf, r0 + li))
        S = sum(pt[0] for pt in parts)
        if not S > 0:
            break
        r_max = max(pt[1] for pt in parts)
        i_max = min(pt[2] for pt in parts if pt[1] == r_max)
        if variant == "mwrbk":
            ik = i_max
        else:
            th = 0.5 if variant == "grbk" else theta
            t = min(th * r_max + (1 - th) * (S / F), r_max)
            adm = rr >= t
            SJs = _gather(float(s[adm].sum()))
            target = _uniform(seed, k) * sum(SJs)
            owner, excl = None, 0.0
            for rk, v in enumerate(SJs):
                if v > 0 and excl + v > target:
                    owner = rk
                    break
                excl += v
            if owner is None:  # rounding left the target uncovered: the last admitted row
                owner, excl = max(rk for rk, v in enumerate(SJs) if v > 0), -np.inf
            pick = None
            if rank == owner:
                run, last = excl, None
                for i in np.nonzero(adm)[0]:
                    last = i
                    if run + s[i] > target:
                        pick = i
                        break
                    run += s[i]
                pick = r0 + int(pick if pick is not None else last)
            box = [pick]
            dist.broadcast_object_list(box, src=owner)
            ik = int(box[0])
        holder = next(rk for rk in range(world) if m * rk // world <= ik < m * (rk + 1) // world)
        row = torch.zeros(B.shape[1] + p, dtype=torch.float64)
        if rank == holder:
            row[:B.shape[1]] = torch.from_numpy(R[ik - r0])
            row[B.shape[1]:] = torch.from_numpy(Al[ik - r0])
        dist.broadcast(row, src=holder)
        Rik, Aik = row[:B.shape[1]].numpy(), row[B.shape[1]:].numpy()
        c = alpha / float(Aik @ Aik)
        w = Rik @ B.T
        X += c * np.outer(Aik, w)
        v = w @ B
        R -= c * np.outer(Al @ Aik, v)
        rows.append(ik)
        Ss.append(S)
    return np.array(rows), np.array(Ss), X


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out_dir, variant, theta, maxit):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads
    A, B, C, _ = workloads.config_small()
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    rows, Ss, X = sharded_solve(A, B, C, variant, theta, alpha, seed=7, maxit=maxit)
    if rank == 0:
        np.savez(os.path.join(out_dir, "shard.npz"), rows=rows, S=Ss, X=X, alpha=alpha)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,variant,theta", [(2, "grbk", 0.5), (2, "rgrbk", 0.8), (2, "mwrbk", 1.0),
                                                 (3, "rgrbk", 0.3)])
def test_row_sharded_exchange_matches_oracle(tmp_path, world, variant, theta):
    import oracle
    import workloads
    maxit = 300
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), variant, theta, maxit), nprocs=world, join=True)
    got = np.load(tmp_path / "shard.npz")
    A, B, C, _ = workloads.config_small()
    alpha = 1.0 / np.linalg.norm(B, 2) ** 2
    assert float(got["alpha"]) == alpha
    orc = oracle.solve(A, B, C, variant, theta=theta, alpha=alpha, seed=7, maxit=maxit,
                       mode=oracle.MODE_FACTORED)
    live = np.nonzero(orc["S"] <= 1e-20 * orc["S"][0])[0]
    n = int(live[0]) if len(live) else maxit
    assert np.array_equal(got["rows"][:n], orc["rows"][:n])
    assert np.max(np.abs(got["S"][:n] - orc["S"][:n]) / orc["S"][:n]) < 1e-9
    assert np.linalg.norm(got["X"] - orc["X"]) <= 1e-9 * np.linalg.norm(orc["X"])
