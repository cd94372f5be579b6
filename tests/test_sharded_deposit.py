"""The sharding property the multi-GPU design relies on (one int64 sum
all-reduce of the charge grid per kick): particles split across ranks in any
proportion, each rank deposits its share, and the all-reduced grid equals the
single-rank deposit bit for bit.  Two gloo ranks on CPU, using the oracle's
fixed-point deposit (Sec. IV-A)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2010_11540_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, split, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = synth.gaussian_bunch(30000, 777, 3e-3, 2e-3, 1e-4, 1e-4)
    g = oracle.Geometry(64, 48, -0.012, 0.012, -0.008, 0.008)
    lo = 0 if rank == 0 else split
    hi = split if rank == 0 else len(parts["x"])
    Q, n_out = oracle.deposit(g, np.ascontiguousarray(parts["x"][lo:hi]), np.ascontiguousarray(parts["y"][lo:hi]))
    t = torch.from_numpy(Q.view(np.int64).copy())  # uint64 sums modulo 2^64 are the same bits
    c = torch.tensor([n_out], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, np.concatenate([t.numpy().view(np.uint64).ravel(), c.numpy().astype(np.uint64)]))
    dist.destroy_process_group()


@pytest.mark.parametrize("split", [15000, 1, 29999])
def test_two_rank_deposit_equals_single_rank(tmp_path, split):
    out = str(tmp_path / "q.npy")
    mp.start_processes(_worker, args=(2, _free_port(), split, out), nprocs=2, join=True, start_method="spawn")
    res = np.load(out)
    parts = synth.gaussian_bunch(30000, 777, 3e-3, 2e-3, 1e-4, 1e-4)
    g = oracle.Geometry(64, 48, -0.012, 0.012, -0.008, 0.008)
    Q, n_out = oracle.deposit(g, parts["x"], parts["y"])
    assert np.array_equal(res[:-1].reshape(Q.shape), Q)
    assert res[-1] == n_out


def _track_worker(rank, world, port, out_path):
    """The sharded turn as the tracked turn runs it (the charge reduction
    between each location's deposit and its solve, the solve normalised by the
    whole bunch), on gloo ranks with the oracle's steps: rank r holds the
    particles r, r + world, ... of the bunch."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts, b, grid, lat = synth.workload("c1", n=6000)
    g = oracle.Geometry(*grid)
    st = {k: np.ascontiguousarray(v[rank::world]) for k, v in parts.items()}
    n_total = len(parts["x"])
    head, kicks = oracle.segments(lat)
    K = oracle.kick_strength(b)
    oracle.push(st, head, b)
    for L, seg in kicks[:20]:
        Q, _ = oracle.deposit(g, st["x"], st["y"])
        t = torch.from_numpy(Q.view(np.int64).copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        Ex, Ey = oracle.solve(g, t.numpy().view(np.uint64).reshape(Q.shape), n_total)
        oracle.kick(g, st, Ex, Ey, K * L)
        oracle.push(st, seg, b)
    np.save(out_path + f".{rank}.npy", np.stack([st[k] for k in ("x", "px", "y", "py", "sigma", "psigma")]))
    dist.destroy_process_group()


def test_two_rank_sharded_turn_equals_single_rank(tmp_path):
    """Twenty space-charge steps of a bunch sharded over two gloo ranks, with
    one charge all-reduce per step, give every particle the same bits as the
    whole bunch tracked on one rank (the reduction point of the sharded
    tracked turn)."""
    out = str(tmp_path / "st")
    mp.start_processes(_track_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    parts, b, grid, lat = synth.workload("c1", n=6000)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, max_kicks=20)
    for rank in range(2):
        got = np.load(out + f".{rank}.npy")
        for i, k in enumerate(("x", "px", "y", "py", "sigma", "psigma")):
            assert np.array_equal(got[i], ref[k][rank::2]), (rank, k)
