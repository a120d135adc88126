"""The multi-GPU path on the CPU: two `gloo` ranks each take their shard of one
population (paper_2606_15622_gb300.shard), run the oracle's moments, exact
closure and velocity update on it with the Philox counters continued from the
slice's first global particle, and the gathered results equal the unsharded
run bit for bit.  The data path has no collective; the test gathers the
results only to compare them."""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2606_15622_gb300 import populations as P
from paper_2606_15622_gb300 import shard as SH

DT, SEED, STEP = 0.3, 77, 5


def _population():
    return P.cavity(seed=8, nx=24, ny=20, mean_ppc=40.0)


def _run(v, offsets, tau, p0):
    m = O.moments(v, offsets)
    y, fl = O.closure(m, tau)
    xi = O.normals(v.shape[1], SEED, STEP, first_index=p0)
    v_new, alpha, fl_out = O.velocity_update(v, offsets, m, y, tau, fl, DT, xi=xi)
    return y, fl_out, v_new


def _worker(rank, world, port, out_path):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    pop = _population()
    v, off, tau, p0, (c0, c1) = SH.shard_arrays(pop.v64, pop.offsets, pop.tau, world, rank)
    y, fl, v_new = _run(v, off, tau, p0)
    parts = [None] * world
    dist.all_gather_object(parts, {"c": (c0, c1), "p0": p0, "y": y, "fl": fl, "v": v_new})
    if rank == 0:
        np.savez(out_path, c=np.array([q["c"] for q in parts]), y=np.concatenate([q["y"] for q in parts]),
                 fl=np.concatenate([q["fl"] for q in parts]), v=np.concatenate([q["v"] for q in parts], axis=1))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_bounds_cover_cells_once_and_balance_particles():
    pop = P.cylinder(nx=64, ny=32, target_particles=200_000)
    for world in (1, 2, 3, 4, 8):
        bounds = [SH.shard_bounds(pop.offsets, world, r) for r in range(world)]
        assert bounds[0][0] == 0 and bounds[-1][1] == pop.n_cells
        for a, b in zip(bounds, bounds[1:]):
            assert a[1] == b[0] and a[3] == b[2]
        for c0, c1, p0, p1 in bounds:
            assert c0 % 32 == 0 and c0 <= c1
            assert abs((p1 - p0) - pop.n_particles / world) <= 0.05 * pop.n_particles / world + 32 * pop.counts.max()
    with pytest.raises(ValueError):
        SH.shard_bounds(pop.offsets, 2, 2)


def test_two_gloo_ranks_equal_the_unsharded_run(tmp_path):
    out = str(tmp_path / "sharded.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    pop = _population()
    y, fl, v_new = _run(pop.v64, pop.offsets, pop.tau, 0)
    c = got["c"]
    assert c[0][0] == 0 and c[-1][1] == pop.n_cells and c[0][1] == c[1][0] and 0 < c[0][1] < pop.n_cells
    np.testing.assert_array_equal(got["y"], y)
    np.testing.assert_array_equal(got["fl"], fl)
    np.testing.assert_array_equal(got["v"], v_new)
