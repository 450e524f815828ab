"""Multi-rank paths on CPU ranks (gloo, world size 2): the element partition
with its interface sum reproduces the full tangent apply, and the benchmark's
max-over-ranks timing and weak-scaling aggregate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _dd_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2408_12479_gb300 import dd
        from paper_2408_12479_gb300 import inputs as I
        from tests import cases
        n, p = 3, 2
        m = I.box_mesh(n, p, jitter=0.1, seed=5, clamp=False)
        M = O.OracleMesh(m)
        mat = cases.oracle_material("cNH")
        X = O.node_coords(M)
        u = I.sine_field(7, strain=0.02)(X).ravel()
        du = I.random_direction(m.n_dofs, 8)
        slabs = dd.slab_partition(n, world)
        z0, z1 = slabs[rank]
        part = O.apply(M, mat, u, du, elems=dd.slab_elements(n, n, z0, z1))
        v = dd.interface_sum(torch.tensor(part), n, n, p, slabs, rank)
        n0, n1 = dd.slab_node_range(n, n, p, z0, z1)
        full = O.apply(M, mat, u, du)
        err = float(np.abs(v.numpy()[3 * n0:3 * n1] - full[3 * n0:3 * n1]).max() / np.abs(full).max())
        out[rank] = err
    finally:
        dist.destroy_process_group()


def test_slab_partition_interface_sum_matches_full_apply():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_dd_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert len(out) == world
    assert max(out.values()) < 1e-13


def _timing_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [1.5, 2.5][rank]
        t_max = bench.max_over_ranks(ms, world)
        out[rank] = (t_max, bench.weak_value(1000, t_max, world))
    finally:
        dist.destroy_process_group()


def test_bench_max_over_ranks_and_weak_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_timing_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 2.5
        assert abs(value - 2 * 1000 / 2.5e-3 / 1e9) < 1e-15
