"""Multi-rank host logic of the batch-axis sharding, on CPU with gloo
(world size 2): every instance is owned by exactly one rank, the dose
all-reduce equals the single-process sum, and the step time is the maximum
over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_12391_gb300 import sharding


def test_blocks_cover_every_item_once():
    for n in (0, 1, 5, 64, 80):
        for world in (1, 2, 3, 8):
            owned = [i for r in range(world) for i in sharding.block(n, r, world)]
            assert owned == list(range(n))
            sizes = [len(sharding.block(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_views, V, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    per_view = rng.uniform(0, 1, size=(n_views, V))           # stand-in per-view doses
    mine = sharding.block(n_views, rank, world)
    dose = torch.tensor(per_view[list(mine)].sum(axis=0), dtype=torch.float64)
    sharding.sum_dose(dose)
    t = sharding.max_time(10.0 + rank)
    if rank == 0:
        np.save(out_path, np.concatenate([dose.numpy(), [t]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_dose_sum_and_max_time(tmp_path):
    n_views, V = 7, 50
    out = str(tmp_path / "r.npy")
    mp.spawn(_worker, args=(2, _free_port(), n_views, V, out), nprocs=2, join=True)
    res = np.load(out)
    ref = np.random.default_rng(0).uniform(0, 1, size=(n_views, V)).sum(axis=0)
    np.testing.assert_allclose(res[:-1], ref, rtol=1e-14)
    assert res[-1] == 11.0


def _physics_worker(rank, world, port, out_path):
    """Each rank solves its block of the views of a small axial scan with the
    oracle and the per-rank doses are summed across ranks."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import solver as osv
    from synth import phantoms as ph
    p = _scan_problem(ph)
    dose = torch.zeros(p.V, dtype=torch.float64)
    for view in sharding.my_items(p.sources, rank, world):
        q = p.with_sources([view])
        dose += torch.from_numpy(osv.dose(q, osv.solve(q, tol=1e-13).phi))
    sharding.sum_dose(dose)
    if rank == 0:
        np.save(out_path, dose.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _scan_problem(ph):
    p = ph.water_cylinder(nx=12, ny=10, nz=4, dx=1.5, dy=1.5, dz=2.0, diameter=14.0, G=2, sn=4, L=1,
                          sid=20.0, fan_deg=60.0, z_width=8.0)
    return p.with_sources(ph.axial_scan_sources(p, 5, sid=20.0, fan_deg=60.0, z_width=8.0))


def test_two_rank_scan_dose_equals_superposed_solve(tmp_path):
    """Five views of an axial scan split over two gloo ranks: the summed
    per-view oracle doses equal the oracle dose of one solve with all five
    sources (the transport problem is linear in its sources)."""
    from oracle import solver as osv
    from synth import phantoms as ph
    out = str(tmp_path / "dose.npy")
    mp.spawn(_physics_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    p = _scan_problem(ph)
    ref = osv.dose(p, osv.solve(p, tol=1e-13).phi)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
