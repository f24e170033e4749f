"""Multi-rank host logic on CPU ranks (gloo): the whole-job rate (units of
all ranks over the slowest rank's time), the partition of a batch's
instances over ranks, and the z-slab decomposition of one grid with halo
exchange, checked on the FP64 oracle against the undivided run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_22221_b300.distributed import (exchange_halos, halo_plan, job_rate, shard_instances, slab_partition,
                                               step_radius)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r did (r+1) * 1e9 units in (1 + r) * 0.5 s
    rate, t = job_rate((rank + 1) * 1e9, (1 + rank) * 0.5)
    out[rank] = (rate, t)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_sums_units_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    for r in range(2):
        assert res[r][1] == pytest.approx(1.0)
        assert res[r][0] == pytest.approx(3e9)


def test_job_rate_single_process():
    assert job_rate(2e9, 0.5) == (4e9, 0.5)


def test_shard_instances_balanced_and_complete():
    rng = np.random.default_rng(0)
    cells = rng.integers(48, 97, size=64) ** 3
    for world in (1, 2, 3, 8):
        sh = shard_instances(cells, world)
        flat = sorted(q for s in sh for q in s)
        assert flat == list(range(64))
        loads = [int(sum(cells[q] for q in s)) for s in sh]
        assert max(loads) - min(loads) <= int(cells.max())
        assert sh == shard_instances(cells, world)       # deterministic


# ------------------------------------------------------------ z slabs

_FIELDS = (("Ex", "face", 0), ("Ey", "face", 0), ("Ez", "cell", 0), ("Hx", "cell", 0), ("Hy", "cell", 0),
           ("Hz", "face", 0), ("M", "cell", 1))
_ITER = 3


def _slab_workload():
    """A 13 x 11 x 30 grid with every feature, and at the cut between two
    ranks (z = 15) a PEC cell, a magnetic region across it and a source."""
    from paper_2510_22221_b300 import workloads as W

    w = W.random_small(21, nx=13, ny=11, nz=30, steps=14, design=True)
    mid = w.mat_id.copy()
    mid[13:18, 4:7, 5:9] = 3
    src = w.sources + [dict(comp=2, i=6, j=8, k=14, J0=2e6, f0=5e12, Tp=1.2e-13, tpk=2.5e-13)]
    import dataclasses

    return dataclasses.replace(w, mat_id=mid, sources=src)


def _slab_oracle(w, ea, eb):
    """The oracle on cells [ea, eb) of the workload along z."""
    import oracle
    from tests.helpers import oracle_from_workload

    full = oracle_from_workload(w, llg_fixed_iter=_ITER)
    mats = full.materials
    srcs = [oracle.Source(comp=s["comp"], ijk=(s["i"], s["j"], s["k"] - ea), J0=s["J0"], f0=s["f0"], Tp=s["Tp"],
                          tpk=s["tpk"]) for s in w.sources if ea <= s["k"] < eb]
    eps = None if full.eps_r_cell is None else full.eps_r_cell[ea:eb]
    return oracle.OracleSim(w.nx, w.ny, eb - ea, w.dx, w.dy, w.dz, full.dt, mats, w.mat_id[ea:eb], w.hbias,
                            sources=srcs, eps_r_cell=eps, llg_fixed_iter=_ITER)


def _slab_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _slab_workload()
    parts = slab_partition(w.nz, world, step_radius(_ITER))
    a, b, ea, eb = parts[rank]
    sub = _slab_oracle(w, ea, eb)
    for _ in range(w.steps):
        sub.run(1)
        exchange_halos([getattr(sub, n) for n, _, _ in _FIELDS], [k for _, k, _ in _FIELDS], parts, rank,
                       z_axes=[ax for _, _, ax in _FIELDS])
    own = {}
    for n, kind, ax in _FIELDS:
        hi = b + 1 if kind == "face" and b == w.nz else b
        own[n] = np.take(getattr(sub, n), range(a - ea, hi - ea), axis=ax)
    out[rank] = own
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_z_slabs_with_halo_exchange_equal_the_whole_grid(world):
    """Each rank steps its slab extended by step_radius ghost planes (cut
    faces as walls) and refreshes the ghosts from their owners after every
    step: the owned planes of every field and of M equal the undivided FP64
    oracle run to the bit, across a PEC cell, a magnetic region (fixed LLG
    iterates) and a source at the cut."""
    from tests.helpers import oracle_from_workload

    w = _slab_workload()
    ref = oracle_from_workload(w, llg_fixed_iter=_ITER)
    ref.run(w.steps)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_slab_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for n, kind, ax in _FIELDS:
        got = np.concatenate([res[r][n] for r in range(world)], axis=ax)
        want = getattr(ref, n)
        assert got.shape == want.shape, n
        np.testing.assert_array_equal(got, want, err_msg=n)
    assert np.abs(ref.M).max() > 0 and np.abs(ref.Ez).max() > 0


def test_halo_plan_covers_every_ghost_plane_once():
    """Every ghost plane of every rank is received once from its owner, and
    what each rank sends is exactly what its peers receive from it."""
    for nz, world, ghost in ((30, 2, 9), (10, 3, 2), (17, 4, 5), (5, 5, 3)):
        parts = slab_partition(nz, world, ghost)
        assert [p[0] for p in parts] == sorted(p[0] for p in parts) and parts[-1][1] == nz
        for kind, top in (("cell", nz), ("face", nz + 1)):
            plans = [halo_plan(parts, r, kind) for r in range(world)]
            for r, (_, recvs) in enumerate(plans):
                a, b, ea, eb = parts[r]
                got = sorted(k for (_, k0, k1) in recvs for k in range(k0, k1))
                hi = min(eb + (1 if kind == "face" and eb == nz else 0), top)
                own_hi = b + (1 if kind == "face" and b == nz else 0)
                assert got == [k for k in range(ea, hi) if not (a <= k < own_hi)]
                for peer, k0, k1 in recvs:
                    assert (r, k0, k1) in plans[peer][0]
            sent = sorted((r, p, k0, k1) for r in range(world) for (p, k0, k1) in plans[r][0])
            recv = sorted((src, r, k0, k1) for r in range(world) for (src, k0, k1) in plans[r][1])
            assert sent == recv


# ------------------------------------------- slabs through plane buffers

class _OracleSlab:
    """An oracle slab seen through the plane-buffer interface of the GPU
    handles (plane_floats / read_planes_device / write_planes_device): the
    planes [k0, k1) of every field and of M, flattened in a fixed order, in
    CPU FP64 tensors."""
    plane_dtype = None
    device = "cpu"

    def __init__(self, sim):
        import torch

        self.sim = sim
        self.plane_dtype = torch.float64

    def _views(self, k0, k1):
        return [np.take(getattr(self.sim, n), range(k0, k1), axis=ax) for n, _, ax in _FIELDS]

    def plane_floats(self, k0, k1):
        return sum(v.size for v in self._views(k0, k1))

    def read_planes_device(self, k0, k1, out):
        import torch

        out.copy_(torch.from_numpy(np.concatenate([v.ravel() for v in self._views(k0, k1)])))

    def write_planes_device(self, k0, k1, data):
        flat = data.numpy()
        o = 0
        for (n, _, ax), v in zip(_FIELDS, self._views(k0, k1)):
            arr = getattr(self.sim, n)
            idx = [slice(None)] * arr.ndim
            idx[ax] = slice(k0, k1)
            arr[tuple(idx)] = flat[o:o + v.size].reshape(v.shape)
            o += v.size


def _far_magnet_workload():
    """The slab workload with its magnetic region moved away from the cuts
    (z 2-4), so that three ghost planes are enough."""
    import dataclasses

    w = _slab_workload()
    mid = w.mat_id.copy()
    mid[mid == 3] = 0
    mid[mid == 4] = 0
    mid[2:5, 4:7, 5:9] = 3
    return dataclasses.replace(w, mat_id=mid)


def _buffer_worker(rank, world, port, far, out):
    import torch.distributed as dist

    from paper_2510_22221_b300.distributed import exchange_slab_planes, slab_ghost

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _far_magnet_workload() if far else _slab_workload()
    mag = sorted({int(k) for k in np.nonzero(np.isin(w.mat_id, (3, 4)))[0]})
    parts = slab_partition(w.nz, world, slab_ghost(w.nz, world, mag, _ITER))
    a, b, ea, eb = parts[rank]
    sub = _OracleSlab(_slab_oracle(w, ea, eb))
    for _ in range(w.steps):
        sub.sim.run(1)
        exchange_slab_planes(sub, parts, rank)
    own = {}
    for n, kind, ax in _FIELDS:
        hi = b + 1 if kind == "face" and b == w.nz else b
        own[n] = np.take(getattr(sub.sim, n), range(a - ea, hi - ea), axis=ax)
    out[rank] = (own, parts[rank][2] - parts[rank][0] if rank else parts[rank][3] - parts[rank][1])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,far", [(2, False), (3, False), (2, True)])
def test_slab_plane_buffers_exchanged_point_to_point_equal_the_whole_grid(world, far):
    """The exchange driver of the GPU slabs (owned planes into buffers, one
    batch of point-to-point sends and receives, buffers into the ghost
    planes), run on CPU ranks with oracle slabs: the owned planes equal the
    undivided FP64 run to the bit, with nine ghost planes where a magnetic
    region lies at a cut and three where none is near one."""
    from tests.helpers import oracle_from_workload

    w = _far_magnet_workload() if far else _slab_workload()
    ref = oracle_from_workload(w, llg_fixed_iter=_ITER)
    ref.run(w.steps)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_buffer_worker, args=(world, _free_port(), far, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert abs(res[0][1]) == (3 if far else 9)
    for n, kind, ax in _FIELDS:
        got = np.concatenate([res[r][0][n] for r in range(world)], axis=ax)
        np.testing.assert_array_equal(got, getattr(ref, n), err_msg=n)
