"""One grid split into z-slabs on the GPU (the box decomposition of section
"Parallelization", along z): the slabs, each extended by ghost planes, run
as the instances of one batch (one launch per kernel per step for all), and
after every step their ghost planes are refreshed from the slabs that own
them with fdtd_llg_planes (exact copies of the stored state, the halo plan
of distributed.py).  The owned planes of E, H, the far-wall H and M equal
the undivided GPU run to the bit."""
import dataclasses

import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import workloads as W
from paper_2510_22221_b300.distributed import halo_plan, slab_partition, step_radius
from tests.test_multirank import _ITER, _slab_workload

pytestmark = pytest.mark.gpu


def _slab(w, ea, eb):
    """The workload restricted to cells [ea, eb) along z (sources shifted,
    the design box clipped, no probes)."""
    src = [dict(s, k=s["k"] - ea) for s in w.sources if ea <= s["k"] < eb]
    box, eps = None, None
    if w.design_box is not None:
        x0, y0, z0, dx_, dy_, dz_ = w.design_box
        lo, hi = max(z0, ea), min(z0 + dz_, eb)
        if lo < hi:
            box = (x0, y0, lo - ea, dx_, dy_, hi - lo)
            eps = w.eps_design[lo - z0:hi - z0]
    return dataclasses.replace(w, name=f"{w.name}_z{ea}_{eb}", nz=eb - ea, mat_id=w.mat_id[ea:eb].copy(),
                               sources=src, probes=[], design_box=box, eps_design=eps)


@pytest.mark.parametrize("world", [2, 3])
def test_gpu_z_slabs_equal_the_whole_grid(world):
    w = _slab_workload()
    parts = slab_partition(w.nz, world, step_radius(_ITER))
    whole = pkg.from_workload(w, llg_fixed_iter=_ITER)
    slabs = [_slab(w, ea, eb) for (_, _, ea, eb) in parts]
    batch = pkg.FdtdLlg.create_batch([(s.nx, s.ny, s.nz) for s in slabs], [(s.dx, s.dy, s.dz) for s in slabs],
                                     dt=whole.dt, llg_fixed_iter=_ITER, probe_capacity=w.steps)
    mem = [batch.batch_member(r) for r in range(world)]
    for m, s in zip(mem, slabs):
        pkg.configure(m, s)
    plans = [halo_plan(parts, r, "cell") for r in range(world)]
    for _ in range(w.steps):
        batch.step(1)
        whole.step(1)
        got = {}
        for r in range(world):
            for peer, k0, k1 in plans[r][1]:
                got[(r, k0)] = (mem[peer].read_planes(k0 - parts[peer][2], k1 - parts[peer][2]), k1)
        for (r, k0), (data, k1) in got.items():
            mem[r].write_planes(k0 - parts[r][2], k1 - parts[r][2], data)
    for r, (a, b, ea, eb) in enumerate(parts):
        np.testing.assert_array_equal(mem[r].read_planes(a - ea, b - ea), whole.read_planes(a, b), err_msg=str(r))
    np.testing.assert_array_equal(mem[-1].get_field("Hz_wall"), whole.get_field("Hz_wall"))
    assert np.abs(whole.get_field("dMx")).max() > 0 and np.abs(whole.get_field("Ez")).max() > 0
    batch.destroy()
    whole.destroy()


def test_planes_round_trip_and_errors():
    w = W.random_small(3, steps=5)
    sim = pkg.from_workload(w)
    sim.step(5)
    a = sim.read_planes(2, 6)
    assert a.size == 4 * (9 * w.nx * w.ny + w.nx + w.ny) and np.abs(a).max() > 0
    before = sim.time_state()
    sim.write_planes(2, 6, a)
    assert sim.time_state() == before                      # the time state is untouched
    np.testing.assert_array_equal(sim.read_planes(2, 6), a)
    for k0, k1 in ((-1, 2), (3, 3), (0, w.nz + 1)):
        with pytest.raises(pkg.LLGError):
            sim.read_planes(k0, k1)
    sim.destroy()


@pytest.mark.parametrize("world,far", [(2, False), (3, False), (2, True)])
def test_gpu_slab_handles_exchange_device_buffers(world, far):
    """The slabs as separate handles on one GPU whose ghost planes are
    refreshed after every step through device buffers (fdtd_llg_planes_device:
    queued copies on the handles' stream, no host round trip), with the ghost
    width that slab_ghost gives (nine planes with a magnet at a cut, three
    with none near one): the owned planes equal the undivided run to the bit."""
    from paper_2510_22221_b300.distributed import exchange_slab_planes_local, slab_ghost
    from tests.test_multirank import _far_magnet_workload

    w = _far_magnet_workload() if far else _slab_workload()
    mag = sorted({int(k) for k in np.nonzero(np.isin(w.mat_id, (3, 4)))[0]})
    ghost = slab_ghost(w.nz, world, mag, _ITER)
    assert ghost == (3 if far else 9)
    parts = slab_partition(w.nz, world, ghost)
    whole = pkg.from_workload(w, llg_fixed_iter=_ITER)
    slabs = []
    for (_, _, ea, eb) in parts:
        s = _slab(w, ea, eb)
        h = pkg.FdtdLlg.create(s.nx, s.ny, s.nz, s.dx, s.dy, s.dz, dt=whole.dt, llg_fixed_iter=_ITER,
                               probe_capacity=w.steps)
        pkg.configure(h, s)
        slabs.append(h)
    for _ in range(w.steps):
        for h in slabs:
            h.step(1)
        whole.step(1)
        exchange_slab_planes_local(slabs, parts)
    for r, (a, b, ea, eb) in enumerate(parts):
        np.testing.assert_array_equal(slabs[r].read_planes(a - ea, b - ea), whole.read_planes(a, b), err_msg=str(r))
    np.testing.assert_array_equal(slabs[-1].get_field("Hz_wall"), whole.get_field("Hz_wall"))
    for h in slabs:
        h.destroy()
