"""Runs over several GPUs, one process per GPU (torchrun): the partition of a
batch's instances over the ranks (no collective on the data path: every rank
advances its own grids), the whole-job rate, and one grid split into z-slabs
(the paper's box decomposition) whose ghost planes are exchanged between
device buffers after every step.
"""
from __future__ import annotations

import heapq


def shard_instances(cells, world: int) -> list:
    """Instance indices per rank, balanced by cell count: largest instance
    first onto the least-loaded rank (ties to the lower rank), each rank's
    list in increasing index order.  Deterministic for given cells and world."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda q: (-int(cells[q]), q))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for q in order:
        load, r = heapq.heappop(heap)
        out[r].append(q)
        heapq.heappush(heap, (load + int(cells[q]), r))
    return [sorted(s) for s in out]


def job_rate(units_local: float, seconds_local: float, group=None):
    """(units of all ranks / slowest rank's time, slowest rank's time) over the
    default process group (one rank: the local values)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return units_local / seconds_local, seconds_local
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / float(t.item()), float(t.item())


# ------------------------------------------------ z-slab domain decomposition
#
# One grid over several ranks (the paper's box decomposition, section
# "Parallelization", along z): rank r owns the cells of planes [a, b) and
# steps the extended slab [a - ghost, b + ghost) clipped to the grid, whose
# cut faces it treats as walls.  One step reaches ``step_radius`` cells, so
# after a step every owned value is exact when ghost >= step_radius; the
# ghost planes are then refreshed from their owners before the next step.
# Arrays come in two plane kinds along z: "cell" arrays have nz planes
# (plane k belongs to cell k) and "face" arrays nz + 1 (plane k is the low z
# face of cell k, plane nz the top wall, which belongs to the last rank).


def step_radius(llg_iterates: int = 0) -> int:
    """An upper bound on how far along z one full step's values depend on
    others: one cell for the E push, and per H/M half-push one for the face
    update plus one per Jacobi iterate of the LLG solve (a fixed count; a
    tolerance-stopped solve couples a whole magnetic region and must not be
    cut).  Errors that enter only at the cut faces, as here, reach less far."""
    return 1 + 2 * (1 + int(llg_iterates))


def slab_partition(nz: int, world: int, ghost: int) -> list:
    """Per rank (a, b, ea, eb): owned cell planes [a, b) (as equal as the
    planes allow, the lower ranks taking the remainder) and the extended slab
    [ea, eb) = [a - ghost, b + ghost) clipped to [0, nz)."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    if ghost < 0:
        raise ValueError("ghost must be >= 0")
    base, extra = divmod(nz, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b, max(0, a - ghost), min(nz, b + ghost)))
        a = b
    return out


def plane_owner(k: int, parts: list, kind: str = "cell") -> int:
    """Rank owning plane k of an array of the given kind."""
    nz = parts[-1][1]
    if kind == "face" and k == nz:
        return len(parts) - 1
    for r, (a, b, _, _) in enumerate(parts):
        if a <= k < b:
            return r
    raise ValueError("plane outside the grid")


def halo_plan(parts: list, rank: int, kind: str = "cell") -> tuple:
    """(sends, recvs): lists of (peer, k0, k1) global plane ranges.  recvs are
    this rank's ghost planes grouped by owner; sends the owned planes that lie
    in another rank's ghost range."""
    nz = parts[-1][1]
    top = nz + 1 if kind == "face" else nz

    def ghosts(r):
        a, b, ea, eb = parts[r]
        hi = eb + 1 if kind == "face" and eb == nz else eb
        own_hi = b + 1 if kind == "face" and b == nz else b
        return [k for k in range(ea, min(hi, top)) if not (a <= k < own_hi)]

    def runs(ks, owner_of):
        out = []
        for k in ks:
            o = owner_of(k)
            if out and out[-1][0] == o and out[-1][2] == k:
                out[-1][2] = k + 1
            else:
                out.append([o, k, k + 1])
        return [tuple(x) for x in out]

    recvs = runs(ghosts(rank), lambda k: plane_owner(k, parts, kind))
    sends = []
    for r in range(len(parts)):
        if r == rank:
            continue
        mine = [k for k in ghosts(r) if plane_owner(k, parts, kind) == rank]
        sends += [(r, k0, k1) for (_, k0, k1) in runs(mine, lambda k: r)]
    return sends, recvs


def exchange_halos(arrays: list, kinds: list, parts: list, rank: int, z_axes=None, group=None) -> None:
    """Refresh this rank's ghost planes of every array from their owners
    (point-to-point over the default process group).  arrays: numpy arrays or
    CPU torch tensors in this rank's extended-slab indexing (local plane k -
    ea along axis z_axes[i], default 0); kinds: "cell" or "face" per array.
    Every rank calls it with the same arrays in the same order."""
    import numpy as np
    import torch
    import torch.distributed as dist

    ea = parts[rank][2]
    z_axes = z_axes or [0] * len(arrays)
    reqs, landing = [], []
    for q, (arr, kind, ax) in enumerate(zip(arrays, kinds, z_axes)):
        t = torch.from_numpy(arr) if isinstance(arr, np.ndarray) else arr
        sends, recvs = halo_plan(parts, rank, kind)
        for peer, k0, k1 in sends:
            buf = t.narrow(ax, k0 - ea, k1 - k0).contiguous()
            reqs.append(dist.isend(buf, dst=peer, group=group, tag=q))
            landing.append(buf)   # kept alive until the waits
        for peer, k0, k1 in recvs:
            buf = torch.empty_like(t.narrow(ax, k0 - ea, k1 - k0).contiguous())
            reqs.append(dist.irecv(buf, src=peer, group=group, tag=q))
            landing.append((t, ax, k0 - ea, k1 - k0, buf))
    for r in reqs:
        r.wait()
    for item in landing:
        if isinstance(item, tuple):
            t, ax, o, n, buf = item
            t.narrow(ax, o, n).copy_(buf)


def slab_ghost(nz: int, world: int, magnetic_planes, llg_iterates: int = 0) -> int:
    """Ghost planes per cut side for a z-slab split of nz planes over `world`
    ranks: step_radius(llg_iterates) when a magnetic cell lies within that
    distance of a cut (the Jacobi iterates of a region couple it across the
    cut), else 3: one plane for the E push and one per H half-push."""
    full = step_radius(llg_iterates)
    cuts = [b for (_, b, _, _) in slab_partition(nz, world, 0)][:-1]
    near = any(abs(k - c) <= full for k in magnetic_planes for c in cuts)
    return full if near else step_radius(0)


def _plane_buffer(slab, k0: int, k1: int):
    """A buffer for the slab's local planes [k0, k1)."""
    import torch

    return torch.empty(slab.plane_floats(k0, k1), dtype=getattr(slab, "plane_dtype", torch.float32),
                       device=getattr(slab, "device", "cuda"))


def exchange_slab_planes(slab, parts: list, rank: int, group=None) -> None:
    """Refresh this rank's ghost planes of one slab from their owners, buffer
    to buffer: the owned planes that other ranks need are copied into buffers
    on the slab's device (fdtd_llg_planes_device: queued on the handle's
    stream, no host round trip), sent and received point-to-point in one
    batch over the process group (NCCL between GPUs), and written into the
    ghost planes.  slab: an instance handle (FdtdLlg) or any object with
    plane_floats, read_planes_device and write_planes_device (and device,
    plane_dtype for its buffers).  Every rank calls it after every step."""
    import torch.distributed as dist

    sends, recvs = halo_plan(parts, rank, "cell")
    ea = parts[rank][2]
    ops, keep, landing = [], [], []
    for peer, k0, k1 in sends:
        buf = _plane_buffer(slab, k0 - ea, k1 - ea)
        slab.read_planes_device(k0 - ea, k1 - ea, buf)
        keep.append(buf)
        ops.append(dist.P2POp(dist.isend, buf, peer, group))
    for peer, k0, k1 in recvs:
        buf = _plane_buffer(slab, k0 - ea, k1 - ea)
        ops.append(dist.P2POp(dist.irecv, buf, peer, group))
        landing.append((k0, k1, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for k0, k1, buf in landing:
        slab.write_planes_device(k0 - ea, k1 - ea, buf)


def exchange_slab_planes_local(slabs: list, parts: list) -> None:
    """The same exchange for slabs that all live in this process (one GPU,
    one stream): each ghost range is copied from its owner's planes through a
    device buffer.  Only owned planes are read and only ghost planes written,
    so the order of the copies does not matter."""
    for r, slab in enumerate(slabs):
        _, recvs = halo_plan(parts, r, "cell")
        for peer, k0, k1 in recvs:
            buf = _plane_buffer(slabs[peer], k0 - parts[peer][2], k1 - parts[peer][2])
            slabs[peer].read_planes_device(k0 - parts[peer][2], k1 - parts[peer][2], buf)
            slab.write_planes_device(k0 - parts[r][2], k1 - parts[r][2], buf)
