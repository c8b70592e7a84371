"""Work decomposition over ranks (Sec. 4 of the iFDK paper), host side.

The paper splits an FDK reconstruction over an R x C grid of workers:
columns split the views (each column back-projects Np / C views into a
partial volume, and the partial volumes are summed, the paper's MPI_Reduce),
rows split the volume into z-slabs (each row back-projects every view into
its own slab; slabs and their z-mirrors are independent, no collective).
The paper's rows take sub-volumes in mirror pairs (a slab and its mirror
slab), which keep Theorem 1 and so the packed back-projector: pair_shard,
gather_pair_slabs.  slab_shard cuts plain contiguous slabs (off-centre plans).
This module computes those partitions and the two collectives they need,
through torch.distributed (NCCL for GPU tensors, gloo for CPU tensors).  The
back-projection itself stays in the CUDA library: a view shard is a call with
[view_begin, view_begin + view_count), a slab shard a plan of the slab's
geometry (vol_off_z = the slab centre's world Z; the general kernel serves
off-centre slabs, a centred slab keeps the mirror paths).

bench.py runs independent problems per rank (weak scaling, no data-path
collective) and uses max_over_ranks for its timing.
"""
from __future__ import annotations

from dataclasses import dataclass

from .geometry import Geometry


def split_range(n: int, parts: int, index: int) -> tuple[int, int]:
    """[begin, end) of part `index` of `parts` near-equal contiguous parts of
    range(n) (the first n % parts parts are one longer)."""
    if parts < 1 or not 0 <= index < parts or n < 0:
        raise ValueError("bad partition")
    q, r = divmod(n, parts)
    begin = index * q + min(index, r)
    return begin, begin + q + (1 if index < r else 0)


def view_shard(geom: Geometry, world: int, rank: int) -> tuple[int, int]:
    """The views a column worker back-projects: (view_begin, view_count)."""
    b, e = split_range(geom.np, world, rank)
    return b, e - b


@dataclass
class Slab:
    k_begin: int      # first voxel index k of the slab in the whole volume
    k_count: int
    geom: Geometry    # the slab as a volume of its own (centre shifted along Z)


def slab_shard(geom: Geometry, world: int, rank: int) -> Slab:
    """The z-slab a row worker reconstructs.  Voxel k of the slab is voxel
    k_begin + k of the whole volume: its world Z, -dz (k_begin + k - (nz-1)/2)
    + vol_off_z (the index flip of M0 in Eq. 2), is the slab's own
    -dz (k - (k_count-1)/2) + slab_off_z with the offset below."""
    b, e = split_range(geom.nz, world, rank)
    n = e - b
    off = geom.vol_off_z - geom.dz * (b + (n - 1) / 2.0 - (geom.nz - 1) / 2.0)
    return Slab(b, n, geom.with_(nz=n, vol_off_z=off))


def max_over_ranks(x: float, device=None) -> float:
    """max of a host scalar over the ranks of the default process group
    (the scalar itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_volume(vol, dst: int = 0):
    """Sums the partial volumes of a view split onto rank dst (the paper's
    MPI_Reduce of the column workers' sub-volumes), in place on dst."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.reduce(vol, dst=dst, op=dist.ReduceOp.SUM)
    return vol


def gather_slabs(slab_vol, full_vol=None, dst: int = 0, nz: int | None = None):
    """Collects the slabs of a row split on rank dst into full_vol [nx][ny][nz]
    (k fastest; made here when None), slab r holding k in split_range(nz, world, r).
    Returns full_vol on dst (on the other ranks whatever they passed); nz is needed when no
    rank passes full_vol."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        if full_vol is not None:
            full_vol.copy_(slab_vol)
            return full_vol
        return slab_vol
    world, rank = dist.get_world_size(), dist.get_rank()
    nz = full_vol.shape[2] if full_vol is not None else nz
    if nz is None:
        raise ValueError("gather_slabs needs full_vol or nz")
    if rank == dst and full_vol is None:
        full_vol = torch.empty(slab_vol.shape[:2] + (nz,), dtype=slab_vol.dtype, device=slab_vol.device)
    # gather wants equal shapes: every slab travels padded to the longest one
    kmax = split_range(nz, world, 0)[1]
    send = torch.zeros(slab_vol.shape[:2] + (kmax,), dtype=slab_vol.dtype, device=slab_vol.device)
    send[:, :, :slab_vol.shape[2]] = slab_vol
    if rank == dst:
        parts = [torch.empty_like(send) for _ in range(world)]
        dist.gather(send, gather_list=parts, dst=dst)
        for r in range(world):
            b, e = split_range(nz, world, r)
            full_vol[:, :, b:e] = parts[r][:, :, :e - b]
    else:
        dist.gather(send, dst=dst)
    return full_vol


def pair_shard(geom: Geometry, world: int, rank: int) -> tuple[int, int]:
    """The mirror pairs a row worker reconstructs (the paper's sub-volumes: a z-slab
    together with its mirror slab): (pair_begin, pair_count) over the (nz + 1) // 2
    pairs (k, nz - 1 - k), for Plan.backproject_packed_pairs."""
    b, e = split_range((geom.nz + 1) // 2, world, rank)
    return b, e - b


def place_pair_slab(full_vol, part, nz: int, pair_begin: int, pair_count: int):
    """Writes a pair-range volume part [nx][ny][nz_out] (direct slab, then its
    mirror) into its voxels of full_vol [nx][ny][nz]."""
    if pair_count == 0:
        return full_vol
    nz_out = part.shape[2]
    full_vol[:, :, pair_begin:pair_begin + pair_count] = part[:, :, :pair_count]
    full_vol[:, :, nz - pair_begin - pair_count:nz - pair_begin] = part[:, :, nz_out - pair_count:]
    return full_vol


def gather_pair_slabs(part, full_vol, nz: int, dst: int = 0):
    """Collects the pair-range volumes of a pair split (pair_shard) on rank dst
    into full_vol [nx][ny][nz] (made here when None); padded to equal shape for
    the gather.  Returns full_vol on dst."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        # one process holds every pair: the part is the whole volume's pair layout
        if part.shape[2] != nz:
            raise ValueError(f"a single process's pair part must hold all {nz} slices, not {part.shape[2]}")
        if full_vol is None:
            full_vol = torch.empty(part.shape[:2] + (nz,), dtype=part.dtype, device=part.device)
        return place_pair_slab(full_vol, part, nz, 0, (nz + 1) // 2)
    world, rank = dist.get_world_size(), dist.get_rank()
    npairs = (nz + 1) // 2
    kmax = 2 * split_range(npairs, world, 0)[1]
    send = torch.zeros(part.shape[:2] + (kmax,), dtype=part.dtype, device=part.device)
    send[:, :, :part.shape[2]] = part
    if rank == dst:
        if full_vol is None:
            full_vol = torch.empty(part.shape[:2] + (nz,), dtype=part.dtype, device=part.device)
        parts = [torch.empty_like(send) for _ in range(world)]
        dist.gather(send, gather_list=parts, dst=dst)
        for r in range(world):
            b, e = split_range(npairs, world, r)
            depth = 2 * (e - b) - (1 if nz % 2 and e == npairs and e > b else 0)
            place_pair_slab(full_vol, parts[r][:, :, :depth], nz, b, e - b)
    else:
        dist.gather(send, dst=dst)
    return full_vol
