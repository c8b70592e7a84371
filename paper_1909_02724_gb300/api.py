"""User-level calls on top of the C-ABI binding.

``fdk`` reconstructs on the device; ``fdk_host`` is the same call on host
buffers: it copies the projections in (from pinned memory), filters,
back-projects and copies the volume out, all on one stream.  When the plan
has packed views (centred volume, 2 v_c integral) and a packed buffer is
given or allowed, the filtered views are packed (ifdk_pack_views) and
back-projected by the packed kernel; otherwise by ifdk_backproject.  Every
step runs in the CUDA library; this module only sequences the calls.
"""
from __future__ import annotations

import torch

from .binding import Plan


def fdk(plan: Plan, E: torch.Tensor, vol: torch.Tensor | None = None, Q: torch.Tensor | None = None,
        dtype=torch.float32, split_terms: int | None = None, Qp: torch.Tensor | None = None,
        packed: bool = True, stream=None) -> torch.Tensor:
    """FDK on the device: vol (+)= backproject(filter(E)).  E: float32 CUDA [np][nv][nu].

    Q (optional): workspace for the filtered views, of the storage dtype.
    Qp (optional): workspace for the packed views (Plan.packed_shape).
    packed: use the packed path when the plan has one.
    vol (optional): the volume to accumulate into; a zeroed one is made if absent."""
    g = plan.geom
    if Q is None:
        Q = torch.empty((g.np, g.nv, g.nu), dtype=dtype, device=E.device)
    plan.filter(E, Q, split_terms=split_terms, stream=stream)
    if vol is None:
        vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=E.device)
    if packed and plan.has_packed(Q.dtype):
        Qp = plan.pack(Q, Qp, stream=stream)
        return plan.backproject_packed(Qp, vol, stream=stream)
    return plan.backproject(Q, vol, stream=stream)


def fdk_host(plan: Plan, E_host: torch.Tensor, vol_host: torch.Tensor, E_dev: torch.Tensor,
             Q_dev: torch.Tensor, vol_dev: torch.Tensor, split_terms: int | None = None,
             Qp_dev: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """FDK from host projections to a host volume through caller-owned device buffers
    (Qp_dev: packed views, used when given).

    E_host / vol_host should be pinned for asynchronous copies; the call returns
    once vol_host holds the result."""
    s = torch.cuda.current_stream() if stream is None else stream
    with torch.cuda.stream(s):
        E_dev.copy_(E_host, non_blocking=True)
        vol_dev.zero_()
        plan.filter(E_dev, Q_dev, split_terms=split_terms, stream=s)
        if Qp_dev is not None:
            plan.pack(Q_dev, Qp_dev, stream=s)
            plan.backproject_packed(Qp_dev, vol_dev, stream=s)
        else:
            plan.backproject(Q_dev, vol_dev, stream=s)
        vol_host.copy_(vol_dev, non_blocking=True)
    s.synchronize()
    return vol_host
