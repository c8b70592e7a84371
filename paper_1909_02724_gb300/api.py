"""User-level calls on top of the C-ABI binding.

``fdk`` reconstructs on the device; ``fdk_host`` is the same call on host
buffers: it copies the projections in (from pinned memory), filters,
back-projects and copies the volume out, all on one stream.  ``BatchFdk``
reconstructs in batches of half-turn view pairs and ``batch_host_pipeline``
streams those batches from host memory.  ``IterativeSolver`` runs SART or MLEM
on the back-projection and its adjoint.  When the plan
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


def fdk_host_pipeline(plan: Plan, E_host: torch.Tensor, vol_host: torch.Tensor, E_dev: list, Q_dev: torch.Tensor,
                      vol_dev: list, Qp_dev: torch.Tensor | None = None, n_steps: int = 1,
                      split_terms: int | None = None) -> torch.Tensor:
    """n_steps FDK reconstructions from host projections to a host volume with the
    copies of one step overlapping the computation of its neighbours.

    Every step copies E_host in (pinned) and its volume out to vol_host; E_dev
    and vol_dev are two device buffers each (double buffering), Q_dev / Qp_dev
    one.  Streams: host-to-device copies, computation (filter, pack,
    back-projection) and device-to-host copies, ordered by events so that a
    buffer is refilled only after the step that used it has finished with it.
    Returns once the last volume is in vol_host."""
    dev = E_dev[0].device
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    s_c = torch.cuda.current_stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    filtered = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    drained = [torch.cuda.Event() for _ in range(2)]
    for k in range(n_steps):
        b = k & 1
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(filtered[b])               # step k-2's filter has read E_dev[b]
            E_dev[b].copy_(E_host, non_blocking=True)
            copied[b].record(s_in)
        s_c.wait_event(copied[b])
        if k >= 2:
            s_c.wait_event(drained[b])                     # step k-2's volume has left vol_dev[b]
        vol_dev[b].zero_()
        plan.filter(E_dev[b], Q_dev, split_terms=split_terms, stream=s_c)
        filtered[b].record(s_c)
        if Qp_dev is not None:
            plan.pack(Q_dev, Qp_dev, stream=s_c)
            plan.backproject_packed(Qp_dev, vol_dev[b], stream=s_c)
        else:
            plan.backproject(Q_dev, vol_dev[b], stream=s_c)
        computed[b].record(s_c)
        with torch.cuda.stream(s_out):
            s_out.wait_event(computed[b])
            vol_host.copy_(vol_dev[b], non_blocking=True)
            drained[b].record(s_out)
    s_out.synchronize()
    s_c.synchronize()
    return vol_host


class BatchFdk:
    """FDK of a scan in batches of half-turn view pairs (group = 2) or
    quarter-turn view quads (group = 4), the way the paper's pipeline (Sec. 4)
    filters and back-projects projections in batches as they arrive: batch b
    holds views [b n, b n + n) and the same range shifted by np / group, ...,
    (group - 1) np / group, n = np / (group batches) (the last batch takes the
    remainder).  One batch is ifdk_filter_views on each part, ifdk_pack_views
    on the group n filtered views and ifdk_backproject_packed_batch (pairs) or
    ifdk_backproject_packed_quads (quads; the plan's view pairing mode decides
    whether one quad launch or pair launches serve them) into the accumulating
    volume (or, without packed views, ifdk_backproject_views on each part).
    The batch buffers (filtered and packed views of one batch) are made here,
    once."""

    def __init__(self, plan: Plan, batches: int, dtype=torch.float32, split_terms: int | None = None,
                 device=None, packed: bool = True, group: int = 2):
        g = plan.geom
        if group not in (2, 4) or g.np % group != 0 or not 1 <= batches <= g.np // group:
            raise ValueError("batches of view groups need group 2 or 4 dividing np and 1 <= batches <= np / group")
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.plan, self.batches, self.dtype, self.split_terms = plan, batches, dtype, split_terms
        self.group = group
        self.part = g.np // group                     # view offset between the parts of a batch
        self.half = self.part                         # (the name used by pairs)
        self.n = -(-self.part // batches)
        self.packed = packed and plan.has_packed(dtype)
        self.Q = torch.empty((group * self.n, g.nv, g.nu), dtype=dtype, device=dev)
        self.Qp = (torch.empty((group * self.n,) + plan.packed_shape(dtype)[1:], dtype=dtype, device=dev)
                   if self.packed else None)

    def views(self, b: int) -> tuple[int, int]:
        """(first view, view count) of the first part of batch b; the other parts are
        the same range shifted by k np / group."""
        s0 = b * self.n
        return s0, max(0, min(self.n, self.part - s0))

    def step(self, E: torch.Tensor, vol: torch.Tensor, b: int, stream=None, ev_bp=None, ev_filter=None) -> None:
        """Batch b of the scan E (float32 CUDA [np][nv][nu], or a buffer holding just this
        batch: its group parts of n views each, n = views(b)[1]) added into vol.  ev_bp,
        ev_filter: optional (start, end) CUDA events recorded around the back-projection
        launch and around the filter calls."""
        g = self.plan.geom
        s0, n = self.views(b)
        if n == 0:
            return
        K = self.group
        s = torch.cuda.current_stream() if stream is None else stream
        if ev_filter is not None:
            ev_filter[0].record(s)
        for k in range(K):
            v0 = s0 + k * self.part
            Ek = E[v0:v0 + n] if E.shape[0] == g.np else E[k * n:(k + 1) * n]
            self.plan.filter_views(Ek, self.Q[k * n:(k + 1) * n], view_begin=v0, split_terms=self.split_terms,
                                   stream=stream)
        if ev_filter is not None:
            ev_filter[1].record(s)
        if self.packed:
            Qpb = self.Qp[:K * n]
            self.plan.pack(self.Q[:K * n], Qpb, stream=stream)
            if ev_bp is not None:
                ev_bp[0].record(s)
            if K == 2:
                self.plan.backproject_packed_batch(Qpb, s0, n, vol, stream=stream)
            else:
                self.plan.backproject_packed_quads(Qpb, s0, n, vol, stream=stream)
        else:
            if ev_bp is not None:
                ev_bp[0].record(s)
            for k in range(K):
                self.plan.backproject_views(self.Q[k * n:(k + 1) * n], vol, view_begin=s0 + k * self.part,
                                            stream=stream)
        if ev_bp is not None:
            ev_bp[1].record(s)

    def reconstruct(self, E: torch.Tensor, vol: torch.Tensor, stream=None) -> torch.Tensor:
        """vol (+)= FDK of the whole scan E, batch by batch."""
        for b in range(self.batches):
            self.step(E, vol, b, stream=stream)
        return vol


def batch_host_pipeline(bf: BatchFdk, E_host: torch.Tensor, vol_host: torch.Tensor, E_dev: list, vol_dev: list,
                        n_steps: int) -> torch.Tensor:
    """n_steps batches (cycling over the scan's batches; every `batches` steps one
    reconstruction) from host projections E_host (pinned float32 [np][nv][nu]) to a
    host volume vol_host: each step copies its batch's views in (E_dev: two device
    buffers of [2 n][nv][nu], double-buffered), and each finished reconstruction
    copies its volume out (vol_dev: two device volumes).  Three streams (in,
    compute, out) ordered by events, so the copies of one step overlap the
    computation of its neighbours.  Returns once the last volume that finished
    is in vol_host (a reconstruction left unfinished stays on the device)."""
    g = bf.plan.geom
    dev = E_dev[0].device
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    s_c = torch.cuda.current_stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    drained = [torch.cuda.Event() for _ in range(2)]
    n_rec = [0, 0]
    for k in range(n_steps):
        e, b = k & 1, k % bf.batches
        r = (k // bf.batches) & 1                          # volume buffer of this reconstruction
        s0, n = bf.views(b)
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(used[e])                   # step k-2's filters have read E_dev[e]
            for q in range(bf.group):
                v0 = s0 + q * bf.part
                E_dev[e][q * n:(q + 1) * n].copy_(E_host[v0:v0 + n], non_blocking=True)
            copied[e].record(s_in)
        s_c.wait_event(copied[e])
        if b == 0:
            if n_rec[r] > 0:
                s_c.wait_event(drained[r])                 # the volume two reconstructions back has left
            vol_dev[r].zero_()
        bf.step(E_dev[e], vol_dev[r], b, stream=s_c)
        used[e].record(s_c)
        if b == bf.batches - 1:
            done[r].record(s_c)
            n_rec[r] += 1
            with torch.cuda.stream(s_out):
                s_out.wait_event(done[r])
                vol_host.copy_(vol_dev[r], non_blocking=True)
                drained[r].record(s_out)
    s_out.synchronize()
    s_c.synchronize()
    return vol_host


def half_turn_subsets(n_views: int, subsets: int) -> list:
    """Ordered subsets of the views for the iterative solvers, each a list of
    (view_begin, view_count) ranges: with an even view count, subset b is the
    block of half-turn pairs [b n, b n + n) and [np/2 + b n, np/2 + b n + n),
    n = ceil(np / (2 subsets)) (so that the packed batch back-projection serves
    it); with an odd count, contiguous blocks of ceil(np / subsets) views."""
    if subsets < 1:
        raise ValueError("subsets must be positive")
    if n_views % 2 == 0:
        h = n_views // 2
        n = -(-h // subsets)
        return [[(b * n, min(n, h - b * n)), (h + b * n, min(n, h - b * n))] for b in range(subsets) if b * n < h]
    m = -(-n_views // subsets)
    return [[(b * m, min(m, n_views - b * m))] for b in range(subsets) if b * m < n_views]


class IterativeSolver:
    """SART or MLEM over ordered view subsets on the GPU, the iterative methods
    the paper names as users of its back-projector (Sec. 1, Sec. 6): A is
    ifdk_project, A^T the back-projection (the packed batch kernel for
    half-turn pair subsets, ifdk_backproject_views otherwise), and the update
    steps are ifdk_iter_ratio / ifdk_iter_update:
        SART:  x <- x + lam A_S^T((p - A x) / R) / C_S     (R = A 1, C_S = A_S^T 1)
        MLEM:  x <- x A_S^T(p / A x) / C_S
    R and the C_S are computed once, here.  Buffers: the forward projection
    (all views, kept zeroed between uses by ifdk_iter_ratio), one subset of
    ratios (and its packed views), the back-projected ratios (kept zeroed by
    ifdk_iter_update), and one C_S volume per subset."""

    def __init__(self, plan: Plan, method: str = "sart", subsets: int = 1, lam: float = 1.0, nonneg: bool = False,
                 device=None, packed: bool = True):
        from .binding import IFDK_MLEM, IFDK_SART
        g = plan.geom
        dev = torch.device("cuda") if device is None else torch.device(device)
        if method not in ("sart", "mlem"):
            raise ValueError("method must be 'sart' or 'mlem'")
        self.plan, self.lam, self.nonneg = plan, float(lam), bool(nonneg)
        self.method = IFDK_SART if method == "sart" else IFDK_MLEM
        self.sets = half_turn_subsets(g.np, subsets)
        self.packed = packed and g.np % 2 == 0 and plan.has_packed(torch.float32)
        nmax = max(sum(c for _, c in S) for S in self.sets)
        self.Ax = torch.zeros((g.np, g.nv, g.nu), dtype=torch.float32, device=dev)
        self.rb = torch.empty((nmax, g.nv, g.nu), dtype=torch.float32, device=dev)
        self.Qp = (torch.empty((nmax,) + plan.packed_shape(torch.float32)[1:], dtype=torch.float32, device=dev)
                   if self.packed else None)
        self.U = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=dev)
        self.R = plan.project(torch.ones((g.nx, g.ny, g.nz), dtype=torch.float32, device=dev)) \
            if self.method == IFDK_SART else None
        self.C = []
        for S in self.sets:
            self.rb.fill_(1.0)
            c = torch.zeros_like(self.U)
            self._backproject(S, c)
            self.C.append(c)

    def _backproject(self, S, vol, stream=None) -> None:
        """vol += A_S^T of the ratios in self.rb (the subset's views in range order)."""
        if self.packed and len(S) == 2 and S[1][0] == S[0][0] + self.plan.geom.np // 2 and S[0][1] == S[1][1]:
            n = S[0][1]
            self.plan.pack(self.rb[:2 * n], self.Qp[:2 * n], stream=stream)
            self.plan.backproject_packed_batch(self.Qp[:2 * n], S[0][0], n, vol, stream=stream)
            return
        o = 0
        for b, c in S:
            self.plan.backproject_views(self.rb[o:o + c], vol, view_begin=b, stream=stream)
            o += c

    def update(self, p: torch.Tensor, x: torch.Tensor, S, C, stream=None) -> None:
        """One subset update of x in place (p: float32 CUDA [np][nv][nu] measured views)."""
        from .binding import ifdk_iter_ratio, ifdk_iter_update
        for b, c in S:
            self.plan.project(x, self.Ax, view_begin=b, view_count=c, stream=stream)
        o = 0
        for b, c in S:
            ifdk_iter_ratio(self.plan.handle, self.method, p[b:b + c], self.Ax[b:b + c],
                            None if self.R is None else self.R[b:b + c], self.rb[o:o + c], c, stream)
            o += c
        self._backproject(S, self.U, stream=stream)
        ifdk_iter_update(self.plan.handle, self.method, x, self.U, C, self.lam, self.nonneg, stream)

    def run(self, p: torch.Tensor, x: torch.Tensor, iterations: int, keep: bool = False, stream=None):
        """iterations passes over the subsets, x updated in place; keep: return a copy of
        x after every pass (else the list is empty)."""
        g = self.plan.geom
        if tuple(p.shape) != (g.np, g.nv, g.nu) or p.dtype != torch.float32 or not p.is_contiguous():
            raise ValueError(f"p must be a contiguous float32 CUDA tensor of shape {(g.np, g.nv, g.nu)}")
        self.plan._check_vol(x)
        out = []
        for _ in range(iterations):
            for S, C in zip(self.sets, self.C):
                self.update(p, x, S, C, stream=stream)
            if keep:
                out.append(x.clone())
        return out


def volume_slices_host(plan: Plan, vol: torch.Tensor, out_host: torch.Tensor, chunk_slices: int = 64,
                       staging: list | None = None) -> torch.Tensor:
    """The output stage to host memory: out_host[k][j][i] = vol[i][j][k] for every slice,
    in out_host's dtype (float32, float16 or bfloat16; pinned for the copies to overlap).

    Slices go in chunks of chunk_slices: ifdk_volume_slices writes chunk c into one of
    two device staging buffers on the current stream while a copy stream moves chunk
    c - 1 to the host, so the transpose of one chunk overlaps the copy of the last.
    staging (optional): two device buffers of at least chunk_slices * ny * nx elements."""
    g = plan.geom
    if tuple(out_host.shape) != (g.nz, g.ny, g.nx) or out_host.is_cuda or not out_host.is_contiguous():
        raise ValueError(f"out_host must be a contiguous host tensor of shape {(g.nz, g.ny, g.nx)}")
    if chunk_slices < 1:
        raise ValueError("chunk_slices must be positive")
    n = min(chunk_slices, g.nz)
    if staging is None:
        staging = [torch.empty(n * g.ny * g.nx, dtype=out_host.dtype, device=vol.device) for _ in range(2)]
    if len(staging) != 2 or any(s.numel() < n * g.ny * g.nx or s.dtype != out_host.dtype for s in staging):
        raise ValueError("staging must be two device buffers of out_host's dtype, chunk_slices slices each")
    compute = torch.cuda.current_stream(vol.device)
    copy = torch.cuda.Stream(vol.device)
    written = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    for c, k0 in enumerate(range(0, g.nz, n)):
        kc = min(n, g.nz - k0)
        b = c % 2
        buf = staging[b][:kc * g.ny * g.nx].view(kc, g.ny, g.nx)
        if c >= 2:
            compute.wait_event(copied[b])          # the copy out of this buffer is done
        plan.slices(vol, buf, k_begin=k0, k_count=kc, stream=compute)
        written[b].record(compute)
        copy.wait_event(written[b])
        with torch.cuda.stream(copy):
            out_host[k0:k0 + kc].copy_(buf, non_blocking=True)
        copied[b].record(copy)
    copy.synchronize()
    return out_host


class FdkGraph:
    """One FDK reconstruction (zero the volume, filter, pack, packed back-projection;
    the standard back-projection where the plan has no packed path) captured as a
    CUDA graph: a replay issues the whole launch sequence at once, which matters
    for small volumes whose kernels take tens of microseconds.

    The graph reads the projections from self.E and writes self.vol (buffers made
    here, fixed for the graph's life): copy new projections into self.E, then
    replay()."""

    def __init__(self, plan: Plan, dtype=torch.float32, split_terms: int | None = None, device=None):
        g = plan.geom
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.plan = plan
        self.E = torch.zeros((g.np, g.nv, g.nu), dtype=torch.float32, device=dev)
        self.Q = torch.empty((g.np, g.nv, g.nu), dtype=dtype, device=dev)
        self.Qp = torch.empty(plan.packed_shape(dtype), dtype=dtype, device=dev) if plan.has_packed(dtype) else None
        self.vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=dev)
        self.split_terms = split_terms
        # warm-up on a side stream (the filter's workspace is allocated here), then capture
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self._step()
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._step()

    def _step(self) -> None:
        self.vol.zero_()
        self.plan.filter(self.E, self.Q, split_terms=self.split_terms)
        if self.Qp is not None:
            self.plan.pack(self.Q, self.Qp)
            self.plan.backproject_packed(self.Qp, self.vol)
        else:
            self.plan.backproject(self.Q, self.vol)

    def replay(self) -> torch.Tensor:
        self.graph.replay()
        return self.vol
