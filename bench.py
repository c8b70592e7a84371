"""Benchmark of the FDK hot path (filter + back-projection) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload fdk512] [--dtype f32|f16|bf16]

A step is one FDK reconstruction of the workload: ifdk_filter (cosine weight +
Ram-Lak Toeplitz product) then ifdk_backproject (Algorithm 4) into a zeroed
volume, inputs resident in HBM.  The metric is GUPS = Nx*Ny*Nz*Np / (T * 2^30)
(Sec. 2.3 of the paper) over the whole step.  Under torchrun each rank
reconstructs its own copy of the workload (independent problems: weak
scaling, no collective on the data path); rank 0 prints one JSON line.

--workload slab4096 (not a default line) times the streamed large-slab case:
a step back-projects the 2048 FP16 filtered views, held in pinned host memory
(only the 272 detector rows the 4096 x 4096 x 256 central slab reads), into a
zeroed slab, copying them to the device in 64-view chunks on a side stream
while the back-projection runs; the copies are inside the timed region.

--impl reference times the FP64 CPU oracle (the reference arm: there is no reference code, only the paper) on
the host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "back-projection GUPS (voxel*view/s / 2^30), whole FDK step"
UNIT = "GUPS"
FP32_OPS_PER_UPDATE = 10   # v FMA, floor, fraction, 3 lerps (sub + FMA), weighted accumulate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fdk512")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-view-pairing", action="store_true",
                    help="back-project every view singly (no half-turn view pairs)")
    ap.add_argument("--view-split", type=int, default=0,
                    help="cap on the view split of small volumes (0 automatic, 1 off)")
    ap.add_argument("--standard", action="store_true",
                    help="back-project the filtered views as filtered (ifdk_backproject), not packed")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload_desc(w):
    g = w.geom
    return (f"{w.name}: {g.nu}x{g.nv}x{g.np} -> {g.nx}x{g.ny}x{g.nz}, d={g.sid:g} mm, D={g.sdd:g} mm, "
            f"voxel {g.dx:g} mm, pixel {g.du:g} mm, {w.n_ellipsoids} seeded ellipsoids"
            + (f" + {w.noise:.0%} Gaussian noise" if w.noise else ""))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_samples(out)


def parse_clock_samples(out: str) -> dict:
    """The `clocks` record from nvidia-smi CSV lines of ClockSampler.Q (no header,
    no units): median SM clock, the largest max clock, and every throttle reason
    seen active in any sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profile_record(kernel_file: str, prof: str) -> dict:
    """The committed ncu summary profiles/<prof>.json of the back-projection kernel,
    if it was taken on the current kernel source (else {})."""
    path = os.path.join(ROOT, "profiles", f"{prof}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        src = open(os.path.join(ROOT, "paper_1909_02724_gb300", "csrc", kernel_file), "rb").read()
        return rec if rec.get("source_sha1") == hashlib.sha1(src).hexdigest() else {}
    except (OSError, ValueError):
        return {}


def oracle_sample_fdk(w, E_rows_fn, n_slices: int, threads: int):
    """Oracle FDK on n_slices z-slices centred on the mid-plane: filters the
    detector rows those voxels touch and back-projects them.  Returns
    (voxels, values, seconds, updates)."""
    import oracle
    g = w.geom
    k0 = g.nz // 2 - n_slices // 2
    ks = np.arange(k0, k0 + n_slices)
    ii, jj, kk = np.meshgrid(np.arange(g.nx), np.arange(g.ny), ks, indexing="ij")
    vox = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1)
    t0 = time.perf_counter()
    need = oracle.rows_needed(g, vox)
    s_idx, r_idx = np.nonzero(need)
    E_rows = E_rows_fn(s_idx, r_idx)
    Qs = oracle.filter_rows(g, E_rows, r_idx)
    rowmap = -np.ones((g.np, g.nv), dtype=np.int64)
    rowmap[s_idx, r_idx] = np.arange(len(s_idx))
    vals = oracle.backproject_voxels(g, Qs, vox, rowmap=rowmap, threads=threads)
    dt = time.perf_counter() - t0
    return vox, vals, dt, vox.shape[0] * g.np


def run_reference(args):
    """The oracle on the host cores, each step a bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1909_02724_gb300.phantom import chord_lengths, pixel_positions, source_positions, workload
    w = workload(args.workload)
    g = w.geom
    ell = w.phantom()
    threads = oracle.default_threads()

    def rows_fn(s_idx, r_idx):   # exact FP64 line integrals of the needed rows only (no noise)
        out = np.empty((len(s_idx), g.nu))
        iu = np.arange(g.nu)
        for s in np.unique(s_idx):
            sel = np.nonzero(s_idx == s)[0]
            beta = g.angles[s]
            src = source_positions(g, [s])[0]
            pix = pixel_positions(g, beta, iu[None, :], r_idx[sel][:, None])
            out[sel] = chord_lengths(ell, src, pix)
        return out

    n_slices = 2
    times, upd = [], 0
    for step in range(args.warmup + args.steps):
        _, _, dt, u = oracle_sample_fdk(w, rows_fn, n_slices, threads)
        if step >= args.warmup:
            times.append(dt)
            upd = u
    value = upd / (float(np.mean(times)) * 2 ** 30)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(w), "storage": "f64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n_slices} mid-plane z-slices ({upd} voxel-view updates) per step, "
                                       "incl. generating and filtering the detector rows they touch"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.api import fdk_host, fdk_host_pipeline
    from paper_1909_02724_gb300.build import build
    from paper_1909_02724_gb300.geometry import gups
    from paper_1909_02724_gb300.parallel import max_over_ranks
    from paper_1909_02724_gb300.phantom import workload, workload_projections_gpu

    # one rank compiles whatever is stale, the others wait and load its output
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    build()
    w = workload(args.workload)
    g = w.geom
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    plan = B.Plan(g)
    plan.set_view_pairing(not args.no_view_pairing)
    plan.set_view_split(args.view_split)
    packed = not args.standard and plan.has_packed(tdt)
    splits = plan.view_split(tdt) if packed else 1
    info = plan.packed_info(tdt) if packed else plan.info(tdt)
    dev = torch.device("cuda", local)
    E = workload_projections_gpu(w)
    Q = torch.empty((g.np, g.nv, g.nu), dtype=tdt, device=dev)
    Qp = torch.empty(plan.packed_shape(tdt), dtype=tdt, device=dev) if packed else None
    vol = torch.empty((g.nx, g.ny, g.nz), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev_bp=None):
        vol.zero_()
        plan.filter(E, Q)
        if packed:
            plan.pack(Q, Qp)
        if ev_bp is not None:
            ev_bp[0].record(stream)
        if packed:
            plan.backproject_packed(Qp, vol)
        else:
            plan.backproject(Q, vol)
        if ev_bp is not None:
            ev_bp[1].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    bp_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.steps):
        step(bp_events[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    bp_ms = float(np.mean([a.elapsed_time(b) for a, b in bp_events]))
    ms = max_over_ranks(ms, device=dev)
    ms_per_step = ms / args.steps
    value = world * g.updates * args.steps / (ms * 1e-3) / 2 ** 30

    # output stage (Algorithm 4's reshape: k-fastest volume -> i-fastest slices), not part
    # of the step; timed alone on the step's volume (512 MiB in, 512 MiB out: above L2)
    slices = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.slices(vol, slices)
    sl_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in sl_events:
        a.record(stream)
        plan.slices(vol, slices)
        b.record(stream)
    torch.cuda.synchronize()
    sl_ms = float(np.mean([a.elapsed_time(b) for a, b in sl_events]))
    sl_bytes = 8 * g.nx * g.ny * g.nz
    del slices

    # launches of our kernels per step: tensor-core filter (a split pre-pass and a GEMM per
    # chunk of rows that fits the preferred workspace), the pack (packed path) and one
    # back-projection (the full scan pairs up, or is one range of single views), plus the
    # sum of the partial volumes when a small volume splits its views
    rows = g.np * g.nv
    terms = 3 if tdt == torch.float32 else 2
    ws_min, ws_pref = B.ifdk_filter_workspace_size(plan.handle, terms)
    cap = ws_pref // (ws_min // 128)
    launches = (2 * -(-rows // cap) + (2 if packed else 1) + (1 if splits > 1 else 0)) * args.steps

    # end to end through host buffers (pinned), copies inside the timed region: every
    # step copies its projections in and its volume out; the copies of one step
    # overlap the computation of its neighbours (two device buffers of each)
    e2e = None
    if not args.no_e2e:
        E_host = torch.empty(E.shape, dtype=torch.float32, pin_memory=True)
        E_host.copy_(E)
        vol_host = torch.empty(vol.shape, dtype=torch.float32, pin_memory=True)
        E2 = [E, torch.empty_like(E)]
        vol2 = [vol, torch.empty_like(vol)]
        e_steps = max(3, min(args.steps, 20))
        fdk_host(plan, E_host, vol_host, E, Q, vol, Qp_dev=Qp)                  # one serial step (warm)
        fdk_host_pipeline(plan, E_host, vol_host, E2, Q, vol2, Qp_dev=Qp, n_steps=2)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a = time.perf_counter()
        fdk_host_pipeline(plan, E_host, vol_host, E2, Q, vol2, Qp_dev=Qp, n_steps=e_steps)
        e_s = max_over_ranks(time.perf_counter() - a, device=dev)
        e2e = {"value": world * g.updates * e_steps / e_s / 2 ** 30, "unit": UNIT,
               "h2d_bytes_per_step": E.numel() * 4, "d2h_bytes_per_step": vol.numel() * 4,
               "steps": e_steps, "overlap": "copies of step k overlap compute of steps k-1, k+1"}
        del E2[1], vol2[1]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_gups = n_sm * 128 * f_max / FP32_OPS_PER_UPDATE / 2 ** 30
    achieved = gups(g, bp_ms * 1e-3)
    if packed:
        kname, kfile = "bp_packed_kernel", "ifdk_bp_packed.cu"
        prof = f"bp_packed_{args.workload}_{args.dtype}" + ("" if info["path"] == 2 else "_single")
    else:
        kname = "bp_pairs_fold_kernel" if info["path"] == 1 else "bp_general_kernel"
        kfile, prof = "ifdk_bp.cu", f"bp_fold_{args.workload}"
    rec = profile_record(kfile, prof)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_gups, "unit": UNIT,
                "frac": achieved / peak_gups, "traffic": rec.get("dram_bytes_per_launch"),
                "ncu": rec.get("ncu"),   # the binding counters of that capture (profiles/<prof>.md)
                "kernel": kname,
                "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz (MEASURED_PEAKS sm_max_mhz) "
                              f"/ {FP32_OPS_PER_UPDATE} FP32 ops per update",
                "frac_at_sampled_clock": (achieved / (peak_gups * ck["sm_mhz"] * 1e6 / f_max)
                                          if ck.get("sm_mhz") else None),
                "bp_ms_per_launch": bp_ms}

    hbm = float(peaks.get("hbm_gbs", 6800.0))
    output_stage = {"kernel": "slices_kernel<float>", "ms_per_launch": sl_ms,
                    "bytes_per_launch": sl_bytes, "achieved": sl_bytes / (sl_ms * 1e-3) / 1e9,
                    "peak": hbm, "unit": "GB/s", "bound": "hbm",
                    "frac": sl_bytes / (sl_ms * 1e-3) / 1e9 / hbm,
                    "peak_basis": "MEASURED_PEAKS hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(w, E, vol, plan, Q)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_desc(w), "storage": args.dtype, "accumulate": "f32",
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (E, Q, vol each >= 256 MiB)",
                       "bp_path": ("packed views" + (", half-turn view pairs" if info["path"] == 2 else ""))
                       if packed else "filtered views as stored",
                       "bp_launch": info, "view_split": splits},
            "e2e": e2e, "gpu_launches": launches, "clocks": ck, "roofline": roofline,
            "cpu_baseline": cpu, "output_stage": output_stage,
            "value_1e9": value * 2 ** 30 / 1e9}   # the same throughput in 10^9 updates/s
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_slab(args):
    """The streamed large-slab workload on one GPU (see the module docstring)."""
    import torch
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.build import build
    from paper_1909_02724_gb300.geometry import gups
    from paper_1909_02724_gb300.phantom import line_integrals_gpu, workload

    rank, world, local = dist_env()
    if rank != 0:
        return                      # one GPU: the other ranks have nothing to do
    torch.cuda.set_device(local)
    build()
    w = workload(args.workload)
    r0, n = B.ifdk_query_rows(w.geom)
    g = w.geom.crop_rows(r0, n)     # the detector rows the slab reads
    plan = B.Plan(g)
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    E = line_integrals_gpu(w.phantom(), g)
    Qd = plan.filter(E, dtype=tdt)
    del E
    Qh = torch.empty(Qd.shape, dtype=tdt, pin_memory=True)
    Qh.copy_(Qd)
    plan.set_view_pairing(not args.no_view_pairing)
    chunk = 64
    packed = not args.standard and plan.has_packed(tdt)
    staging = torch.empty(plan.staging_elems(tdt, chunk, packed), dtype=tdt, device="cuda")
    vol = torch.empty((g.nx, g.ny, g.nz), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        vol.zero_()
        plan.backproject_host(Qh, vol, staging, chunk_views=chunk, packed=packed)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    value = g.updates / (ms * 1e-3) / 2 ** 30
    # the same back-projection from device-resident views (kernel only)
    Qpd = plan.pack(Qd) if packed else None
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms = []
    for _ in range(3):
        vol.zero_()
        k0.record(stream)
        if packed:
            plan.backproject_packed(Qpd, vol)
        else:
            plan.backproject(Qd, vol)
        k1.record(stream)
        torch.cuda.synchronize()
        kms.append(k0.elapsed_time(k1))
    del Qpd
    bp_ms = float(np.median(kms))
    # end to end: the streamed step plus reading the slab back to pinned host memory
    vol_host = torch.empty(vol.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    a = time.perf_counter()
    step()
    vol_host.copy_(vol, non_blocking=True)
    torch.cuda.synchronize()
    e_s = time.perf_counter() - a
    props = torch.cuda.get_device_properties(torch.device("cuda", local))
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_gups = props.multi_processor_count * 128 * f_max / FP32_OPS_PER_UPDATE / 2 ** 30
    achieved = gups(g, bp_ms * 1e-3)
    es = Qh.element_size()
    line = {"metric": METRIC.replace("whole FDK step", "back-projection streamed from pinned host views"),
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_desc(w) + f"; detector rows {r0}..{r0 + n - 1} of {w.geom.nv}",
                       "storage": args.dtype, "accumulate": "f32", "chunk_views": chunk,
                       "h2d_bytes_per_step": Qh.numel() * es, "l2": "inputs larger than L2",
                       "bp_path": ("views packed per chunk on the device" +
                                   (", half-turn view pairs" if plan.packed_info(tdt)["path"] == 2 else ""))
                       if packed else "filtered views as stored",
                       "bp_launch": plan.packed_info(tdt) if packed else plan.info(tdt)},
            "kernel_only": {"value": achieved, "unit": UNIT, "bp_ms": bp_ms},
            "e2e": {"value": g.updates / e_s / 2 ** 30, "unit": UNIT, "h2d_bytes_per_step": Qh.numel() * es,
                    "d2h_bytes_per_step": vol.numel() * 4},
            "gpu_launches": (2 if packed else 1) * -(-g.np // chunk) * args.steps, "clocks": ck,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gups, "unit": UNIT,
                         "frac": achieved / peak_gups, "traffic": None,
                         "kernel": "bp_packed_kernel" if packed else "bp_pairs_fold_kernel"},
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, E, vol_gpu_unused, plan, Q):
    """The oracle on the host cores on a bounded sample (mid-plane slab), plus the
    accuracy of this run's GPU volume on the same voxels."""
    import torch
    import oracle
    g = w.geom
    threads = oracle.default_threads()
    E_cpu = None

    def rows_fn(s_idx, r_idx):
        nonlocal E_cpu
        return E[torch.from_numpy(s_idx).to(E.device), torch.from_numpy(r_idx).to(E.device)].double().cpu().numpy()

    # calibrate on one slice, then size the sample to about 12 s
    _, _, dt1, _ = oracle_sample_fdk(w, rows_fn, 1, threads)
    n_slices = int(max(1, min(g.nz, round(12.0 / max(dt1, 1e-3)))))
    vox, vals, dt, upd = oracle_sample_fdk(w, rows_fn, n_slices, threads)
    # GPU FDK of the same inputs (FP32 storage, as timed), compared on the sample
    vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=E.device)
    Qf = torch.empty(E.shape, dtype=torch.float32, device=E.device)
    plan.filter(E, Qf)
    plan.backproject(Qf, vol)
    v = vol.cpu().numpy()[vox[:, 0], vox[:, 1], vox[:, 2]].astype(np.float64)
    rel = float(np.linalg.norm(v - vals) / np.linalg.norm(vals))
    mx = float(np.max(np.abs(v - vals)) / np.max(np.abs(vals)))
    return {"value": upd / dt / 2 ** 30, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_slices} mid-plane z-slices of {g.nx}x{g.ny} ({upd} voxel-view updates), "
                      "incl. filtering the detector rows they touch (FP64 C, pthreads)",
            "seconds": dt, "gpu_f32_vs_oracle_on_sample": {"rel_l2": rel, "max_abs_over_max": mx}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "slab4096":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
