"""Benchmark of the FDK hot path (filter + back-projection) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload fdk2048] [--dtype f32|f16|bf16] [--batches 4]

The workload is fdk2048 (2048^3 from 2048 views of 2048 x 2048), the largest
that fits one GPU.  A step is one batch of the paper's pipeline (Sec. 4:
projections are filtered and back-projected in batches): ifdk_filter_views
(cosine weight + Ram-Lak Toeplitz product on the tensor cores) on the batch's
views, ifdk_pack_views, and ifdk_backproject_packed_batch (Algorithm 4, the
batch's half-turn view pairs) into the accumulating volume; --batches steps
make one reconstruction, whose first step zeroes the volume.  Inputs are
resident in HBM.  The metric is GUPS = Nx*Ny*Nz*Np / (T * 2^30) (Sec. 2.3)
over the timed steps (each step contributes Nx*Ny*Nz times its views).

The same line carries: the back-projection kernel's roofline against the
arithmetic rates measured on this GPU (ifdk_arith_rate); the other storage
types (FP16 / BF16 filtered views, FP32 accumulation) as `storage_arms`,
each one reconstruction on the same projections, with their error against
the main arm's volume and the FP64 oracle; `e2e`, the same steps with each
batch's projections copied in from pinned host memory and each finished
volume copied out; and `cpu_baseline`, the oracle on the host cores (one
thread and every core) with the accuracy of the timed volume on a sample of
voxels.  Under torchrun each rank reconstructs its own copy of the workload
(independent problems: weak scaling, no collective on the data path); rank 0
prints one JSON line.

--workload slab4096 (not a default line) times the streamed large-slab case:
a step back-projects the 2048 FP16 filtered views, held in pinned host memory
(only the 272 detector rows the 4096 x 4096 x 256 central slab reads), into a
zeroed slab, copying them to the device in 64-view chunks on a side stream
while the back-projection runs; the copies are inside the timed region.

--impl reference times the FP64 CPU oracle (the reference arm: there is no
reference code, only the paper) on the host cores, each step a bounded
sample of the same workload.
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
    ap.add_argument("--workload", default="fdk2048")
    ap.add_argument("--batches", type=int, default=4,
                    help="batches of half-turn view pairs per reconstruction (a step is one batch)")
    ap.add_argument("--no-arms", action="store_true", help="skip the other storage types' arms")
    ap.add_argument("--solver", choices=["sart", "mlem"], default=None,
                    help="time iterations of an iterative solver instead of FDK (e.g. --workload grad256)")
    ap.add_argument("--subsets", type=int, default=10, help="ordered view subsets of --solver")
    ap.add_argument("--unrolled", type=int, default=0,
                    help="time this many unrolled gradient-descent steps (forward + backward, e.g. grad256)")
    ap.add_argument("--filter-views", type=int, default=0,
                    help="time only the filtering stage on this many views of the workload")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-view-pairing", action="store_true",
                    help="back-project every view singly (no half-turn view pairs)")
    ap.add_argument("--pairing", type=int, default=1, choices=[1, 2],
                    help="1: half-turn view pairs (the faster); 2: quarter-turn quads where they apply (FP16), "
                         "pairs elsewhere")
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


def host_memory_available() -> int:
    """MemAvailable of /proc/meminfo in bytes (a large number where it cannot be read)."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 1 << 62


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


def midplane_sample(g, n_vox: int, seed: int) -> np.ndarray:
    """A seeded random subset of n_vox voxels of the two z-slices around the mid-plane."""
    ks = np.array([max(0, g.nz // 2 - 1), g.nz // 2])
    n_all = g.nx * g.ny * len(ks)
    idx = np.random.default_rng(seed).choice(n_all, size=min(n_vox, n_all), replace=False)
    kk, rest = np.divmod(idx, g.nx * g.ny)
    ii, jj = np.divmod(rest, g.ny)
    return np.stack([ii, jj, ks[kk]], 1).astype(np.int64)


def midplane_rows(g):
    """(view, row) indices of the detector rows that any voxel of the two mid-plane
    z-slices can tap: per view, every row between the lowest and the highest row
    the slices' corner columns tap (v - v_c is (B2 k' + B3) / z with z affine in
    (i, j), so the columns' v lie between the corners'; Eq. 3, Theorems 2-3)."""
    import oracle
    ks = sorted({max(0, g.nz // 2 - 1), g.nz // 2})
    cor = np.array([[i, j, k] for i in (0, g.nx - 1) for j in (0, g.ny - 1) for k in ks], dtype=np.int64)
    need = oracle.rows_needed(g, cor)
    lo = need.argmax(1)
    hi = g.nv - 1 - need[:, ::-1].argmax(1)
    s_idx = np.concatenate([np.full(hi[s] - lo[s] + 1, s) for s in range(g.np) if need[s].any()])
    r_idx = np.concatenate([np.arange(lo[s], hi[s] + 1) for s in range(g.np) if need[s].any()])
    return s_idx.astype(np.int64), r_idx.astype(np.int64)


def accuracy_sample(g) -> np.ndarray:
    """Voxels on which the GPU volumes are compared with the oracle: the slices
    k = 0, nz/2 - 1, nz/2, nz - 1 (the ends and the middle of the mirror pairs),
    subsampled to at most 128 x 128 columns each."""
    st = max(1, g.nx // 128)
    ks = sorted({0, max(0, g.nz // 2 - 1), g.nz // 2, g.nz - 1})
    ii, jj, kk = np.meshgrid(np.arange(0, g.nx, st), np.arange(0, g.ny, st), np.asarray(ks), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1).astype(np.int64)


def oracle_rows(g, vox):
    """(view index, row index) of every detector row the voxels' taps touch."""
    import oracle
    return np.nonzero(oracle.rows_needed(g, vox))


def oracle_sample_fdk(g, E_rows, s_idx, r_idx, vox, threads: int):
    """Oracle FDK at the voxels vox from the raw rows E_rows of (view s_idx, row
    r_idx): Algorithm 1 on those rows, then Algorithm 2 at each voxel.  Returns
    (values, seconds)."""
    vals, t_f, t_b = oracle_sample_fdk_parts(g, E_rows, s_idx, r_idx, vox, threads)
    return vals, t_f + t_b


def oracle_sample_fdk_parts(g, E_rows, s_idx, r_idx, vox, threads: int):
    """oracle_sample_fdk with the two stages timed apart: (values, filter s, back-projection s)."""
    import oracle
    t0 = time.perf_counter()
    Qs = oracle.filter_rows(g, E_rows, r_idx, threads=threads)
    t1 = time.perf_counter()
    rowmap = -np.ones((g.np, g.nv), dtype=np.int64)
    rowmap[s_idx, r_idx] = np.arange(len(s_idx))
    vals = oracle.backproject_voxels(g, Qs, vox, rowmap=rowmap, threads=threads)
    return vals, t1 - t0, time.perf_counter() - t1


def run_reference(args):
    """The oracle on the host cores, each step a bounded sample of the workload:
    Algorithm 1 on the detector rows that a seeded set of mid-plane voxels
    touches, then Algorithm 2 at those voxels.  The rows' line integrals are
    generated once, before the timed steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1909_02724_gb300.phantom import line_integral_rows, workload
    w = workload(args.workload)
    g = w.geom
    threads = oracle.default_threads()
    vox_all = midplane_sample(g, 1 << 20, 7)
    s_idx, r_idx = midplane_rows(g)
    E_rows = line_integral_rows(w.phantom(), g, s_idx, r_idx)   # exact FP64 line integrals, no noise
    # size the sample for about 6 s per step from one calibration run
    n = min(len(vox_all), 16384)
    _, dt = oracle_sample_fdk(g, E_rows, s_idx, r_idx, vox_all[:n], threads)
    n = int(min(len(vox_all), max(1024, n * 6.0 / max(dt, 1e-3))))
    vox = vox_all[:n]
    times = []
    for step in range(args.warmup + args.steps):
        _, dt = oracle_sample_fdk(g, E_rows, s_idx, r_idx, vox, threads)
        if step >= args.warmup:
            times.append(dt)
    upd = n * g.np
    value = upd / (float(np.mean(times)) * 2 ** 30)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(w), "storage": "f64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} seeded voxels of the two mid-plane z-slices x {g.np} views "
                                       f"({upd} voxel-view updates) per step, incl. filtering the "
                                       f"{len(s_idx)} detector rows they touch"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rel_l2_chunked(a, b) -> float:
    """||a - b|| / ||b|| over two equal CUDA volumes, in FP64, slab by slab (no full temporary)."""
    import torch
    num = den = 0.0
    step = max(1, a.shape[0] // 64)
    for i in range(0, a.shape[0], step):
        x, y = a[i:i + step].double(), b[i:i + step].double()
        num += float(((x - y) ** 2).sum())
        den += float((y ** 2).sum())
        del x, y
    return (num / den) ** 0.5 if den > 0 else float("nan")


def sample_errors(vol, vox, ref) -> dict:
    import torch
    idx = [torch.from_numpy(vox[:, c]).to(vol.device) for c in range(3)]
    v = vol[idx[0], idx[1], idx[2]].double().cpu().numpy()
    return {"rel_l2": float(np.linalg.norm(v - ref) / np.linalg.norm(ref)),
            "max_abs_over_max": float(np.max(np.abs(v - ref)) / np.max(np.abs(ref)))}


def path_ceilings(rates: dict, n_sm: int, f_hz: float) -> dict:
    """Arithmetic ceilings of the back-projection (GUPS) from the measured per-SM rates:
    'alu10': the ten FP32 operations per update of Algorithms 3 and 4 (v, floor,
    fraction, three lerps of sub + FMA, weighted accumulate) at the best measured
    FP32 lane rate (FFMA or the packed FFMA2); per storage type, the minimal
    instruction mix that storage's path needs per update, at the measured rates
    (times of the different kinds added: they share the FMA issue):
      f32:  the ten FP32 operations;
      bf16: the ten FP32 operations, the u-lerp's two among them as FP32 FMAs
            of BF16 inputs (fma.rn.f32.bf16 rate: weights 1 - du and du on the
            stored taps, which are never widened);
      f16:  v, floor, fraction in FP32 (3), the three lerps in half2 (6 FP16
            lanes) and the accumulate as one FP16-product FP32 FMA."""
    r32 = max(rates["ffma"]["lane_ops_per_clk_sm"], rates["ffma2"]["lane_ops_per_clk_sm"])
    rh = rates["hfma2"]["lane_ops_per_clk_sm"]
    rm = rates["fma_f32_f16"]["lane_ops_per_clk_sm"]
    rb = rates["fma_f32_bf16"]["lane_ops_per_clk_sm"]
    per_clk = {"f32": 1.0 / (FP32_OPS_PER_UPDATE / r32),
               "bf16": 1.0 / ((FP32_OPS_PER_UPDATE - 2) / r32 + 2.0 / rb),
               "f16": 1.0 / (3.0 / r32 + 6.0 / rh + 1.0 / rm)}
    scale = n_sm * f_hz / 2 ** 30
    return {"alu10": r32 / FP32_OPS_PER_UPDATE * scale, "fp32_lane_ops_per_clk_sm": r32,
            **{k: v * scale for k, v in per_clk.items()},
            "updates_per_clk_sm": per_clk}


class Arm:
    """One storage type's FDK in batches: the batch runner, its volume and its
    back-projection events."""

    def __init__(self, plan, batches, tdt, dev, standard):
        from paper_1909_02724_gb300.api import BatchFdk
        g = plan.geom
        # quarter-turn quads where the plan serves this storage type with them
        group = 4 if (not standard and plan.packed_info(tdt)["path"] == 4) else 2
        self.bf = BatchFdk(plan, batches, dtype=tdt, device=dev, packed=not standard, group=group)
        self.vol = torch_empty_vol(g, dev)

    def step(self, E, k, ev=None, ev_filter=None):
        b = k % self.bf.batches
        if b == 0:
            self.vol.zero_()
        self.bf.step(E, self.vol, b, ev_bp=ev, ev_filter=ev_filter)

    def updates(self, k) -> int:
        g = self.bf.plan.geom
        return g.nx * g.ny * g.nz * self.bf.group * self.bf.views(k % self.bf.batches)[1]

    def finish(self, E, k_next):
        """Runs the batches left in the current reconstruction (untimed), so that the
        volume holds a whole reconstruction."""
        k = k_next
        while k % self.bf.batches != 0:
            self.step(E, k)
            k += 1


def torch_empty_vol(g, dev):
    import torch
    return torch.empty((g.nx, g.ny, g.nz), dtype=torch.float32, device=dev)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.api import batch_host_pipeline
    from paper_1909_02724_gb300.build import build
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
    dts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    tdt = dts[args.dtype]
    dev = torch.device("cuda", local)
    plan = B.Plan(g)
    plan.set_view_pairing(0 if args.no_view_pairing else args.pairing)
    plan.set_view_split(args.view_split)
    packed = not args.standard and plan.has_packed(tdt)
    info = plan.packed_info(tdt) if packed else plan.info(tdt)
    batches = max(1, min(args.batches, g.np // 2))
    stream = torch.cuda.current_stream()
    E = workload_projections_gpu(w)

    # measured arithmetic rates of this GPU (the roofline's denominator)
    rates = B.arith_rates(dev)

    arm = Arm(plan, batches, tdt, dev, args.standard)
    for k in range(max(3, args.warmup)):
        arm.step(E, k)
    arm.finish(E, max(3, args.warmup))
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    bp_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    f_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.steps):
        arm.step(E, k, bp_events[k], f_events[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    arm.finish(E, args.steps)            # the volume holds one whole reconstruction
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    upd_steps = sum(arm.updates(k) for k in range(args.steps))
    bp_ms = [a.elapsed_time(b) for a, b in bp_events]
    f_ms = float(np.mean([a.elapsed_time(b) for a, b in f_events]))
    bp_gups = float(np.mean([arm.updates(k) / (t * 1e-3) / 2 ** 30 for k, t in enumerate(bp_ms)]))
    ms = max_over_ranks(ms, device=dev)
    ms_per_step = ms / args.steps
    value = world * upd_steps / (ms * 1e-3) / 2 ** 30

    # launches of our kernels per step: per half of the batch the tensor-core filter (a
    # split pre-pass and a GEMM per chunk of rows that fits the preferred workspace),
    # then the pack (packed path) and the back-projection (one launch of half-turn
    # pairs, else one per half), plus the sum of the partial volumes when a small
    # volume splits its views
    terms = 3 if tdt == torch.float32 else 2
    ws_min, ws_pref = B.ifdk_filter_workspace_size(plan.handle, terms)
    cap = ws_pref // (ws_min // 128)
    half_rows = arm.bf.n * g.nv
    bp_launches = 1 if (packed and info["path"] in (2, 4)) else 2
    splits = plan.view_split(tdt) if packed else 1
    per_step = 2 * 2 * -(-half_rows // cap) + (1 if packed else 0) + bp_launches * (2 if splits > 1 else 1)
    launches = per_step * args.steps

    # output stage (Algorithm 4's reshape: k-fastest volume -> i-fastest slices), not part
    # of the step; timed alone on the step's volume
    slices = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.slices(arm.vol, slices)
    sl_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in sl_events:
        a.record(stream)
        plan.slices(arm.vol, slices)
        b.record(stream)
    torch.cuda.synchronize()
    sl_ms = float(np.mean([a.elapsed_time(b) for a, b in sl_events]))
    sl_bytes = 8 * g.nx * g.ny * g.nz
    del slices

    # end to end through host buffers (pinned), copies inside the timed region: every
    # step copies its batch of projections in; every finished reconstruction copies its
    # volume out; the copies overlap the computation of the neighbouring steps
    e2e = None
    # the host leg pins the scan and one volume per rank: skip it (and say so) where the
    # host cannot hold that for every rank of this node
    pin_bytes = (E.numel() + arm.vol.numel()) * 4
    local_world = int(os.environ.get("LOCAL_WORLD_SIZE", world))
    need = pin_bytes * local_world + (8 << 30)
    host_ok = host_memory_available() > need
    if not args.no_e2e and not host_ok:
        e2e = {"skipped": f"host memory below {need / 2**30:.0f} GiB for the pinned buffers of {local_world} ranks"}
    if not args.no_e2e and host_ok:
        E_host = torch.empty(E.shape, dtype=torch.float32, pin_memory=True)
        E_host.copy_(E)
        vol_host = torch.empty(arm.vol.shape, dtype=torch.float32, pin_memory=True)
        E_b = [torch.empty((arm.bf.group * arm.bf.n, g.nv, g.nu), dtype=torch.float32, device=dev)
               for _ in range(2)]
        vol2 = [arm.vol, torch.empty_like(arm.vol)]
        e_steps = max(batches, min(args.steps, 2 * batches))
        batch_host_pipeline(arm.bf, E_host, vol_host, E_b, vol2, batches)          # warm
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a = time.perf_counter()
        batch_host_pipeline(arm.bf, E_host, vol_host, E_b, vol2, e_steps)
        e_s = max_over_ranks(time.perf_counter() - a, device=dev)
        e_upd = sum(arm.updates(k) for k in range(e_steps))
        h2d = sum(arm.bf.group * arm.bf.views(k % batches)[1] for k in range(e_steps)) * g.nv * g.nu * 4
        d2h = (e_steps // batches) * arm.vol.numel() * 4
        e2e = {"value": world * e_upd / e_s / 2 ** 30, "unit": UNIT,
               "h2d_bytes_per_step": h2d // e_steps, "d2h_bytes_per_step": d2h // e_steps,
               "steps": e_steps,
               "overlap": "batch copies in and volume copies out overlap the computation of neighbouring steps",
               "d2h": "one volume per finished reconstruction (every %d steps), averaged per step" % batches}
        del E_b, vol2, E_host, vol_host
        arm.finish(E, 0)
        arm.vol.zero_()
        for k in range(batches):              # the timed volume again (the pipeline reused it)
            arm.step(E, k)
        torch.cuda.synchronize()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    n_sm = rates["n_sm"]
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    ceil = path_ceilings(rates, n_sm, f_max)
    nominal = n_sm * 128 * f_max / FP32_OPS_PER_UPDATE / 2 ** 30
    if packed:
        kname, kfile = "bp_packed_kernel", "ifdk_bp_packed.cu"
        prof = f"bp_packed_{args.workload}_{args.dtype}" + {2: "", 4: "_quads"}.get(info["path"], "_single")
    else:
        kname = "bp_pairs_fold_kernel" if info["path"] == 1 else "bp_general_kernel"
        kfile, prof = "ifdk_bp.cu", f"bp_fold_{args.workload}"
    rec = profile_record(kfile, prof)

    def roofline_of(gups_bp, dtype_key):
        return {"bound": "alu", "achieved": gups_bp, "peak": ceil["alu10"], "unit": UNIT,
                "frac": gups_bp / ceil["alu10"],
                "peak_basis": f"{n_sm} SMs x {ceil['fp32_lane_ops_per_clk_sm']:.1f} FP32 lane ops per SM clock "
                              f"(measured: best of FFMA / FFMA2, ifdk_arith_rate) x {f_max / 1e6:.0f} MHz "
                              f"(MEASURED_PEAKS sm_max_mhz) / {FP32_OPS_PER_UPDATE} FP32 ops per update",
                "peak_path": ceil[dtype_key], "frac_path": gups_bp / ceil[dtype_key],
                "path_basis": f"minimal instruction mix of the {dtype_key} storage path at the measured rates",
                "peak_nominal_128lane": nominal, "frac_nominal_128lane": gups_bp / nominal,
                "frac_at_sampled_clock": (gups_bp / (ceil["alu10"] * ck["sm_mhz"] * 1e6 / f_max)
                                          if ck.get("sm_mhz") else None)}

    roofline = roofline_of(bp_gups, args.dtype)
    roofline.update({"traffic": rec.get("dram_bytes_per_launch"), "ncu": rec.get("ncu"), "kernel": kname,
                     "bp_ms_per_launch": float(np.mean(bp_ms)),
                     "units_per_launch": arm.updates(0)})

    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the filtering stage of a step (split pre-pass + tensor-core Toeplitz GEMM per row chunk):
    # dense FLOPs 2 rows Nu (Nu + 1) per BF16 term product (6 products for 3 terms, 3 for 2)
    rows_step = arm.bf.group * arm.bf.n * g.nv
    products = {3: 6, 2: 3, 1: 1}[terms]
    f_flops = 2.0 * rows_step * g.nu * (g.nu + 1) * products
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    filter_stage = {"kernels": "filter_split_kernel + filter_tc_kernel per row chunk", "ms_per_step": f_ms,
                    "split_terms": terms, "term_products": products, "flops_per_step": f_flops,
                    "achieved": f_flops / (f_ms * 1e-3) / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
                    "bound": "tensor", "frac": f_flops / (f_ms * 1e-3) / 1e12 / bf16_peak,
                    "frac_split_terms_count": f_flops / products * terms / (f_ms * 1e-3) / 1e12 / bf16_peak,
                    "peak_basis": "MEASURED_PEAKS bf16_tflops (burst)" if "bf16_tflops" in peaks
                    else "fallback 1900 TFLOP/s"}
    output_stage = {"kernel": "slices_kernel<float>", "ms_per_launch": sl_ms,
                    "bytes_per_launch": sl_bytes, "achieved": sl_bytes / (sl_ms * 1e-3) / 1e9,
                    "peak": hbm, "unit": "GB/s", "bound": "hbm",
                    "frac": sl_bytes / (sl_ms * 1e-3) / 1e9 / hbm,
                    "peak_basis": "MEASURED_PEAKS hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}

    # oracle on a sample of voxels: the accuracy of every arm's volume
    acc = None
    if not args.no_cpu and world == 1:
        acc = oracle_accuracy(w, E, accuracy_sample(g))

    main_bf_group, main_bf_n = arm.bf.group, arm.bf.n
    storage_arms = {}
    if not args.no_arms and world == 1:
        others = [d for d in ("f16", "bf16", "f32") if d != args.dtype]
        vol_main = arm.vol
        main_bf = arm.bf
        del arm
        for key in others:
            main_bf.Q = main_bf.Qp = None      # the main arm's batch buffers are not needed any more
            storage_arms[key] = run_arm(plan, batches, dts[key], dev, args.standard, E, vol_main, acc,
                                        roofline_of, key)
            if packed and storage_arms[key]["bp_path"] == "half-turn view pairs":
                # DRAM bytes of one launch of this arm's kernel (committed ncu summary)
                arm_rec = profile_record(kfile, f"bp_packed_{args.workload}_{key}")
                storage_arms[key]["roofline"]["traffic"] = arm_rec.get("dram_bytes_per_launch")
        torch.cuda.synchronize()
        vol_for_acc = vol_main
    else:
        vol_for_acc = arm.vol

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(w, E)
        cpu["accuracy_of_timed_volume"] = sample_errors(vol_for_acc, acc["vox"], acc["ref"])
        cpu["accuracy_sample"] = acc["desc"]
        cpu["oracle_seconds_for_accuracy_sample"] = acc["seconds"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_desc(w), "storage": args.dtype, "accumulate": "f32",
                       "step": f"one batch: filter + pack + back-project {main_bf_group * main_bf_n} views "
                               f"({main_bf_n} {'half-turn pairs' if main_bf_group == 2 else 'quarter-turn quads'}) "
                               f"of the "
                               f"{g.np}-view scan; "
                               f"{batches} steps = one reconstruction (volume zeroed at its first)",
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (E, Q, Qp and the volume each >= 256 MiB)",
                       "bp_path": ("packed views" + {2: ", half-turn view pairs", 4: ", quarter-turn view quads"}
                                   .get(info["path"], ""))
                       if packed else "filtered views as stored",
                       "bp_launch": info, "view_split": splits},
            "e2e": e2e, "gpu_launches": launches, "clocks": ck, "roofline": roofline,
            "storage_arms": storage_arms, "cpu_baseline": cpu, "filter_stage": filter_stage,
            "output_stage": output_stage,
            "arith_rates": {k: (v if k == "n_sm" else {"lane_ops_per_clk_sm": round(v["lane_ops_per_clk_sm"], 2),
                                                        "warp_instr_per_clk_sm": round(v["warp_instr_per_clk_sm"], 3)})
                            for k, v in rates.items()},
            "value_1e9": value * 2 ** 30 / 1e9}   # the same throughput in 10^9 updates/s
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_arm(plan, batches, tdt, dev, standard, E, vol_ref, acc, roofline_of, key) -> dict:
    """Another storage type on the same inputs: one warm-up batch, then one timed
    reconstruction (every batch); its volume against the main arm's and the oracle."""
    import torch
    arm = Arm(plan, batches, tdt, dev, standard)
    arm.step(E, 0)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(batches)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    t0.record(stream)
    for k in range(batches):
        arm.step(E, k, ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    upd = sum(arm.updates(k) for k in range(batches))
    bp = float(np.mean([arm.updates(k) / (a.elapsed_time(b) * 1e-3) / 2 ** 30 for k, (a, b) in enumerate(ev)]))
    out = {"step_gups": upd / (t0.elapsed_time(t1) * 1e-3) / 2 ** 30, "bp_gups": bp,
           "bp_path": {2: "half-turn view pairs", 4: "quarter-turn view quads"}.get(arm.bf.group),
           "roofline": {k2: v for k2, v in roofline_of(bp, key).items()
                        if k2 in ("frac", "peak_path", "frac_path", "frac_nominal_128lane")},
           "rel_l2_vs_main_volume": rel_l2_chunked(arm.vol, vol_ref),
           "split_terms": 3 if tdt == torch.float32 else 2}
    if acc is not None:
        out["vs_oracle_sample"] = sample_errors(arm.vol, acc["vox"], acc["ref"])
    arm.bf.Q = arm.bf.Qp = None
    del arm
    torch.cuda.empty_cache()
    return out


def oracle_accuracy(w, E, vox) -> dict:
    """Oracle values at the accuracy sample, from this run's projections E (the rows
    the voxels touch, read back from the device in FP32 and widened)."""
    import torch
    import oracle
    g = w.geom
    s_idx, r_idx = oracle_rows(g, vox)
    rows = []
    for a in range(0, len(s_idx), 65536):
        s = torch.from_numpy(s_idx[a:a + 65536]).to(E.device)
        r = torch.from_numpy(r_idx[a:a + 65536]).to(E.device)
        rows.append(E[s, r].double().cpu().numpy())
    ref, dt = oracle_sample_fdk(g, np.concatenate(rows), s_idx, r_idx, vox, oracle.default_threads())
    ks = sorted(set(int(k) for k in vox[:, 2]))
    return {"vox": vox, "ref": ref, "seconds": dt,
            "desc": f"{len(vox)} voxels: z-slices {ks}, every {max(1, g.nx // 128)}th column in i and j"}


def cpu_baseline(w, E) -> dict:
    """The oracle on the host cores on a bounded sample (seeded mid-plane voxels, all
    views), with one thread and with every core, about 10 s each."""
    import torch
    import oracle
    g = w.geom
    cores = oracle.default_threads()
    vox_all = midplane_sample(g, 1 << 20, 7)
    s_idx, r_idx = midplane_rows(g)
    E_rows = E[torch.from_numpy(s_idx).to(E.device), torch.from_numpy(r_idx).to(E.device)].double().cpu().numpy()
    out = {"unit": UNIT, "kind": "oracle"}
    for label, threads, budget in (("all_cores", cores, 10.0), ("one_thread", 1, 20.0)):
        # size the back-projection part of the sample to about `budget` seconds
        n = min(len(vox_all), 4096 * threads)
        _, t_f, t_b = oracle_sample_fdk_parts(g, E_rows, s_idx, r_idx, vox_all[:n], threads)
        n = int(min(len(vox_all), max(256, n * max(budget - t_f, 1.0) / max(t_b, 1e-3))))
        _, t_f, t_b = oracle_sample_fdk_parts(g, E_rows, s_idx, r_idx, vox_all[:n], threads)
        out[label] = {"value": n * g.np / (t_f + t_b) / 2 ** 30, "threads": threads, "voxels": n,
                      "seconds": t_f + t_b, "filter_seconds": t_f, "rows_filtered": int(len(s_idx)),
                      "backprojection_gups": n * g.np / t_b / 2 ** 30}
    out["value"] = out["all_cores"]["value"]
    out["cores"] = cores
    out["sample"] = (f"seeded voxels of the two mid-plane z-slices x all {g.np} views (all_cores: "
                     f"{out['all_cores']['voxels']}, one_thread: {out['one_thread']['voxels']} voxels), incl. "
                     f"filtering the {len(s_idx)} detector rows they touch (FP64 C, pthreads); "
                     f"backprojection_gups leaves the filtering out")
    return out


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


def run_solver(args):
    """--solver sart|mlem: iterations of the iterative solver on the workload's
    projections (one GPU); a step is one iteration (a pass over the subsets)."""
    import torch
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.api import IterativeSolver
    from paper_1909_02724_gb300.build import build
    from paper_1909_02724_gb300.phantom import workload, workload_projections_gpu

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build()
    w = workload(args.workload)
    g = w.geom
    plan = B.Plan(g)
    p = workload_projections_gpu(w)
    if args.solver == "mlem":
        p.clamp_(min=0.0)
    solver = IterativeSolver(plan, args.solver, args.subsets, lam=1.0, nonneg=args.solver == "sart")
    x = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device="cuda")
    x0 = 0.0 if args.solver == "sart" else 1.0
    x.fill_(x0)
    solver.run(p, x, max(1, args.warmup))
    x.fill_(x0)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    solver.run(p, x, args.steps)
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    # one subset update timed stage by stage
    S, C = solver.sets[0], solver.C[0]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ev[0].record(stream)
    for b, c in S:
        plan.project(x, solver.Ax, view_begin=b, view_count=c)
    ev[1].record(stream)
    o = 0
    for b, c in S:
        B.ifdk_iter_ratio(plan.handle, solver.method, p[b:b + c], solver.Ax[b:b + c],
                          None if solver.R is None else solver.R[b:b + c], solver.rb[o:o + c], c)
        o += c
    ev[2].record(stream)
    solver._backproject(S, solver.U)
    ev[3].record(stream)
    B.ifdk_iter_update(plan.handle, solver.method, x, solver.U, C, 1.0, solver.nonneg)
    ev[4].record(stream)
    torch.cuda.synchronize()
    stages = dict(zip(("project", "ratio", "backproject", "update"),
                      (ev[i].elapsed_time(ev[i + 1]) for i in range(4))))
    upd = 2 * g.nx * g.ny * g.nz * g.np
    views_s = sum(c for _, c in S)
    line = {"metric": f"{args.solver} iteration GUPS (forward + back-projection updates, 2 Nx Ny Nz Np per "
                      "iteration / T / 2^30)",
            "value": upd / (ms * 1e-3) / 2 ** 30, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(w), "solver": args.solver, "subsets": len(solver.sets),
                       "bp_path": "packed batch" if solver.packed else "filtered views as stored",
                       "step": "one iteration: every subset's project, ratio, back-projection and update"},
            "first_subset_ms": stages, "first_subset_views": views_s,
            "project_gups": g.nx * g.ny * g.nz * views_s / (stages["project"] * 1e-3) / 2 ** 30,
            "backproject_gups": g.nx * g.ny * g.nz * views_s / (stages["backproject"] * 1e-3) / 2 ** 30,
            "clocks": ck}
    print(json.dumps(line), flush=True)


def run_filter(args):
    """--filter-views N: the filtering stage alone (ifdk_filter_views, tensor cores) on the
    first N views of the workload (a small case of the step's filter, for profiling)."""
    import torch
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.build import build
    from paper_1909_02724_gb300.phantom import line_integrals_gpu, workload

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build()
    w = workload(args.workload)
    g = w.geom
    n = min(args.filter_views, g.np)
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    plan = B.Plan(g)
    E = line_integrals_gpu(w.phantom(), g, view_count=n)
    Q = torch.empty(E.shape, dtype=tdt, device="cuda")
    terms = 3 if tdt == torch.float32 else 2
    for _ in range(max(3, args.warmup)):
        plan.filter_views(E, Q, view_begin=0, split_terms=terms)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        plan.filter_views(E, Q, view_begin=0, split_terms=terms)
        b.record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    products = {3: 6, 2: 3, 1: 1}[terms]
    flops = 2.0 * n * g.nv * g.nu * (g.nu + 1) * products
    peak = float(measured_peaks().get("bf16_tflops", 1900.0))
    print(json.dumps({"metric": "filtering stage TFLOP/s (dense Toeplitz, BF16 term products)",
                      "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": args.dtype,
                      "config": {"workload": workload_desc(w) + f"; first {n} views", "split_terms": terms,
                                 "term_products": products},
                      "roofline": {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak,
                                   "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / peak}}), flush=True)


def run_unrolled(args):
    """--unrolled T: the differentiation workload (grad256): T unrolled gradient-descent
    steps on ||A x - y||^2 (A = ifdk_project, A^T the back-projection) with per-step
    recomputation, forward and backward; a step is one such forward + backward.  Also
    times one application of each operator on a dense volume."""
    import torch
    from paper_1909_02724_gb300 import autograd as A
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.build import build
    from paper_1909_02724_gb300.phantom import workload, workload_projections_gpu

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build()
    w = workload(args.workload)
    g = w.geom
    plan = B.Plan(g)
    y = workload_projections_gpu(w)
    y = y / y.abs().max()
    v = torch.randn((g.nx, g.ny, g.nz), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    for _ in range(8):                    # power iteration on A^T A for the step size
        v = plan.backproject(plan.project(v))
        lam = float(v.norm())
        v /= lam
    T = args.unrolled

    def once():
        alphas = torch.full((T,), 0.5 / lam, device="cuda", requires_grad=True)
        x = A.unrolled_gd(plan, y, torch.zeros((g.nx, g.ny, g.nz), device="cuda"), alphas, recompute=True)
        r = A.project(x, plan) - y
        (r * r).sum().backward()
        return alphas.grad

    for _ in range(max(1, args.warmup)):
        once()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        once()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    ops = T * 6 + 2          # forward, recomputed forward, the two transposes per step; the loss
    # one application of each operator on a dense volume / dense views
    xd = plan.backproject(plan.filter(workload_projections_gpu(w)))
    P = torch.zeros_like(y)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    plan.project(xd, P)
    P.zero_()
    ev[0].record(stream)
    plan.project(xd, P)
    ev[1].record(stream)
    A.backproject(P, plan)
    ev[2].record(stream)
    torch.cuda.synchronize()
    pj, bp = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    print(json.dumps({"metric": "unrolled gradient descent GUPS (operator updates: (6 T + 2) Nx Ny Nz Np per "
                                "forward + backward / T / 2^30)",
                      "value": ops * g.updates / (ms * 1e-3) / 2 ** 30, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": workload_desc(w), "unrolled_steps": T, "recompute": True},
                      "project_ms_per_application": pj, "backproject_ms_per_application": bp,
                      "project_gups": g.updates / (pj * 1e-3) / 2 ** 30,
                      "backproject_gups": g.updates / (bp * 1e-3) / 2 ** 30}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.unrolled:
        run_unrolled(args)
    elif args.filter_views:
        run_filter(args)
    elif args.solver:
        run_solver(args)
    elif args.workload == "slab4096":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
