"""Benchmark of the DENSER hot path on one GB300 (or N, one independent street per rank).

One step = the whole hot path over one synthetic driving street: reset the map;
for each of 200 depth maps (1241x376, f = 718 px, poses 0.5 m apart along a 100 m
road) allocate blocks and fuse; 200 primal-dual iterations with the FP64 energy
and gap at the end; extract keys, f, w, Omega and u.  Inputs are resident in HBM
when the timed region starts.

value = allocated voxels x primal-dual iterations / step time (voxel-updates/s per
primal-dual iteration, fusion and extraction included in the time).

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload (the first frames of the same street, as many iterations as frames).
"""

from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_VOXEL_ITER = {0: 48, 1: 28, 2: 28}  # FP32 / FP16 / BF16 storage of u, u_bar, p
WORKLOAD = "driving street 100 m: 200 depth maps 1241x376, f=718 px, 0.1 m voxels, 8^3 blocks, mu 0.3 m, 200 PD iters"


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_rows_street100_traffic.json")
SWEEP_SOURCE = os.path.join(ROOT, "paper_1604_03734_gb300", "csrc", "regularize.cu")


def sweep_fingerprint() -> str:
    """sha256 of the row-sweep kernel's source and of the stencil arithmetic it calls."""
    import hashlib
    src = open(SWEEP_SOURCE).read()
    parts = []
    for start, end in (("// Arithmetic shared by every sweep variant", "// Dual step at tile position"),
                       ("// --------------------------------------------------------------- row sweep",
                        "template <typename T>\nconstexpr size_t sweep_pipe_smem")):
        i, j = src.find(start), src.find(end)
        parts.append(src[i:j] if 0 <= i < j else "")
    return hashlib.sha256("".join(parts).encode()).hexdigest()


def measured_traffic(kernel: str, precision: int, nvox: int, schedule=None):
    """DRAM bytes per launch from the committed ncu capture of the same kernel and workload,
    or None when the capture is missing, of another workload, or the kernel changed since."""
    try:
        with open(TRAFFIC_FILE) as fh:
            j = json.load(fh)
    except (OSError, ValueError):
        return None
    if kernel != "sweep_rows_kernel" or precision != 0 or j.get("source_fingerprint") != sweep_fingerprint():
        return None
    if schedule is not None and list(j.get("schedule", [])) != [schedule["sweep_kernel"], schedule["order"],
                                                                 schedule["ctas_per_sm"]]:
        return None
    if int(j.get("voxels", -1)) != nvox:
        return None
    return float(j["dram_read_bytes"]) + float(j["dram_write_bytes"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms.  The sampler is started before the
    warm-up (so that nvidia-smi's own start-up does not fall into the timed region) and
    the summary keeps the samples whose timestamps lie inside the timed region."""

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index
        self.t0 = self.t1 = None

    def wait_ready(self, timeout=5.0):
        """Waits until the first sample is written (or the timeout)."""
        t_end = time.time() + timeout
        while self.proc is not None and time.time() < t_end:
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.05)

    def start(self):
        self.t0 = datetime.datetime.now()

    def stop(self):
        self.t1 = datetime.datetime.now()

    def __enter__(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(parts[2]), float(parts[3]),
                             [nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
        window = "timed region"
        if not inside and rows and self.t0 is not None:
            # a region shorter than the sampling period: the first sample after it began
            after = [r for r in rows if r[0] >= self.t0]
            inside, window = (after[:1] or rows[-1:]), "first sample after the start of the timed region"
        if not inside:
            return None
        reasons = sorted({nm for r in inside for nm in r[3]})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": float(max(r[2] for r in inside)),
                "samples": len(inside), "window": window, "reasons": reasons}


def make_inputs(seed, frames=None, length=100.0):
    from synth.scenes import street_scene
    scene = street_scene(seed=seed, length=length)
    depths = scene.depth_maps(frames, workers=min(16, os.cpu_count() or 1) if length > 100.0 else 1)
    return scene, depths


# ------------------------------------------------------------- reference arm
def oracle_sample(scene, depths, n, iters):
    """Oracle alloc+fuse of n frames then ``iters`` iterations; returns (voxel-updates, seconds)."""
    from oracle import denser_oracle as O
    cam = scene.camera
    K = O.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    t0 = time.perf_counter()
    g = O.SparseGrid(O.Params())
    for k in range(n):
        O.alloc_blocks(g, depths[k], K, scene.poses[k])
        O.fuse_depth(g, depths[k], K, scene.poses[k])
    O.regularize(g, iters)
    dt = time.perf_counter() - t0
    return g.n_blocks * 512 * iters, dt, g.n_blocks


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    # a step is n frames of allocation and fusion and n iterations (the workload's 1:1
    # ratio); one frame when many steps are asked for, so that the run stays within minutes
    n = 1 if args.steps + args.warmup > 8 else 2
    scene, depths = make_inputs(0, range(n))
    for _ in range(args.warmup):
        oracle_sample(scene, depths, n, n)
    tot_u, tot_t, nb = 0, 0.0, 0
    for _ in range(args.steps):
        u, t, nb = oracle_sample(scene, depths, n, n)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    sample = f"first {n} frames of the street (alloc+fuse) then {n} PD iterations on their {nb} blocks, FP64 numpy"
    line = {"impl": "reference", "metric": "voxel-updates/s per primal-dual iteration", "value": v,
            "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "voxel-updates/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- multi-rank
def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (timings: the job ends with its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    """x summed over all ranks (work units: every rank fuses and solves its own street)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="denser", choices=["denser", "reference"])
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--frames", type=int, default=None, help="depth maps fused per step (default: the whole street)")
    ap.add_argument("--length", type=float, default=100.0, help="street length in metres (a pose every 0.5 m)")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--batch", type=int, default=16,
                    help="depth maps per allocation + fusion launch (1: one denser_integrate call per map)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default=None, help="sweep_kernel,order,ctas_per_sm,use_graph (default: the library's)")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the warm-start time-to-gap comparison")
    ap.add_argument("--no-surface", action="store_true", help="skip the surface-extraction measurement")
    ap.add_argument("--no-laser", action="store_true", help="skip the laser-scan fusion measurement")
    ap.add_argument("--no-stereo", action="store_true", help="skip the stereo depth-map measurement")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.frames is None:
        args.frames = int(round(args.length / 0.5))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_1604_03734_gb300 import build as B
    B.build()
    from paper_1604_03734_gb300 import native as N

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # inputs: each rank fuses its own street (independent problems: weak scaling)
    scene, depths_np = make_inputs(seed=rank, frames=range(args.frames), length=args.length)
    cam = scene.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    depths_host = torch.from_numpy(depths_np).pin_memory()
    depths_dev = depths_host.to(dev)
    poses = scene.poses[:args.frames]
    poses_arr = np.asarray(poses, dtype=np.float64)
    stream = torch.cuda.current_stream(dev)

    # pool and hash sized for the street: about 250 blocks per metre at 10 cm voxels
    mb = 1 << max(17, int(np.ceil(np.log2(300 * args.length))))
    m = N.DenserMap(device=local, max_blocks=mb, hash_slots=2 * mb if mb > (1 << 19) else 1 << 20,
                    precision=args.precision)
    ctx = m.ctx
    if args.schedule:
        N.denser_set_schedule(ctx, *[int(v) for v in args.schedule.split(",")])

    def pipeline(depth_src, outs):
        N.denser_reset(ctx, stream)
        if args.batch > 1:
            for first in range(0, args.frames, args.batch):
                N.denser_integrate_batch(ctx, depth_src[first:first + args.batch], K,
                                         poses_arr[first:first + args.batch], 0, stream)
        else:
            for k in range(args.frames):
                N.denser_integrate(ctx, depth_src[k], K, poses[k], 0, stream)
        st = N.denser_regularize(ctx, args.iters, 0.0, 0, stream)
        N.denser_extract(ctx, outs["coords"], outs["f"], outs["w"], outs["omega"], outs["u"],
                         outs["cap"], stream)
        return st

    def outputs(nb, device):
        pin = device.type == "cpu"
        mk = (lambda *s, dt: torch.empty(*s, dtype=dt, pin_memory=True)) if pin else \
            (lambda *s, dt: torch.empty(*s, dtype=dt, device=device))
        return {"coords": mk(nb, 4, dt=torch.int32), "f": mk(nb, 512, dt=torch.float32),
                "w": mk(nb, 512, dt=torch.float32), "omega": mk(nb, 512, dt=torch.uint8),
                "u": mk(nb, 512, dt=torch.float32), "cap": nb}

    # size the outputs with one untimed pass
    probe = {"coords": None, "f": None, "w": None, "omega": None, "u": None, "cap": 0}
    pipeline(depths_dev, probe)
    nb = N.denser_num_blocks(ctx, stream)
    out_dev = outputs(nb, dev)
    out_host = outputs(nb, torch.device("cpu"))

    with ClockSampler(local) as clk:
        clk.wait_ready()
        for _ in range(args.warmup):
            pipeline(depths_dev, out_dev)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

        l0 = N.denser_launch_count(ctx)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sweep_ms, sweep_launches = 0.0, 0
        torch.cuda.synchronize()
        clk.start()
        ev0.record(stream)
        for _ in range(args.steps):
            st = pipeline(depths_dev, out_dev)
            sweep_ms += st.sweep_ms
            sweep_launches += st.sweep_launches
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.stop()
    launches = N.denser_launch_count(ctx) - l0
    step_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    if world > 1:
        dist.barrier()

    nvox = nb * 512
    updates = nvox * args.iters
    updates_all = sum_over_ranks(updates, world, dev)  # each rank's street has its own block count
    value = updates_all / (step_ms / 1e3)

    # end to end: host depth maps (pinned) in, host results out, through the C ABI; one
    # untimed pass first (the library's host staging buffers are allocated on first use)
    pipeline(depths_host, out_host)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        pipeline(depths_host, out_host)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0)) / e2e_steps, world, dev)
    h2d = args.frames * cam.width * cam.height * 4   # each map staged once (allocation and fusion)
    d2h = nb * (16 + 512 * (4 + 4 + 1 + 4))

    hbm, peak_kind = peaks()
    sweep_avg_ms = sweep_ms / max(sweep_launches, 1)
    bpv = BYTES_PER_VOXEL_ITER[args.precision]
    achieved = bpv * nvox / (sweep_avg_ms / 1e3) / 1e9
    kernel_name = ["sweep_kernel", "sweep_pipe_kernel", "sweep_rows_kernel", "sweep_rows_tma_kernel",
                   "sweep_rows_kernel"][N.denser_get_schedule(ctx)["sweep_kernel"]]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # second metric: time to a relative gap of 1e-4, learned warm start against the plain
    # cold start, on held-out scenes of the tiny workload's generator (seeds 200-219)
    ttg = None
    if not args.no_warmstart:
        from paper_1604_03734_gb300 import warmstart as WS
        net = WS.load_default(device=dev)
        if net is not None:
            ttg = WS.evaluate(net, range(200, 220))

    # surface extraction of the regularised street, outside the step: time per call with
    # device outputs (count, scan, host read of the total, emit), L2 flushed before each
    surface = None
    if not args.no_surface:
        ntri = N.denser_extract_surface(ctx, stream=stream)
        tp = torch.empty((max(ntri, 1), 3, 3), dtype=torch.float32, device=dev)
        ti = torch.empty((max(ntri, 1), 3), dtype=torch.int64, device=dev)
        bf = torch.empty(nb + 1, dtype=torch.int64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for _ in range(3):
            N.denser_extract_surface(ctx, tp, ti, ntri, bf, stream)
        reps, tot = 10, 0.0
        for _ in range(reps):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            N.denser_extract_surface(ctx, tp, ti, ntri, bf, stream)
            s1.record(stream)
            torch.cuda.synchronize()
            tot += s0.elapsed_time(s1)
        sms = tot / reps
        elem = 4 if args.precision == 0 else 2
        alg = nvox * (elem + 4) + ntri * 60 + (nb + 1) * 8
        surface = {"ms_per_call": sms, "triangles": int(ntri), "algorithmic_bytes": int(alg),
                   "achieved_gbs": alg / (sms / 1e3) / 1e9, "frac_of_measured_hbm": alg / (sms / 1e3) / 1e9 / hbm,
                   "bytes": "u and w read once per voxel, 36 B positions + 24 B ids per triangle",
                   "l2": "256 MB written before each call"}
        del tp, ti, bf, flush

    # laser ray fusion (a separate map, outside the step): 64-beam x 2000-azimuth scans
    # every 5 m along the same street, allocation + march + finalize per scan
    laser = None
    if not args.no_laser:
        from synth.scenes import Lidar
        lid = Lidar()
        lframes = list(range(0, args.frames, 10))
        pts = [torch.from_numpy(np.ascontiguousarray(scene.lidar_scan(k, lid))).to(dev) for k in lframes]
        ml = N.DenserMap(device=local, max_blocks=1 << 17, hash_slots=1 << 20)

        def laser_pass():
            N.denser_reset(ml.ctx, stream)
            for p, k in zip(pts, lframes):
                N.denser_integrate_points(ml.ctx, p, poses[k], 0, stream)

        laser_pass()
        torch.cuda.synchronize()
        snap = ml.snapshot()
        obs = float(snap["w"].sum())
        reps, tot = 3, 0.0
        for _ in range(reps):
            l0e, l1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0e.record(stream)
            laser_pass()
            l1e.record(stream)
            torch.cuda.synchronize()
            tot += l0e.elapsed_time(l1e)
        lms = tot / reps
        rays = sum(int(p.shape[0]) for p in pts)
        lbytes = 12 * rays + 16 * obs
        laser = {"scans": len(pts), "rays_per_scan": int(pts[0].shape[0]), "ms_per_scan": lms / len(pts),
                 "rays_per_s": rays / (lms / 1e3), "observations_per_s": obs / (lms / 1e3),
                 "blocks": int(len(snap["coords"])), "achieved_gbs": lbytes / (lms / 1e3) / 1e9,
                 "frac_of_measured_hbm": lbytes / (lms / 1e3) / 1e9 / hbm,
                 "bytes": "12 B per ray (point) + 16 B per voxel observation (64-bit accumulator read and write)"}
        ml.close()
        del pts

    # stereo depth map (Section IV) of one street pair, outside the step: the whole
    # estimate with inputs resident, and the share of its primal-dual kernels
    stereo = None
    if not args.no_stereo:
        IL, IR, _, _ = scene.stereo_pair(10)
        Hs, Ws = IR.shape
        sprm = N.denser_stereo_default_params(max_disp=256)
        ws = torch.zeros(N.denser_stereo_workspace_size(Ws, Hs), dtype=torch.uint8, device=dev)
        il, ir = torch.from_numpy(IL).to(dev), torch.from_numpy(IR).to(dev)
        disp = torch.zeros((Hs, Ws), device=dev)
        N.denser_stereo_estimate(il, ir, sprm, ws, disp, stream)
        torch.cuda.synchronize()
        reps, tot = 3, 0.0
        for _ in range(reps):
            s0e, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0e.record(stream)
            N.denser_stereo_estimate(il, ir, sprm, ws, disp, stream)
            s1e.record(stream)
            torch.cuda.synchronize()
            tot += s0e.elapsed_time(s1e)
        sms = tot / reps
        pd_iters = sprm.outer * sprm.inner
        stereo = {"width": Ws, "height": Hs, "max_disp": sprm.max_disp, "outer": sprm.outer, "inner": sprm.inner,
                  "ms_per_depth_map": sms, "megapixels_per_s": Ws * Hs / (sms / 1e3) / 1e6,
                  "pd_bytes_per_pixel_iteration": 148,
                  "pd_algorithmic_gbs": 148.0 * Ws * Hs * pd_iters / (sms / 1e3) / 1e9,
                  "note": "12 state planes ping-ponged (2 x 22 MB) plus tensor and a: about half the reads "
                          "hit L2; the GB/s figure divides by the whole estimate's time, a lower bound on the "
                          "primal-dual kernel's rate"}
        del ws, il, ir, disp

    cpu = None
    if not args.no_cpu_baseline:
        n = 3
        sc, dn = make_inputs(0, range(n))
        u, t, nbs = oracle_sample(sc, dn, n, n)
        cpu = {"value": u / t, "unit": "voxel-updates/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"first {n} frames of the street (alloc+fuse) then {n} PD iterations on their "
                         f"{nbs} blocks, FP64 numpy, {t:.1f} s"}

    line = {
        "metric": "voxel-updates/s per primal-dual iteration", "value": value, "unit": "voxel-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "f16-storage/f32", 2: "bf16-storage/f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.length == 100.0 else WORKLOAD.replace("100 m: 200", f"{args.length:g} m: {args.frames}"),
                   "frames": args.frames, "fusion_batch": args.batch, "iters": args.iters, "blocks": nb,
                   "voxels": nvox, "parallelism": f"{world} independent streets" if world > 1 else "1 GPU",
                   "l2": f"working set {bpv * nvox / 1e9:.2f} GB per sweep > 129 MB L2, no flush",
                   "pd_only_voxel_updates_per_s": nvox / (sweep_avg_ms / 1e3),
                   "pd_share_of_step": sweep_ms / args.steps / step_ms,
                   "time_to_gap_1e-4_warm_vs_plain": ttg, "surface_extraction": surface, "laser_fusion": laser,
                   "stereo_depth": stereo},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": measured_traffic(kernel_name, args.precision, nvox, N.denser_get_schedule(ctx)),
                     "traffic_unit": "bytes per launch (ncu dram read + write)", "kernel": kernel_name,
                     "peak_kind": peak_kind, "bytes_per_voxel": bpv,
                     "schedule": N.denser_get_schedule(ctx)},
        "e2e": {"value": updates_all / (e2e_ms / 1e3), "unit": "voxel-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
