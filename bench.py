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


def peaks_bf16() -> float:
    """Measured dense BF16 tensor throughput (TFLOP/s, the burst figure) or the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except Exception:
        return 1900.0


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
def oracle_sample(scene, depths, n, iters, threads=0):
    """C FP64 oracle: alloc+fuse of n frames then ``iters`` iterations on their blocks with
    ``threads`` threads (0: one per processor); returns (voxel-updates, seconds, blocks)."""
    from oracle import denser_oracle as O
    from oracle import oracle_c as C
    cam = scene.camera
    K = O.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    C.set_threads(threads)
    t0 = time.perf_counter()
    m = C.CMap(O.Params(), 1 << 17)
    for k in range(n):
        m.alloc_blocks(depths[k], K, scene.poses[k])
        m.fuse_depth(depths[k], K, scene.poses[k])
    m.regularize(iters)
    dt = time.perf_counter() - t0
    nb = m.n_blocks
    m.close()
    return nb * 512 * iters, dt, nb


def cpu_threads():
    return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return
    # a step is n frames of allocation and fusion and n iterations on their blocks (the
    # workload's 1:1 ratio of frames to iterations), the C oracle on every host core
    n = 32
    scene, depths = make_inputs(0, range(n))
    for _ in range(args.warmup):
        oracle_sample(scene, depths, n, n)
    tot_u, tot_t, nb = 0, 0.0, 0
    for _ in range(args.steps):
        u, t, nb = oracle_sample(scene, depths, n, n)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    sample = (f"first {n} frames of the street (alloc+fuse) then {n} PD iterations on their {nb} blocks, "
              f"C FP64 oracle, {cpu_threads()} threads ({cpu_model()})")
    line = {"impl": "reference", "metric": "voxel-updates/s per primal-dual iteration", "value": v,
            "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "voxel-updates/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
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



# ------------------------------------------------------- extra workloads
def synth_workers(args) -> int:
    return args.workers if args.workers > 0 else max(1, min(16, os.cpu_count() or 1))


def device_maps(specs, workers, dev):
    """Depth maps of the streets ``specs`` [(seed, length)], made by a process pool and
    copied into one device tensor as they arrive; returns (tensor [n, H, W], per-spec
    first frame)."""
    import torch
    from synth.scenes import street_depth_maps, street_scene
    cam = street_scene(seed=specs[0][0], length=specs[0][1]).camera
    counts = [int(round(length / 0.5)) for _, length in specs]
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(int)
    out = torch.empty((sum(counts), cam.height, cam.width), dtype=torch.float32, device=dev)
    stage = torch.empty((cam.height, cam.width), dtype=torch.float32).pin_memory()
    for i, k, d in street_depth_maps(specs, workers=workers):
        stage.copy_(torch.from_numpy(d))
        out[first[i] + k].copy_(stage)
    torch.cuda.synchronize(dev)
    return out, first


def time_steps(pipeline, steps, warmup, stream):
    """(ms per step, sweep ms summed, sweep launches) over ``steps`` timed steps."""
    import torch
    for _ in range(warmup):
        pipeline()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweep_ms, launches = 0.0, 0
    e0.record(stream)
    for _ in range(steps):
        st = pipeline()
        sweep_ms += st.sweep_ms
        launches += st.sweep_launches
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, sweep_ms, launches


def precision_street(args, dev, stream, N, hbm, K, workers):
    """The 1 km street (2000 depth maps, the same generator) fused and regularised (200
    iterations) with u, u_bar and p stored in FP32, FP16 and BF16, each with the sweep
    schedule the autotuner picks on that map and storage type."""
    import torch
    from paper_1604_03734_gb300 import autotune as AT
    from synth.scenes import street_scene
    length = 1000.0
    sc = street_scene(seed=0, length=length)
    depths, _ = device_maps([(0, length)], workers, dev)
    poses = np.asarray(sc.poses, dtype=np.float64)
    rows = {}
    for prec, name in ((0, "fp32"), (1, "fp16"), (2, "bf16")):
        m = N.DenserMap(device=dev.index or 0, max_blocks=1 << 18, hash_slots=1 << 20, precision=prec)

        def pipeline():
            N.denser_reset(m.ctx, stream)
            for first in range(0, len(poses), 16):
                N.denser_integrate_batch(m.ctx, depths[first:first + 16], K, poses[first:first + 16], 0, stream)
            st = N.denser_regularize(m.ctx, args.iters, 0.0, 0, stream)
            N.denser_extract(m.ctx, None, None, None, None, u_out, nb, stream)
            return st

        nb = 0
        u_out = None
        pipeline()
        nb = N.denser_num_blocks(m.ctx, stream)
        u_out = torch.empty((nb, 512), dtype=torch.float32, device=dev)
        tune = AT.autotune(m.ctx, prec, iters=10, use_cache=False, stream=stream)
        ms, sweep_ms, launches = time_steps(pipeline, 3, 1, stream)
        bpv = BYTES_PER_VOXEL_ITER[prec]
        nvox = nb * 512
        sweep_avg = sweep_ms / max(launches, 1)
        gbs = bpv * nvox / (sweep_avg / 1e3) / 1e9
        rows[name] = {"ms_per_step": ms, "voxel_updates_per_s": nvox * args.iters / (ms / 1e3),
                      "sweep_ms": sweep_avg, "sweep_voxel_updates_per_s": nvox / (sweep_avg / 1e3),
                      "bytes_per_voxel": bpv, "sweep_gbs": gbs, "frac_of_measured_hbm": gbs / hbm,
                      "schedule": N.denser_get_schedule(m.ctx),
                      "autotune": {"schedule": tune["schedule"], "ms_per_iter": tune["ms_per_iter"],
                                   "candidates": len(tune["table"])}}
        m.close()
    del depths
    torch.cuda.empty_cache()
    return {"workload": "driving street 1 km: 2000 depth maps 1241x376, 200 PD iters (storage precision variant)",
            "blocks": nb, "voxels": nb * 512, "steps": 3, "warmup": 1,
            "by_storage": rows, "note": "u, u_bar, p stored as named; f, w FP32; FP32 stencil arithmetic; "
                                        "FP64 energies"}


def batched_segments(args, dev, stream, N, hbm, K, workers):
    """64 independent street segments of lengths uniform in 50-500 m (seeds 1-64), all
    fused into one map (segment = its index) and regularised together: one sweep
    launch per iteration covers every segment, the loop runs as one CUDA graph, and
    the sweep schedule is the autotuner's pick on this map."""
    import torch
    from paper_1604_03734_gb300 import autotune as AT
    from synth.scenes import segment_scenes
    scenes = segment_scenes()
    specs = [(s.seed, len(s.poses) * 0.5) for s in scenes]
    frames = [len(s.poses) for s in scenes]
    total_len = float(sum(l for _, l in specs))
    cam = scenes[0].camera
    max_blocks = int(np.ceil(290.0 * total_len / 1024.0)) * 1024
    need = sum(frames) * cam.width * cam.height * 4 + max_blocks * (46 * 512 + 600) + max_blocks * 2048
    free = torch.cuda.mem_get_info(dev)[0]
    if need > 0.92 * free:
        return {"skipped": f"needs about {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free"}
    t0 = time.perf_counter()
    depths, first = device_maps(specs, workers, dev)
    synth_s = time.perf_counter() - t0
    poses = [np.asarray(s.poses, dtype=np.float64) for s in scenes]
    m = N.DenserMap(device=dev.index or 0, max_blocks=max_blocks, hash_slots=1 << 23)
    u_out = None
    nb = 0

    def pipeline():
        N.denser_reset(m.ctx, stream)
        for seg in range(len(scenes)):
            for f0 in range(0, frames[seg], 16):
                n = min(16, frames[seg] - f0)
                N.denser_integrate_batch(m.ctx, depths[first[seg] + f0:first[seg] + f0 + n], K,
                                         poses[seg][f0:f0 + n], seg, stream)
        st = N.denser_regularize(m.ctx, args.iters, 0.0, 0, stream)
        if u_out is not None:
            N.denser_extract(m.ctx, None, None, None, None, u_out, nb, stream)
        return st

    pipeline()
    nb = N.denser_num_blocks(m.ctx, stream)
    u_out = torch.empty((nb, 512), dtype=torch.float32, device=dev)
    tune = AT.autotune(m.ctx, 0, iters=10, use_cache=False, stream=stream)
    ms, sweep_ms, launches = time_steps(pipeline, 2, 1, stream)
    nvox = nb * 512
    sweep_avg = sweep_ms / max(launches, 1)
    gbs = 48 * nvox / (sweep_avg / 1e3) / 1e9
    out = {"workload": "64 street segments, lengths uniform in 50-500 m (seeds 1-64), one map, 200 PD iters, FP32",
           "segments": len(scenes), "frames": int(sum(frames)), "length_m": total_len,
           "shortest_m": min(l for _, l in specs), "longest_m": max(l for _, l in specs),
           "blocks": nb, "voxels": nvox, "steps": 2, "warmup": 1, "ms_per_step": ms,
           "voxel_updates_per_s": nvox * args.iters / (ms / 1e3),
           "sweep_ms": sweep_avg, "sweep_voxel_updates_per_s": nvox / (sweep_avg / 1e3),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                        "bytes_per_voxel": 48, "kernel": "sweep (autotuned schedule)"},
           "autotune": {"schedule": tune["schedule"], "ms_per_iter": tune["ms_per_iter"],
                        "table": tune["table"]},
           "graph_loop": bool(N.denser_get_schedule(m.ctx)["use_graph"]),
           "synthesis_s": synth_s, "inputs": "depth maps resident in HBM",
           "l2": f"working set {48 * nvox / 1e9:.0f} GB per sweep > 129 MB L2, no flush"}
    m.close()
    del depths, u_out
    torch.cuda.empty_cache()
    return out


def guarded(fn, *a):
    """Runs one extra measurement; an error is reported in its field instead of ending the run."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        return {"error": f"{type(e).__name__}: {e}"[:300]}


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
    ap.add_argument("--no-precision-street", action="store_true",
                    help="skip the 1 km street in FP32 / FP16 / BF16 storage")
    ap.add_argument("--no-segments", action="store_true", help="skip the 64 batched street segments")
    ap.add_argument("--workers", type=int, default=0, help="depth-map synthesis processes (0: all cores, at most 16)")
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

    side = torch.cuda.Stream(dev)
    fused = torch.cuda.Event()

    def pipeline(depth_src, outs, overlap=False, ev=None):
        """One step; ev: a pair of timing events recorded on the stream around the
        iteration loop (the loop then runs without the host waiting for its statistics)."""
        N.denser_reset(ctx, stream)
        if args.batch > 1:
            for first in range(0, args.frames, args.batch):
                N.denser_integrate_batch(ctx, depth_src[first:first + args.batch], K,
                                         poses_arr[first:first + args.batch], 0, stream)
        else:
            for k in range(args.frames):
                N.denser_integrate(ctx, depth_src[k], K, poses[k], 0, stream)
        if not overlap:
            if ev is not None:
                # the call waits for the fusion before it queues the loop, so the first
                # event lands after the fusion and the second after the loop; then the
                # FP64 primal and dual energies (the gap) of the result, as the
                # statistics would give them
                ev[0].record(stream)
                N.denser_regularize(ctx, args.iters, 0.0, 0, stream, stats=False)
                ev[1].record(stream)
                N.denser_energy(ctx, stream)
                st = None
            else:
                st = N.denser_regularize(ctx, args.iters, 0.0, 0, stream)
            N.denser_extract(ctx, outs["coords"], outs["f"], outs["w"], outs["omega"], outs["u"],
                             outs["cap"], stream)
            return st
        # host outputs: coords, f, w and Omega are final once the maps are fused, so they
        # travel to the host on a second stream while the iterations run; u follows them
        fused.record(stream)
        N.denser_regularize(ctx, args.iters, 0.0, 0, stream, stats=False)
        side.wait_event(fused)
        N.denser_extract(ctx, outs["coords"], outs["f"], outs["w"], outs["omega"], None, outs["cap"], side)
        N.denser_energy(ctx, stream)
        N.denser_extract(ctx, None, None, None, None, outs["u"], outs["cap"], stream)
        return None

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
        loop_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        torch.cuda.synchronize()
        clk.start()
        ev0.record(stream)
        for k in range(args.steps):
            pipeline(depths_dev, out_dev, ev=loop_ev[k])
        ev1.record(stream)
        torch.cuda.synchronize()
        # the sweeps' device time: the loop's events (they also hold the loop's short
        # set-up: Omega bits, neighbour rows, zeroed state), all iterations being sweeps
        sweep_ms = sum(a.elapsed_time(b) for a, b in loop_ev)
        sweep_launches = args.steps * args.iters
        clk.stop()
    launches = N.denser_launch_count(ctx) - l0
    step_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    if world > 1:
        dist.barrier()

    nvox = nb * 512
    updates = nvox * args.iters
    updates_all = sum_over_ranks(updates, world, dev)  # each rank's street has its own block count
    value = updates_all / (step_ms / 1e3)

    # end to end: host depth maps (pinned) in, host results out, through the C ABI, over
    # the same K steps as the device-resident measurement; one untimed pass first (the
    # library's host staging buffers are allocated on first use)
    pipeline(depths_host, out_host, overlap=True)
    torch.cuda.synchronize()
    e2e_steps = max(1, args.steps)
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        pipeline(depths_host, out_host, overlap=True)
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
                   "sweep_rows_kernel", "sweep_rows_prefetch_kernel",
                   "sweep_rows_pipelined_kernel", "sweep_rows_kernel",
                   "sweep_rows_kernel", "sweep_rows_pipelined_kernel"][N.denser_get_schedule(ctx)["sweep_kernel"]]

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

    # the warm-start network's convolution on the tensor cores (tcgen05): one 16 -> 16
    # channel 3^3 layer over 4096 blocks (10^3 voxels each), BF16 in, FP32 accumulate
    conv = None
    if not args.no_warmstart:
        ns = 4096
        xs = torch.randn(ns, 1000, 16, device=dev).to(torch.bfloat16)
        wts = (torch.randn(27, 16, 16, device=dev) * 0.1).to(torch.bfloat16)
        ys = torch.empty(ns, 1000, 16, dtype=torch.bfloat16, device=dev)
        for _ in range(3):
            N.denser_conv3(xs, wts, None, 1, ys, None, ns, stream)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        c0.record(stream)
        for _ in range(reps):
            N.denser_conv3(xs, wts, None, 1, ys, None, ns, stream)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / reps
        flops = 2.0 * ns * 1000 * 16 * 16 * 27
        peak_tf = peaks_bf16()
        conv = {"samples": ns, "ms_per_layer": cms, "useful_tflops": flops / (cms / 1e3) / 1e12,
                "frac_of_measured_bf16": flops / (cms / 1e3) / 1e12 / peak_tf, "peak_tflops": peak_tf,
                "kernel": "conv3_tc_kernel (tcgen05.mma M128 N16 K16, accumulators in TMEM)",
                "flops": "2 x 1000 voxels x 16 x 16 x 27 per sample (the padded rows the kernel also computes "
                         "are not counted)", "net_check": N.denser_net_check(stream)}
        del xs, wts, ys

    # fusion roofline: the same 200 maps allocated and fused with the library's fusion
    # profiling on (CUDA events around the key pass, the rest of the allocation, culling
    # and the fusion kernel; the call waits after each group, so this is not the step above)
    fusion = None
    if args.batch > 1:
        N.denser_set_fusion_profiling(ctx, True)
        reps = 3
        for _ in range(reps):
            N.denser_reset(ctx, stream)
            for first in range(0, args.frames, args.batch):
                N.denser_integrate_batch(ctx, depths_dev[first:first + args.batch], K,
                                         poses_arr[first:first + args.batch], 0, stream)
        pr = N.denser_get_fusion_profile(ctx)
        N.denser_set_fusion_profiling(ctx, False)
        npix = cam.width * cam.height
        fuse_bytes = 16.0 * 512 * pr["listed_blocks"] + 4.0 * npix * pr["maps"]
        key_bytes = 4.0 * npix * pr["maps"] + 16.0 * pr["new_blocks"]
        fusion = {"maps": pr["maps"] // reps, "groups": pr["groups"] // reps,
                  "listed_blocks_per_group": pr["listed_blocks"] / max(pr["groups"], 1),
                  "ms_per_pass": (pr["key_pass_ms"] + pr["alloc_rest_ms"] + pr["cull_ms"] + pr["fuse_ms"]) / reps,
                  "key_pass": {"ms_per_map": pr["key_pass_ms"] / pr["maps"],
                               "achieved_gbs": key_bytes / (pr["key_pass_ms"] / 1e3) / 1e9,
                               "frac_of_measured_hbm": key_bytes / (pr["key_pass_ms"] / 1e3) / 1e9 / hbm,
                               "bytes": "4 B of depth per pixel + 16 B per new block key"},
                  "fuse_kernel": {"ms_per_map": pr["fuse_ms"] / pr["maps"],
                                  "achieved_gbs": fuse_bytes / (pr["fuse_ms"] / 1e3) / 1e9,
                                  "frac_of_measured_hbm": fuse_bytes / (pr["fuse_ms"] / 1e3) / 1e9 / hbm,
                                  "bytes": "16 B per listed voxel per launch (f, w read and written once for the "
                                           "group's maps) + 4 B of depth per pixel and map"},
                  "alloc_rest_ms_per_map": pr["alloc_rest_ms"] / pr["maps"],
                  "cull_ms_per_map": pr["cull_ms"] / pr["maps"],
                  "timing": "CUDA events inside the library, fusion profiling on (waits after each group)"}

    # the 1 km street in each storage type, and the 64 batched segments (one GPU, rank 0)
    workers = synth_workers(args)
    prec_street = None if args.no_precision_street or world > 1 else \
        guarded(precision_street, args, dev, stream, N, hbm, K, workers)
    segments = None if args.no_segments or world > 1 else guarded(batched_segments, args, dev, stream, N, hbm, K,
                                                                   workers)

    # the C FP64 oracle on the host cores: the whole workload (the same 200 maps, 200
    # iterations) on every core, and a sample on one thread
    cpu = None
    if not args.no_cpu_baseline:
        u, t, nbs = oracle_sample(scene, depths_np, args.frames, args.iters, 0)
        n1 = 8
        u1, t1, nb1 = oracle_sample(scene, depths_np, n1, n1, 1)
        cpu = {"value": u / t, "unit": "voxel-updates/s", "cores": cpu_threads(), "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"the whole workload: {args.frames} maps alloc+fuse then {args.iters} PD iterations on "
                         f"their {nbs} blocks, C FP64 oracle (OpenMP over blocks), {t:.1f} s",
               "single_thread": {"value": u1 / t1, "cores": 1,
                                 "sample": f"first {n1} maps alloc+fuse then {n1} PD iterations on their {nb1} "
                                           f"blocks, {t1:.1f} s"}}
        from oracle import oracle_c as C
        C.set_threads(0)

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
                   "stereo_depth": stereo, "warmstart_conv": conv, "fusion_roofline": fusion,
                   "precision_street_1km": prec_street,
                   "batched_segments": segments},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": measured_traffic(kernel_name, args.precision, nvox, N.denser_get_schedule(ctx)),
                     "traffic_unit": "bytes per launch (ncu dram read + write)", "kernel": kernel_name,
                     "peak_kind": peak_kind, "bytes_per_voxel": bpv,
                     "schedule": N.denser_get_schedule(ctx)},
        "e2e": {"value": updates_all / (e2e_ms / 1e3), "unit": "voxel-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "pinned host depth maps staged per batch on the library's copy stream; coords, f, w and "
                            "Omega copied to pinned host memory on a second stream while the iterations run, u "
                            "after them"},
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
