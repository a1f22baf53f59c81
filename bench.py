#!/usr/bin/env python3
"""Benchmark of the RealLiFe hot path on GB300: MPI refinements/s at 512x384, D=32.

One step = one HSGD refinement (3 iterations at pyramid levels 2, 1, 0; N=4 source
views, k=5 kept planes) of a seeded synthetic scene plus 9 novel views rendered from the
refined MPI, all through the C ABI.  Inputs are resident in HBM before the timed region;
before every timed step the MPI is reset from a pristine copy and L2 is flushed by
writing a 512 MB buffer (both outside the step's CUDA events).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (a bounded
sample per step, on the host cores).  Under torchrun every rank refines its own scene
(independent problems, no collective on the data path) and rank 0 reports the aggregate.

``--stage volume`` times instead the sparsified gradient volume of Sec. 3.3 at the three
levels of the schedule (one step = three volumes), and ``--stage lgd`` the learned HSGD
refinement (one step = one learned iteration at each of the three levels: volume, tensor-core
network, restore update), each with the roofline of its dominant kernel.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MPI refinements/s and HBM GB/s at 512x384 D=32; p50/p99 serve latency"
UNIT = "refinements/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper", choices=["paper", "paper_bf16", "display", "small", "serve"])
    ap.add_argument("--requests", type=int, default=2000, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--slots", type=int, default=8, help="serve: concurrent request slots")
    ap.add_argument("--arena-gb", type=float, default=24.0, help="serve: device memory arena (GB)")
    ap.add_argument("--graphs", action="store_true", help="serve: replay captured CUDA graphs")
    ap.add_argument("--serve-mode", choices=["batched", "streams"], default="streams",
                    help="serve: one batched launch per stage for all active requests, or a stream per slot")
    ap.add_argument("--lanes", type=int, default=2, help="serve, batched: size classes batched separately")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--direct", action="store_true",
                    help="launch the step's kernels directly instead of replaying a CUDA graph of the step "
                         "(graph replay measured 3%% faster: 0.608 against 0.628 ms per step)")
    ap.add_argument("--trace-every", type=int, default=10,
                    help="record per-kernel CUDA events on every E-th timed step only (each kernel boundary "
                         "with events costs about 2 us of device time); kernel durations and the roofline "
                         "come from those steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="paper workload: skip the BF16, display and serving keys of the default line")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-quality", action="store_true", help="skip the PSNR / SSIM / kept-mass report")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--stage", choices=["hsgd", "volume", "lgd"], default="hsgd",
                    help="hsgd: refinement + renders (default); volume: gradient volumes; lgd: learned refinement")
    ap.add_argument("--kernel-path", type=int, default=0,
                    help="warp-kernel family: 0 automatic, 2 per-pixel gather, 3-5 plane-parallel (3 and 5: 8 warps a "
                         "block, 4: 4 warps where D <= 32)")
    args = ap.parse_args()
    args.graph = not args.direct
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def csrc_digest() -> str:
    """Digest of everything that decides the compiled kernels: every file of the CUDA sources,
    the public header and the build script (its nvcc flags).  A stored ncu counter is used only
    while it matches."""
    paths = sorted(glob.glob(os.path.join(ROOT, "paper_2307_03017_gb300", "csrc", "*")))
    paths += sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
    paths.append(os.path.join(ROOT, "paper_2307_03017_gb300", "build.py"))
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def stored_traffic(key: str):
    """ncu DRAM bytes per launch of a kernel (profiles/traffic.json), or None once any kernel
    source, the header or the build flags differ from those the counters were taken on."""
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tf):
        return None
    try:
        tr = json.load(open(tf)).get(key)
        if tr and tr.get("csrc_digest") == csrc_digest():
            return tr["dram_bytes_per_launch"]
    except Exception:
        return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        self.first.wait(timeout=3.0)  # the samples cover the timed region from its start

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- workload

def load_scene(name: str, seed: int):
    import scenegen as sg
    sc, cfg = sg.workload(name, seed)
    return sc, cfg


def k3_algorithmic_bytes(cfg, sc, level: int, elt: int) -> int:
    """Minimal DRAM bytes of one fused warp/composite/adjoint launch at `level`:
    read the level MPI once, the level source images once (the full-resolution images at
    level 0; the pyramid pass writes the coarser ones), the selection mask once, write the
    compact gradient once."""
    h, w = sc.H >> level, sc.W >> level
    return (sc.D * h * w * 4 * elt + cfg["N"] * h * w * 3 * 4 + h * w * 8 + cfg["k"] * h * w * 16)


RENDER_VIEWS_PER_LAUNCH = 16  # RL_MAX_VIEWS: target views per render launch


def render_algorithmic_bytes(sc, elt: int, n_views: int) -> int:
    """Minimal DRAM bytes of rendering n_views: the MPI read once per launch of up to 16
    views (their blocks share it through L2) and every view's RGB output written once."""
    Mb = sc.D * sc.H * sc.W * 4 * elt
    launches = -(-n_views // RENDER_VIEWS_PER_LAUNCH)
    return launches * Mb + n_views * sc.H * sc.W * 12


def step_algorithmic_bytes(cfg, sc, elt: int) -> int:
    """Minimal DRAM bytes of one step: per level-l iteration read M (select / pyramid),
    write M_l and read the full-resolution images and write the level images (l > 0), the
    fused kernel's traffic, read-modify-write the kept k/D of M; then the renders."""
    Mb = sc.D * sc.H * sc.W * 4 * elt
    Ib = cfg["N"] * sc.H * sc.W * 3 * 4
    tot = 0
    for l in cfg["schedule"]:
        tot += Mb + ((Mb >> (2 * l)) + Ib + (Ib >> (2 * l)) if l else 0) + k3_algorithmic_bytes(cfg, sc, l, elt) \
            + 2 * cfg["k"] * Mb // sc.D
    return tot + render_algorithmic_bytes(sc, elt, len(sc.novel))


def kernel_algorithmic_bytes(cfg, sc, elt: int) -> dict:
    """Minimal DRAM bytes per step of each kernel family of the step (the trace names' prefixes):
    the fused gradient (all levels), the renders, the coarse pyramid + selection passes (read M
    and the full-resolution images, write M_l, the level images, S, the slot map and the zeroed
    compact gradient), the level-0 selection (read M, write S, the slot map and the zeroed compact
    gradient) and the masked updates (read-modify-write the kept k/D of M, read G_s and S)."""
    Mb = sc.D * sc.H * sc.W * 4 * elt
    Ib = cfg["N"] * sc.H * sc.W * 3 * 4
    k, D = cfg["k"], sc.D
    out = {"grad": 0, "render": render_algorithmic_bytes(sc, elt, len(sc.novel)), "pyramid_select": 0, "select": 0,
           "update": 0}
    for l in cfg["schedule"]:
        hw = (sc.H >> l) * (sc.W >> l)
        out["grad"] += k3_algorithmic_bytes(cfg, sc, l, elt)
        sel = k * hw + D * hw + 16 * k * hw
        if l:
            out["pyramid_select"] += Mb + (Mb >> (2 * l)) + Ib + (Ib >> (2 * l)) + sel
        else:
            out["select"] += Mb + sel
        out["update"] += 2 * k * Mb // D + 16 * k * hw + k * hw
    return out


def run_ours(args, world, rank, local):
    import torch
    import paper_2307_03017_gb300 as rl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rl.reallife_set_kernel_path(args.kernel_path)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sc, cfg = load_scene(args.workload, args.seed + rank)
    dtype = torch.bfloat16 if cfg["dtype"] == "bf16" else torch.float32
    elt = 2 if dtype == torch.bfloat16 else 4
    k, sched = cfg["k"], tuple(cfg["schedule"])
    N = len(sc.src)
    M0 = torch.from_numpy(sc.coarse_mpi).to(dev).to(dtype).contiguous()
    M = M0.clone()
    images = torch.from_numpy(sc.images).to(dev)
    mpi = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    ws = rl.workspace(N, sc.D, sc.H, sc.W, k, dtype, dev)
    out = torch.empty((len(sc.novel), sc.H, sc.W, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(len(sched), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rl.reallife_refine(mpi, images, sc.src, k, sched, loss_per_iter=loss, ws=ws)
        rl.reallife_render(mpi, sc.novel, out=out)

    for _ in range(max(args.warmup, 1 if args.graph else 0)):  # kernels load before any capture
        M.copy_(M0)
        step()
    torch.cuda.synchronize()

    every = max(1, args.trace_every)
    traced = lambda i: i % every == 0  # steps whose kernels are bracketed by CUDA events
    n_traced = sum(1 for i in range(args.steps) if traced(i))
    graph = graph_plain = None
    capture_error = None
    if args.graph:
        # one step captured as a CUDA graph with the tracer's event nodes around each kernel, and
        # one without them for the untraced steps.  Only this thread's CUDA calls are checked
        # during capture (other threads of the process, such as a process group's watchdog, may
        # keep polling); should capture fail all the same, the steps are launched directly.
        try:
            rl.reallife_trace_enable(True)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, capture_error_mode="thread_local"):
                step()
            rl.reallife_trace_enable(False)
            graph_plain = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph_plain, capture_error_mode="thread_local"):
                step()
            rl.reallife_trace_read()
            for g in (graph, graph_plain):  # first replays (untimed)
                M.copy_(M0)
                g.replay()
            torch.cuda.synchronize()
            rl.reallife_trace_read()
        except Exception as e:  # noqa: BLE001 -- any capture failure falls back to direct launches
            rl.reallife_trace_enable(False)
            graph = graph_plain = None
            capture_error = (str(e).splitlines() or [type(e).__name__])[0][:200]
            torch.cuda.synchronize()
            rl.reallife_trace_read()
            rl.reallife_trace_release_captured()

    clocks = ClockSampler(local) if not args.no_clocks else None
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    trace = {}

    def add_trace(tr):
        for name, (n, ms) in tr.items():
            c, t = trace.get(name, (0, 0.0))
            trace[name] = (c + n, t + ms)

    rl.reallife_trace_read()  # reset counters
    for i in range(args.steps):
        M.copy_(M0)  # reset and L2 flush are not part of the step
        flush.fill_(i & 0xFF)
        if graph is not None:
            starts[i].record(stream)
            (graph if traced(i) else graph_plain).replay()
            stops[i].record(stream)
            if traced(i):
                torch.cuda.synchronize()
                add_trace(rl.reallife_trace_read())  # this replay's kernel durations
        else:
            rl.reallife_trace_enable(traced(i))
            starts[i].record(stream)
            step()
            stops[i].record(stream)
            rl.reallife_trace_enable(False)
    torch.cuda.synchronize()
    if graph is None:
        add_trace(rl.reallife_trace_read())
    clk = clocks.stop() if clocks else None
    ms_steps = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    total_ms = reduce_max(sum(ms_steps), dist, dev)
    if dist:
        dist.barrier()
    value = world * args.steps / (total_ms / 1e3)

    # dominant kernel: roofline from its live CUDA-event durations on the traced steps of the
    # timed region; every step launches the same kernels, so the launch count scales by steps
    launches = sum(v[0] for v in trace.values()) * args.steps // n_traced
    dom = max(trace.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_n, dom_ms) = dom
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    peak_gbs, peak_src = (peaks["hbm_gbs"], "measured") if "hbm_gbs" in peaks else (6800.0, "fallback")
    if dom_name.startswith("grad"):
        per_step = sum(k3_algorithmic_bytes(cfg, sc, l, elt) for l in sched)
        alg_bytes = per_step * n_traced
    elif dom_name.startswith("render"):
        alg_bytes = n_traced * render_algorithmic_bytes(sc, elt, len(sc.novel))
    else:
        alg_bytes = None
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9 if alg_bytes else None
    traffic = stored_traffic(f"{args.workload}:{dom_name}")
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1) if achieved else None,
                "peak": peak_gbs, "unit": "GB/s", "frac": round(achieved / peak_gbs, 4) if achieved else None,
                "traffic": traffic, "alg_bytes_per_launch": int(alg_bytes / dom_n) if alg_bytes else None,
                "avg_launch_us": round(dom_ms / dom_n * 1e3, 2), "peak_source": peak_src}
    step_bytes = step_algorithmic_bytes(cfg, sc, elt)
    kernels = {n: {"launches": c, "ms_per_step": round(t / n_traced, 4)} for n, (c, t) in sorted(trace.items())}
    # per-kernel useful bandwidth: algorithmic bytes per step over the traced steps' time
    fam_bytes = kernel_algorithmic_bytes(cfg, sc, elt)
    for n, kd in kernels.items():
        fam = next((f for f in ("pyramid_select", "select", "grad", "render", "update") if n.startswith(f)), None)
        if fam and kd["ms_per_step"] > 0:
            gbs = fam_bytes[fam] / (kd["ms_per_step"] / 1e3) / 1e9
            kd["alg_gbs"] = round(gbs, 1)
            kd["alg_frac"] = round(gbs / peak_gbs, 4)
    render_ms = sum(kd["ms_per_step"] for n, kd in kernels.items() if n.startswith("render"))
    render_views_per_s = round(len(sc.novel) / (render_ms / 1e3), 1) if render_ms > 0 else None

    qual = None
    if rank == 0 and args.workload in ("paper", "paper_bf16", "small") and not args.no_quality:
        qual = quality(rl, sc, k, sched, M0, mpi, out, loss, dev)

    launch_mode = "CUDA graph replay of the step" if graph is not None else (
        f"direct (graph capture failed: {capture_error})" if capture_error else "direct")
    if graph is not None:
        del graph, graph_plain
        torch.cuda.synchronize()
        rl.reallife_trace_release_captured()
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, rl, sc, cfg, dtype, dev, world, dist)

    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            # the arithmetic is FP32 for either storage type (BF16 values are widened on load)
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ray-cast layered scenes; no dataset)",
            "config": {"workload": f"{args.workload}: {sc.W}x{sc.H} D={sc.D} N={N} k={k} levels={list(sched)} "
                                   f"+ {len(sc.novel)} novel views", "storage": cfg["dtype"],
                       "kernel_path": args.kernel_path,
                       "launch": launch_mode,
                       "trace": f"per-kernel CUDA events on {n_traced} of the {args.steps} timed steps (every "
                                f"{every}th); kernels' ms_per_step and launches are theirs",
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas{world}"},
            "hbm_gbs_step": round(step_bytes / (total_ms / args.steps / 1e3) / 1e9, 1),
            "render_views_per_s": render_views_per_s,
            "roofline": roofline, "kernels": kernels, "gpu_launches": int(launches),
            "clocks": clk, "e2e": e2e,
        }
        if qual is not None:
            result["quality"] = qual
    if dist:
        dist.destroy_process_group()
    return result


def quality(rl, sc, k, sched, M0, mpi, out, loss, dev) -> dict:
    """Render quality of the coarse and the refined MPI on the novel views against noise-free
    ray casts of the scene (PSNR, SSIM), the share of the reference view's alpha weight that
    the level-0 top-k selection keeps, and the loss of each iteration of the last refinement.
    Runs after the timed region on the refined MPI that the last step left."""
    import numpy as np
    import scenegen as sg
    import torch
    truth = np.stack([sg.raycast(sc.layers, sc.ref.K, c, sc.H, sc.W)[0] for c in sc.novel]).astype(np.float32)
    truth = torch.from_numpy(truth).to(dev)
    coarse = rl.make_mpi(M0, sc.near, sc.far, sc.ref)
    res = {}
    for name, m, r in (("coarse", coarse, rl.reallife_render(coarse, sc.novel)), ("refined", mpi, out)):
        q = rl.reallife_image_metrics(r, truth).cpu().tolist()
        _, mask = rl.reallife_select(m, k)
        km = rl.reallife_kept_mass(m, mask).cpu().tolist()
        res[name] = {"psnr_db": round(10.0 * math.log10(1.0 / q[0]), 3), "ssim": round(q[1], 5),
                     "kept_mass": round(km[0] / km[1], 5)}
    res["loss_per_iteration"] = [round(v, 6) for v in loss.cpu().tolist()]
    res["levels"] = list(sched)
    res["reference"] = (f"{len(sc.novel)} novel views against noise-free ray casts of the scene; SSIM 11x11 "
                        "Gaussian window (sigma 1.5); kept mass = top-k alpha weight / all alpha weight at level 0")
    return res


def volume_kernel_bytes(sc, k: int, level: int, elt: int) -> dict:
    """Algorithmic bytes per launch of the gradient-volume kernels at one level."""
    N, D = len(sc.src), sc.D
    h, w = sc.H >> level, sc.W >> level
    hw = h * w
    return {
        # read the level MPI once, write the view alpha weights
        "view_alpha": D * hw * 4 * elt + N * D * hw * 4,
        # write V, read S, the kept voxels of M_l, one alpha-weight sample and the images once
        "volume": (4 * N + 4) * k * hw * 4 + k * hw + k * hw * 4 * elt + N * k * hw * 4 + N * sc.H * sc.W * 12,
    }


def lgd_conv_flops(k: int, h: int, w: int) -> int:
    """FLOPs of one 3x3x3, 32 -> 32 channel block over k x h x w voxels."""
    return 2 * k * h * w * 27 * 32 * 32


def lgd_net_flops(k: int, h: int, w: int, c_in: int) -> int:
    """Algorithmic FLOPs of the whole network over k x h x w voxels: the first 3x3x3 block from
    the volume's c_in channels, four 32 -> 32 blocks and the 1x1x1 layer to 4 channels."""
    vox = k * h * w
    return 2 * vox * 27 * 32 * c_in + 4 * lgd_conv_flops(k, h, w) + 2 * vox * 32 * 4


def run_stage(args, world, rank, local):
    """Timed steps of the gradient volume (--stage volume) or the learned refinement (--stage lgd)."""
    import torch
    import paper_2307_03017_gb300 as rl
    import scenegen as sg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sc, cfg = load_scene(args.workload, args.seed + rank)
    dtype = torch.bfloat16 if cfg["dtype"] == "bf16" else torch.float32
    elt = 2 if dtype == torch.bfloat16 else 4
    k, sched = cfg["k"], tuple(cfg["schedule"])
    N = len(sc.src)
    M0 = torch.from_numpy(sc.coarse_mpi).to(dev).to(dtype).contiguous()
    M = M0.clone()
    images = torch.from_numpy(sc.images).to(dev)
    mpi = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    if args.stage == "volume":
        ws = torch.empty(rl.reallife_gradient_volume_workspace_bytes(N, sc.D, sc.H, sc.W, k, dtype), dtype=torch.uint8,
                         device=dev)
        Vs = {l: torch.empty((4 * N + 4, k, sc.H >> l, sc.W >> l), device=dev) for l in sched}
        Ss = {l: torch.empty((k, sc.H >> l, sc.W >> l), dtype=torch.uint8, device=dev) for l in sched}

        def step():
            for l in sched:
                rl.reallife_gradient_volume(mpi, images, sc.src, k, l, V=Vs[l], S_out=Ss[l], ws=ws)
        metric = "gradient volumes/s (Sec. 3.3 V_s at levels 2, 1, 0) at 512x384 D=32"
        unit = "volume sets/s"
    else:
        net = rl.LgdNet(sg.lgd_weights(args.seed, 4 * N + 4), device=dev)
        ws = torch.empty(rl.reallife_lgd_step_workspace_bytes(N, sc.D, sc.H, sc.W, k, dtype), dtype=torch.uint8,
                         device=dev)

        def step():
            for l in sched:
                rl.reallife_lgd_step(mpi, images, sc.src, k, net, level=l, ws=ws)
        metric = "learned MPI refinements/s (Sec. 3.3 learned update at levels 2, 1, 0) at 512x384 D=32"
        unit = "learned refinements/s"

    for _ in range(args.warmup):
        M.copy_(M0)
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if not args.no_clocks else None
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    every = max(1, args.trace_every)
    n_traced = sum(1 for i in range(args.steps) if i % every == 0)
    rl.reallife_trace_read()
    for i in range(args.steps):
        M.copy_(M0)
        flush.fill_(i & 0xFF)
        rl.reallife_trace_enable(i % every == 0)
        starts[i].record(stream)
        step()
        stops[i].record(stream)
        rl.reallife_trace_enable(False)
    torch.cuda.synchronize()
    trace = rl.reallife_trace_read()
    clk = clocks.stop() if clocks else None
    total_ms = reduce_max(sum(a.elapsed_time(b) for a, b in zip(starts, stops)), dist, dev)
    if dist:
        dist.barrier()
    value = world * args.steps / (total_ms / 1e3)
    assert rl.reallife_device_status(clear=True) == 0
    launches = sum(v[0] for v in trace.values()) * args.steps // n_traced
    dom_name, (dom_n, dom_ms) = max(trace.items(), key=lambda kv: kv[1][1])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    if args.stage == "lgd" and dom_name.startswith("lgd_conv"):
        # one launch runs the whole network of a level
        flops = n_traced * sum(lgd_net_flops(k, sc.H >> l, sc.W >> l, 4 * len(sc.src) + 4) for l in sched)
        achieved = flops / (dom_ms / 1e3) / 1e12
        peak, src = (peaks["bf16_tflops"], "measured (burst)") if "bf16_tflops" in peaks else (1900.0, "fallback")
        roofline = {"bound": "tensor", "kernel": dom_name, "achieved": round(achieved, 1), "peak": peak,
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": stored_traffic(f"{args.workload}:{dom_name}"),
                    "alg_flops_per_launch": int(flops / dom_n), "avg_launch_us": round(dom_ms / dom_n * 1e3, 2),
                    "peak_source": src}
    else:
        key = "volume" if dom_name.startswith("volume") else ("view_alpha" if dom_name.startswith("view_alpha")
                                                              else None)
        alg = n_traced * sum(volume_kernel_bytes(sc, k, l, elt)[key] for l in sched) if key else None
        achieved = alg / (dom_ms / 1e3) / 1e9 if alg else None
        peak, src = (peaks["hbm_gbs"], "measured") if "hbm_gbs" in peaks else (6800.0, "fallback")
        roofline = {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1) if achieved else None,
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
                    "traffic": stored_traffic(f"{args.workload}:{dom_name}"),
                    "alg_bytes_per_launch": int(alg / dom_n) if alg else None,
                    "avg_launch_us": round(dom_ms / dom_n * 1e3, 2), "peak_source": src}
    kernels = {n: {"launches": c, "ms_per_step": round(t / n_traced, 4)} for n, (c, t) in sorted(trace.items())}
    result = None
    if rank == 0:
        result = {
            "metric": metric, "value": round(value, 3), "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            # the network multiplies BF16 operands (FP32 accumulation); everything else is FP32
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.stage == "lgd" else "f32",
            "data": "synthetic (seeded ray-cast layered scenes; random network weights; no dataset)",
            "config": {"workload": f"{args.workload}: {sc.W}x{sc.H} D={sc.D} N={N} k={k} levels={list(sched)}",
                       "stage": args.stage, "storage": cfg["dtype"],
                       "network": "5 x (3x3x3 conv 32 ch + BN + ReLU) + 1x1x1, BF16 on tcgen05"
                       if args.stage == "lgd" else None,
                       "trace": f"per-kernel CUDA events on {n_traced} of the {args.steps} timed steps (every "
                                f"{every}th); kernels' ms_per_step and launches are theirs",
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas{world}"},
            "roofline": roofline, "kernels": kernels, "gpu_launches": int(launches), "clocks": clk, "e2e": None,
        }
    if dist:
        dist.destroy_process_group()
    return result


def cpu_baseline_stage(sc, cfg, stage: str, seed: int) -> dict:
    """The FP64 oracle on the coarsest level of the stage's step, scaled by that level's share of
    the step's pixels (levels 2, 1, 0 hold 1/21, 4/21 and 16/21 of them)."""
    import oracle
    from oracle import lgd as olgd
    import scenegen as sg
    oracle.build()
    k, sched = cfg["k"], tuple(cfg["schedule"])
    lvl = max(sched)
    share = (1 << (2 * (max(sched) - lvl))) / sum(1 << (2 * (max(sched) - l)) for l in sched)
    t0 = time.perf_counter()
    if stage == "volume":
        oracle.gradient_volume(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k, lvl)
    else:
        olgd.lgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images,
                      sg.lgd_weights(seed, 4 * len(sc.src) + 4), k, lvl)
    dt = time.perf_counter() - t0
    return {"value": round(share / dt, 5), "unit": "volume sets/s" if stage == "volume" else "learned refinements/s",
            "cores": 1, "kind": "oracle",
            "sample": f"the level-{lvl} {'gradient volume' if stage == 'volume' else 'learned iteration'} of one step "
                      f"({share:.4f} of the step's pixels), FP64, single thread, {dt:.2f} s; value scaled by the "
                      f"pixel share", "cpu": platform_cpu()}


def run_e2e(args, rl, sc, cfg, dtype, dev, world, dist):
    """Same metric through the public API from pinned host memory: H2D of the coarse MPI and
    the source images, refine + render, D2H of the rendered views, every step.  Successive
    steps are pipelined as a caller streaming reconstructions would run them: two device
    buffer sets, the copies in and out on their own streams, so that step i+1's inputs travel
    while step i computes.  The timed region runs from the first copy in to the last copy out."""
    import torch
    k, sched = cfg["k"], tuple(cfg["schedule"])
    N = len(sc.src)
    h_M = torch.from_numpy(sc.coarse_mpi).to(dtype).pin_memory()
    h_I = torch.from_numpy(sc.images).pin_memory()
    h_out = [torch.empty((len(sc.novel), sc.H, sc.W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    M = [torch.empty_like(h_M, device=dev) for _ in range(2)]
    images = [torch.empty_like(h_I, device=dev) for _ in range(2)]
    out = [torch.empty_like(h_out[0], device=dev) for _ in range(2)]
    ws = rl.workspace(N, sc.D, sc.H, sc.W, k, dtype, dev)  # the compute stream runs one step at a time
    mpi = [rl.make_mpi(M[b], sc.near, sc.far, sc.ref) for b in range(2)]
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def step(i):
        b = i & 1
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_comp[b])  # step i-2 is done with this buffer set
            M[b].copy_(h_M, non_blocking=True)
            images[b].copy_(h_I, non_blocking=True)
            ev_in[b].record(s_in)
        comp.wait_event(ev_in[b])
        comp.wait_event(ev_out[b])  # step i-2's views have left
        rl.reallife_refine(mpi[b], images[b], sc.src, k, sched, ws=ws)
        rl.reallife_render(mpi[b], sc.novel, out=out[b])
        ev_comp[b].record(comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[b])
            h_out[b].copy_(out[b], non_blocking=True)
            ev_out[b].record(s_out)

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    s_in.wait_event(a)
    s_out.wait_event(a)
    for i in range(args.steps):
        step(i)
    comp.wait_event(ev_out[(args.steps - 1) & 1])
    comp.wait_event(ev_out[args.steps & 1])
    e.record(comp)
    torch.cuda.synchronize()
    ms = reduce_max(a.elapsed_time(e), dist, dev)
    return {"value": round(world * args.steps / (ms / 1e3), 3), "unit": UNIT,
            "h2d_bytes_per_step": int(h_M.numel() * h_M.element_size() + h_I.numel() * 4),
            "d2h_bytes_per_step": int(h_out[0].numel() * 4),
            "pipelined": "two buffer sets; copies in and out on their own streams"}


# ----------------------------------------------------------------------- serving

SERVE_RES = [(192, 256), (384, 512), (576, 768), (768, 1024)]
SERVE_D = [16, 32, 48, 64]


def _serve_scene(args):
    import scenegen as sg
    seed, H, W, D, n_views = args
    sc = sg.make_scene(seed, H, W, D, n_views, n_layers=(3, 8), novel="none")
    return (H, W, D), sc


def serve_scene_pool(seed: int = 7, n_views: int = 6):
    """One seeded scene per (resolution, D) of the serving workload, with 6 source views
    (requests with fewer views use the first N), coarse MPI BF16 in pinned host memory.  The
    scenes are drawn in parallel processes (spawned: safe beside a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    jobs = []
    for (H, W) in SERVE_RES:
        for D in SERVE_D:
            jobs.append((seed + len(jobs), H, W, D, n_views))
    workers = max(1, min(len(jobs), len(os.sched_getaffinity(0))))
    pool = {}
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for key, sc in ex.map(_serve_scene, jobs):
            M = torch.from_numpy(sc.coarse_mpi).to(torch.bfloat16).pin_memory()
            I = torch.from_numpy(sc.images).pin_memory()
            sc.coarse_mpi = None  # host copy no longer needed
            pool[key] = (sc, M, I)
    return pool


def serve_requests_from_pool(pool, draws):
    from paper_2307_03017_gb300.serve import Request
    out = []
    for r in draws:
        sc, M, I = pool[(r["H"], r["W"], r["D"])]
        N = r["N"]
        out.append(Request(id=r["id"], arrival=r["arrival"], coarse=M, images=I[:N], ref=sc.ref, src=sc.src[:N],
                           near=sc.near, far=sc.far, schedule=(2, 1, 0) if r["iters"] == 3 else (2, 0), k=5))
    return out


def run_serve(args, world, rank, local, pool=None):
    import torch
    import scenegen as sg
    from paper_2307_03017_gb300.serve import ServeEngine, latency_stats
    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    if pool is None:
        pool = serve_scene_pool()
    t_gen = time.perf_counter() - t_gen
    draws = sg.serve_requests(args.requests, args.rate, seed=12345)
    max_elems = max(M.numel() for (_, M, _) in pool.values())
    eng = ServeEngine(int(args.arena_gb * (1 << 30)), max_slots=args.slots, graphs=args.graphs,
                      max_result_elems=max_elems, batched=args.serve_mode == "batched", lanes=args.lanes)
    # warm-up: one request of every (resolution, D) so first-use costs stay out of the run
    warm = serve_requests_from_pool(pool, [dict(id=-1, arrival=0.0, H=H, W=W, D=D, N=4, iters=3)
                                           for (H, W) in SERVE_RES for D in SERVE_D])
    eng.run(warm, realtime=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if not args.no_clocks else None
    if clocks:
        clocks.start()
    done = eng.run(serve_requests_from_pool(pool, draws), realtime=True)
    poisson = latency_stats(done)
    closed = latency_stats(eng.run(serve_requests_from_pool(pool, draws[: max(1, args.requests // 4)]),
                                   realtime=False))
    clk = clocks.stop() if clocks else None
    mean_px = float(np.mean([d["H"] * d["W"] for d in draws]))
    return {
        "metric": "p50/p99 serve latency and reconstructions/s (Poisson arrivals, BF16 MPIs)",
        "value": round(poisson["p99_ms"], 3), "unit": "ms (p99 latency)", "higher_is_better": False,
        "n_gpus": world, "p50_ms": round(poisson["p50_ms"], 3), "p99_ms": round(poisson["p99_ms"], 3),
        "mean_ms": round(poisson["mean_ms"], 3), "max_ms": round(poisson["max_ms"], 3),
        "queue_p50_ms": round(poisson["queue_p50_ms"], 3), "queue_p99_ms": round(poisson["queue_p99_ms"], 3),
        "reconstructions_per_s": round(poisson["reconstructions_per_s"], 2),
        "closed_loop_reconstructions_per_s": round(closed["reconstructions_per_s"], 2),
        "dtype": "f32", "data": "synthetic (seeded ray-cast layered scenes; no dataset)",
        "config": {"workload": f"serve: {args.requests} requests, Poisson {args.rate}/s, res in {SERVE_RES}, "
                               f"D in {SERVE_D}, N 2-6, 2-3 iterations, k=5, BF16",
                   "storage": "bf16", "slots": args.slots, "arena_gb": args.arena_gb, "graphs": bool(args.graphs),
                   "mode": args.serve_mode, "lanes": args.lanes if args.serve_mode == "batched" else None,
                   "latency": "arrival -> refined MPI and losses on the host (queueing, H2D, compute, D2H)",
                   "mean_pixels": mean_px, "scene_pool_s": round(t_gen, 1)},
        "graph_captures": eng.captures, "graph_replays": eng.replays, "clocks": clk,
        "batched_steps": eng.steps, "max_requests_per_step": eng.max_items_per_step,
    }


# ------------------------------------------------------------------- CPU oracle

def crop_scene(sc, rows: int):
    """Rows [y0, y0 + rows) of the scene (MPI, images, cameras with the principal point
    shifted): the same problem on a horizontal band, for bounded CPU samples."""
    import copy
    import scenegen as sg
    y0 = ((sc.H - rows) // 2) & ~7
    out = copy.copy(sc)
    out.H = rows
    out.coarse_mpi = np.ascontiguousarray(sc.coarse_mpi[:, y0:y0 + rows])
    out.images = np.ascontiguousarray(sc.images[:, y0:y0 + rows])

    def shift(c):
        K = c.K.copy()
        K[1, 2] -= y0
        return sg.Camera(K, c.R, c.t)
    out.ref = shift(sc.ref)
    out.src = [shift(c) for c in sc.src]
    out.novel = [shift(c) for c in sc.novel]
    return out


def oracle_step(sc, cfg):
    import oracle
    M, _, _ = oracle.refine(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, cfg["k"],
                            tuple(cfg["schedule"]))
    for cam in sc.novel:
        oracle.render(M, sc.near, sc.far, sc.ref, cam)


def sample_rows(sc, frac: float) -> int:
    """Band height for a CPU sample: about frac of the rows, a multiple of 8 (pyramid levels)."""
    return max(8, int(sc.H * frac) // 8 * 8)


BASELINE_BAND = 1.0 / 8.0  # share of the rows the oracle's samples take (both legs)


def cpu_baseline(sc, cfg, frac: float = BASELINE_BAND) -> dict:
    """The FP64 oracle as it stands on one step of a band of the same workload (1/8 of its rows,
    the reference arm's band), timed single-threaded and on all the host cores this process may
    use (the OpenMP build, bit-identical results), scaled to refinements/s by the band's share of
    pixels.  ``value`` is the all-core figure."""
    import oracle
    oracle.build()
    rows = sample_rows(sc, frac)
    band = crop_scene(sc, rows)
    share = rows / sc.H
    out = {}
    for threads in (False, True):
        oracle.set_threads(threads)
        n = oracle.num_threads()
        t0 = time.perf_counter()
        oracle_step(band, cfg)
        out[threads] = (time.perf_counter() - t0, n)
    oracle.set_threads(False)
    (t1, _), (tn, n) = out[False], out[True]
    return {"value": round(share / tn, 5), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"one step ({len(cfg['schedule'])}-level refine + {len(sc.novel)} renders) on a {sc.W}x{rows} "
                      f"band ({share:.3f} of the pixels) of the same scene, FP64, OpenMP on {n} cores, {tn:.2f} s; "
                      f"value scaled by the pixel share",
            "single_thread": {"value": round(share / t1, 5), "cores": 1, "seconds": round(t1, 2)},
            "cpu": platform_cpu()}


def platform_cpu() -> str:
    try:
        import platform
        m = platform.processor() or platform.machine()
        if os.path.exists("/proc/cpuinfo"):
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    return f"{platform.machine()} {ln.split(':', 1)[1].strip()}"
        return m
    except Exception:
        return "unknown"


def reference_band_rows(H: int, unit: int, t_unit: float, n_steps: int, budget_s: float = 120.0) -> int:
    """Rows of the reference arm's band: the CPU-baseline band (1/8 of the H rows, a multiple of 8),
    or fewer (a multiple of `unit`, the coarsest level's block, at least one unit) when n_steps
    steps of t_unit seconds per unit of rows would exceed budget_s."""
    units = int(budget_s / max(1, n_steps) / max(t_unit, 1e-6))
    cap = max(1, (max(8, int(H * BASELINE_BAND) // 8 * 8)) // unit)
    return unit * max(1, min(cap, units))


def run_reference(args, world, rank):
    """The oracle on the host cores (the OpenMP build on every core this process may use), each
    step a horizontal band of the workload scaled by its share of the pixels: the CPU-baseline
    band of 1/8 of the rows, unless an untimed calibration step on a 4-row band (the least height
    the coarsest pyramid level allows) shows that the warm-up and timed steps would take more
    than about two minutes, in which case the band is narrowed to fit."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    oracle.set_threads(True)
    cores = oracle.num_threads()
    sc, cfg = load_scene(args.workload, args.seed)
    unit = 1 << max(cfg["schedule"])
    t0 = time.perf_counter()
    oracle_step(crop_scene(sc, unit), cfg)
    rows = reference_band_rows(sc.H, unit, time.perf_counter() - t0, args.steps + args.warmup)
    band = crop_scene(sc, rows)
    share = rows / sc.H
    for _ in range(args.warmup):
        oracle_step(band, cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(band, cfg)
    dt = time.perf_counter() - t0
    v = share * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ray-cast layered scenes; no dataset)",
            "config": {"workload": f"{args.workload}: {sc.W}x{sc.H} D={sc.D} N={len(sc.src)} k={cfg['k']} "
                                   f"levels={list(cfg['schedule'])} + {len(sc.novel)} novel views"},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step = one step on a {sc.W}x{rows} band ({share:.3f} of the pixels) "
                                       f"of the workload, FP64 oracle, OpenMP on {cores} cores; value scaled by "
                                       f"the share",
                             "cpu": platform_cpu()},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _summary(r: dict) -> dict:
    """The keys of a secondary workload's line that the default line carries."""
    keep = ("value", "unit", "ms_per_step", "steps", "dtype", "config", "roofline", "kernels", "gpu_launches",
            "hbm_gbs_step", "render_views_per_s", "e2e", "quality")
    return {k: r[k] for k in keep if k in r}


def run_extras(args, world, rank, local) -> dict:
    """The default line's secondary keys: the same step with BF16 storage, the 1920x1080 display
    workload and the serving stream (shortened; per-stream and batched engines)."""
    import copy
    out = {}
    a = copy.copy(args)
    a.no_clocks = True
    a.workload = "paper_bf16"
    out["bf16"] = _summary(run_ours(a, world, rank, local))
    a = copy.copy(args)
    a.no_clocks = True
    a.workload = "display"
    a.steps = max(20, min(args.steps, 50))
    a.warmup = max(3, min(args.warmup, 5))
    out["display"] = _summary(run_ours(a, world, rank, local))
    a = copy.copy(args)
    a.no_clocks = True
    a.requests = min(args.requests, 500)
    pool = serve_scene_pool()
    serve = {}
    for mode in ("streams", "batched"):
        a.serve_mode = mode
        r = run_serve(a, world, rank, local, pool=pool)
        serve[mode] = {k: r[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "queue_p50_ms", "queue_p99_ms",
                                         "reconstructions_per_s", "closed_loop_reconstructions_per_s",
                                         "batched_steps", "max_requests_per_step")}
    serve["config"] = r["config"]["workload"]
    serve["unit"] = "ms (latency), reconstructions/s"
    out["serve"] = serve
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload == "serve":
        res = run_serve(args, world, rank, local) if rank == 0 else None
    elif args.stage != "hsgd":
        res = run_stage(args, world, rank, local)
        if res is not None and not args.no_cpu_baseline and world == 1:
            sc, cfg = load_scene(args.workload, args.seed)
            res["cpu_baseline"] = cpu_baseline_stage(sc, cfg, args.stage, args.seed)
        elif res is not None:
            res["cpu_baseline"] = None
    else:
        res = run_ours(args, world, rank, local)
        if res is not None and not args.no_cpu_baseline and world == 1:
            sc, cfg = load_scene(args.workload, args.seed)
            res["cpu_baseline"] = cpu_baseline(sc, cfg)
        elif res is not None:
            res["cpu_baseline"] = None
        if res is not None and world == 1 and args.workload == "paper" and not args.no_extras:
            res.update(run_extras(args, world, rank, local))
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
