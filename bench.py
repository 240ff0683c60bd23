#!/usr/bin/env python3
"""Benchmark: shortest-path-map throughput (Mpixel/s) on one or more GB300s.

Default workload: the 4096 x 4096 maze (64 x 64 cells, 16-unit walls, one
exit segment + 4 point sources, seed 0). One step = one spm_compute: the
vertex-cost fixpoint, tile culling and the pixel pass for the whole grid, with
the scene already resident in HBM. The L2 is flushed (a 256 MiB write)
between timed steps; each step is timed with CUDA events on the compute
stream. Under torchrun every rank computes its own replica (the path has no
exchange step), so per-GPU work is fixed ("weak" scaling) and value is the
pixels of all ranks over the slowest rank's time.

--impl reference times the CPU FP64 oracle on the host cores instead (a
bounded pixel sample per step, extrapolated to the full grid).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen as sg  # noqa: E402

METRIC = "SPM Mpixel/s at 4096^2"
UNIT = "Mpixel/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP32 lanes per SM x SMs x 2 flops per FMA; clock from the measured peaks file
FP32_LANES, N_SMS = 128, 152
FLOPS_PER_PIXEL = 7  # winning-generator distance: 2 sub, mul, fma(2), sqrt, add
# One pixel-kernel launch per workload, from a single-pass ncu capture of a
# full-size launch (dram__bytes_read.sum + dram__bytes_write.sum,
# smsp__issue_active and the ALU / FMA pipe shares; the first timed step,
# right after the L2 flush) and from the instrumentation build's work
# counters (orientation tests and exact polygon tests per pixel); valid for
# those workloads and that kernel version only (re-captured after a change).
KPIXELS_TRAFFIC = {"maze4096": 104_169_728, "batched256": 1_310_612_480, "polys1024": 6_548_736}
KPIXELS_UTIL = {"maze4096": {"issue_frac": 0.437, "alu_pipe_frac": 0.304, "fma_pipe_frac": 0.131,
                             "orient_per_px": 0.254, "exact_tests_per_px": 0.0636},
                "batched256": {"issue_frac": 0.414, "alu_pipe_frac": 0.289, "fma_pipe_frac": 0.123},
                "polys1024": {"issue_frac": 0.452, "alu_pipe_frac": 0.296, "fma_pipe_frac": 0.117,
                              "orient_per_px": 0.360, "exact_tests_per_px": 0.0611}}


def fixpoint_start(spm, s, args, tuning):
    """--fixpoint-start: where the vertex fixpoint starts (auto, sources, or
    the tree of the scene's table of obstacle-vertex geodesic distances), for
    A/B runs; returns the tuning as the scene now holds it."""
    choice = {"auto": 0, "sources": 1, "tree": 2}[getattr(args, "fixpoint_start", "auto")]
    if choice:
        spm.spm_scene_set_tuning(s.handle, tuning["flood_mode"], tuning["hidden_chunk"], tuning["tile"],
                                 tuning["maps"], fixpoint_start=choice)
    return dict(tuning, **s.tuning())


def workload(name: str):
    if name == "maze4096":
        return sg.maze(0), "maze 64x64 cells, 4096^2 px, 16384^2 world, 1 segment + 4 points"
    if name == "dynamic4096":
        return sg.maze(0), ("maze 64x64 cells, 4096^2 px, 16384^2 world, 1 segment + 4 points moving "
                            "every frame, 100k agents")
    if name == "maze2048":
        return sg.maze(0, cells=32, N=2048), "maze 32x32 cells, 2048^2 px, 8192^2 world, 1 segment + 4 points"
    if name == "batched256":
        return sg.batched(0), "256 scenes, side uniform in {128,256,512,1024} over 4096^2, 10-500 convex polygons, 1-6 point/segment sources"
    if name == "polys1024":
        return sg.plain_polys(0), "200 convex polygons, 1024^2 px, 4096^2 world, 3 points + 2 segments"
    if name == "rects256":
        return sg.plain_rects(0), "8 rectangles, 256^2 px, 256^2 world, 1 point"
    if name == "diff2048":
        return sg.differentiable(0, n_agents=10), "150 convex polygons, 2048^2 px, 8192^2 world"
    if name == "diff2048_grad":
        return sg.differentiable(0), ("150 convex polygons, 2048^2 px, 8192^2 world, 4 FP32 points + "
                                      "1 FP32 segment, 100k agents")
    raise SystemExit(f"unknown workload {name}")


def metric_for(Nx: int, Ny: int) -> str:
    """The headline metric's name, with the workload's own grid."""
    return METRIC if (Nx, Ny) == (4096, 4096) else f"SPM Mpixel/s at {Nx}x{Ny}"


def rank_env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (x itself on one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Units all ranks processed (each rank the same amount) over the slowest rank's time."""
    return world * units_per_rank / slowest_seconds


def shard_lpt(weights, world: int, rank: int):
    """Longest-processing-time-first assignment of items to ranks (heaviest
    item to the least loaded rank, ties to the lower index); the indices of
    this rank's items, in input order."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0.0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += weights[i]
    return [i for i in range(len(weights)) if owner[i] == rank]


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(scene, n_pixels: int, seed: int, nthreads: int):
    """Oracle throughput estimate on the host: vertex phase + a seeded pixel
    sample, extrapolated to the full grid. Returns (Mpixel/s, seconds used)."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(scene, nthreads=nthreads)
    t_build = time.perf_counter() - t0
    Nx, Ny = scene.grid
    rng = np.random.default_rng(seed)
    ij = np.stack([rng.integers(0, Nx, n_pixels), rng.integers(0, Ny, n_pixels)], 1).astype(np.int32)
    t1 = time.perf_counter()
    o.pixels(ij)
    t_pix = time.perf_counter() - t1
    full = t_build + t_pix * (Nx * Ny) / n_pixels
    return (Nx * Ny) / full / 1e6, t_build + t_pix


def _reference_line(args, metric, value, unit, higher, ms_step, config, nthreads, sample):
    return {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": higher,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _oracle_scene_seconds(scene, n_pixels, seed, nthreads):
    """Oracle time for one whole map: vertex phase + a seeded pixel sample,
    extrapolated to the grid."""
    rate, _ = cpu_oracle_rate(scene, n_pixels, seed, nthreads)
    return scene.grid[0] * scene.grid[1] / (rate * 1e6)


def run_reference_other(args, nthreads):
    """The oracle on the workloads that are not a single map per step."""
    import oracle
    steps = range(args.warmup + args.steps)
    if args.workload == "batched256":
        scenes, cfg_desc = workload("batched256")
        k = 8  # scenes sampled per step, extrapolated to the batch
        per_step = []
        for st in steps:
            pick = [scenes[(st * k + i) % len(scenes)] for i in range(k)]
            t = sum(_oracle_scene_seconds(sc, max(1000, args.ref_pixels // k), st, nthreads) for sc in pick)
            per_step.append(t * len(scenes) / k)
        batch_s = float(np.mean(per_step[args.warmup:]))
        value = len(scenes) / batch_s
        return _reference_line(args, "SPM batched scenes/s", value, "scenes/s", True, 1e3 * batch_s,
                               {"workload": args.workload, "scene": cfg_desc}, nthreads,
                               f"per step: {k} of the {len(scenes)} scenes (oracle vertex phase + "
                               f"{max(1000, args.ref_pixels // k)} seeded pixels each, extrapolated to their "
                               f"grids), scaled to the batch")
    if args.workload == "diff2048_grad":
        scene, cfg_desc = workload("diff2048_grad")
        n_ag = 2000  # agents sampled per step, extrapolated to all
        per_step = []
        for st in steps:
            t0 = time.perf_counter()
            o = oracle.Oracle(scene, nthreads=nthreads)
            t_build = time.perf_counter() - t0
            rng = np.random.default_rng(st)
            sub = np.asarray(scene.agents)[rng.integers(0, len(scene.agents), n_ag)]
            t1 = time.perf_counter()
            o.agent_loss_and_grad(sub)
            per_step.append(t_build + (time.perf_counter() - t1) * len(scene.agents) / n_ag)
        ms = 1e3 * float(np.mean(per_step[args.warmup:]))
        return _reference_line(args, "SPM differentiable step ms (forward + backward), 2048^2, 100k agents", ms,
                               "ms", False, ms, {"workload": args.workload, "scene": cfg_desc}, nthreads,
                               f"per step: oracle vertex phase + loss and root-link gradients of {n_ag} seeded "
                               f"agents, extrapolated to all {len(scene.agents)}")
    # profiling1000: the paper's Profiling3 map, one seeded source per step
    k = 8
    srcs = sg.profiling_sources(k, max(1, args.warmup + args.steps))
    per_step = []
    for st in steps:
        sc = sg.profiling_map(k)
        sc = sg.Scene(sc.world, sc.grid, sc.polys, srcs[st:st + 1], sc.segs)
        per_step.append(_oracle_scene_seconds(sc, args.ref_pixels, st, nthreads))
    ms = 1e3 * float(np.mean(per_step[args.warmup:]))
    return _reference_line(args, "SPM ms per map, Profiling3 (64 squares), 1000^2, one source", ms, "ms", False,
                           ms, {"workload": args.workload, "scene": "k x k uniform squares (k = 8), 1000^2"},
                           nthreads, f"per step: one seeded source, oracle vertex phase + {args.ref_pixels} "
                                     f"seeded pixels extrapolated to the 1000x1000 grid")


def run_reference(args, cfg_desc, scene):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    nthreads = oracle.default_threads()
    if args.workload in ("batched256", "diff2048_grad", "profiling1000"):
        print(json.dumps(run_reference_other(args, nthreads)), flush=True)
        return
    for w in range(args.warmup):
        cpu_oracle_rate(scene, args.ref_pixels, 1000 + w, nthreads)
    rates, used = [], 0.0
    for k in range(args.steps):
        r, t = cpu_oracle_rate(scene, args.ref_pixels, k, nthreads)
        rates.append(r)
        used += t
    value = float(np.mean(rates))
    Nx, Ny = scene.grid
    sample = (f"per step: oracle vertex phase + {args.ref_pixels} seeded pixels of the "
              f"{Nx}x{Ny} grid, extrapolated to the full grid")
    metric, unit, ms_step = metric_for(Nx, Ny), UNIT, 1e3 * Nx * Ny / (value * 1e6)
    if args.workload == "dynamic4096":  # one frame = one full map
        metric, unit = "SPM frames/s with sources moving every frame, maze 4096^2", "frames/s"
        value = value * 1e6 / (Nx * Ny)
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "scene": cfg_desc, "grid": [Nx, Ny]},
        "cpu_baseline": {"value": value, "unit": unit, "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tune_by_size_class(spm, objs, scenes, prefix, culling):
    """Culling per size class (grid side) of a batch: the autotuner on the
    class's scene of median polygon count (cached per class and GPU), then
    applied to every scene of the class. Fixed modes when culling is not
    'autotune'."""
    tunings = {}
    for side in sorted({sc.grid[0] for sc in scenes}):
        idx = sorted((k for k, sc in enumerate(scenes) if sc.grid[0] == side), key=lambda k: len(scenes[k].polys))
        rep = idx[len(idx) // 2]
        if culling == "autotune":
            t = objs[rep].autotune(cache_key=f"{prefix}-side{side}")
        else:
            t = {"flood_mode": {"auto": 0, "flood": 1, "scan": 2}[culling], "hidden_chunk": 32, "tile": 0, "maps": 0,
                 "source": "fixed"}
        tunings[side] = t
    for k, o in enumerate(objs):
        t = tunings[scenes[k].grid[0]]
        spm.spm_scene_set_tuning(o.handle, t["flood_mode"], t["hidden_chunk"], t["tile"], t["maps"])
    return {str(side): t for side, t in tunings.items()}


def run_batched(args, cfg_desc, scenes):
    """Batched form: all scenes in one batch (batched vertex phase, one
    persistent pixel kernel, replayed from a CUDA graph); value = scenes/s.
    Culling is tuned per size class. Under torchrun the job is 256 scenes per
    rank (seeded set of 256 x world scenes), dealt to ranks longest-first by
    pixel count; ranks share no data."""
    import torch
    import torch.distributed as dist
    import paper_1805_08500_gb300 as spm
    world, rank, local = rank_env()
    all_scenes = scenes
    if world > 1:
        dist.init_process_group("nccl")
        all_scenes = sg.batched(0, n_scenes=len(scenes) * world)
        mine = shard_lpt([sc.grid[0] * sc.grid[1] for sc in all_scenes], world, rank)
        scenes = [all_scenes[i] for i in mine]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", torch.cuda.current_device())
    objs = [spm.Scene(sc) for sc in scenes]
    tunings = tune_by_size_class(spm, objs, scenes, "batched256", args.culling)  # set-up, not timed
    batch = spm.Batch(objs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    npx = sum(sc.grid[0] * sc.grid[1] for sc in scenes)
    for _ in range(args.warmup):
        batch.compute(stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            batch.compute(stream)
            ev[k][1].record(stream)
            phases.append(batch.phase_ms())  # events inside the batch's graph
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for o in objs:
        o.sync()
    total_ms = max_over_ranks(float(np.sum([a.elapsed_time(b) for a, b in ev])), world, dev)
    ms = total_ms / args.steps
    npx_all = sum(sc.grid[0] * sc.grid[1] for sc in all_scenes)
    vert_ms = float(np.mean([p[0] for p in phases]))
    pix_ms = float(np.mean([p[1] for p in phases]))
    # end to end through the public API: every scene's sources up from
    # page-locked host memory (one copy, then a device-side move per scene),
    # the batch, and every output plane down into page-locked host memory
    src = [np.concatenate([np.asarray(sc.points, np.float32).reshape(-1), np.asarray(sc.segs, np.float32).reshape(-1)])
           for sc in scenes]
    offs = np.cumsum([0] + [len(a) for a in src])
    h_src = torch.tensor(np.concatenate(src) if offs[-1] else np.zeros(1, np.float32)).pin_memory()
    d_src = torch.empty_like(h_src, device=dev)
    outs = batch.outputs
    h_out = [(torch.empty(d.shape, dtype=d.dtype).pin_memory(), torch.empty(p.shape, dtype=p.dtype).pin_memory())
             for d, p in outs]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d_src.copy_(h_src, non_blocking=True)
        for k, (sc, o) in enumerate(zip(scenes, objs)):
            npt = 2 * len(sc.points)
            a, b2 = int(offs[k]), int(offs[k + 1])
            spm.spm_scene_update_sources_device(o.handle, stream, d_src[a:a + npt] if npt else None,
                                                d_src[a + npt:b2] if b2 > a + npt else None)
        batch.compute(stream)
        for (d, p), (hd, hp) in zip(outs, h_out):
            hd.copy_(d, non_blocking=True)
            hp.copy_(p, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    peaks, peak_src = load_peaks()
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = FP32_LANES * N_SMS * 2 * clock_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_PIXEL * npx / (pix_ms * 1e-3) / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    write_gbs = 8.0 * npx / (pix_ms * 1e-3) / 1e9
    line = {"metric": "SPM batched scenes/s", "value": len(all_scenes) / (ms * 1e-3), "unit": "scenes/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i32 (f64 vertex costs)", "data": "synthetic",
            "config": {"workload": "batched256", "scene": cfg_desc, "scenes": len(all_scenes),
                       "pixels": npx_all, "l2": "flushed between timed steps (256 MiB write)",
                       "launch": "one CUDA graph per step", "tuning_by_grid_side": tunings},
            "mpixel_per_s": npx_all / (ms * 1e-3) / 1e6, "clocks": clk.summary(),
            "phases_ms": {"vertex_and_lists": vert_ms, "pixel": pix_ms},
            "roofline": {"bound": "alu", "kernel": "k_pixels_batched", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": KPIXELS_TRAFFIC.get("batched256"), **KPIXELS_UTIL.get("batched256", {}),
                         "note": f"algorithmic = {FLOPS_PER_PIXEL} FP32 flops/pixel (winning distance) over the "
                                 f"persistent pixel kernel's event-timed duration; peak = FP32 lanes x SMs x 2 x max "
                                 f"SM clock ({peak_src}); issue_frac and the pipe shares: ncu on one launch; "
                                 f"traffic above the 8 B/pixel writes is the scenes' depth maps (several GB "
                                 f"for 256 scenes, beyond L2) read bin by bin"},
            "hbm_write": {"achieved": write_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": write_gbs / hbm_peak,
                          "bytes_per_pixel": 8, "peak_source": peak_src},
            "e2e": {"value": len(all_scenes) / e2e_s, "unit": "scenes/s",
                    "h2d_bytes_per_step": int(4 * offs[-1]), "d2h_bytes_per_step": int(8 * npx),
                    "host_buffers": "page-locked"},
            # vertex phase (7), list reset, flood, scan, fill, the persistent pixel kernel
            "gpu_launches": 12 * args.steps}
    if world > 1:
        line["config"]["parallelism"] = f"scenes sharded longest-first over {world} ranks"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        nthreads = oracle.default_threads()
        k = 8  # scenes sampled, extrapolated to the batch
        t0 = time.perf_counter()
        t = sum(_oracle_scene_seconds(scenes[(i * 31) % len(scenes)], 20000, i, nthreads) for i in range(k))
        used = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k / t, "unit": "scenes/s", "cores": nthreads, "kind": "oracle",
                                "sample": f"{k} of the {len(scenes)} scenes (oracle vertex phase + 20000 seeded "
                                          f"pixels each, extrapolated to their grids; {used:.1f} s wall on "
                                          f"{nthreads} threads)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        dist.destroy_process_group()


# Table 1 of the paper (GTX 970, OpenGL, 1000^2, single source, mean of 100
# random sources): Profiling0..6, compute seconds. Context only.
PAPER_PROFILING_S = {4: 0.0014, 16: 0.0054, 36: 0.0456, 64: 0.1251, 100: 0.2701, 196: 0.8564, 400: 2.7371}


def run_profiling(args):
    """The paper's Profiling maps (k x k uniform squares, P = k^2, 1000^2
    grid, one point source): per map, the mean device time of spm_compute
    over 100 seeded free source positions (each moved in with
    spm_scene_update_sources before its timed compute). value = the
    Profiling3 map (P = 64, V = 256, the configuration Table 2 also quotes)."""
    import torch
    import paper_1805_08500_gb300 as spm
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n_src = 100
    rows = []
    with ClockSampler(local) as clk:
        for k in (2, 4, 6, 8, 10, 14, 20):
            scene = sg.profiling_map(k)
            s = spm.Scene(scene)
            tuning = s.autotune(cache_key=f"profiling{k * k}")
            d, p = s.empty_outputs()
            srcs = sg.profiling_sources(k, n_src)
            empty = np.zeros((0, 4), np.float32)
            for i in range(max(args.warmup, 3)):
                spm.spm_scene_update_sources(s.handle, srcs[i:i + 1].astype(np.float32), empty)
                s.compute(d, p, stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_src)]
            for i in range(n_src):
                spm.spm_scene_update_sources(s.handle, srcs[i:i + 1].astype(np.float32), empty)
                ev[i][0].record(stream)
                s.compute(d, p, stream)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            s.sync(stream)
            ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
            # A/B: the paper's generator-sequential schedule on the same maps
            # and sources (first n_seq sources), same outputs
            n_seq = 10
            ev_seq = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(n_seq)]
            spm.spm_scene_update_sources(s.handle, srcs[0:1].astype(np.float32), empty)
            s.compute_sequential(d, p, stream)  # warm-up
            for i in range(n_seq):
                spm.spm_scene_update_sources(s.handle, srcs[i:i + 1].astype(np.float32), empty)
                ev_seq[i][0].record(stream)
                s.compute_sequential(d, p, stream)
                ev_seq[i][1].record(stream)
            torch.cuda.synchronize()
            s.sync(stream)
            seq_ms = float(np.mean([a.elapsed_time(b) for a, b in ev_seq]))
            P = k * k
            rows.append({"P": P, "V": 4 * P, "ms": ms, "mpixel_per_s": 1.0e6 / (ms * 1e-3) / 1e6,
                         "sequential_ms": seq_ms, "culled_speedup_over_sequential": seq_ms / ms,
                         "paper_gtx970_ms": 1e3 * PAPER_PROFILING_S[P], "tuning": tuning})
    ref = next(r for r in rows if r["P"] == 64)
    line = {"metric": "SPM ms per map, Profiling3 (64 squares), 1000^2, one source", "value": ref["ms"],
            "unit": "ms", "n_gpus": 1, "steps": n_src, "warmup": max(args.warmup, 3), "ms_per_step": ref["ms"],
            "higher_is_better": False, "scaling": "weak",
            "vs_baseline": ref["ms"] / ref["paper_gtx970_ms"],
            "dtype": "f32+i32 (f64 vertex costs)", "data": "synthetic",
            "config": {"workload": "profiling1000", "scene": "k x k uniform squares (half the cell pitch), 1000^2 world "
                       "and grid, one seeded free point source per compute, mean of 100 sources",
                       "l2": "inputs resident; no flush (the paper times back-to-back frames)"},
            "maps": rows, "clocks": clk.summary(),
            "note": "vs_baseline divides by the paper's GTX 970 OpenGL time (Table 1): context, not a target; "
                    "sequential_ms = the paper's generator-sequential schedule (spm_compute_sequential) on "
                    "this GPU, mean of the first 10 sources"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_differentiable(args, cfg_desc, scene):
    """Differentiable form: one step = spm_compute + agent loss (forward) +
    its adjoint w.r.t. the sources (backward), 100k agents; value = forward +
    backward ms per step (lower is better)."""
    import torch
    import torch.distributed as dist
    import paper_1805_08500_gb300 as spm
    world, rank, local = rank_env()
    if world > 1:  # replicas: every rank runs its own step; the time is the slowest rank's
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = spm.Scene(scene)
    tuning = s.autotune(cache_key="diff2048_grad")  # set-up, not timed
    tuning = fixpoint_start(spm, s, args, tuning)
    agents = torch.tensor(np.asarray(scene.agents, np.int32), device=dev)
    n_p, n_s = len(scene.points), len(scene.segs)
    d_out, p_out = s.empty_outputs()
    loss = torch.empty((), dtype=torch.float32, device=dev)
    gp = torch.empty(2 * n_p, dtype=torch.float32, device=dev)
    gs = torch.empty(4 * max(n_s, 1), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    n_ag = int(agents.shape[0])
    tape = spm.empty_tape(n_ag, dev)  # the forward's record for the backward

    def step():
        s.compute(d_out, p_out, stream)
        spm.spm_agents_forward(s.handle, stream, agents, d_out, p_out, loss, tape)

    def backward():
        spm.spm_agents_backward(s.handle, stream, tape, n_ag, gp, gs)

    for _ in range(args.warmup):
        step()
        backward()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    phases = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            backward()
            ev[k][2].record(stream)
            phases.append(s.phase_ms())  # this step's map: vertex phase, culling, pixel pass
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s.sync(stream)
    fwd = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b, _ in ev])), world, dev)
    bwd = max_over_ranks(float(np.mean([b.elapsed_time(c) for _, b, c in ev])), world, dev)
    # end to end: FP32 sources up from the host, the step, loss and gradients back
    pts = np.asarray(scene.points, np.float32)
    segs = np.asarray(scene.segs, np.float32)
    h_out = torch.empty(1 + 2 * n_p + 4 * max(n_s, 1), dtype=torch.float32).pin_memory()
    h_src = torch.tensor(np.concatenate([pts.reshape(-1), segs.reshape(-1)])).pin_memory()
    d_src = torch.empty_like(h_src, device=dev)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d_src.copy_(h_src, non_blocking=True)
        spm.spm_scene_update_sources_device(s.handle, stream, d_src[:2 * n_p] if n_p else None,
                                            d_src[2 * n_p:] if n_s else None)
        step()
        backward()
        h_out[:1].copy_(loss.reshape(1), non_blocking=True)
        h_out[1:1 + 2 * n_p].copy_(gp, non_blocking=True)
        h_out[1 + 2 * n_p:].copy_(gs, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, world, dev)
    info = s.info()
    Nx, Ny = scene.grid
    npx = Nx * Ny
    peaks, peak_src = load_peaks()
    pix_ms = float(np.mean([p[2] for p in phases]))  # the map's pixel pass, the step's dominant kernel
    peak_tflops = FP32_LANES * N_SMS * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = FLOPS_PER_PIXEL * npx / (pix_ms * 1e-3) / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    write_gbs = 8.0 * npx / (pix_ms * 1e-3) / 1e9
    line = {"metric": "SPM differentiable step ms (forward + backward), 2048^2, 100k agents",
            "value": fwd + bwd, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": fwd + bwd, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i32 (f64 vertex costs, f64 gradient sums)", "data": "synthetic",
            "config": {"workload": "diff2048_grad", "scene": cfg_desc, "agents": int(agents.shape[0]),
                       "l2": "flushed between timed steps (256 MiB write)", "tuning": tuning,
                       "parallelism": f"replicas x{world} (the slowest rank's step)"},
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "phases_ms": {"vertex": float(np.mean([p[0] for p in phases])),
                          "cull": float(np.mean([p[1] for p in phases])), "pixel": pix_ms},
            "fixpoint_rounds": s.info()["rounds"],
            "roofline": {"bound": "alu", "kernel": "k_pixels", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": None,
                         "note": f"the forward's map: algorithmic = {FLOPS_PER_PIXEL} FP32 flops/pixel (winning "
                                 f"distance) over the pixel pass's event-timed duration; peak = FP32 lanes x SMs "
                                 f"x 2 x max SM clock ({peak_src})"},
            "hbm_write": {"achieved": write_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": write_gbs / hbm_peak,
                          "bytes_per_pixel": 8, "peak_source": peak_src},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(pts.nbytes + segs.nbytes),
                    "d2h_bytes_per_step": int(h_out.numel() * 4)},
            "gpu_launches": (info["kernels_per_compute"] + 5) * args.steps}  # + 3 forward, 2 backward kernels
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        nthreads = oracle.default_threads()
        t0 = time.perf_counter()
        o = oracle.Oracle(scene, nthreads=nthreads)
        o.agent_loss_and_grad(scene.agents)
        used = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": used * 1e3, "unit": "ms", "cores": nthreads, "kind": "oracle",
                                "sample": f"the full step: oracle vertex phase + all {len(scene.agents)} agents "
                                          f"+ root-link gradients ({used:.1f} s wall)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_dynamic(args, cfg_desc, scene):
    """Maps of moving sources (Sec. 6): every frame the maze's point sources
    take a step of their seeded random walk and the exit segment slides, the
    new coordinates are validated and committed on the device
    (spm_scene_update_sources_device) and the map is recomputed. value =
    frames/s from the CUDA-event time of (source update + compute) per frame,
    L2 flushed between frames. e2e = frames/s of the wall-clock frame loop a
    user runs: the frame's sources copied up from pinned host memory, update,
    compute, 100k agents read their distance (spm_agents_forward) and the mean
    comes back to the host; the same loop with host-side source updates and
    one CUDA graph of all frames are reported beside it."""
    import torch
    import torch.distributed as dist
    import paper_1805_08500_gb300 as spm
    world, rank, local = rank_env()
    if world > 1:  # replicas: every rank runs its own frame stream
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = spm.Scene(scene)
    if args.culling == "autotune":
        tuning = s.autotune(cache_key="maze4096")  # the same scene class as the static map
    else:
        spm.spm_scene_set_tuning(s.handle, {"auto": 0, "flood": 1, "scan": 2}[args.culling], 32)
        tuning = dict(s.tuning(), source="fixed")
    Nx, Ny = scene.grid
    npx = Nx * Ny
    F = args.warmup + args.steps
    pts, segs = sg.maze_source_frames(scene, F, seed=1)
    n_p, n_s = pts.shape[1], segs.shape[1]
    P = torch.tensor(pts.reshape(F, -1), device=dev)
    Q = torch.tensor(segs.reshape(F, -1), device=dev)
    agents = torch.tensor(sg.maze_agents(scene, 100_000, seed=2), device=dev)
    d_out, p_out = s.empty_outputs()
    loss = torch.empty((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    info = s.info()

    for f in range(args.warmup):
        spm.spm_scene_update_sources_device(s.handle, stream, P[f], Q[f])
        s.compute(d_out, p_out, stream)
    s.sync(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            f = args.warmup + k
            flush.zero_()
            ev[k][0].record(stream)
            spm.spm_scene_update_sources_device(s.handle, stream, P[f], Q[f])
            s.compute(d_out, p_out, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s.sync(stream)
    total_ms = max_over_ranks(float(np.sum([a.elapsed_time(b) for a, b in ev])), world, dev)
    ms = total_ms / args.steps  # per frame on the slowest rank

    # wall-clock frame loops (no flush: frames follow each other as in an application)
    h_pts = torch.tensor(pts.reshape(F, -1)).pin_memory()
    h_segs = torch.tensor(segs.reshape(F, -1)).pin_memory()
    h_loss = torch.zeros(F, dtype=torch.float32).pin_memory()
    p_dev = torch.empty(2 * n_p, dtype=torch.float32, device=dev)
    s_dev = torch.empty(4 * n_s, dtype=torch.float32, device=dev)

    def frame(f, st):
        p_dev.copy_(h_pts[f], non_blocking=True)
        s_dev.copy_(h_segs[f], non_blocking=True)
        spm.spm_scene_update_sources_device(s.handle, st, p_dev, s_dev)
        spm.spm_compute(s.handle, st, d_out, p_out)
        spm.spm_agents_forward(s.handle, st, agents, d_out, p_out, loss)
        h_loss[f:f + 1].copy_(loss.reshape(1), non_blocking=True)

    def loop(body):  # whole-job frames/s: every rank's frames over the slowest rank's wall time
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        body()
        torch.cuda.synchronize()
        return whole_job_rate(F, world, max_over_ranks(time.perf_counter() - t0, world, dev))

    frame(0, stream)
    e2e_fps = loop(lambda: [frame(f, stream) for f in range(F)])
    s.sync(stream)
    device_losses = h_loss.clone()

    def host_frames():
        for f in range(F):
            spm.spm_scene_update_sources(s.handle, pts[f], segs[f])
            spm.spm_compute(s.handle, stream, d_out, p_out)
            spm.spm_agents_forward(s.handle, stream, agents, d_out, p_out, loss)
            h_loss[f:f + 1].copy_(loss.reshape(1), non_blocking=True)
    host_fps = loop(host_frames)
    s.sync(stream)
    host_losses = h_loss.clone()

    gst = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=gst):
        for f in range(F):
            frame(f, gst)
    graph_fps = loop(g.replay)
    s.sync(stream)
    same = bool(torch.equal(device_losses, host_losses) and torch.equal(h_loss, host_losses))

    line = {"metric": "SPM frames/s with sources moving every frame, maze 4096^2",
            "value": whole_job_rate(args.steps, world, total_ms * 1e-3),
            "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i32 (f64 vertex costs)", "data": "synthetic",
            "config": {"workload": "dynamic4096", "scene": cfg_desc, "grid": [Nx, Ny],
                       "motion": "point sources: integer random walk (<= 6 units per axis per frame) in their "
                                 "cells; exit segment: sideways walk within 3 units",
                       "agents": int(agents.shape[0]), "frames": F,
                       "l2": "flushed between timed frames (256 MiB write)", "tuning": tuning,
                       "parallelism": f"replicas x{world}"},
            "mpixel_per_s": world * npx * 1e3 / ms / 1e6,
            "clocks": clk.summary(),
            "e2e": {"value": e2e_fps, "unit": "frames/s",
                    "h2d_bytes_per_step": int(4 * (2 * n_p + 4 * n_s)), "d2h_bytes_per_step": 4},
            "e2e_host_update_fps": host_fps, "e2e_cuda_graph_fps": graph_fps,
            "losses_identical_across_loops": same,
            "gpu_launches": (info["kernels_per_compute"] + 1) * args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        nthreads = oracle.default_threads()
        moved = sg.Scene(scene.world, scene.grid, scene.polys, pts[-1].astype(np.float64),
                         segs[-1].astype(np.float64))
        rate, used = cpu_oracle_rate(moved, args.cpu_pixels, 4321, nthreads)
        line["cpu_baseline"] = {
            "value": rate * 1e6 / npx, "unit": "frames/s", "cores": nthreads, "kind": "oracle",
            "sample": (f"one frame's sources: oracle vertex phase + {args.cpu_pixels} seeded pixels, "
                       f"extrapolated to {Nx}x{Ny} ({used:.1f} s wall on {nthreads} threads)")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="maze4096",
                    choices=["maze4096", "maze2048", "polys1024", "rects256", "diff2048", "diff2048_grad",
                             "batched256", "profiling1000", "dynamic4096"])
    ap.add_argument("--cpu-pixels", type=int, default=3_000_000,
                    help="oracle pixel sample for the cpu_baseline leg")
    ap.add_argument("--ref-pixels", type=int, default=40_000,
                    help="oracle pixel sample per step for --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fixpoint-start", default="auto", choices=["auto", "sources", "tree"],
                    help="where the vertex fixpoint starts (A/B of the warm start)")
    ap.add_argument("--culling", default="autotune", choices=["autotune", "flood", "scan", "auto"],
                    help="culling mode: autotuned at set-up (default) or fixed")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.impl == "reference":
        scene, cfg_desc = (None, None) if args.workload == "profiling1000" else workload(args.workload)
        run_reference(args, cfg_desc, scene)
        return
    if args.workload == "profiling1000":
        run_profiling(args)
        return
    scene, cfg_desc = workload(args.workload)
    if args.workload == "batched256":
        run_batched(args, cfg_desc, scene)
        return
    if args.workload == "diff2048_grad":
        run_differentiable(args, cfg_desc, scene)
        return
    if args.workload == "dynamic4096":
        run_dynamic(args, cfg_desc, scene)
        return

    import torch
    import torch.distributed as dist

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1805_08500_gb300 as spm

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = spm.Scene(scene)  # returns once the scene's device structures are built
    create_ms = (time.perf_counter() - t0) * 1e3
    if args.culling == "autotune":
        tuning = s.autotune(cache_key=args.workload)  # set-up, not timed
    else:
        spm.spm_scene_set_tuning(s.handle, {"auto": 0, "flood": 1, "scan": 2}[args.culling], 32)
        tuning = dict(s.tuning(), source="fixed")
    tuning = fixpoint_start(spm, s, args, tuning)
    # cold start: a fresh scene with the chosen tuning, created and computed once
    # (scene creation, the obstacles' static structures and the first map)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s_cold = spm.Scene(scene)
    spm.spm_scene_set_tuning(s_cold.handle, tuning["flood_mode"], tuning["hidden_chunk"], tuning["tile"],
                             tuning["maps"], tuning.get("fixpoint_start", 0))
    s_cold.compute()
    s_cold.sync()
    cold_ms = (time.perf_counter() - t0) * 1e3
    s_cold.close()
    del s_cold
    Nx, Ny = scene.grid
    npx = Nx * Ny
    d_out, p_out = s.empty_outputs()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    info = s.info()
    launches_per_step = info["kernels_per_compute"]

    for _ in range(args.warmup):
        s.compute(d_out, p_out, stream)
    s.sync(stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phases = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            s.compute(d_out, p_out, stream)
            ev[k][1].record(stream)
            phases.append(s.phase_ms())  # waits for this step's pixel pass
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s.sync(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(npx * args.steps, world, total_ms * 1e-3) / 1e6

    # end to end through the C ABI with host buffers: source upload + compute +
    # copy of both output planes into pinned host memory
    pts = np.asarray(scene.points, np.float32)
    segs = np.asarray(scene.segs, np.float32)
    hd = torch.empty((Ny, Nx), dtype=torch.float32).pin_memory()
    hp = torch.empty((Ny, Nx), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    spm.spm_compute_host(s.handle, stream, hd, hp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        spm.spm_scene_update_sources(s.handle, pts, segs)
        spm.spm_compute_host(s.handle, stream, hd, hp)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = whole_job_rate(npx, world, max_over_ranks(e2e_s, world, dev)) / 1e6
    # the same into pageable host memory (numpy arrays): row slabs through the
    # scene's page-locked bounce buffers
    nd = np.empty((Ny, Nx), np.float32)
    npar = np.empty((Ny, Nx), np.int32)
    spm.spm_compute_host(s.handle, stream, nd, npar)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        spm.spm_scene_update_sources(s.handle, pts, segs)
        spm.spm_compute_host(s.handle, stream, nd, npar)
    e2e_pageable = whole_job_rate(npx, world, max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)) / 1e6
    del nd, npar

    peaks, peak_src = load_peaks()
    vert_ms = float(np.mean([p[0] for p in phases]))
    cull_ms = float(np.mean([p[1] for p in phases]))
    pix_ms = float(np.mean([p[2] for p in phases]))  # k_pixels, one launch per step
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = FP32_LANES * N_SMS * 2 * clock_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_PIXEL * npx / (pix_ms * 1e-3) / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    write_gbs = 8.0 * npx / (pix_ms * 1e-3) / 1e9

    line = {
        "metric": metric_for(Nx, Ny), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32 (f64 vertex costs)", "data": "synthetic",
        "config": {"workload": args.workload, "scene": cfg_desc, "grid": [Nx, Ny],
                   "generators": info["n_gen"], "polygons": info["n_polys"],
                   "l2": "flushed between timed steps (256 MiB write)",
                   "tuning": tuning,
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"vertex": vert_ms, "cull": cull_ms, "pixel": pix_ms},
        "fixpoint_rounds": s.info()["rounds"],
        "setup_ms": {"scene_create": create_ms, "cold_create_and_first_compute": cold_ms,
                     "note": "host wall clock, outside the timed steps: validation, lattice, device "
                             "upload and the obstacles' static structures (free-space mask, vertex depth "
                             "maps, obstacle-vertex visibility and edges, the table of geodesic distances "
                             "between obstacle vertices; the obstacle vertices' flood at the first compute)"},
        "roofline": {"bound": "alu", "kernel": "k_pixels", "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": KPIXELS_TRAFFIC.get(args.workload),
                     **KPIXELS_UTIL.get(args.workload, {}),
                     "note": f"algorithmic = {FLOPS_PER_PIXEL} FP32 flops/pixel (winning distance); "
                             f"peak = FP32 lanes x SMs x 2 x max SM clock ({peak_src}); issue_frac and the "
                             f"pipe shares: ncu on one launch of this kernel; orient_per_px: counted "
                             f"orientation tests of the exact visibility per pixel"},
        "hbm_write": {"achieved": write_gbs, "peak": hbm_peak, "unit": "GB/s",
                      "frac": write_gbs / hbm_peak, "bytes_per_pixel": 8,
                      "peak_source": peak_src},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(pts.nbytes + segs.nbytes),
                "d2h_bytes_per_step": int(8 * npx), "host_buffers": "page-locked (torch pin_memory)",
                "pageable_value": e2e_pageable},
        "gpu_launches": launches_per_step * args.steps,
        "step_ms_stats": {"median": float(np.median(step_ms)), "p10": float(np.percentile(step_ms, 10)),
                          "p90": float(np.percentile(step_ms, 90)), "rank": rank},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        nthreads = oracle.default_threads()
        rate, used = cpu_oracle_rate(scene, args.cpu_pixels, 12345, nthreads)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": (f"oracle vertex phase + {args.cpu_pixels} seeded pixels, extrapolated "
                       f"to {Nx}x{Ny} ({used:.1f} s wall on {nthreads} threads)")}
        if npx <= 65536:  # a small grid: the whole map on one host thread as well
            t0 = time.perf_counter()
            oracle.Oracle(scene, nthreads=1).field()
            line["cpu_baseline"]["single_thread_full_map"] = {
                "value": npx / (time.perf_counter() - t0) / 1e6, "unit": UNIT, "cores": 1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
