#!/usr/bin/env python
"""Benchmark: batched 3DGS RGB-D rendering, env-frames/s on one GB300.

Workload (default): 2048 envs x 640x480, a 500k-Gaussian static room-shell
background plus a 20-link robot with 5k Gaussians per link, per-env joint
angles and jittered head cameras (seeded synthetic stand-in for the paper's
scenes; paper Sec. III-C "Throughput Scaling": 2048 environments at 640x480).
One step renders the whole batch (RGB + depth) through gs_render_batch with
inputs resident in HBM.  `e2e` times the same batch through
gs_render_batch_host (pinned host poses in, RGB + depth copied back).

`--impl reference` times the CPU oracle (plain FP64 renderer) on a bounded
sample of the same workload on the host cores.

Multi-GPU (torchrun): envs are independent, so every rank renders its own
replica batch (weak scaling, no data-path collective); the step time is the
max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-frames/s at 2048x640x480 RGB-D"
UNIT = "env-frames/s"

# DRAM traffic of the compositor per env of a launch, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over a 32-env launch, divided
# by 32), valid only for the compositor sources it was taken on (the hash
# below; sources that differ from the captured ones in comments only keep it).
COMPOSITE_TRAFFIC_PER_ENV = (0.680517e9 + 0.523335e9) / 32
COMPOSITE_TRAFFIC_SOURCES = ("paper_2604_25459_gb300/csrc/gs_composite.cu",)
COMPOSITE_TRAFFIC_SHA = "05cb60c8cec62bb9"


def _sources_sha(paths) -> str:
    import hashlib

    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--envs", type=int, default=2048)
    ap.add_argument("--width", type=int, default=640)
    ap.add_argument("--height", type=int, default=480)
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="c1: skip the other forms measured in the same run (128x128, BF16/FP16, c3 plan, c4 rate)")
    ap.add_argument("--oracle-seconds", type=float, default=12.0,
                    help="CPU-baseline sample: oracle envs rendered one by one until this much time has passed")
    ap.add_argument("--workload", choices=["c1", "c3", "c4", "prune", "lidar"], default="c1",
                    help="c1: uniform 640x480 batch (headline); c3: batched uneven form through a plan")
    ap.add_argument("--no-graph", action="store_true", help="c3: eager plan launches instead of a CUDA graph")
    ap.add_argument("--obs", action="store_true",
                    help="c1 in the observation form: 8-bit RGB after per-env appearance randomisation + half depth")
    ap.add_argument("--rates", default="1000,3000,10000,30000", help="c4: offered request rates (req/s)")
    ap.add_argument("--prune-envs", type=int, default=64, help="prune: envs whose cameras rank the Gaussians")
    ap.add_argument("--beams", type=int, default=64, help="lidar: beams (rows)")
    ap.add_argument("--rays", type=int, default=0,
                    help="lidar: rays per env of a non-repetitive (rosette) pattern within +-0.6 rad of the sensor's "
                         "x axis instead of a grid scan; --beams x --azimuth then only bins them over +-0.65 rad")
    ap.add_argument("--azimuth", type=int, default=1024, help="lidar: azimuth steps across the window (columns)")
    ap.add_argument("--az-window", default="0,6.283185307179586",
                    help="lidar: azimuth window az_min,az_max in radians (a full turn: rotating; narrower: solid-state)")
    ap.add_argument("--duration", type=float, default=2.0, help="c4: seconds of arrivals per rate")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="c4: HBM budget of the request loop")
    ap.add_argument("--scene-budget-gb", type=float, default=0.0,
                    help="c1: the scene's scratch budget in GiB (0: the library default of 64 GiB)")
    ap.add_argument("--slots", type=int, default=4, help="c4: stream slots (batches in flight)")
    ap.add_argument("--max-batch", type=int, default=512, help="c4: requests per batch")
    return ap.parse_args()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over the ranks of the process group (x itself on one
    rank): the job's time is that of its slowest rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_sample(w, envs, threads=None, budget_s=None):
    """Time the plain FP64 oracle on `envs` of workload w, one env after the
    other, stopping early once budget_s seconds have passed; returns (seconds,
    cores, envs rendered)."""
    from oracle import oracle

    if threads:
        oracle.set_num_threads(threads)
    cores = oracle.num_threads()
    S = oracle.scene_arrays(w)
    t0 = time.perf_counter()
    done = 0
    for e in envs:
        oracle.render_env(w, e, S=S)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 >= budget_s:
            break
    return time.perf_counter() - t0, cores, done


def run_reference(a, rank, world):
    if rank != 0:
        return
    from paper_2604_25459_gb300 import synth

    w = synth.make_c1(n_envs=a.envs, width=a.width, height=a.height, f=500.0 * a.width / 640)
    for k in range(a.warmup):
        oracle_sample(w, [k % a.envs])
    ts = []
    cores = 1
    for k in range(a.steps):
        t, cores, _ = oracle_sample(w, [(a.warmup + k) % a.envs])
        ts.append(t)
    tot = sum(ts)
    val = a.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c1: {a.envs} envs x {a.width}x{a.height}, 500k bg + 20x5k link Gaussians",
                       "step": "one env rendered by the plain FP64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "1 env per step of the c1 workload, plain FP64 oracle"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def time_uniform(a, w, scene, step, E, W, H, dev, local_rank, world, steps, warmup, dtype="f32", obs=False,
                 tile="16x16"):
    """Warm-up, an untimed counting pass (composited pairs, visible records),
    then `steps` timed steps bracketed by CUDA events on the launching stream
    with the clocks sampled in between; returns the timings and the
    compositor's roofline (plain-ALU bound) and the whole step's."""
    import torch
    import torch.distributed as dist

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    scene.sync_status()
    # algorithmic work of one batch: composited (pixel, Gaussian) pairs (untimed pass)
    scene.set_counters(True)
    step()
    torch.cuda.synchronize()
    st = scene.stats()
    n_eval = st["composited"]
    n_vis = st["visible"]
    n_pairs = st["n_gaussians"] * E  # (env, Gaussian) pairs tested
    intersections = st["intersections"]
    launches_per_step = st["kernel_launches"]
    scene.set_counters(False)

    scene.set_profile(True)
    scene.timings(reset=True)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    scene.set_profile(False)
    tim = scene.timings(reset=True)
    lat = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(steps))
    total_ms = evs[0].elapsed_time(evs[-1])
    scene.sync_status()
    t_max = max_over_ranks(total_ms, world, dev)
    ms_step = t_max / steps
    value = world * E * steps / (t_max / 1e3)

    # roofline of the dominant kernel (compositing): plain-ALU bound.
    comp_ms, comp_launches = tim["composite"]
    per_launch_ms = comp_ms / max(comp_launches, 1)
    launches_per_batch = comp_launches / steps
    evals_per_launch = n_eval / max(launches_per_batch, 1)
    ops_per_eval = 20.0  # quadratic form, ex2, alpha, T, 3 colour + 1 depth FMA (lane-ops)
    sm_mhz = ck.get("sm_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak_lane_ops = props.multi_processor_count * 128 * sm_mhz * 1e6
    achieved = evals_per_launch * ops_per_eval / (per_launch_ms / 1e3)
    traffic = None
    # the captured traffic holds for the captured form only: 640x480 camera images, 16x16 tiles
    if (_sources_sha(COMPOSITE_TRAFFIC_SOURCES) == COMPOSITE_TRAFFIC_SHA and (W, H) == (640, 480)
            and tile == "16x16" and not obs and dtype == "f32"):
        traffic = COMPOSITE_TRAFFIC_PER_ENV * E / max(launches_per_batch, 1)  # bytes per launch
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_lane_ops / 1e9, "unit": "Glane-op/s",
                "frac": achieved / peak_lane_ops, "traffic": traffic,
                "kernel": "k_composite", "per_launch_ms": per_launch_ms,
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x median {sm_mhz:.0f} MHz "
                              "(1 lane-op per lane per clock, FMA counted once)"}
    phase_ms = {k: v[0] / steps for k, v in tim.items()}

    # whole-step roofline: algorithmic HBM bytes vs FP32 work (paper's hot path, all steps)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    attr_bytes = (w.background.n + w.links.n) * (236 if dtype == "f32" else 132)
    out_bytes = E * H * W * (6 if obs else 16)
    io_bytes = attr_bytes + E * (w.n_links * 28 + 56) + out_bytes
    # whole step: time floor = max(algorithmic bytes / HBM peak, algorithmic FP32 work / ALU peak), the
    # work being N_eval x 20 (compositing) + E G x 20 (culling every pair) + E V x 300 (projecting the
    # visible pairs: covariance, conic, SH degree 3)
    fp32_ops = n_eval * 20.0 + n_pairs * 20.0 + n_vis * 300.0
    hbm_floor_ms = io_bytes / (hbm * 1e9) * 1e3
    alu_floor_ms = fp32_ops / peak_lane_ops * 1e3
    step_roofline = {"io_bytes": io_bytes, "hbm_floor_ms": hbm_floor_ms, "hbm_gbs_peak": hbm,
                     "fp32_lane_ops": fp32_ops, "alu_floor_ms": alu_floor_ms,
                     "bound": "alu" if alu_floor_ms > hbm_floor_ms else "hbm",
                     "frac": max(alu_floor_ms, hbm_floor_ms) / ms_step,
                     "composited_pairs": n_eval, "visible_pairs": n_vis, "tested_pairs": n_pairs,
                     "intersections": intersections}
    return {"value": value, "ms_per_step": ms_step, "steps": steps, "warmup": warmup,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": _pct(lat, 0.99), "mean": sum(lat) / len(lat)},
            "clocks": ck, "roofline": roofline, "step_roofline": step_roofline, "phase_ms_per_step": phase_ms,
            "gpu_launches": int(launches_per_step * steps), "mpix_per_s": value * H * W / 1e6}


def measure_uniform(a, w, dtype, dev, local_rank, world, steps, warmup, tile="16x16"):
    """One uniform-resolution batch of workload w in storage dtype, timed as
    the headline is; the scene and images are released afterwards."""
    import torch

    from paper_2604_25459_gb300 import gsbatch

    tw, th = (int(x) for x in tile.split("x"))
    E, H, W = w.n_envs, int(w.cams["height"][0]), int(w.cams["width"][0])
    scene = gsbatch.scene_from_workload(w, dtype)
    scene.set_tile(tw, th)
    poses = torch.from_numpy(w.link_poses).to(dev)
    rgb = torch.empty((E, H, W, 3), dtype=torch.float32, device=dev)
    depth = torch.empty((E, H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        scene.render(poses, w.cams, rgb=rgb, depth=depth, want_alpha=False, stream=stream)

    r = time_uniform(a, w, scene, step, E, W, H, dev, local_rank, world, steps, warmup, dtype=dtype, tile=tile)
    scene.close()
    del rgb, depth, poses
    torch.cuda.empty_cache()
    r["config"] = {"workload": f"{w.name}: {E} envs x {W}x{H} RGB-D, {dtype} storage, tile {tile}",
                   "l2": f"outputs of {E * H * W * 16 / 1e9:.1f} GB written per step (> 129 MB L2)"}
    return r


def run_ours(a, rank, world, local_rank):
    import torch

    import __graft_entry__
    from paper_2604_25459_gb300 import gsbatch, synth

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    tw, th = (int(x) for x in a.tile.split("x"))
    f = 500.0 * a.width / 640
    w = synth.make_c1(n_envs=a.envs, width=a.width, height=a.height, f=f)
    E, H, W = a.envs, a.height, a.width
    scene = gsbatch.scene_from_workload(w, a.dtype)
    scene.set_tile(tw, th)
    if a.scene_budget_gb > 0:
        scene.set_budget(int(a.scene_budget_gb * (1 << 30)))
    poses = torch.from_numpy(w.link_poses).to(dev)
    stream = torch.cuda.current_stream()
    if a.obs:  # observation form: per-env exposure, contrast, brightness
        arng = np.random.default_rng([a.envs, 91])
        ap_h = np.stack([arng.uniform(-0.5, 0.5, E), arng.uniform(0.7, 1.3, E), arng.uniform(-0.1, 0.1, E)],
                        1).astype(np.float32)
        ap_d = torch.from_numpy(ap_h).to(dev)
        rgb8 = torch.empty((E, H, W, 3), dtype=torch.uint8, device=dev)
        depth16 = torch.empty((E, H, W), dtype=torch.float16, device=dev)

        def step():
            scene.render_obs(poses, w.cams, appearance=ap_d, rgb8=rgb8, depth16=depth16, stream=stream)
    else:
        rgb = torch.empty((E, H, W, 3), dtype=torch.float32, device=dev)
        depth = torch.empty((E, H, W), dtype=torch.float32, device=dev)

        def step():
            scene.render(poses, w.cams, rgb=rgb, depth=depth, want_alpha=False, stream=stream)

    r = time_uniform(a, w, scene, step, E, W, H, dev, local_rank, world, a.steps, a.warmup, dtype=a.dtype,
                     obs=a.obs, tile=a.tile)
    try:  # measured plain-ALU rates, reported beside the derived peak
        alu = gsbatch.measure_alu_peak(stream)
    except Exception as ex:  # noqa: BLE001
        alu = {"error": str(ex)}
    r["roofline"]["measured_fma_glane_ops"] = alu.get("fma_lane_ops_per_s", 0.0) / 1e9
    r["roofline"]["measured_ex2_glane_ops"] = alu.get("ex2_lane_ops_per_s", 0.0) / 1e9

    e2e = None
    if not a.no_e2e:
        pin = lambda shape, dt=torch.float32: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        poses_h = torch.from_numpy(w.link_poses).pin_memory().numpy()
        if a.obs:
            rgb_h, depth_h = pin((E, H, W, 3), torch.uint8), pin((E, H, W), torch.float16)
            host_step = lambda: scene.render_obs_host(poses_h, w.cams, ap_h, rgb_h, depth_h)
        else:
            rgb_h, depth_h = pin((E, H, W, 3)), pin((E, H, W))
            host_step = lambda: scene.render_host(poses_h, w.cams, rgb_h, depth_h)
        host_step()
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            host_step()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": world * E * a.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(poses_h.nbytes + w.cams.nbytes),
               "d2h_bytes_per_step": int(rgb_h.nbytes + depth_h.nbytes),
               "ms_per_step": 1e3 * dt / a.e2e_steps,
               "api": "gs_render_batch_obs_host" if a.obs else "gs_render_batch_host"}
        del rgb_h, depth_h, poses_h
    scene.close()
    if a.obs:
        del rgb8, depth16
    else:
        del rgb, depth
    del poses
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        t, cores, done = oracle_sample(w, list(range(E)), budget_s=a.oracle_seconds)
        cpu = {"value": done / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"envs 0..{done - 1} of the same c1 batch rendered one by one by the plain FP64 oracle "
                         f"({t:.1f} s of CPU time budgeted at {a.oracle_seconds:.0f} s)"}

    # The other forms of the path, measured in the same run on the same GPU
    # (one process, N=1 only): the RL-typical 128x128 image, the BF16/FP16
    # storage forms of the headline batch, a short replay of the batched
    # uneven plan and the request loop at one offered rate.
    sub = None
    headline = (E, W, H, a.dtype, a.obs, a.tile) == (2048, 640, 480, "f32", False, "16x16")
    if world == 1 and headline and not a.no_sub:
        sub = {}
        sub_steps, sub_warm = 5, 3
        w128 = synth.make_c2(n_envs=E, res="128x128")
        sub["c2_128x128_f32"] = measure_uniform(a, w128, "f32", dev, local_rank, world, sub_steps, sub_warm)
        del w128
        for dt in ("bf16", "f16"):
            sub[f"c1_{dt}"] = measure_uniform(a, w, dt, dev, local_rank, world, sub_steps, sub_warm)
        sub["c3_plan"] = measure_c3(a, dev, local_rank, world, steps=3, warmup=1)
        sub["c4_served"] = measure_c4(a, dev, local_rank, world, rates=[1e4], duration=2.0, plain=False)

    if rank == 0:
        line = {
            "metric": METRIC if (E, W, H) == (2048, 640, 480) else f"env-frames/s at {E}x{W}x{H} RGB-D",
            "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.dtype if a.dtype != "f32" else "f32", "data": "synthetic",
            "config": {"workload": f"c1: {E} envs x {W}x{H} RGB-D, 500k room-shell background + 20 links x 5k "
                                   f"Gaussians, SH degree 3, tile {a.tile}"
                                   + (", observation form: u8 RGB after per-env exposure/contrast/brightness + f16 depth"
                                      if a.obs else ""),
                       "envs_per_gpu": E, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"outputs of {E * H * W * (6 if a.obs else 16) / 1e9:.1f} GB written per step "
                             "(> 129 MB L2)"},
            "mpix_per_s": r["mpix_per_s"],
            "latency_ms": r["latency_ms"],
            "clocks": r["clocks"],
            "roofline": r["roofline"],
            "step_roofline": r["step_roofline"],
            "phase_ms_per_step": r["phase_ms_per_step"],
            "gpu_launches": r["gpu_launches"],
            "e2e": e2e,
            "cpu_baseline": cpu,
            "sub_results": sub,
        }
        print(json.dumps(line), flush=True)


def measure_c3(a, dev, local_rank, world, steps, warmup, envs_n=4096):
    """Batched uneven form: 4096 envs, per-env objects of 10k-200k Gaussians on a
    shared 300k background, resolutions {64^2, 128^2, 320x240, 640x480} with
    probabilities {.3, .3, .2, .2}; one plan (autotuned tile shape, claim
    size and compositor form, replayed from a captured CUDA graph); a step is
    one plan launch.  The compositor's roofline comes from an eager,
    profiled render of the same batch (gs_render_batch_v) after the timing."""
    import torch
    import torch.distributed as dist

    from paper_2604_25459_gb300 import gsbatch, synth

    E = envs_n
    t0 = time.perf_counter()
    w = synth.make_c3(n_envs=E, threads=os.cpu_count() or 8)
    gen_s = time.perf_counter() - t0
    scene = gsbatch.Scene(w.background)
    scene.attach_links(w.link_offsets, w.links)
    envs = gsbatch.make_envs(w.cams, link_ranges=np.stack([np.arange(E), np.arange(E) + 1], 1),
                             pose_offsets=np.arange(E))
    npx = int((w.cams["width"].astype(np.int64) * w.cams["height"]).sum())
    rgb = torch.empty(npx * 3, device=dev)
    depth = torch.empty(npx, device=dev)
    poses = torch.from_numpy(w.link_poses).to(dev)
    stream = torch.cuda.current_stream()
    plan = scene.plan(envs, autotune=True, graph=not a.no_graph)
    t0 = time.perf_counter()
    plan.launch(poses, rgb, depth, stream=stream)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    for _ in range(warmup):
        plan.launch(poses, rgb, depth, stream=stream)
    torch.cuda.synchronize()
    scene.sync_status()
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        plan.launch(poses, rgb, depth, stream=stream)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    scene.sync_status()
    lat = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(steps))
    total_ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), world, dev)
    info = plan.info()
    plan.close()
    # eager pass: composited pairs, then the compositor's time per launch
    scene.set_tile(info["tile_w"], info["tile_h"])
    scene.set_counters(True)
    scene.render_v(envs, poses, rgb, depth, stream=stream)
    torch.cuda.synchronize()
    n_eval = scene.stats()["composited"]
    scene.set_counters(False)
    scene.set_profile(True)
    scene.timings(reset=True)
    scene.render_v(envs, poses, rgb, depth, stream=stream)
    tim = scene.timings(reset=True)
    scene.set_profile(False)
    scene.sync_status()
    comp_ms, comp_launches = tim["composite"]
    sm_mhz = ck.get("sm_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * sm_mhz * 1e6
    per_launch = comp_ms / max(comp_launches, 1)
    achieved = n_eval / max(comp_launches, 1) * 20.0 / (per_launch / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Glane-op/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_composite", "per_launch_ms": per_launch,
                "basis": "eager gs_render_batch_v of the same batch with the plan's tile shape (the plan's own "
                         "launches are graph replays without per-kernel events); composited pairs x 20 lane-ops"}
    scene.close()
    del rgb, depth, poses
    torch.cuda.empty_cache()
    value = world * E * steps / (total_ms / 1e3)
    res, cnt = np.unique(w.cams["width"], return_counts=True)
    return {"metric": "env-frames/s, batched uneven RGB-D (4096 mixed-resolution envs)", "value": value,
            "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
            "config": {"workload": f"c3: {E} envs, 300k background + per-env objects log-uniform 10k-200k "
                                   f"({w.links.n} object Gaussians), widths {dict(zip(res.tolist(), cnt.tolist()))}",
                       "l2": f"{npx * 16 / 1e9:.2f} GB of outputs per step"},
            "mpix_per_s": value * npx / E / 1e6,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": _pct(lat, 0.99)},
            "clocks": ck, "plan": info, "roofline": roofline, "composited_pairs": n_eval,
            "eager_phase_ms": {k: v[0] for k, v in tim.items()}, "generate_s": gen_s, "first_launch_s": tune_s}


def run_c3(a, rank, world, local_rank):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    r = measure_c3(a, dev, local_rank, world, a.steps, a.warmup, envs_n=a.envs if a.envs != 2048 else 4096)
    if rank == 0:
        line = dict(r)
        line.update({"n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                     "dtype": "f32", "data": "synthetic", "gpu_launches": None, "e2e": None, "cpu_baseline": None})
        print(json.dumps(line), flush=True)


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))] if xs else None


def measure_c4(a, dev, local_rank, world, rates, duration, plain=True, envs_n=4096):
    """Served form: 8 resident scenes (room-shell backgrounds of 200k..1M
    Gaussians plus the 20-link robot) and 4096 env instances at the c3
    resolution mix.  Requests (one env's link poses, from the host) arrive as
    a Poisson stream at each offered rate and are served by the library's
    request loop (continuous batching under a 120 GB HBM budget on a pool of
    streams); reported per rate: served env-frames/s and p50/p99 latency
    (arrival to completion on the device).  With `plain`, the plain per-batch
    path (every env of every scene rendered by gs_render_batch_v, scene by
    scene) is timed beside it."""
    import torch

    from paper_2604_25459_gb300 import gsbatch, synth

    E = envs_n
    t0 = time.perf_counter()
    w = synth.make_c4(n_envs=E)
    gen_s = time.perf_counter() - t0
    S, L = len(w.backgrounds), w.n_links
    tw, th = (int(x) for x in a.tile.split("x"))
    scenes = []
    for k in range(S):
        sc = gsbatch.Scene(w.backgrounds[k])
        sc.attach_links(w.link_offsets, w.links)
        sc.set_tile(tw, th)
        sc.set_budget(8 << 30)
        scenes.append(sc)
    npx = int((w.cams["width"].astype(np.int64) * w.cams["height"]).sum())
    stream = torch.cuda.current_stream()

    plain_ms = None
    if plain:  # plain per-batch path: all envs, scene by scene, one step = every env once
        poses_all = torch.from_numpy(w.request_poses(E, stream=99).reshape(E * L, 7)).to(dev)
        rgb = torch.empty(npx * 3, device=dev)
        depth = torch.empty(npx, device=dev)
        envs_all = gsbatch.make_envs(w.cams, link_ranges=np.tile([0, L], (E, 1)), pose_offsets=np.arange(E) * L)
        per_scene = [envs_all[w.env_scene == k] for k in range(S)]

        def plain_step():
            for k in range(S):
                scenes[k].render_v(per_scene[k], poses_all, rgb, depth, stream=stream)

        for _ in range(a.warmup):
            plain_step()
        torch.cuda.synchronize()
        for sc in scenes:
            sc.sync_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            plain_step()
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1) / a.steps
        del rgb, depth, poses_all
        torch.cuda.empty_cache()

    # the request loop
    sv = gsbatch.Server(budget_bytes=int(a.budget_gb * (1 << 30)), max_inflight=a.slots,
                        max_batch_envs=a.max_batch, tile=(tw, th))
    ids = [sv.add_scene(sc) for sc in scenes]
    for i in range(E):
        sv.add_env(ids[int(w.env_scene[i])], w.cams[i], 0, L)
    sv.start()
    warm = w.request_poses(E, stream=98)
    for rep in range(2):  # grows every slot's scratch, seeds the key estimates
        for i in range(E):
            sv.submit(i, warm[i])
        sv.drain(600.0)
        while sv.poll(1 << 16):
            pass
    rng = np.random.default_rng([7, E])
    sweep = []
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    for ri, rate in enumerate(rates):
        n = max(1, int(rate * duration))
        arr = np.cumsum(rng.exponential(1.0 / rate, n))
        env = rng.integers(0, E, n)
        poses = w.request_poses(n, stream=ri)
        st0 = sv.stats()
        base = sv.now() + 0.3 + 8e-6 * n
        for j in range(n):
            sv.submit(int(env[j]), poses[j], base + float(arr[j]))
        sv.drain(600.0)
        res = []
        while True:
            got = sv.poll(1 << 16)
            if not got:
                break
            res += got
        st1 = sv.stats()
        ok = [r for r in res if r["status"] == 0]
        lat = [(r["done_s"] - r["arrival_s"]) * 1e3 for r in ok]
        span = max(r["done_s"] for r in ok) - min(r["arrival_s"] for r in ok)
        nb = st1["batches"] - st0["batches"]
        sweep.append({"offered_req_s": rate, "requests": n, "served_env_frames_s": len(ok) / span,
                      "p50_ms": _pct(lat, 0.50), "p99_ms": _pct(lat, 0.99), "max_ms": max(lat),
                      "batches": nb, "mean_batch": len(ok) / max(nb, 1), "max_batch": st1["max_batch"],
                      "max_concurrent": st1["max_concurrent"], "retried": st1["retried"] - st0["retried"],
                      "peak_inflight_gb": st1["peak_inflight_bytes"] / 1e9})
        print("c4 rate", json.dumps(sweep[-1]), file=sys.stderr, flush=True)
    ck = clocks.stop()
    sv.close()
    for sc in scenes:
        sc.sync_status()
        sc.close()
    torch.cuda.empty_cache()
    sustained = [x for x in sweep if x["served_env_frames_s"] >= 0.95 * x["offered_req_s"]]
    top = max(sustained, key=lambda x: x["offered_req_s"]) if sustained else sweep[0]
    res_w, cnt = np.unique(w.cams["width"], return_counts=True)
    out = {"metric": "served env-frames/s and p99 latency (8 resident scenes, 4096 envs, Poisson arrivals)",
           "value": top["served_env_frames_s"], "unit": UNIT,
           "config": {"workload": f"c4: {S} scenes, backgrounds "
                                  f"{[b.n for b in w.backgrounds]} + 20x5k robot, {E} envs, widths "
                                  f"{dict(zip(res_w.tolist(), cnt.tolist()))}",
                      "budget_gb": a.budget_gb, "slots": a.slots, "max_batch": a.max_batch, "tile": a.tile,
                      "arrivals_s_per_rate": duration},
           "latency_ms": {"p50": top["p50_ms"], "p99": top["p99_ms"], "at_offered_req_s": top["offered_req_s"]},
           "sweep": sweep, "clocks": ck, "generate_s": gen_s}
    if plain_ms is not None:
        out["ms_per_step"] = plain_ms
        out["plain_per_batch"] = {"ms_per_step": plain_ms, "env_frames_s": E / (plain_ms / 1e3),
                                  "latency_ms_one_step": plain_ms,
                                  "l2": f"{npx * 16 / 1e9:.2f} GB of outputs per plain step"}
    return out


def run_c4(a, rank, world, local_rank):
    """The served form (see measure_c4) at every offered rate of --rates.
    Replicas only under torchrun: each rank serves its own copy."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    r = measure_c4(a, dev, local_rank, world, [float(x) for x in a.rates.split(",")], a.duration, plain=True,
                   envs_n=a.envs if a.envs != 2048 else 4096)
    if rank == 0:
        line = dict(r)
        line.update({"n_gpus": world, "steps": a.steps, "warmup": a.warmup, "higher_is_better": True,
                     "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                     "gpu_launches": None, "e2e": None, "cpu_baseline": None})
        print(json.dumps(line), flush=True)


def run_prune(a, rank, world, local_rank):
    """Pruning as a scene transform on c1: rank every Gaussian by its summed
    blending weight over the cameras of the first --prune-envs envs of the
    batch (the contribution pass), keep the top 30 % of the background and 10 %
    of each link's cluster, then time the full 2048-env batch on the pruned
    scene; error: PSNR of the pruned render against the FP64 oracle of the
    unpruned scene on sampled envs."""
    import torch

    import __graft_entry__
    from oracle import oracle
    from paper_2604_25459_gb300 import gsbatch, synth

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    E, H, W = a.envs, a.height, a.width
    w = synth.make_c1(n_envs=E, width=W, height=H, f=500.0 * W / 640)
    poses = torch.from_numpy(w.link_poses).to(dev)
    stream = torch.cuda.current_stream()
    scene = gsbatch.scene_from_workload(w)
    ns = min(a.prune_envs, E)
    t0 = time.perf_counter()
    scores = scene.contribution(poses[:ns], w.cams[:ns], stream=stream)
    torch.cuda.synchronize()
    score_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    pscene, _ = scene.prune(scores, keep_bg=0.3, keep_links=0.1)  # selection + new scene on the device
    torch.cuda.synchronize()
    prune_s = time.perf_counter() - t0
    rgb = torch.empty((E, H, W, 3), dtype=torch.float32, device=dev)
    depth = torch.empty((E, H, W), dtype=torch.float32, device=dev)

    def timed(sc):
        for _ in range(a.warmup):
            sc.render(poses, w.cams, rgb=rgb, depth=depth, want_alpha=False, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            sc.render(poses, w.cams, rgb=rgb, depth=depth, want_alpha=False, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sc.sync_status()
        return e0.elapsed_time(e1) / a.steps

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    full_ms = timed(scene)
    pruned_ms = timed(pscene)
    ck = clocks.stop()
    # error on sampled envs (the last rendered batch holds the pruned images)
    S = oracle.scene_arrays(w)
    errs = []
    for e in (0, E // 2, E - 1):
        ref = oracle.render_env(w, e, S=S)
        diff = rgb[e].cpu().numpy().astype(np.float64) - ref["rgb"]
        mse = float((diff ** 2).mean())
        errs.append({"env": e, "psnr_db": 10 * math.log10(1.0 / max(mse, 1e-20)),
                     "max_abs": float(np.abs(diff).max())})
    if rank == 0:
        line = {"metric": "env-frames/s at 2048x640x480 RGB-D, pruned scene (30 % background, 10 % per link)",
                "value": E / (pruned_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": pruned_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"c1 pruned by contribution over the cameras of {ns} envs: "
                                       f"{pscene.n_background} of {w.background.n} background and "
                                       f"{pscene.stats()['n_gaussians'] - pscene.n_background} of "
                                       f"{w.links.n} link Gaussians kept"},
                "unpruned": {"ms_per_step": full_ms, "env_frames_s": E / (full_ms / 1e3)},
                "speedup": full_ms / pruned_ms, "error_vs_unpruned_fp64_oracle": errs,
                "contribution_pass_s": score_s, "prune_s": prune_s, "clocks": ck,
                "gpu_launches": None, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    pscene.close()
    scene.close()



def run_lidar(a, rank, world, local_rank):
    """Batch-LiDAR on the c1 scene: every env carries a LiDAR at its jittered
    head position, a rotating one of --beams x --azimuth rays (elevation
    -0.4..0.3 rad; --az-window narrower: solid-state), or with --rays R a
    non-repetitive rosette pattern of R rays per env (a different phase per
    env); a step scans all envs (range + hit per ray) with the links posed per
    env.  Reported in rays/s, with the compositor's roofline: composited
    (ray, Gaussian) pairs x 40 lane-ops (the ray-space evaluation: three dot
    products with the rows of G, a cross product, a reciprocal, q and t*,
    ex2, alpha, then transmittance and range) per launch time, against the
    FP32 lane peak."""
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2604_25459_gb300 import gsbatch, synth

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    E = a.envs
    w = synth.make_c1(n_envs=E)
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).to(dev)
    rng = np.random.default_rng([E, 53])
    sens = np.zeros(E, dtype=gsbatch.LIDAR_DTYPE)
    sens["q_ws"] = [1.0, 0.0, 0.0, 0.0]
    sens["t_ws"] = -(np.array([-1.0, 0.0, 1.4]) + rng.uniform(-0.2, 0.2, (E, 3)))
    sens["rows"], sens["cols"] = a.beams, a.azimuth
    sens["near_range"] = 0.05
    R, Cc = a.beams, a.azimuth
    stream = torch.cuda.current_stream()
    if a.rays > 0:
        sens["elev_min"], sens["elev_max"] = -0.65, 0.65
        sens["az_min"], sens["az_max"] = -0.65, 0.65
        dirs = torch.from_numpy(synth.rosette_rays(E, a.rays, seed=7)).to(dev)
        out_r = torch.empty((E, a.rays), dtype=torch.float32, device=dev)
        out_h = torch.empty((E, a.rays), dtype=torch.float32, device=dev)
        rays = E * a.rays

        def step():
            scene.render_rays(poses, sens, dirs, out_r, out_h, stream=stream)
        desc = (f"non-repetitive rosette LiDAR, {a.rays} rays per env within 0.6 rad of the sensor axis, binned on a "
                f"{R}x{Cc} grid over +-0.65 rad")
    else:
        sens["elev_min"], sens["elev_max"] = -0.4, 0.3
        az0, az1 = (float(x) for x in a.az_window.split(","))
        sens["az_min"], sens["az_max"] = az0, az1  # a full turn: rotating; narrower: solid-state
        out_r = torch.empty((E, R, Cc), dtype=torch.float32, device=dev)
        out_h = torch.empty((E, R, Cc), dtype=torch.float32, device=dev)
        rays = E * R * Cc

        def step():
            scene.render_lidar(poses, sens, out_r, out_h, stream=stream)
        desc = (f"{'rotating' if az1 - az0 >= 6.28318 else 'solid-state'} LiDAR {R} beams x {Cc} azimuth steps over "
                f"azimuth {az0:.3f}..{az1:.3f} rad, elevation -0.4..0.3 rad")
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    scene.sync_status()
    scene.set_counters(True)  # untimed: composited (ray, Gaussian) pairs
    step()
    torch.cuda.synchronize()
    n_eval = scene.stats()["composited"]
    scene.set_counters(False)
    scene.set_profile(True)
    scene.timings(reset=True)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    tim = scene.timings(reset=True)
    scene.set_profile(False)
    scene.sync_status()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, world, dev)
    hit_frac = float((out_h > 0.5).float().mean())
    comp_ms, comp_launches = tim["composite"]
    per_launch = comp_ms / max(comp_launches, 1)
    launches_per_step = comp_launches / a.steps
    sm_mhz = ck.get("sm_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * sm_mhz * 1e6
    achieved = n_eval / max(launches_per_step, 1) * 40.0 / (per_launch / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Glane-op/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_composite (LiDAR form)",
                "per_launch_ms": per_launch, "composited_pairs": n_eval, "lane_ops_per_pair": 40}
    if rank == 0:
        line = {"metric": f"LiDAR rays/s ({E} envs x {rays // E} rays, c1 scene)", "value": world * rays / (ms / 1e3),
                "unit": "rays/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"c1 scene (500k room-shell background + 20x5k robot), {E} envs, {desc}",
                           "rays_hit_over_half": hit_frac},
                "env_scans_per_s": world * E / (ms / 1e3),
                "phase_ms_per_step": {k: v[0] / a.steps for k, v in tim.items()},
                "roofline": roofline,
                "clocks": ck, "gpu_launches": None, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    scene.close()


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if a.impl == "ours":
            import torch

            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if a.impl == "reference":
        run_reference(a, rank, world)
    elif a.workload == "c3":
        run_c3(a, rank, world, local_rank)
    elif a.workload == "c4":
        run_c4(a, rank, world, local_rank)
    elif a.workload == "prune":
        run_prune(a, rank, world, local_rank)
    elif a.workload == "lidar":
        run_lidar(a, rank, world, local_rank)
    else:
        run_ours(a, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
