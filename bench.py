#!/usr/bin/env python3
"""Benchmark of the Adaptive Multi-NeRF rendering hot path on one GB300 (or N ranks).

Workload (one "step"): the paper-scale scene -- 8 anisotropic Gaussians plus a thin
shell on a 128^3 guidance grid, KD tree of depth <= 8 with leaf mass <= total/256,
one 4 x 64 MLP per leaf (frequency encoding L=10 / L=4), 8 views of 800 x 800 rays,
8 samples per leaf crossing, cap 192 samples per ray -- rendered end to end through
the library: traversal, grouping, per-leaf networks and compositing.  Inputs are
synthetic and seeded; the per-step working set (5.12 M rays, ~10 GB of per-sample
records) is far larger than L2, so no extra flush is needed.

Two network paths are timed: the plain FP32 SIMT path and the BF16 tcgen05 grouped
path (the headline `value`).  Pixels of a seeded ray subset are compared with the
FP64 oracle (PSNR, max abs), and the same oracle, timed on the host cores on that
subset, is reported as `cpu_baseline`.

--impl reference runs the oracle itself (the CPU program the GPU path is checked
against) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_01881_gb300 import scenes as S  # noqa: E402

METRIC = "Msamples/s, Mrays/s at 800x800: plain FP32 vs BF16 grouped @ PSNR≥45dB vs FP64"
# DRAM bytes (read + write) per generated sample of the BF16 network kernel, from one
# ncu capture of a one-view 400x400 case of the c2 workload, valid only for the kernel
# sources whose SHA-256 prefix is recorded here: the bench reports roofline.traffic as
# this figure times the step's samples while the sources are unchanged, else null.
NETWORK_DRAM_PER_SAMPLE = {"sha256_16": "fbc7cbd6659f912c", "bytes_per_sample": 10.6394}
NETWORK_SOURCES = ("k_mlp_tc.cu", "tc_common.cuh")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
FP32_LANES = 128  # FP32 lanes per SM (sm_100 class)


def _network_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in NETWORK_SOURCES:
        with open(os.path.join(ROOT, "paper_2310_01881_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons.  Each row carries
    nvidia-smi's own timestamp, so a sampler started before the warm-up keeps only
    the rows taken between mark_start() and mark_stop() (the timed region), with the
    first row after the region as a stand-in when the region is shorter than the
    sampling interval."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 100

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()
        if self.proc is not None:   # let the row that follows the region arrive
            time.sleep(2.5 * self.INTERVAL_MS / 1000)

    @staticmethod
    def _stamp(x: str):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(x, fmt).timestamp()
            except ValueError:
                pass
        return None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append([self._stamp(parts[0])] + parts[1:])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self) -> dict:
        rows, window = self.rows, "whole sampler"
        if self.t0 is not None and self.t1 is not None and all(r[0] is not None for r in rows):
            inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
            after = [r for r in rows if r[0] > self.t1]
            if inside:
                rows, window = inside, "timed region"
            else:
                rows, window = after[:1], "first sample after the timed region"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(cfg, rank: int, views: int | None = None, px: int | None = None):
    """Scene, rays of this rank's views (rank r renders views V r .. V r + V - 1).
    `views` / `px` shrink the workload for profiling runs (defaults: the config's)."""
    grid = S.density_grid(S.scene_for(cfg.scene, 0), cfg.G)
    nv = views or cfg.views
    os_, ds_ = [], []
    for v in range(nv):
        o, d = S.view_rays(cfg, 0, rank * nv + v, px, px)
        os_.append(o)
        ds_.append(d)
    return grid, np.concatenate(os_), np.concatenate(ds_)


def workload_name(cfg, args) -> str:
    """The benchmark workload, as both arms name it in `config`."""
    return (f"{cfg.name}: {args.px or cfg.px_w}x{args.px or cfg.px_h} x {args.views or cfg.views} views per GPU, "
            f"{cfg.G}^3 guidance grid, depth<={cfg.max_depth}"
            + (f" (mass<=1/{round(1 / cfg.leaf_mass_frac)})" if cfg.leaf_mass_frac > 0 else "")
            + f", {cfg.hidden}x{cfg.width} MLP per leaf, {cfg.steps} samples/crossing, cap {cfg.cap}"
            + (f", stratified jitter (seed {args.jitter})" if getattr(args, "jitter", 0) else "")
            + (f", empty-space skipping (density > {args.skip_empty:g})"
               if getattr(args, "skip_empty", None) is not None else "")
            + (f", early ray termination in waves of {args.ert_wave} crossings"
               if getattr(args, "ert_wave", 0) else "")
            + (f", adaptive hierarchical sampling (nodes refined while wider than {args.lod_px:g} pixels)"
               if getattr(args, "lod_px", 0) else ""))


def pixel_angle(cfg, px=None) -> float:
    """Vertical angle of one pixel of the workload's camera (radians)."""
    return 2.0 * math.tan(math.radians(cfg.fov_deg / 2.0)) / (px or cfg.px_h)


def barrier():
    """Barrier over the ranks of the default process group (no-op for one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _reduce(x: float, op: str, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device="cuda") -> float:
    """The slowest rank's time: the whole job's step time."""
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device="cuda") -> float:
    """Units of all ranks (each rank renders different views, so counts differ)."""
    return _reduce(x, "sum", device)


def _algorithmic(cfg, st, slot_bytes=16):
    """Algorithmic work of one step (bytes / flops), per the unit counts of the step.

    slot_bytes: per-sample output (sigma, rgb) as written by the network and read by the
    compositing: 16 (FP32 path) or 8 (4 x FP16, tensor-core paths)."""
    rays, xs, samples = st["rays"], st["crossings"], st["samples_generated"]
    k0 = S.mlp_input_width(cfg.lx, cfg.ld)
    w, h = cfg.width, cfg.hidden
    flops_per_sample = 2 * (k0 * w + (h - 1) * w * w + 4 * w)
    return {
        "traverse_bytes": 24 * rays + 1 * rays + 10 * xs,
        "group_bytes": 1 * rays + 6 * xs,
        "network_bytes": 24 * rays + 12 * xs + slot_bytes * samples,
        "composite_bytes": 21 * rays + 8 * xs + slot_bytes * samples,
        "network_flops": flops_per_sample * samples,
        "flops_per_sample": flops_per_sample,
    }


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2310_01881_gb300 import amnerf, build

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    cfg = S.CONFIGS[args.config]
    grid, o_np, d_np = workload(cfg, rank, args.views, args.px)
    n = len(o_np)
    R = amnerf.Renderer(local)
    R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    lod = args.lod_px * pixel_angle(cfg, args.px) if args.lod_px else 0.0
    cells = R.network_cells() if lod > 0 else R.leaf_cells()   # one network per node with hierarchical sampling
    P = S.xavier_weights(0, S.leaf_mean_density(grid, cells), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o = torch.from_numpy(o_np).cuda()
    d = torch.from_numpy(d_np).cuda()
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    stream = torch.cuda.current_stream()
    peaks, peak_src = _peaks()

    def load_prec(prec):
        if prec == "fp8s":  # E4M3 with static scales, calibrated on a view outside the timed set
            R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "fp32")
            oc, dc = S.view_rays(cfg, 0, 1000 + rank, args.px, args.px)
            amax = R.calibrate_fp8(torch.from_numpy(oc).cuda(), torch.from_numpy(dc).cuda(), cfg.hidden,
                                   steps=cfg.steps, cap=cfg.cap, t_term=cfg.t_term, lod=lod)
            R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
        else:
            R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, prec)

    results = {}
    precs = [p for p in args.prec.split(",") if p]
    for prec in precs:  # a precision that fails to load fails the run
        load_prec(prec)
        with ClockSampler(local) as clk:       # started before the warm-up: sampling when the timed region opens
            for _ in range(args.warmup):
                R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out, jitter=args.jitter,
                         skip_empty=args.skip_empty, ert_wave=args.ert_wave, lod=lod)
            _, _, _, st = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out, jitter=args.jitter,
                                   skip_empty=args.skip_empty, ert_wave=args.ert_wave, lod=lod)
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            clk.mark_start()
            e0.record(stream)
            for _ in range(args.steps):
                R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out, jitter=args.jitter, skip_empty=args.skip_empty,
                         ert_wave=args.ert_wave, lod=lod)
            e1.record(stream)
            torch.cuda.synchronize()
            clk.mark_stop()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        R.sync()
        # per-stage CUDA-event times on the launching stream (second pass, synchronised per step)
        amnerf.amnerf_set_timing(R.ctx, True)
        stage = np.zeros(4)
        for _ in range(args.steps):
            *_, s2 = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out, jitter=args.jitter,
                              skip_empty=args.skip_empty, ert_wave=args.ert_wave, lod=lod)
            stage += np.array(s2["ms"])
        amnerf.amnerf_set_timing(R.ctx, False)
        stage /= args.steps
        pix = [t.cpu().numpy() for t in out]
        results[prec] = {"ms": ms, "stats": st, "stage_ms": stage.tolist(), "pixels": pix, "clocks": clk.summary()}

    if not results:
        raise RuntimeError("no network precision could be loaded")
    head = "bf16" if "bf16" in results else next(iter(results))
    hr = results[head]
    st = hr["stats"]
    samples_all = int(sum_over_ranks(float(st["samples_generated"])))
    rays_all = int(sum_over_ranks(float(n)))
    value = samples_all / (hr["ms"] * 1e-3) / 1e6

    # end to end through the host-buffer entry point (pinned host memory, copies timed)
    load_prec(head)
    ho = torch.from_numpy(o_np).pin_memory().numpy()
    hd = torch.from_numpy(d_np).pin_memory().numpy()
    hout = [torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy(),
            torch.empty(n, dtype=torch.float32).pin_memory().numpy(),
            torch.empty(n, dtype=torch.float32).pin_memory().numpy()]
    for _ in range(max(1, args.warmup)):
        amnerf.amnerf_render_host(R.ctx, ho, hd, *hout, steps=cfg.steps, cap=cfg.cap, t_term=cfg.t_term,
                                  jitter=args.jitter, skip_empty=args.skip_empty, ert_wave=args.ert_wave, lod=lod)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        amnerf.amnerf_render_host(R.ctx, ho, hd, *hout, steps=cfg.steps, cap=cfg.cap, t_term=cfg.t_term,
                                  jitter=args.jitter, skip_empty=args.skip_empty, ert_wave=args.ert_wave, lod=lod)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
    barrier()

    if rank != 0:
        R.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # accuracy against the FP64 oracle on a seeded ray subset + the oracle's own speed
    import oracle as O
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    cells_or = tree.network_cells() if lod > 0 else tree.leaf_cells()
    P_or = S.xavier_weights(0, S.leaf_mean_density(grid, cells_or), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    idx = S.ray_subset(n, args.psnr_rays, 7)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = O.render(tree, P_or, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps, cfg.cap,
                   cfg.t_term, mode=0, threads=cores, jitter=args.jitter,
                   skip=(grid, args.skip_empty) if args.skip_empty is not None else None, lod=lod)
    cpu_s = time.perf_counter() - t0
    cpu_samples = int(ref["n_gen"].sum())
    acc = {}
    for prec, r in results.items():
        rgb = r["pixels"][0][idx].astype(np.float64)
        mse = float(np.mean((rgb - ref["rgb"]) ** 2))
        acc[prec] = {"psnr_db": 10 * np.log10(1.0 / max(mse, 1e-30)),
                     "max_abs_rgb": float(np.abs(rgb - ref["rgb"]).max()),
                     "max_abs_opacity": float(np.abs(r["pixels"][2][idx] - ref["opacity"]).max())}

    alg = _algorithmic(cfg, st, 16 if head == "fp32" else 8)
    net_ms = hr["stage_ms"][2]
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if head == "fp32":
        peak = n_sm * FP32_LANES * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": alg["network_flops"] / (net_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": f"derived: {n_sm} SMs x {FP32_LANES} FP32 lanes x 2 x max SM clock"}
    else:
        # the network kernel is one launch of ~13 ms per step, timed as such: the burst peak
        peak = peaks["bf16_tflops"] if head == "bf16" else 2 * peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": alg["network_flops"] / (net_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": f"{peak_src} burst bf16" + (" x2 (fp8)" if head in ("fp8", "fp8s") else "")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = "k_mlp_tc" if head != "fp32" else "k_mlp_simt"
    roof["kernel_ms"] = net_ms
    rec = NETWORK_DRAM_PER_SAMPLE
    same_kernel = rec["sha256_16"] is not None and rec["sha256_16"] == _network_sources_sha()
    roof["traffic"] = (rec["bytes_per_sample"] * st["samples_generated"]
                       if (head == "bf16" and cfg.name == "c2" and same_kernel) else None)
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a 400x400 c2 view, scaled by "
                              "samples" if roof["traffic"] is not None else
                              "none for these kernel sources (no capture since they changed)")
    roof["algorithmic_bytes"] = alg["network_bytes"]
    hbm = peaks["hbm_gbs"]
    stages = {}
    for i, (name, key) in enumerate((("traverse", "traverse_bytes"), ("group", "group_bytes"),
                                     ("network", "network_bytes"), ("composite", "composite_bytes"))):
        ms_i = hr["stage_ms"][i]
        gbs = alg[key] / (ms_i * 1e-3) / 1e9 if ms_i > 0 else None
        stages[name] = {"ms": ms_i, "algorithmic_bytes": alg[key], "GB/s": gbs,
                        "frac_hbm": gbs / hbm if gbs else None}

    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "Msamples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(hr["ms"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3", "fp8s": "e4m3"}[head],
        "data": "synthetic",
        "config": {"workload": workload_name(cfg, args),
                   "rays_per_step": rays_all, "samples_per_step": samples_all, "leaves": R.n_leaves,
                   "l2": "inputs larger than L2 (per-step working set ~10 GB)", "parallelism": f"replicas x{world}"},
        "mrays_per_s": round(rays_all / (hr["ms"] * 1e-3) / 1e6, 3),
        "paths": {p: {"Msamples/s": round(samples_all / (r["ms"] * 1e-3) / 1e6, 3),
                      "Mrays/s": round(rays_all / (r["ms"] * 1e-3) / 1e6, 3), "ms_per_step": round(r["ms"], 4),
                      "stage_ms": [round(x, 4) for x in r["stage_ms"]], "vs_fp64": acc[p]}
                  for p, r in results.items()},
        "roofline": roof,
        "stages_hbm": stages,
        "e2e": {"value": round(samples_all / (e2e_ms * 1e-3) / 1e6, 3), "unit": "Msamples/s",
                "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(24 * n), "d2h_bytes_per_step": int(20 * n)},
        "gpu_launches": 5 * args.steps,
        "clocks": hr["clocks"],
        "cpu_baseline": {"value": round(cpu_samples / cpu_s / 1e6, 6), "unit": "Msamples/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"FP64 oracle on {len(idx)} seeded rays of view set 0 ({cpu_samples} samples, "
                                   f"{cpu_s:.1f} s)"},
    }
    if "fp32" in results and head != "fp32":
        line["speedup_vs_fp32"] = round(results["fp32"]["ms"] / hr["ms"], 3)
    R.close()
    if world == 1 and cfg.name == "c2" and args.views is None and args.px is None and not args.no_extras:
        line.update(_extras(args))
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_ahs(args, grid=None, lods_px=(64.0, 128.0)) -> dict:
    """Adaptive hierarchical sampling on the 4096-leaf workload (16 views of 1920x1080,
    one network per node, BF16): leaf-only against nodes refined only while wider than
    K pixels at the ray's entry distance.  Per setting: time per step, samples per ray,
    and PSNR against the FP64 oracle of the same method on a seeded ray subset."""
    import torch

    from paper_2310_01881_gb300 import amnerf, build

    torch.cuda.set_device(0)
    build.build()
    cfg = S.CONFIGS["c4"]
    if grid is None:
        grid = S.density_grid(S.scene_for(cfg.scene, 0), cfg.G)
    rays = [S.view_rays(cfg, 0, v) for v in range(cfg.views)]
    o_np = np.concatenate([r[0] for r in rays]); d_np = np.concatenate([r[1] for r in rays])
    del rays
    n = len(o_np)
    R = amnerf.Renderer(0)
    R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, R.network_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "bf16")
    o = torch.from_numpy(o_np).cuda(); d = torch.from_numpy(d_np).cuda()
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    stream = torch.cuda.current_stream()
    import oracle as O
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P_or = S.xavier_weights(0, S.leaf_mean_density(grid, tree.network_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    idx = S.ray_subset(n, 4096, 13)
    rows = []
    with ClockSampler(0) as clk:
        for k in (0.0,) + tuple(lods_px):
            lod = k * pixel_angle(cfg)
            for _ in range(args.warmup):
                R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out, lod=lod)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out, lod=lod)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            *_, st = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out, lod=lod)
            rgb = out[0].cpu().numpy().astype(np.float64)
            ref = O.render(tree, P_or, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps,
                           cfg.cap, cfg.t_term, mode=0, threads=os.cpu_count() or 1, lod=lod)
            mse = float(np.mean((rgb[idx] - ref["rgb"]) ** 2))
            rows.append({"refine_above_px": k, "lod": lod, "ms": round(ms, 3),
                         "Mrays/s": round(n / (ms * 1e-3) / 1e6, 3),
                         "Msamples/s": round(st["samples_generated"] / (ms * 1e-3) / 1e6, 3),
                         "samples_per_ray": round(st["samples_generated"] / n, 3),
                         "psnr_vs_fp64_same_method": round(10 * np.log10(1.0 / max(mse, 1e-30)), 2)})
    base = rows[0]
    for r in rows[1:]:
        r["spr_reduction"] = round(base["samples_per_ray"] / r["samples_per_ray"], 3)
        r["speedup"] = round(base["ms"] / r["ms"], 3)
    R.close()
    return {"workload": f"c4: {cfg.views} views x {cfg.px_w}x{cfg.px_h}, {tree.n_leaves} leaves, one 4x64 BF16 "
                        f"network per node ({tree.n_nodes})", "settings": rows, "clocks": clk.summary()}


def _extras(args) -> dict:
    """The batching (c4) and learned-proposal (c5) workloads, summarised for the default
    line: one GPU, 16 views of 1920x1080 each, the 4096-leaf scene."""
    import torch
    a = argparse.Namespace(**vars(args))
    a.steps = min(args.steps, 10)
    a.views, a.px = None, None
    a.c5_scene, a.leaf_net, a.density_scale, a.ert_wave = "c4", "", 1.0, 0
    cfg4 = S.CONFIGS["c4"]
    grid = S.density_grid(S.scene_for(cfg4.scene, 0), cfg4.G)
    c4 = run_c4(a, emit=False, grid=grid)
    torch.cuda.empty_cache()
    c5 = run_c5(a, emit=False, grid=grid)
    torch.cuda.empty_cache()
    ahs = run_ahs(a, grid=grid)
    torch.cuda.empty_cache()
    keep4 = ("value", "unit", "ms_per_step", "mrays_per_s", "graph_ms", "stream_ms", "per_leaf_launch_ms",
             "speedup_vs_per_leaf", "stage_ms", "stage_ms_per_leaf", "autotuned", "leaf_counts", "vs_fp64",
             "zipf_network_microbench", "clocks")
    keep5 = ("value", "unit", "ms_per_step", "plain", "proposal", "spr_reduction", "delta_psnr_vs_fp64_db",
             "training", "clocks")
    return {"c4": {"workload": c4["config"]["workload"], **{k: c4[k] for k in keep4 if k in c4}},
            "c5": {"workload": c5["config"]["workload"], **{k: c5[k] for k in keep5 if k in c5}},
            "hierarchical_sampling": ahs}


def _zipf_exponent(counts: np.ndarray) -> float:
    """Least-squares slope of log(count) against log(rank) over the non-empty leaves."""
    c = np.sort(np.asarray(counts, np.float64))[::-1]
    c = c[c > 0]
    r = np.arange(1, len(c) + 1, dtype=np.float64)
    slope = np.polyfit(np.log(r), np.log(c), 1)[0]
    return float(-slope)


def run_c4(args, emit: bool = True, grid=None) -> dict:
    """Imbalanced batching workload: 4096-leaf tree, 16 views of 1920x1080 (33.2 M rays)
    rendered as ONE batch (one persistent grouped network launch), autotuned, replayed
    from a CUDA graph, next to the per-leaf-launch baseline.  Returns the JSON line
    (printed when `emit`)."""
    import ctypes

    import torch

    from paper_2310_01881_gb300 import amnerf, build

    torch.cuda.set_device(0)
    build.build()
    cfg = S.CONFIGS["c4"]
    views = args.views or cfg.views
    if grid is None:
        grid = S.density_grid(S.scene_for(cfg.scene, 0), cfg.G)
    rays = [S.view_rays(cfg, 0, v, args.px, args.px) for v in range(views)]
    o_np = np.concatenate([r[0] for r in rays]); d_np = np.concatenate([r[1] for r in rays])
    del rays
    n = len(o_np)
    R = amnerf.Renderer(0)
    nl = R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "bf16")
    o = torch.from_numpy(o_np).cuda()
    d = torch.from_numpy(d_np).cuda()
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    # autotune on the first view, then fix the configuration
    nv = n // views
    g_best, s_best, ws_best, ms_best = amnerf.amnerf_autotune(R.ctx, o[:nv], d[:nv], out[0][:nv], out[1][:nv], out[2][:nv],
                                                     steps=cfg.steps, cap=cfg.cap, t_term=cfg.t_term, reps=2)
    _, _, _, st = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out)
    # realised per-leaf crossing counts
    counts = torch.zeros(nl, dtype=torch.int32, device="cuda")
    dbg = amnerf.amnerf_debug(None, None, None, None, counts.data_ptr(), None, None, None)
    p = amnerf._params(cfg.steps, cfg.cap, cfg.t_term, (0.0, 0.0, 0.0))
    rc = amnerf.load().amnerf_render_debug(R.ctx, o.data_ptr(), d.data_ptr(), n, ctypes.byref(p), out[0].data_ptr(),
                                          out[1].data_ptr(), out[2].data_ptr(), ctypes.byref(dbg), None)
    assert rc == 0
    cnt = counts.cpu().numpy().astype(np.int64)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    graph, gout = R.capture(o, d, cfg.steps, cfg.cap, cfg.t_term)
    with ClockSampler(0) as clk:
        ms_graph = timed(graph.replay, args.steps)
    ms_plain = timed(lambda: R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out), args.steps)
    amnerf.amnerf_set_timing(R.ctx, True)
    stage = np.zeros(4)
    for _ in range(2):
        *_, s2 = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out)
        stage += np.array(s2["ms"]) / 2
    # per-leaf-launch baseline (one network launch per leaf)
    amnerf.amnerf_set_tuning(R.ctx, g_best, amnerf.SCHED_PER_LEAF, ws_best)
    stage_pl = np.zeros(4)
    for _ in range(2):
        *_, s3 = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, out=out)
        stage_pl += np.array(s3["ms"]) / 2
    amnerf.amnerf_set_timing(R.ctx, False)
    ms_pl = timed(lambda: R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out), max(1, args.steps // 2))
    # network microbench: crossing lists whose per-leaf counts are drawn from Zipf s = 1.1
    # over the 4096 leaves (seeded rank permutation), grouped launch vs per-leaf launches
    zn = min(n, 2_000_000)
    maxc = cfg.cap // cfg.steps
    zx, zl, za, zb = S.zipf_crossings(zn, maxc, nl, 1.1, 0)
    zc = np.bincount(zl.reshape(-1).astype(np.int64), minlength=nl)
    zargs = (o[:zn], d[:zn], torch.from_numpy(zx).cuda(), torch.from_numpy(zl.view(np.int16).reshape(-1)).cuda(),
             torch.from_numpy(za.reshape(-1)).cuda(), torch.from_numpy(zb.reshape(-1)).cuda())
    del zx, zl, za, zb
    zout = (out[0][:zn], out[1][:zn], out[2][:zn])
    zipf = {"rays": zn, "crossings": zn * maxc, "samples": zn * maxc * cfg.steps, "zipf_s": 1.1,
            "zipf_exponent_fit": round(_zipf_exponent(zc), 3), "max_leaf_crossings": int(zc.max()),
            "min_leaf_crossings": int(zc.min())}
    amnerf.amnerf_set_timing(R.ctx, True)
    for name_, sched_ in (("grouped", s_best), ("per_leaf", amnerf.SCHED_PER_LEAF)):
        amnerf.amnerf_set_tuning(R.ctx, g_best, sched_, ws_best)
        amnerf.amnerf_render_crossings(R.ctx, *zargs, *zout, steps=cfg.steps, cap=cfg.cap, t_term=cfg.t_term)
        net = []
        for _ in range(3):
            zst = amnerf.amnerf_render_crossings(R.ctx, *zargs, *zout, steps=cfg.steps, cap=cfg.cap,
                                                 t_term=cfg.t_term, stats=True)
            net.append(zst["ms"][2])
        nm = float(np.median(net))
        zipf[name_] = {"network_ms": round(nm, 3), "network_Msamples/s": round(zipf["samples"] / (nm * 1e-3) / 1e6, 1)}
    amnerf.amnerf_set_timing(R.ctx, False)
    zipf["speedup_vs_per_leaf"] = round(zipf["per_leaf"]["network_ms"] / zipf["grouped"]["network_ms"], 3)
    del zargs
    amnerf.amnerf_set_tuning(R.ctx, g_best, s_best, ws_best)
    R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, out=out)
    rgb = out[0].cpu().numpy().astype(np.float64)
    import oracle as O
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P_or = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    idx = S.ray_subset(n, args.psnr_rays // 4, 9)
    ref = O.render(tree, P_or, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps, cfg.cap,
                   cfg.t_term, mode=0, threads=os.cpu_count() or 1)
    mse = float(np.mean((rgb[idx] - ref["rgb"]) ** 2))
    samples = st["samples_generated"]
    names = {0: "contiguous", 1: "interleaved", 2: "dynamic"}
    line = {
        "metric": "Msamples/s (c4 batching: one persistent grouped launch under CUDA graph vs per-leaf launches)",
        "value": round(samples / (ms_graph * 1e-3) / 1e6, 3), "unit": "Msamples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_graph, 3), "higher_is_better": True,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"c4: {views} views x {o_np.shape[0] // views} rays, 256^3 grid, depth<=12, "
                               f"{nl} leaves, 4x64 MLP, cap 192", "rays_per_step": n, "samples_per_step": samples},
        "mrays_per_s": round(n / (ms_graph * 1e-3) / 1e6, 3),
        "graph_ms": round(ms_graph, 3), "stream_ms": round(ms_plain, 3), "per_leaf_launch_ms": round(ms_pl, 3),
        "speedup_vs_per_leaf": round(ms_pl / ms_graph, 3),
        "stage_ms": [round(x, 3) for x in stage], "stage_ms_per_leaf": [round(x, 3) for x in stage_pl],
        "autotuned": {"groups": g_best, "schedule": names.get(s_best, s_best), "width_split": ws_best,
                      "ms_one_view": round(ms_best, 3)},
        "leaf_counts": {"leaves": nl, "nonempty": int((cnt > 0).sum()), "max": int(cnt.max()),
                        "median_nonempty": float(np.median(cnt[cnt > 0])), "zipf_exponent_fit": round(_zipf_exponent(cnt), 3)},
        "vs_fp64": {"psnr_db": round(10 * np.log10(1.0 / max(mse, 1e-30)), 2),
                    "max_abs_rgb": float(np.abs(rgb[idx] - ref["rgb"]).max()), "rays": int(len(idx))},
        "zipf_network_microbench": zipf,
        "clocks": clk.summary(),
    }
    if emit:
        print(json.dumps(line))
    R.close()
    return line


def run_c5(args, emit: bool = True, grid=None) -> dict:
    """Learned proposal with BF16 leaves: trained on plain-rendered views, evaluated on
    held-out views against the plain sampler, the FP64 oracle, and the oracle's own
    bound -- the samples per ray when the kept bins come from the true (plain-render)
    weights.  The scene is the 4096-leaf imbalanced one (--c5-scene c4, the default,
    with its 4 x 64 leaf networks) or the config-1 scene (--c5-scene c1, 2 x 32 leaves),
    optionally with every density scaled.  Returns the JSON line (printed when `emit`)."""
    import torch

    from paper_2310_01881_gb300 import amnerf, build

    torch.cuda.set_device(0)
    build.build()
    cfg = S.CONFIGS[args.c5_scene]
    if args.leaf_net:  # another leaf network shape, e.g. "4x64" (the scene is unchanged)
        h, w = (int(v) for v in args.leaf_net.lower().split("x"))
        cfg = dataclasses.replace(cfg, hidden=h, width=w)
    if grid is None:
        grid = S.density_grid(S.scene_for(cfg.scene, 0), cfg.G)
    grid = grid * np.float32(args.density_scale)
    R = amnerf.Renderer(0)
    R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "bf16")
    n_train_views, tw, th = args.train_views, 480, 270
    tr = [S.view_rays(cfg, 0, 1000 + v, tw, th) for v in range(n_train_views)]
    o_tr = torch.from_numpy(np.concatenate([t[0] for t in tr])).cuda()
    d_tr = torch.from_numpy(np.concatenate([t[1] for t in tr])).cuda()
    del tr
    n_tr = o_tr.shape[0]
    out_tr = (torch.empty((n_tr, 3), device="cuda"), torch.empty(n_tr, device="cuda"), torch.empty(n_tr, device="cuda"))
    tg = torch.empty((n_tr, 65), device="cuda")
    root = torch.empty((n_tr, 2), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amnerf.amnerf_proposal_targets(R.ctx, o_tr, d_tr, *out_tr, tg, root, steps=cfg.steps, cap=cfg.cap,
                                   t_term=cfg.t_term)
    t_targets = time.perf_counter() - t0
    amnerf.amnerf_proposal_set(R.ctx, S.proposal_init(1))
    t0 = time.perf_counter()
    losses = amnerf.amnerf_proposal_train(R.ctx, o_tr, d_tr, root, tg, steps=args.train_steps, batch=8192, lr=3e-3,
                                          seed=7)
    t_train = time.perf_counter() - t0
    del o_tr, d_tr, out_tr, tg, root
    torch.cuda.empty_cache()
    views = args.views or 16
    px_w, px_h = (args.px, args.px) if args.px else (1920, 1080)
    te = [S.view_rays(cfg, 0, 2000 + v, px_w, px_h) for v in range(views)]
    o_np = np.concatenate([t[0] for t in te]); d_np = np.concatenate([t[1] for t in te])
    del te
    n = len(o_np)
    o = torch.from_numpy(o_np).cuda(); d = torch.from_numpy(d_np).cuda()
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    stream = torch.cuda.current_stream()
    points = [(0.99, 64), (0.99, 16), (0.95, 64)]   # (coverage, max_bins); the first is the headline

    def timed(prop, cov=0.99, mb=64, waves=0):
        kw = dict(out=out, proposal=prop, coverage=cov, max_bins=mb, ert_wave=waves)
        for _ in range(args.warmup):
            R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        amnerf.amnerf_set_timing(R.ctx, True)
        *_, st = R.render(o, d, cfg.steps, cfg.cap, cfg.t_term, stats=True, **kw)
        amnerf.amnerf_set_timing(R.ctx, False)
        return e0.elapsed_time(e1) / args.steps, st, out[0].cpu().numpy().astype(np.float64)

    with ClockSampler(0) as clk:
        ms_plain, st_plain, rgb_plain = timed(False)
        runs = [timed(True, cov, mb) for cov, mb in points]
        # early ray termination in waves (--ert-wave W): the same renders, evaluating
        # only the crossings before each ray's termination
        wave_runs = [timed(prop, cov, mb, args.ert_wave) for prop, cov, mb in
                     [(False, 0.99, 64)] + [(True, c, b) for c, b in points]] if args.ert_wave else []
    import oracle as O
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P_or = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    idx = S.ray_subset(n, args.psnr_rays // (16 if cfg.width * cfg.hidden > 64 else 4), 11)
    threads = os.cpu_count() or 1
    ref = O.render(tree, P_or, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps, cfg.cap,
                   cfg.t_term, mode=0, threads=threads, bins=True)

    def psnr(a, b):
        return round(10 * np.log10(1.0 / max(float(np.mean((a - b) ** 2)), 1e-30)), 2)

    def spr(st):
        return round(st["samples_generated"] / n, 3)

    p_plain = psnr(rgb_plain[idx], ref["rgb"])
    spr_plain_or = float(ref["n_gen"].mean())
    res = []
    for (cov, mb), (ms, st, rgb) in zip(points, runs):
        m, fb = O.prop_select(ref["bins"], cov, mb)
        bound = O.render(tree, P_or, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps,
                         cfg.cap, cfg.t_term, mode=0, threads=threads, mask=m, fallback=fb.astype(np.int32))
        p = psnr(rgb[idx], ref["rgb"])
        res.append({"coverage": cov, "max_bins": mb, "Mrays/s": round(n / (ms * 1e-3) / 1e6, 3),
                    "ms": round(ms, 3), "stage_ms": [round(x, 3) for x in st["ms"]],
                    "proposal_ms": round(st["proposal_ms"], 3),
                    "samples_per_ray": spr(st), "spr_reduction": round(spr(st_plain) / spr(st), 3),
                    "fallback_frac": round(st["fallback_rays"] / n, 4), "psnr_vs_plain": psnr(rgb, rgb_plain),
                    "psnr_vs_fp64": p, "delta_psnr_vs_fp64_db": round(p_plain - p, 2),
                    "true_weight_bound": {"spr_reduction": round(spr_plain_or / max(float(bound["n_gen"].mean()), 1e-9),
                                                                 3),
                                          "fallback_frac": round(float(fb.mean()), 4),
                                          "psnr_vs_plain_fp64": psnr(bound["rgb"], ref["rgb"])}})
    waves = []
    for i, (ms, st, rgb) in enumerate(wave_runs):
        ref_rgb = rgb_plain if i == 0 else runs[i - 1][2]
        waves.append({"sampler": "plain" if i == 0 else f"proposal {points[i - 1][0]}/{points[i - 1][1]}",
                      "ert_wave": args.ert_wave, "ms": round(ms, 3), "Mrays/s": round(n / (ms * 1e-3) / 1e6, 3),
                      "evaluated_per_ray": round(st["samples_evaluated"] / n, 3),
                      "generated_per_ray": spr(st), "composited_per_ray": round(st["samples_composited"] / n, 3),
                      "identical_to_one_pass": bool(np.array_equal(rgb, ref_rgb))})
    head = res[0]
    line = {
        "metric": "Mrays/s and samples per ray (learned proposal vs plain sampler)",
        "value": head["Mrays/s"], "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"{cfg.name} scene x{args.density_scale:g} density ({R.n_leaves} leaves, "
                               f"{cfg.hidden}x{cfg.width} BF16 MLPs, cap {cfg.cap}); "
                               f"proposal trained on {n_train_views} views at {tw}x{th}, evaluated on {views} "
                               f"held-out views at {px_w}x{px_h}",
                   "rays_per_step": n, "density_scale": args.density_scale, "oracle_rays": len(idx)},
        "plain": {"Mrays/s": round(n / (ms_plain * 1e-3) / 1e6, 3), "ms": round(ms_plain, 3),
                  "stage_ms": [round(x, 3) for x in st_plain["ms"]],
                  "samples_per_ray": spr(st_plain), "psnr_vs_fp64": p_plain,
                  "composited_frac": round(st_plain["samples_composited"] / max(st_plain["samples_generated"], 1), 4)},
        "proposal": res,
        **({"ert_waves": waves} if waves else {}),
        "spr_reduction": head["spr_reduction"],
        "delta_psnr_vs_fp64_db": head["delta_psnr_vs_fp64_db"],
        "training": {"rays": n_tr, "steps": args.train_steps, "batch": 8192, "lr": 3e-3,
                     "loss_first": round(float(losses[:50].mean()), 4), "loss_last": round(float(losses[-50:].mean()), 4),
                     "targets_s": round(t_targets, 2), "train_s": round(t_train, 2)},
        "clocks": clk.summary(),
    }
    if emit:
        print(json.dumps(line))
    R.close()
    return line


def run_reference(args):
    """The oracle (FP64 CPU program) on a bounded sample of the same workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    cfg = S.CONFIGS[args.config]
    grid, o_np, d_np = workload(cfg, 0)
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    cores = os.cpu_count() or 1
    per_step = args.ref_rays
    times, samples = [], []
    for i in range(args.warmup + args.steps):
        idx = S.ray_subset(len(o_np), per_step, 100 + i)
        t0 = time.perf_counter()
        ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o_np[idx], d_np[idx], cfg.steps, cfg.cap,
                       cfg.t_term, mode=0, threads=cores, jitter=args.jitter,
                       skip=(grid, args.skip_empty) if args.skip_empty is not None else None)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            samples.append(int(ref["n_gen"].sum()))
    tot_t, tot_s = sum(times), sum(samples)
    value = tot_s / tot_t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Msamples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t * 1e3 / len(times), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(cfg, args), "sample_rays_per_step": per_step},
        "mrays_per_s": round(per_step * len(times) / tot_t / 1e6, 6),
        "cpu_baseline": {"value": round(value, 6), "unit": "Msamples/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} seeded rays per step of the 800x800x8 workload"},
        "e2e": {"value": round(value, 6), "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--prec", default="fp32,bf16,fp8,fp8s")
    ap.add_argument("--psnr-rays", type=int, default=262144)
    ap.add_argument("--ref-rays", type=int, default=16384)
    ap.add_argument("--views", type=int, default=None, help="views per GPU (default: the config's)")
    ap.add_argument("--train-views", type=int, default=64, help="c5: plain-rendered training views")
    ap.add_argument("--train-steps", type=int, default=3000, help="c5: Adam steps")
    ap.add_argument("--density-scale", type=float, default=1.0, help="c5: factor on every density of the scene")
    ap.add_argument("--leaf-net", default="", help="c5: leaf network shape HxW (default: the scene config's)")
    ap.add_argument("--c5-scene", default="c4", choices=["c4", "c1"],
                    help="c5: the scene the proposal is trained and evaluated on (default: the 4096-leaf one)")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2: skip the c4 batching and c5 proposal summaries of the default line")
    ap.add_argument("--px", type=int, default=None, help="square image size (default: the config's)")
    ap.add_argument("--skip-empty", type=float, default=None,
                    help="empty-space skipping: density threshold of the guidance grid (c1/c2); default off")
    ap.add_argument("--ert-wave", type=int, default=0,
                    help="early ray termination in waves of this many crossings (0: one pass)")
    ap.add_argument("--lod-px", type=float, default=0.0,
                    help="adaptive hierarchical sampling: an inner node is refined only while wider than this "
                         "many pixels at the ray's entry distance (0: leaves only)")
    ap.add_argument("--jitter", type=int, default=0,
                    help="sample placement: 0 = stratum midpoints, else the stratified jitter's seed (c1/c2)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "c4":
        run_c4(args)
    elif args.config == "c5":
        run_c5(args)
    elif args.config == "ahs":
        print(json.dumps(run_ahs(args)))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
