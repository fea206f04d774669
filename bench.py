#!/usr/bin/env python
"""Benchmark of the Beta-splatting rasterizer hot path on GB300.

One step = forward + backward of every view of a batch through the whole hot
path (project -> bin/sort -> raster fwd -> L1 loss -> raster bwd -> project
bwd) on seeded synthetic inputs: 1M Betas (256 planar sheets, 3 spherical-Beta
lobes), views of 1920x1080 on a ring of radius 4.  The batched path runs
every view in the same launches; the plain per-view path (the baseline of the
batched speedup) runs the same entry points one view at a time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--views V] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank renders its own
views (weak scaling) and the parameter gradients are summed with one NCCL
all-reduce per step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/view and Mpixels/s at 1M Betas 1080p; batched vs per-view speedup"
UNIT = "Mpixel/s"
FWD_FLOPS_PER_EVAL = 24   # r^2 (11), 1 - r^2, beta lg2 + log2 o, min, T alpha, C += (6), T update
BWD_FLOPS_PER_EVAL = 60   # recompute alpha, T recovery, dL/dalpha, 10 gradient terms
FP32_LANES_PER_SM = 128
# raster_fwd includes the per-view L1 loss (computed in the forward's epilogue);
# with the one-launch raster kernel (every tile shape but 8x4) the stage
# "raster" is the forward, the L1 term and the backward together
STAGES = ["project", "bin_sort", "raster_fwd", "raster_bwd", "project_bwd"]
STAGES_FUSED = ["project", "bin_sort", "raster", "project_bwd"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--n", type=int, default=None, help="Betas (default: the workload's, 1M for workload 3)")
    ap.add_argument("--width", type=int, default=None, help="view width (default: the workload's)")
    ap.add_argument("--height", type=int, default=None, help="view height (default: the workload's)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip per-view, e2e and CPU legs (profiling runs)")
    ap.add_argument("--cpu-pixels", type=int, default=16384)
    ap.add_argument("--workload", type=int, default=3, choices=[3, 4, 5],
                    help="scene recipe: 3 = 1M Betas (default), 4 = 3M Betas, 5 = 6M Betas")
    ap.add_argument("--raster", choices=["fused", "split"], default="fused",
                    help="fused: the autotuner (or --config) may run the raster forward + L1 + backward in one "
                         "launch per tile; split: always two launches (8x4 tiles always split)")
    ap.add_argument("--hit-masks", choices=["on", "off"], default="on",
                    help="the forward keeps its cover pass for the backward (on), or the backward recomputes "
                         "it (off)")
    ap.add_argument("--config", default=None,
                    help="pin the raster configuration instead of autotuning, e.g. 16x16/256/P (P persistent, G one CTA per tile)")
    return ap.parse_args()


def _size(args):
    """An explicit --width/--height pair, else None (the workload's sizes)."""
    if (args.width is None) != (args.height is None):
        raise SystemExit("give both --width and --height, or neither")
    return (args.width, args.height) if args.width is not None else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows]
        out["samples"] = len(rows)
        out["sm_mhz"] = statistics.median(sm)
        out["sm_max_mhz"] = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for k, name in enumerate(names):
            if any(r[5 + k].lower().startswith("active") for r in rows):
                out["reasons"].append(name)
        return out


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("beta_raster.cu", "beta_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2501_18630_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, launch_units: float):
    """dram bytes per launch of `kernel` from the committed ncu summary, scaled
    to this launch; None if absent or if the kernel source changed since."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
        e = d["kernels"][kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_unit"]) * launch_units
    except Exception:
        return None


def ncu_metric(kernel: str, name: str):
    """A per-kernel figure from the committed ncu summary, or None if absent or
    if the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        e = json.load(open(p))["kernels"][kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e.get(name)
    except Exception:
        return None


REC_BYTES = 48          # raster record read per (tile, Beta) pair
PROJ_BYTES = 64         # record + tile rectangle + depth key + tile mask written per (view, Beta)
GRAD2D_BYTES = 48       # 2D-gradient slot per (view, Beta)


def hbm_roofline(stage_ms, ms_step, n, param_bytes, n_rec, K, px, peak, peak_src):
    """Algorithmic bytes of every stage (each stream counted once) over its
    CUDA-event time, against the measured HBM copy bandwidth:
      project      params read + records written         n P + n_rec 64
      bin_sort     rectangles and tile masks twice,      n_rec 28 + K 20
                   keys once per record,
                   item written + read + id written per pair
      raster_fwd   record + list index per pair, colour, K 52 + px (20 + 12 + 12)
                   T, n_contrib written, target read, dL/dC written
      raster_bwd   record + index per pair, dL/dC, T,    K 52 + px 20 + n_rec 48
                   n_contrib read, 2D-gradient slots accumulated
      project_bwd  2D-gradient slots read and cleared,   n_rec 96 + 2 n P
                   params read, gradients written
      raster       (the one-launch forward + L1 + backward) charged the sum
                   of raster_fwd and raster_bwd above: the method's streams,
                   although T, n_contrib and dL/dC stay in registers there"""
    b = {"project": n * param_bytes + n_rec * PROJ_BYTES,
         "bin_sort": n_rec * 28 + K * 20,
         "raster_fwd": K * (REC_BYTES + 4) + px * (20 + 12 + 12),
         "raster_bwd": K * (REC_BYTES + 4) + px * 20 + n_rec * GRAD2D_BYTES,
         "project_bwd": n_rec * 2 * GRAD2D_BYTES + 2 * n * param_bytes}
    if "raster" in stage_ms:
        b = {"project": b["project"], "bin_sort": b["bin_sort"], "raster": b["raster_fwd"] + b["raster_bwd"],
             "project_bwd": b["project_bwd"]}
    out = {"peak_gbs": peak, "peak_kind": f"{peak_src} copy bandwidth", "stages": {}}
    for k, v in b.items():
        ms = stage_ms.get(k, 0.0)
        gbs = v / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        out["stages"][k] = {"bytes": v, "ms": ms, "gbs": gbs, "frac": gbs / peak}
    tot = sum(b.values())
    out["step"] = {"bytes": tot, "ms": ms_step, "gbs": tot / (ms_step * 1e-3) / 1e9,
                   "frac": tot / (ms_step * 1e-3) / 1e9 / peak}
    out["target_frac"] = 0.5
    out["target_met"] = out["step"]["frac"] >= 0.5
    return out


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_leg(args, cams, sc, pixels_per_step, steps, warmup):
    import numpy as np

    import oracle
    from paper_2501_18630_gb300 import scenes
    oracle.build()
    cores = os.cpu_count() or 1
    times = []
    for s in range(warmup + steps):
        cam = cams[s % len(cams)]
        xs, ys = scenes.sample_pixels(cam, pixels_per_step, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.render(sc.planes, sc.n, sc.n_lobes, cam, xs, ys, n_threads=cores)
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
    total = sum(times)
    value = pixels_per_step * len(times) / total / 1e6
    return value, cores, total


def oracle_full_frame():
    """The oracle on the small workload, full frame: 4,096 Betas at 256x256,
    one view, forward only, all host cores."""
    import oracle
    from paper_2501_18630_gb300 import scenes
    oracle.build()
    sc1 = scenes.config_scene(1)
    cam = sc1.cameras[0]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.render_full(sc1.planes, sc1.n, sc1.n_lobes, cam, n_threads=cores)
    dt = time.perf_counter() - t0
    px = cam.width * cam.height
    return {"ms_per_view": dt * 1e3, "value": px / dt / 1e6, "unit": UNIT, "cores": cores,
            "what": f"{sc1.n} Betas, {cam.width}x{cam.height}, every pixel, forward only"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2501_18630_gb300 import scenes
    sc = scenes.config_scene(args.workload, n=args.n, n_views=args.views)
    cams = scenes.ring_cameras(args.views, 4.0, 15.0, scenes.workload_sizes(args.workload, args.views, _size(args)))
    px = 1024
    value, cores, total = oracle_leg(args, cams, sc, px, args.steps, args.warmup)
    ms = total / args.steps * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{sc.n} Betas (256 sheets, 3 SB lobes), {args.views} views "
                               f"{scenes.describe_sizes(cams)}; FP64 oracle forward on {px} sampled pixels per step",
                   "n_betas": sc.n, "views": args.views},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{px} seeded pixels of one view per step, forward only (the oracle has no backward)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2501_18630_gb300 import _lib, distributed, render, scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    _lib.load()

    V = args.views
    sc = scenes.config_scene(args.workload, n=args.n, n_views=V)
    ring = scenes.ring_cameras(V * world, 4.0, 15.0, scenes.workload_sizes(args.workload, V * world, _size(args)))
    cams = distributed.shard_views(ring, rank, world)
    planes = torch.from_numpy(sc.planes).to(dev)
    targets_np = scenes.target_images(cams, seed=77 + rank)
    target = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets_np])).to(dev)
    grad = torch.zeros_like(planes)

    # ---- autotuned batched step, captured as one CUDA graph -----------------
    from paper_2501_18630_gb300 import autotune, batched
    hit_masks = args.hit_masks == "on"
    t_tune = time.perf_counter()
    if args.config:
        shape, bsz, mode = args.config.split("/")
        tw_, th_ = (int(x) for x in shape.split("x"))
        best, tune_ms = (tw_, th_, int(bsz), mode.upper() == "P", args.raster == "fused"), {}
    else:
        best, tune_ms = autotune.tune(planes, sc.n, sc.n_lobes, cams, target, reps=3, hit_masks=hit_masks,
                                      fused=args.raster == "fused",
                                      log=(lambda m: print(m, file=sys.stderr)) if rank == 0 else None)
    t_tune = time.perf_counter() - t_tune
    tw, th, bs, persist = best[:4]
    opts = _lib.default_opts(tile_w=tw, tile_h=th, batch_s=bs)
    # on several GPUs the projection backward runs after the replay in chunks,
    # each chunk's gradient all-reduce overlapping the next chunks
    bstep = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, target, opts=opts, persistent=persist,
                                hit_masks=hit_masks, graph_project_bwd=world == 1, fused=autotune.fused_of(best))
    rast = bstep.rast
    grad = bstep.grad

    def step():
        bstep.step()
        if world > 1:
            bstep.project_bwd_reduced()

    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return distributed.max_over_ranks(x, dev)

    for _ in range(args.warmup):
        step()
    K = bstep.check()

    # ---- timed region: K replays of the captured batched step --------------
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    clocks = clk.summary()
    st, K = rast.device_status()
    if st != 0:
        raise SystemExit(f"device status {st} in the timed region")
    pix_per_step = rast.total_pixels * world
    value = pix_per_step / (ms_step * 1e-3) / 1e6

    # ---- per-stage times (separate loop, events between the entry points) ---
    fused = bstep.fused
    stages = STAGES_FUSED if fused else STAGES
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
    stage_ms = {s: 0.0 for s in stages}
    for _ in range(args.steps):
        ev[0].record(stream)
        rast.project(planes); ev[1].record(stream)
        rast.bin_sort(planes)
        if rast.persistent:
            rast.schedule()
        ev[2].record(stream)
        if fused:
            rast.raster_fwd_bwd_l1(planes, target); ev[3].record(stream)
        else:
            rast.raster_fwd_l1(planes, target); ev[3].record(stream)
            rast.raster_bwd(planes, rast.dL_dcolor); ev[4].record(stream)
        rast.project_bwd(planes, grad); ev[len(stages)].record(stream)
        torch.cuda.synchronize()
        for k, s in enumerate(stages):
            stage_ms[s] += ev[k].elapsed_time(ev[k + 1]) / args.steps

    # ---- roofline of the dominant kernel -----------------------------------
    hbm_peak, sm_max_mhz, peak_src = peaks()
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    dom = max(stage_ms, key=stage_ms.get)
    rec = rast.proj[: V * rast.pitch * 48].view(torch.float32).view(V, rast.pitch, 12)
    keys = rast.proj[V * rast.pitch * 56: V * rast.pitch * 60].view(torch.int32).view(V, rast.pitch)
    binned = keys != -1
    area = math.pi / (rec[..., 4] * rec[..., 5]).clamp_min(1e-30)          # pi sqrt(det Sigma')
    view_px = torch.tensor([float(c.width * c.height) for c in cams], device=area.device).view(V, 1)
    evals = float(torch.where(binned, torch.minimum(area, view_px), torch.zeros_like(area)).sum().item())
    alu_peak = n_sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12    # TFLOP/s
    n_planes = scenes.n_planes(sc.n_lobes)
    hbm = hbm_roofline(stage_ms, ms_step, sc.n, n_planes * 4, V * sc.n, K, rast.total_pixels, hbm_peak,
                       peak_src)
    if dom in ("raster_fwd", "raster_bwd", "raster"):
        fl = {"raster_fwd": FWD_FLOPS_PER_EVAL, "raster_bwd": BWD_FLOPS_PER_EVAL,
              "raster": FWD_FLOPS_PER_EVAL + BWD_FLOPS_PER_EVAL}[dom]
        achieved = evals * fl / (stage_ms[dom] * 1e-3) / 1e12
        kname = {"raster_fwd": "k_raster_fwd", "raster_bwd": "k_raster_bwd", "raster": "k_raster_step"}[dom]
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": ncu_traffic(kname, rast.total_pixels),
                "peak_source": f"{n_sms} SMs x 128 FP32 lanes x 2 flop x max SM clock",
                "algorithmic": f"{fl} flop x {evals:.4g} (pixel, Beta) evaluations inside the support (ellipse areas)"}
    else:
        nrec = V * sc.n
        bytes_alg = {"project": sc.n * n_planes * 4 + nrec * PROJ_BYTES,
                     "bin_sort": nrec * 28 + K * 20,
                     "l1": rast.total_pixels * 3 * 4 * 3,
                     "project_bwd": nrec * 48 * 2 + sc.n * n_planes * 8}.get(dom, 0)
        achieved = bytes_alg / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None}
    roof["peak_kind"] = f"{peak_src} (max SM clock {sm_max_mhz:.0f} MHz)" if roof["bound"] == "alu" else peak_src
    roof["hbm"] = hbm
    roof["issue_active"] = {k: ncu_metric(k, "issue_active_pct")
                            for k in (("k_raster_step",) if fused else ("k_raster_fwd", "k_raster_bwd"))}

    extras = {}
    if not args.no_extras:
        # ---- plain per-view path (baseline of the batched speedup) ----------
        singles = [render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, [c], device=dev) for c in cams]
        gview = [torch.zeros_like(planes) for _ in cams]
        tv = [target[3 * rast.pix_off[v]: 3 * rast.pix_off[v] + 3 * c.width * c.height] for v, c in enumerate(cams)]
        for s in singles:
            s.forward(planes, check_capacity=True)
            _, k = s.device_status()
            s._alloc_pairs(int(k * 1.1) + 65536)

        def step_views():
            for v, s in enumerate(singles):
                s.project(planes)
                s.bin_sort(planes)
                s.raster_fwd(planes)
                s.l1_loss(tv[v])
                s.raster_bwd(planes, s.dL_dcolor)
                s.project_bwd(planes, gview[v])

        for _ in range(args.warmup):
            step_views()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step_views()
        e1.record(stream)
        barrier()
        ms_views = max_over_ranks(e0.elapsed_time(e1)) / args.steps
        extras["per_view_path"] = {"ms_per_step": ms_views, "ms_per_view": ms_views / V,
                                   "value": pix_per_step / (ms_views * 1e-3) / 1e6}
        extras["batched_speedup"] = ms_views / ms_step
        del singles, gview

        # ---- end to end through host buffers --------------------------------
        # Every step copies its inputs (parameters, targets) from pinned host
        # memory and reads its results (gradients, losses) back, inside the
        # timed region.  Two captured steps with their own input and output
        # buffers alternate, so that step i+1's inputs land (copy-in stream)
        # while step i runs and step i's results leave (copy-out stream) while
        # step i+1 runs, with no device-side staging copies.
        h_planes = torch.from_numpy(sc.planes).pin_memory()
        h_target = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets_np])).pin_memory()
        h_grad = torch.empty(planes.shape, dtype=torch.float32).pin_memory()
        h_loss = torch.empty(V, dtype=torch.float32).pin_memory()
        twin = batched.BatchedStep(torch.empty_like(planes).copy_(planes), sc.n, sc.n_lobes, cams,
                                   torch.empty_like(target).copy_(target), opts=opts, persistent=persist,
                                   hit_masks=hit_masks, graph_project_bwd=world == 1, fused=bstep.fused)
        twin.capture()
        steps2 = [bstep, twin]
        cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_sent = [torch.cuda.Event() for _ in range(2)]
        for e in ev_free + ev_sent:
            e.record(stream)

        def h2d(i):
            b = i % 2
            with torch.cuda.stream(cin):
                cin.wait_event(ev_free[b])          # the step that last read these inputs is done
                steps2[b].planes.copy_(h_planes, non_blocking=True)
                steps2[b].target.copy_(h_target, non_blocking=True)
                ev_in[b].record(cin)

        def step_e2e(i, n):
            b = i % 2
            stream.wait_event(ev_in[b])             # inputs landed
            stream.wait_event(ev_sent[b])           # the previous results of these buffers left
            if i + 1 < n:
                h2d(i + 1)
            steps2[b].step()
            if world > 1:
                steps2[b].project_bwd_reduced()
            ev_free[b].record(stream)
            ev_out[b].record(stream)
            with torch.cuda.stream(cout):
                cout.wait_event(ev_out[b])
                h_grad.copy_(steps2[b].grad, non_blocking=True)
                h_loss.copy_(steps2[b].loss, non_blocking=True)
                ev_sent[b].record(cout)

        h2d(0)
        for i in range(args.warmup):
            step_e2e(i, args.warmup)
        stream.wait_stream(cin)
        stream.wait_stream(cout)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        h2d(0)
        for i in range(args.steps):
            step_e2e(i, args.steps)
        stream.wait_stream(cout)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1)) / args.steps
        st_tw, k_tw = twin.rast.device_status()
        if st_tw != _lib.BETA_OK:
            raise _lib.BetaError("e2e step", st_tw, _lib.load().beta_status_string(st_tw).decode())
        extras["e2e"] = {"value": pix_per_step / (ms_e2e * 1e-3) / 1e6, "unit": UNIT,
                         "h2d_bytes_per_step": (h_planes.numel() + h_target.numel()) * 4 * world,
                         "d2h_bytes_per_step": (h_grad.numel() + h_loss.numel()) * 4 * world,
                         "ms_per_step": ms_e2e,
                         "copies": "pipelined on copy-in / copy-out streams, two alternating captured steps"}
        del twin, steps2

        # ---- the optimiser step after the backward (Sec. 3.4), HBM-bound ----
        from paper_2501_18630_gb300.optim import BetaAdam
        opt_planes = planes.clone()
        adam = BetaAdam(opt_planes, sc.n, sc.n_lobes)
        eta = torch.randn(3, sc.pitch, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            adam.step(opt_planes, grad, eta)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        t_opt = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)                       # inputs do not stay in L2 between steps
            e0.record(stream)
            adam.step(opt_planes, grad, eta)
            e1.record(stream)
            torch.cuda.synchronize()
            t_opt += e0.elapsed_time(e1)
        ms_opt = t_opt / args.steps
        opt_bytes = sc.n * (7 * 4 * n_planes + 12)
        extras["optimizer_step"] = {
            "ms": ms_opt, "n_betas": sc.n, "algorithmic_bytes": opt_bytes,
            "achieved_gbs": opt_bytes / (ms_opt * 1e-3) / 1e9,
            "frac_of_measured_hbm": opt_bytes / (ms_opt * 1e-3) / 1e9 / hbm_peak,
            "what": "beta_adam_step: Adam + regulariser gradients + Beta-scaled position noise on all raw "
                    "parameters (reads params, grads, 2 moments, noise; writes params, 2 moments); L2 flushed "
                    "before each timed launch"}
        # relocation of dead primitives (the scene's opacity logits, threshold 0.005)
        n_dead = 0
        for _ in range(2):
            reloc_planes = planes.clone()
            radam = BetaAdam(reloc_planes, sc.n, sc.n_lobes)
            torch.cuda.synchronize()
            e0.record(stream)
            cnt, _ = radam.relocate(reloc_planes, 0.005)
            e1.record(stream)
            torch.cuda.synchronize()
            n_dead = int(cnt.item())
        extras["relocation"] = {"ms": e0.elapsed_time(e1), "n_betas": sc.n, "relocated": n_dead,
                                "what": "beta_relocate: fixed-rule opacities, 64-bit cumulative weights, one "
                                        "binary search per dead primitive, opacity-only update, copies"}
        del opt_planes, adam, flush, reloc_planes, radam

        # ---- the composite loss with the DSSIM term (Sec. 3.4), HBM-bound ---
        for _ in range(args.warmup):
            rast.dssim_loss(target, 0.2)
        t_ss = 0.0
        for _ in range(args.steps):
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev).fill_(1.0)
            e0.record(stream)
            rast.dssim_loss(target, 0.2)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ss += e0.elapsed_time(e1)
            del flush
        ms_ss = t_ss / args.steps
        # the L1 term's share of the step: forward with it minus forward without it
        t_fl = {"plain": 0.0, "l1": 0.0}
        for _ in range(args.steps):
            for kind in ("plain", "l1"):
                flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev).fill_(1.0)
                e0.record(stream)
                if kind == "plain":
                    rast.raster_fwd(planes)
                else:
                    rast.raster_fwd_l1(planes, target)
                e1.record(stream)
                torch.cuda.synchronize()
                t_fl[kind] += e0.elapsed_time(e1) / args.steps
                del flush
        l1_ms = max(0.0, t_fl["l1"] - t_fl["plain"])
        ss_bytes = rast.total_pixels * 3 * 44
        extras["dssim_loss"] = {
            "ms": ms_ss, "l1_ms": l1_ms, "step_ms_with_dssim": ms_step - l1_ms + ms_ss,
            "algorithmic_bytes": ss_bytes, "achieved_gbs": ss_bytes / (ms_ss * 1e-3) / 1e9,
            "frac_of_measured_hbm": ss_bytes / (ms_ss * 1e-3) / 1e9 / hbm_peak,
            "what": "beta_l1_dssim_loss, lambda 0.2: Gaussian-window SSIM statistics, loss and gradient "
                    "(x, y read twice, three partial-derivative planes written and read once, dL/dC "
                    "written: 44 B per channel-pixel); L2 flushed before each timed launch"}

        # ---- the oracle on the host cores (bounded sample) -------------------
        if rank == 0 and world == 1:
            v_cpu, cores, tot = oracle_leg(args, cams[:1], sc, args.cpu_pixels, 1, 0)
            view_px = cams[0].width * cams[0].height
            c1 = oracle_full_frame()
            extras["cpu_baseline"] = {
                "value": v_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{args.cpu_pixels} seeded pixels of view 0 of the same workload, forward only "
                          f"(FP64, every Beta per pixel), {tot:.1f} s on {cores} threads",
                "ms_per_view_extrapolated": tot * 1e3 * view_px / args.cpu_pixels,
                "extrapolation": f"linear in pixels: the sample's time x {view_px} / {args.cpu_pixels} "
                                 f"(one {cams[0].width}x{cams[0].height} view, forward only)",
                "full_frame_4096_betas_256x256": c1}

    # kernel launches of ours inside the timed region (all inside the replayed graph on
    # one GPU): project 3 (worklist reset, projection, rule-B2 tiles); bin_sort 5 (prep,
    # tile counts, scan, scatter, list sort); schedule 3 (persistent); raster fwd with
    # the L1 term 2 and raster bwd 1, or the one-launch raster kernel and the L1
    # reduce 2; project bwd 1 (one per chunk on several GPUs)
    from paper_2501_18630_gb300.distributed import chunk_ranges
    n_pbwd = len(chunk_ranges(sc.n, max(4, (sc.n + 7) // 8))) if world > 1 else 1
    per_step = 3 + 5 + (3 if rast.persistent else 0) + (2 if fused else 3) + n_pbwd
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{sc.n} Betas (256 planar sheets, 3 SB lobes), {V} views {scenes.describe_sizes(cams)} "
                               f"per GPU, fwd+bwd with per-view L1 loss, one CUDA-graph replay per step",
                   "tile": f"{tw}x{th}", "batch_s": bs, "persistent": persist,
                   "raster": "one launch (forward + L1 + backward)" if fused else "forward + L1, backward",
                   "hit_masks": hit_masks and not fused,
                   "autotune": {"s": round(t_tune, 1),
                                "ms": {f"{c[0]}x{c[1]}/S{c[2]}/{'P' if c[3] else 'G'}"
                                       f"{'' if autotune.fused_of(c) else '/split'}": round(v, 3)
                                       for c, v in tune_ms.items()}},
                   "n_betas": sc.n, "views_per_gpu": V, "resolution": scenes.describe_sizes(cams),
                   "pairs_per_step": K, "l2": f"inputs larger than L2: {sc.n * n_planes * 4 / 1e6:.0f} MB params + "
                                               f"{V * sc.pitch * 64 / 1e6:.0f} MB records per step",
                   "parallelism": f"dp{world} over views"},
        "ms_per_view": ms_step / V,
        "stage_ms": stage_ms,
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": per_step * args.steps,
        "kernel_source": kernel_source_hash(),
    }
    line.update({k: v for k, v in extras.items()})
    if "cpu_baseline" not in line and world == 1 and not args.no_extras:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
