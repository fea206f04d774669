"""Autotuner for the batched raster step: picks the tile shape, the number of
records staged per batch, persistent vs one-CTA-per-tile scheduling and the
raster forward + backward as one launch or two, by timing each candidate's
captured CUDA graph on the actual workload.

Results are cached in a JSON file keyed by (primitive count, lobes, view
resolutions, device name), so a workload is tuned once per machine.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import _lib
from .batched import BatchedStep

# (tile_w, tile_h, batch_s, persistent[, fused]): fused (default True) runs the
# raster forward, L1 loss and backward as one launch where the tile shape has
# pixel pairs (all but 8x4), False as two launches with hit masks
CANDIDATES = [
    (16, 16, 256, False), (16, 16, 128, True), (16, 8, 128, False), (16, 8, 64, False),
    (8, 8, 64, False), (8, 8, 128, False), (8, 4, 64, False),
    (16, 16, 256, False, False), (16, 8, 64, False, False),
]


def fused_of(cand) -> bool:
    return bool(cand[4]) if len(cand) > 4 else True


def cache_path() -> str:
    base = os.environ.get("BETA_AUTOTUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2501_18630_gb300", "autotune.json")


def workload_key(n: int, n_lobes: int, cameras, device) -> str:
    res = ",".join(f"{c.width}x{c.height}" for c in cameras)
    return f"v5;n={n};M={n_lobes};views={res};dev={torch.cuda.get_device_name(device)}"


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _save(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_candidate(planes, n, n_lobes, cameras, target, cand, reps=5, hit_masks=True):
    tw, th, s, persist = cand[:4]
    opts = _lib.default_opts(tile_w=tw, tile_h=th, batch_s=s)
    step = BatchedStep(planes, n, n_lobes, cameras, target, opts=opts, persistent=persist, hit_masks=hit_masks,
                       fused=fused_of(cand))
    step.step()
    step.check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del step
    torch.cuda.empty_cache()
    return ms


def tune(planes, n, n_lobes, cameras, target, candidates=None, reps=5, use_cache=True, log=None,
         hit_masks=True, fused=True):
    """Returns (best candidate, {candidate: ms}).  Candidates are tuples
    (tile_w, tile_h, batch_s, persistent[, fused]) (see CANDIDATES); with
    fused=False only two-launch candidates are timed."""
    cands = [tuple(c) for c in (candidates or CANDIDATES)]
    if not fused:
        cands = list(dict.fromkeys(c[:4] + (False,) for c in cands))
    key = (workload_key(n, n_lobes, cameras, planes.device) + f";hm={int(hit_masks)}"
           + ";cands=" + "|".join(",".join(str(int(x)) for x in c) for c in cands))
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        e = cache[key]
        return tuple(e["best"]), {tuple(json.loads(k)): v for k, v in e["times"].items()}
    times = {}
    for cand in cands:
        t0 = time.perf_counter()
        times[tuple(cand)] = time_candidate(planes, n, n_lobes, cameras, target, cand, reps, hit_masks)
        if log:
            log(f"autotune {cand}: {times[tuple(cand)]:.3f} ms ({time.perf_counter() - t0:.1f} s)")
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"best": list(best), "times": {json.dumps(list(k)): v for k, v in times.items()}}
        _save(cache)
    return best, times
