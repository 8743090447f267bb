"""Autotuner for the batched build + trace launch.

Times the persistent launch (grtBatchBuildTrace through its CUDA graph) over a grid
of launch shapes and keeps the fastest: threads per block, traversal stack entries
in shared memory, the warp refill (compaction) threshold, then, one knob at a time
from that point, the scenes per scheduling group, the rays per trace item, the radix
tiles per sort item and the largest scene built by a single block. Every candidate is a batch over the same
geometries and rays, so each run also rebuilds and retraces everything; the hit
records of every candidate are checked against the first one (all options give
bit-identical results). The winner is stored in a JSON cache keyed by the device
name and a signature of the workload.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import torch

from . import batch_options, grtGetLastDeviceError, GRT_SUCCESS
from .objects import Batch

GRID = dict(block_size=[64, 128, 256], shared_depth=[8, 16, 32], compact=[0.25, 0.5, 0.75])
REFINE = dict(scene_group=[8, 16, 64, 256], trace_chunk=[4096, 16384, 65536], sort_chunk_tiles=[2, 8, 32],
              small_scene_prims=[2048, 8192, 32768])
DEFAULTS = dict(block_size=128, shared_depth=16, compact=0.75, trace_chunk=16384, sort_chunk_tiles=8,
                small_scene_prims=8192, scene_group=32)


def default_cache_path() -> str:
    return os.environ.get("GRT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "grt", "autotune.json"))


def workload_key(scenes) -> str:
    """Device name plus the scene count, total primitives and total rays (rounded to
    two significant digits, so reruns of the same workload share an entry)."""
    def sig(x):
        return float(f"{float(x):.2g}")
    prims = sum(int(g.input.triangleMesh.triangleCount) for g, _, _ in scenes)
    rays = sum(int(r.shape[0]) for _, r, _ in scenes)
    return f"{torch.cuda.get_device_name()}|scenes={len(scenes)}|prims={sig(prims)}|rays={sig(rays)}"


def _time_batch(ctx, scenes, opts: dict, repeats: int, reference=None):
    B = Batch(ctx, scenes, batch_options(graph=True, **opts))
    try:
        B.run()  # capture + first run
        torch.cuda.synchronize()
        if grtGetLastDeviceError(ctx.handle) != GRT_SUCCESS:
            return None
        if reference is not None:
            for ref, (_, _, h) in zip(reference, scenes):
                if not torch.equal(ref, h):
                    raise RuntimeError(f"batch options {opts} changed the hit records")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        best = float("inf")
        for _ in range(repeats):
            ev[0].record()
            B.run()
            ev[1].record()
            ev[1].synchronize()
            best = min(best, ev[0].elapsed_time(ev[1]))
        return best
    finally:
        B.close()


def tune(ctx, scenes, repeats: int = 3, cache_path: str | None = None, use_cache: bool = True,
         log=None) -> tuple[dict, dict]:
    """Best batch options for `scenes` (a list of (Geometry, rays, hits)), and a report
    {tried: [(options, ms)], seconds, key, cached}. The scenes' hit tensors are
    overwritten by the trial runs."""
    cache_path = cache_path or default_cache_path()
    key = workload_key(scenes)
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return dict(cache[key]["options"]), {"key": key, "cached": True, "ms": cache[key]["ms"], "tried": []}
    t0 = time.time()
    tried = []
    base = _time_batch(ctx, scenes, DEFAULTS, 1)
    reference = [h.clone() for _, _, h in scenes]

    def trial(opts):
        ms = _time_batch(ctx, scenes, opts, repeats, reference)
        tried.append((dict(opts), ms))
        if log:
            log(f"autotune {opts} -> {ms}")
        return ms if ms is not None else float("inf")

    best, best_ms = dict(DEFAULTS), float("inf")
    for values in itertools.product(*GRID.values()):
        opts = dict(DEFAULTS, **dict(zip(GRID.keys(), values)))
        ms = trial(opts)
        if ms < best_ms:
            best, best_ms = opts, ms
    for name, values in REFINE.items():
        for v in values:
            if v == best[name]:
                continue
            opts = dict(best, **{name: v})
            ms = trial(opts)
            if ms < best_ms:
                best, best_ms = opts, ms
    report = {"key": key, "cached": False, "ms": best_ms, "default_ms": base, "tried": tried,
              "seconds": round(time.time() - t0, 1)}
    cache[key] = {"options": best, "ms": best_ms}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return best, report
