#!/usr/bin/env python3
"""Throughput benchmark of the GPU ray tracer on the two-level ambient-occlusion workload.

Workload (synthetic, seeded): one procedural terrain mesh (256x256 cells, 131,072
triangles, 4-octave value noise of amplitude 0.2) instanced 64 times under random SRT
frames (uniform rotation, per-axis scale in [0.5, 2], translation in [-10, 10]^3);
a 1920x1080 pinhole camera at the scene centre + (0, 0, 1.5 * extent) with 60 degree
vertical field of view; at every primary hit 8 cosine-weighted hemisphere rays of
length 0.05 * extent traced as any-hit queries.

One step = the whole hot path: bottom-level LBVH build (primitive boxes, centroid
bounds, Morton codes, radix sort, Karras emission, bottom-up fit, 8-wide nodes),
top-level build over the instances (8-wide nodes), camera ray generation, closest-hit
traversal of the primary rays, and the fused ambient-occlusion kernel (ray generation +
any-hit traversal).
value = (primary rays + AO rays) / step time, in Mrays/s, all ranks together; each
rank runs its own replica (the path shards by independent replicas, so no collective
touches the data path). L2 is flushed (512 MB write) between timed steps, outside the
timed region.

`--impl reference` times the CPU oracle (FP64, oracle/) on a bounded sample of the
same workload on the host cores.

`--workload batched-soups-256` times 256 uneven triangle soups (1e3 to 2e6 triangles,
4,096 to 2^20 rays each): all builds and closest-hit traces in one persistent launch
(CUDA graph, autotuned options) against 256 sequential per-scene build + trace calls.

`--workload lambert-adjoint-1080p` prints a second kind of line instead: differentiable
Lambert shading of a 642-vertex icosphere at 1920x1080 (closest hit, shading with one
shadow any-hit ray per lit pixel), forward alone against forward + adjoint backward,
with the hit records stored (21 bytes per pixel) or recomputed by the backward pass.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s closest/any-hit, % of mem roofline; batched & adjoint vs plain same GPU"
UNIT = "Mrays/s"
WORKLOAD = dict(workload="terrain64-ao-1080p", instances=64, terrain_cells=256, triangles_per_instance=131072,
                width=1920, height=1080, ao_samples=8, ao_length="0.05*extent", seed=20260301)
RAY_BYTES, HIT_BYTES = 32, 20
NODE_BYTES, TRI_BYTES, INST_BYTES = 112, 48, 128  # a 4-wide node visit reads 7 of its 8 float4
NODE8_BYTES = 224  # an 8-wide node visit reads 14 of its 16 float4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="grt", choices=["grt", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--workload", default=WORKLOAD["workload"],
                   choices=[WORKLOAD["workload"], "icosphere-512", "spheres-1m", "lambert-adjoint-1080p",
                            "batched-soups-256"],
                   help="the two-level ambient-occlusion throughput workload (default), the single-icosphere "
                        "primary-ray one, the million-sphere custom-primitive one, the differentiable-shading one, "
                        "or the batched many-scenes one")
    p.add_argument("--image", default=None, metavar="WxH",
                   help="terrain workload: another image size (a smaller case, e.g. for a profiler)")
    p.add_argument("--no-autotune", action="store_true", help="batched workload: default launch options")
    p.add_argument("--scenes", type=int, default=256, help="batched workload: the first N soups (a smaller case)")
    p.add_argument("--no-sequential", action="store_true",
                   help="batched workload: skip the 256 sequential per-scene calls (e.g. under a profiler)")
    p.add_argument("--no-clustered", action="store_true",
                   help="batched workload: skip the second run with subtree-clustered builds")
    p.add_argument("--no-quantized", action="store_true",
                   help="batched workload: skip the run with quantised 64-byte nodes")
    p.add_argument("--no-split", action="store_true",
                   help="batched workload: skip the per-scene run with split triangles")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, dist=None, device: str = "cuda"):
    """Element-wise maximum of per-rank timings over all ranks (each rank runs its own
    replica; the job takes as long as its slowest rank). Without a process group the
    values are returned as they are."""
    values = [float(v) for v in values]
    if dist is None:
        return values
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank processed units_per_rank (weak
    scaling) in at most `seconds`."""
    return world * units_per_rank / seconds


def workload():
    import scenegen

    sc = scenegen.terrain_instances(WORKLOAD["instances"], WORKLOAD["terrain_cells"], 0.2, WORKLOAD["seed"])
    cam = scenegen.overview_camera(sc, WORKLOAD["width"], WORKLOAD["height"])
    return sc, cam


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# The translation unit that holds each kernel whose DRAM traffic bench.py reports.
KERNEL_UNITS = {"aoTraceKernel": "trace.cu", "traceKernel<closest, scene>": "trace.cu",
                "traceKernel<closest, geometry> icosphere-512": "trace.cu",
                "traceKernel<closest, geometry> spheres-1m": "trace.cu",
                "traceKernel<any, geometry> spheres-1m": "trace.cu",
                "shadeBackwardKernel<false, true>": "trace.cu", "batchKernel": "batch.cu"}


def code_only(src: str) -> str:
    """C/C++ source without its comments and without blank space (runs of spaces and tabs
    collapsed, lines trimmed, empty lines dropped); string and character literals kept."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (re.sub(r"[ \t]+", " ", line).strip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def source_hash(unit: str) -> str:
    """Hash of a translation unit of the library as compiled: the code (comments and blank
    space removed) of the .cu file and of every header it includes (transitively, by
    #include "..."), and the build script with its flags. A change to comments alone leaves
    the hash, and the DRAM traffic recorded under it, as they were."""
    csrc = os.path.join(ROOT, "paper_2603_00292_gb300", "csrc")
    seen, todo = [], [os.path.join(csrc, unit)]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in seen:
            continue
        seen.append(f)
        with open(f) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith('#include "'):
                    todo.append(os.path.join(os.path.dirname(f), line.split('"')[1]))
    h = hashlib.sha256()
    for f in sorted(seen):
        with open(f) as fh:
            h.update(os.path.relpath(f, ROOT).encode() + code_only(fh.read()).encode())
    with open(os.path.join(ROOT, "paper_2603_00292_gb300", "build.py"), "rb") as fh:
        h.update(b"paper_2603_00292_gb300/build.py" + fh.read())
    return h.hexdigest()[:16]


def ncu_record(kernel: str):
    """The committed ncu record of `kernel` (profiles/ncu_traffic.json), if it was taken
    from the kernel's current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(KERNEL_UNITS[kernel]):
        return None
    return e


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu record, if it was taken
    from the kernel's current sources (else None)."""
    e = ncu_record(kernel)
    return None if e is None else e.get("dram_bytes_per_launch")


# What bounds each traversal kernel when no current ncu record says so: the unit with
# the highest ncu utilisation in the last capture (profiles/): instruction issue for
# the terrain kernels, L1 for the sphere and icosphere traversals, DRAM for the batch.
STATIC_BOUND = {"aoTraceKernel": "issue", "traceKernel<closest, scene>": "issue",
                "traceKernel<closest, geometry> icosphere-512": "l1",
                "traceKernel<closest, geometry> spheres-1m": "l1", "traceKernel<any, geometry> spheres-1m": "l1",
                "shadeBackwardKernel<false, true>": "issue", "batchKernel": "issue"}


def kernel_bound(kernel: str, peak_gbs: float):
    """(bound, counters): the unit with the highest utilisation in the kernel's current
    ncu record among L1, L2, DRAM and instruction issue, with those percentages; or the
    static label and None without a current record."""
    e = ncu_record(kernel)
    if not e or "l1_pct" not in e:
        return STATIC_BOUND.get(kernel, "hbm"), None
    dram_pct = e.get("dram_pct")  # recorded where the capture was scaled to a larger launch
    if dram_pct is None:
        dram_pct = 100.0 * e["dram_bytes_per_launch"] / (e["duration_ns"] * 1e-9) / 1e9 / peak_gbs
    util = {"l1": e["l1_pct"], "l2": e["l2_pct"], "hbm": round(dram_pct, 2), "issue": e["issue_pct"]}
    counters = dict(util, memory_sol_pct=e.get("mem_sol_pct"), l2_hit_pct=e.get("l2_hit_pct"),
                    warps_active_pct=e.get("warps_active_pct"), lanes_per_instruction=e.get("lanes_per_inst"))
    return max(util, key=util.get), counters


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU arm
def run_grt(args, rank, world, local):
    import torch

    import paper_2603_00292_gb300 as grt
    from paper_2603_00292_gb300 import build as grt_build
    from paper_2603_00292_gb300.objects import Context, FuncTable, Geometry, Scene, device_tensor, new_hits, new_rays

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        grt_build.build()
    if dist:
        dist.barrier()

    sc, cam = workload()
    W, H, spp = WORKLOAD["width"], WORKLOAD["height"], WORKLOAD["ao_samples"]
    npix = W * H
    length = float(np.float32(0.05 * sc.extent))
    seed = WORKLOAD["seed"]
    mesh = sc.meshes[0]
    ctx = Context(local)
    verts = device_tensor(mesh.vertices)
    idx = device_tensor(mesh.indices)
    frames = device_tensor(sc.frames.packed())
    # the terrain and its instances in 8-wide nodes (GRT_BUILD_WIDE8_NODES): measured faster
    # than 4-wide on this workload for both queries (features.build_options)
    W8 = grt.GRT_BUILD_WIDE8_NODES
    geom = Geometry(ctx, vertices=verts, indices=idx, build_flags=W8)
    scene = Scene(ctx, [geom.handle] * WORKLOAD["instances"], frames, build_flags=W8)
    rays = new_rays(npix)
    hits = new_hits(npix)
    ao = torch.empty(npix, dtype=torch.float32, device="cuda")
    c = cam.packed()
    gcam = grt.camera(c[0:3], c[3:6], c[6:9])
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ev = {k: torch.cuda.Event(enable_timing=True) for k in ("b0", "b1", "b2", "c0", "c1", "a0", "a1", "s0", "s1")}

    def step(timed_kernels: bool):
        if timed_kernels:
            ev["b0"].record(stream)
        geom.build(sh)
        if timed_kernels:
            ev["b1"].record(stream)
        scene.build(sh)
        if timed_kernels:
            ev["b2"].record(stream)
        grt.grtGenerateCameraRays(ctx.handle, gcam, W, H, rays, sh)
        if timed_kernels:
            ev["c0"].record(stream)
        grt.grtTraceClosest(ctx.handle, scene.handle, None, rays, npix, hits, None, None, sh)
        if timed_kernels:
            ev["c1"].record(stream)
            ev["a0"].record(stream)
        grt.grtTraceAmbientOcclusion(ctx.handle, scene.handle, rays, hits, npix, spp, seed, length, ao, None, sh)
        if timed_kernels:
            ev["a1"].record(stream)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    nhit = int((hits[:, 1].view(torch.int32) != -1).sum().item())
    rays_per_step = npix + spp * nhit

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    step_ms, closest_ms, ao_ms, blas_ms, tlas_ms = [], [], [], [], []
    clocks = ClockSampler(local)
    launches0 = grt.grtGetLaunchCount()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        ev["s0"].record(stream)
        step(True)
        ev["s1"].record(stream)
        ev["s1"].synchronize()
        step_ms.append(ev["s0"].elapsed_time(ev["s1"]))
        closest_ms.append(ev["c0"].elapsed_time(ev["c1"]))
        ao_ms.append(ev["a0"].elapsed_time(ev["a1"]))
        blas_ms.append(ev["b0"].elapsed_time(ev["b1"]))
        tlas_ms.append(ev["b1"].elapsed_time(ev["b2"]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = grt.grtGetLaunchCount() - launches0
    total_s = sum(step_ms) / 1e3
    (total_s,) = max_over_ranks([total_s], dist)
    value = job_throughput(rays_per_step * args.steps, world, total_s) / 1e6

    # --------------------------------------------------- the traversal features on the same scene
    # (device-resident, L2 flushed before each timed launch, CUDA events, median of 10):
    # instance masks (alternate instances carry mask 1 or 2; the rays carry mask 1),
    # a primitive-mask intersection filter that rejects every other triangle, and every
    # hit of each primary ray (up to 4 stored per ray).
    def timed(fn, reps=10):
        out = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            fn()
        for _ in range(reps):
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    masked = Scene(ctx, [geom.handle] * WORKLOAD["instances"], frames,
                   masks=[1 + (k & 1) for k in range(WORKLOAD["instances"])], build_flags=W8).build(sh)
    mopt = grt.trace_options(ray_mask=1)
    mhits = new_hits(npix)

    def masked_step():
        grt.grtTraceClosest(ctx.handle, masked.handle, None, rays, npix, mhits, None, mopt, sh)
        grt.grtTraceAmbientOcclusion(ctx.handle, masked.handle, rays, mhits, npix, spp, seed, length, ao, mopt, sh)

    keep = torch.full(((mesh.indices.shape[0] + 31) // 32,), 0x55555555, dtype=torch.int32, device="cuda")
    table = FuncTable(ctx)  # triangles 0, 2, 4, ... stand
    table.set(0, 0, grt.GRT_INTERSECT_NONE, None, grt.GRT_FILTER_PRIMITIVE_MASK, keep)
    fhits = new_hits(npix)
    kmax = 4
    ahits = new_hits(npix * kmax)
    acount = torch.empty(npix, dtype=torch.int32, device="cuda")
    # path tracing with next event estimation (Sec. 5): the 64 terrain instances plus an
    # emitting 4x4 quad above the scene's centre; per-triangle albedo 0.7, sky (0.3, 0.4, 0.6);
    # three path vertices, one sample per pixel from the camera rays
    quad_v = device_tensor(np.array([[-1, 0, -1], [1, 0, -1], [1, 0, 1], [-1, 0, 1]], np.float32))
    quad_i = device_tensor(np.array([[0, 1, 2], [0, 2, 3]], np.uint32))
    quad = Geometry(ctx, vertices=quad_v, indices=quad_i, build_flags=W8).build(sh)
    ctr = 0.5 * (sc.lo + sc.hi)
    light_frame = np.array([0, 0, 0, 1, 2, 1, 2, ctr[0], sc.hi[1] + 0.5 * sc.extent, ctr[2]], np.float32)
    pt_frames = device_tensor(np.concatenate([sc.frames.packed(), light_frame[None, :]]))
    pt_scene = Scene(ctx, [geom.handle] * WORKLOAD["instances"] + [quad.handle], pt_frames, build_flags=W8).build(sh)
    ntri = mesh.indices.shape[0]
    pt_alb = device_tensor(np.concatenate([np.full((ntri, 3), 0.7), np.zeros((2, 3))]).astype(np.float32))
    pt_emi = device_tensor(np.concatenate([np.zeros((ntri, 3)), np.full((2, 3), 20.0)]).astype(np.float32))
    pt_off = device_tensor(np.array([0] * WORKLOAD["instances"] + [ntri], np.uint32))
    pt_lights = device_tensor(np.array([[WORKLOAD["instances"], 0], [WORKLOAD["instances"], 1]], np.uint32))
    pt_in = grt.path_trace_input(pt_alb, pt_emi, pt_off, pt_lights, 2, 3, 1, seed, (0.3, 0.4, 0.6))
    pt_ws = torch.empty(grt.grtGetPathTraceWorkspaceSize(npix), dtype=torch.uint8, device="cuda")
    pt_out = torch.empty((npix, 3), dtype=torch.float32, device="cuda")
    ms_pt = timed(lambda: grt.grtPathTrace(ctx.handle, pt_scene.handle, rays, npix, pt_in, pt_ws, pt_out, None, sh),
                  reps=5)
    ms_mask = timed(masked_step)
    ms_filter = timed(lambda: grt.grtTraceClosest(ctx.handle, scene.handle, None, rays, npix, fhits, table.handle,
                                                  None, sh))
    ms_all = timed(lambda: grt.grtTraceAllHits(ctx.handle, scene.handle, None, rays, npix, ahits, kmax, acount,
                                               None, None, sh))
    # the same scene framed densely: the overview camera moved to 0.35 extent from the
    # scene centre, where most pixels hit (closest hit + fused AO, as in the step)
    import scenegen
    dcam = scenegen.close_camera(sc, W, H).packed()
    drays, dhits = new_rays(npix), new_hits(npix)
    grt.grtGenerateCameraRays(ctx.handle, grt.camera(dcam[0:3], dcam[3:6], dcam[6:9]), W, H, drays, sh)
    ms_dc = timed(lambda: grt.grtTraceClosest(ctx.handle, scene.handle, None, drays, npix, dhits, None, None, sh))
    ms_da = timed(lambda: grt.grtTraceAmbientOcclusion(ctx.handle, scene.handle, drays, dhits, npix, spp, seed, length,
                                                       ao, None, sh))
    dhit = int((dhits[:, 1].view(torch.int32) != -1).sum().item())
    dense = {"camera": "scene centre + (0, 0, 0.35 extent), looking down -z", "primary_hits": dhit,
             "hit_fraction": round(dhit / npix, 4), "closest_ms": round(ms_dc, 4), "ao_ms": round(ms_da, 4),
             "rays": npix + spp * dhit, "mrays_per_s": round((npix + spp * dhit) / (ms_dc + ms_da) / 1e3, 1),
             "closest_mrays_per_s": round(npix / ms_dc / 1e3, 1),
             "ao_mrays_per_s": round(spp * dhit / ms_da / 1e3, 1)}
    # the build options of the terrain geometry (linear BVH, clustering with search
    # radius 8 and 32, clustering inside the linear BVH's subtrees): build time,
    # surface-area cost of the tree, the closest + AO traces and the whole step over it
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS  # the features above
    builds = {}
    for name, flags in (("fast_lbvh", grt.GRT_BUILD_PREFER_FAST), ("balanced_ploc8", grt.GRT_BUILD_PREFER_BALANCED),
                        ("high_quality_ploc32", grt.GRT_BUILD_PREFER_HIGH_QUALITY),
                        ("subtree_cluster16", grt.GRT_BUILD_CLUSTER_SUBTREES),
                        ("fast_lbvh_quantized_nodes", grt.GRT_BUILD_PREFER_FAST | grt.GRT_BUILD_QUANTIZED_NODES),
                        ("fast_lbvh_wide8_nodes", grt.GRT_BUILD_PREFER_FAST | grt.GRT_BUILD_WIDE8_NODES),
                        ("fast_lbvh_wide8_split_triangles", grt.GRT_BUILD_PREFER_FAST | grt.GRT_BUILD_WIDE8_NODES |
                         grt.GRT_BUILD_SPLIT_TRIANGLES)):
        gq = Geometry(ctx, vertices=verts, indices=idx, build_flags=flags).build(sh)
        sq = Scene(ctx, [gq.handle] * WORKLOAD["instances"], frames,
                   build_flags=flags & grt.GRT_BUILD_WIDE8_NODES).build(sh)
        qhits = new_hits(npix)

        def q_trace(sq=sq, qhits=qhits):
            grt.grtTraceClosest(ctx.handle, sq.handle, None, rays, npix, qhits, None, None, sh)
            grt.grtTraceAmbientOcclusion(ctx.handle, sq.handle, rays, qhits, npix, spp, seed, length, ao, None, sh)

        def q_step(gq=gq, sq=sq, q_trace=q_trace):
            gq.build(sh)
            sq.build(sh)
            grt.grtGenerateCameraRays(ctx.handle, gcam, W, H, rays, sh)
            q_trace()

        ms_b = timed(lambda gq=gq: gq.build(sh))
        ms_t = timed(q_trace)
        ms_s = timed(q_step)
        ms_c = timed(lambda sq=sq, qhits=qhits: grt.grtTraceClosest(ctx.handle, sq.handle, None, rays, npix, qhits,
                                                                     None, None, sh))
        ms_a = timed(lambda sq=sq, qhits=qhits: grt.grtTraceAmbientOcclusion(ctx.handle, sq.handle, rays, qhits, npix,
                                                                              spp, seed, length, ao, None, sh))
        torch.cuda.synchronize()
        qhit = int((qhits[:, 1].view(torch.int32) != -1).sum().item())
        builds[name] = {"blas_build_ms": round(ms_b, 4), "sah_cost": round(sah_cost(gq), 3),
                        "closest_plus_ao_ms": round(ms_t, 4), "closest_ms": round(ms_c, 4), "ao_ms": round(ms_a, 4),
                        "step_ms": round(ms_s, 4), "primary_hits": qhit}
        sq.close()
        gq.close()
    torch.cuda.synchronize()
    # a clustering build that could not keep its blocks co-resident reports a timeout
    # instead of a tree: record it here rather than fail the line
    build_err = grt.grtGetLastDeviceError(ctx.handle, sh)
    if build_err != grt.GRT_SUCCESS:
        builds["device_error"] = int(build_err)
    mhit = int((mhits[:, 1].view(torch.int32) != -1).sum().item())
    all_found = int(acount.sum().item())
    features = {"instance_mask_half": {"closest_plus_ao_ms": round(ms_mask, 4), "primary_hits": mhit,
                                       "mrays_per_s": round((npix + spp * mhit) / ms_mask / 1e3, 1)},
                "filter_half_closest_ms": round(ms_filter, 4),
                "all_hits_primary": {"ms": round(ms_all, 4), "hits_found": all_found,
                                     "mrays_per_s": round(npix / ms_all / 1e3, 1)},
                "dense_view": dense,
                "path_trace_nee": {"ms": round(ms_pt, 4), "max_depth": 3, "spp": 1,
                                   "mpaths_per_s": round(npix / ms_pt / 1e3, 1),
                                   "mean_radiance": round(float(pt_out.mean().item()), 5)},
                "build_options": builds}
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS

    # --------------------------------------------------- traversal work per ray (counting pass)
    cnt = grt.trace_options(flags=grt.GRT_TRACE_FLAG_COUNT)
    grt.grtGetTraceStatistics(ctx.handle, sh)
    grt.grtTraceClosest(ctx.handle, scene.handle, None, rays, npix, hits, None, cnt, sh)
    st_c = grt.grtGetTraceStatistics(ctx.handle, sh)
    grt.grtTraceAmbientOcclusion(ctx.handle, scene.handle, rays, hits, npix, spp, seed, length, ao, cnt, sh)
    st_a = grt.grtGetTraceStatistics(ctx.handle, sh)
    bytes_closest = (npix * (RAY_BYTES + HIT_BYTES) + NODE8_BYTES * st_c["nodesVisited"] +
                     TRI_BYTES * st_c["trianglesTested"] + INST_BYTES * st_c["instancesEntered"])
    # AO: per pixel the primary ray and hit in, the AO value out; per hit pixel the
    # instance record, geometry header, leaf index, triangle record and frame rows
    bytes_ao = (npix * (RAY_BYTES + HIT_BYTES + 4) + nhit * (128 + 64 + 4 + 48 + 48) +
                NODE8_BYTES * st_a["nodesVisited"] + TRI_BYTES * st_a["trianglesTested"] +
                INST_BYTES * st_a["instancesEntered"])
    kern = {"closest": (statistics.mean(closest_ms), bytes_closest, "traceKernel<closest, scene>"),
            "ao": (statistics.mean(ao_ms), bytes_ao, "aoTraceKernel")}
    dom = max(kern, key=lambda k: kern[k][0])
    ms, nbytes, kname = kern[dom]
    roofline = roofline_entry(kname, nbytes, ms, st_c if dom == "closest" else st_a)
    roofline_closest = roofline_entry(kern["closest"][2], kern["closest"][1], kern["closest"][0], st_c)

    # --------------------------------------------------- end to end through the C ABI, host buffers
    vh = torch.from_numpy(mesh.vertices).pin_memory()
    ih = torch.from_numpy(mesh.indices.view(np.int32)).pin_memory()
    fh = torch.from_numpy(sc.frames.packed()).pin_memory()
    ao_h = torch.empty(npix, dtype=torch.float32).pin_memory()
    hits_h = torch.empty((npix, 5), dtype=torch.int32).pin_memory()
    # the hit records go back on a second stream while the AO kernel runs
    copy_stream = torch.cuda.Stream()
    hits_done = torch.cuda.Event()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        ev["s0"].record(stream)
        verts.copy_(vh, non_blocking=True)
        idx.copy_(ih, non_blocking=True)
        frames.copy_(fh, non_blocking=True)
        geom.build(sh)
        scene.build(sh)
        grt.grtGenerateCameraRays(ctx.handle, gcam, W, H, rays, sh)
        grt.grtTraceClosest(ctx.handle, scene.handle, None, rays, npix, hits, None, None, sh)
        hits_done.record(stream)
        copy_stream.wait_event(hits_done)
        with torch.cuda.stream(copy_stream):
            hits_h.copy_(hits, non_blocking=True)
        grt.grtTraceAmbientOcclusion(ctx.handle, scene.handle, rays, hits, npix, spp, seed, length, ao, None, sh)
        ao_h.copy_(ao, non_blocking=True)
        stream.wait_stream(copy_stream)
        ev["s1"].record(stream)
        ev["s1"].synchronize()
        if k >= args.warmup:
            e2e_ms.append(ev["s0"].elapsed_time(ev["s1"]))
    e2e_s = sum(e2e_ms) / 1e3
    (e2e_s,) = max_over_ranks([e2e_s], dist)
    h2d = vh.numel() * 4 + ih.numel() * 4 + fh.numel() * 4
    d2h = ao_h.numel() * 4 + hits_h.numel() * 4
    e2e = {"value": round(job_throughput(rays_per_step * args.steps, world, e2e_s) / 1e6, 2), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD, node_format="8-wide (GRT_BUILD_WIDE8_NODES)", rays_per_step=rays_per_step,
                           primary_hits=nhit, l2="flushed between steps",
                           parallelism=f"replicas{world}"),
            "roofline": roofline, "roofline_closest": roofline_closest, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk,
            "kernel_ms": {"closest": round(statistics.mean(closest_ms), 4), "ao": round(statistics.mean(ao_ms), 4),
                          "blas_build": round(statistics.mean(blas_ms), 4),
                          "tlas_build": round(statistics.mean(tlas_ms), 4)},
            "build": {"blas_prims": int(mesh.indices.shape[0]), "tlas_instances": WORKLOAD["instances"],
                      "ms": round(statistics.mean(blas_ms) + statistics.mean(tlas_ms), 4),
                      "mprims_per_s": round((mesh.indices.shape[0] + WORKLOAD["instances"]) /
                                            (statistics.mean(blas_ms) + statistics.mean(tlas_ms)) / 1e3, 1),
                      "blas_mprims_per_s": round(mesh.indices.shape[0] / statistics.mean(blas_ms) / 1e3, 1)},
            "features": features}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle(sc, cam, length, seed, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle
def oracle_scene(sc):
    import oracle

    S = oracle.Scene()
    g = S.add_mesh(sc.meshes[0].vertices, sc.meshes[0].indices)
    for k in range(len(sc.geom_of_instance)):
        S.add_instance(g, sc.frames.packed()[k])
    S.build()
    return S


def oracle_sample(S, sc, cam, length, seed, stride: int, offset: int = 0):
    """Trace every `stride`-th pixel's primary ray (closest) and its AO rays (any-hit)
    with the FP64 oracle. Returns (rays traced, seconds)."""
    import oracle

    W, H, spp = WORKLOAD["width"], WORKLOAD["height"], WORKLOAD["ao_samples"]
    rays = oracle.camera_rays(cam.packed(), W, H)[offset::stride]
    t0 = time.perf_counter()
    hits = S.trace(rays)
    ao = oracle.ao_rays(S, rays, hits, spp, seed, length)
    valid = ao[:, 7] > 0
    S.trace(ao[valid], any_hit=True)
    dt = time.perf_counter() - t0
    return rays.shape[0] + int(valid.sum()), dt


def cpu_oracle(sc, cam, length, seed, target_s: float):
    S = oracle_scene(sc)
    n, dt = oracle_sample(S, sc, cam, length, seed, stride=2003)
    stride = max(1, int(2003 * dt / max(target_s, 1e-3)))
    n, dt = oracle_sample(S, sc, cam, length, seed, stride=stride, offset=1)
    return {"value": round(n / dt / 1e6, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"every {stride}th pixel of the 1920x1080 image: closest hit + 8 AO any-hit rays per hit, "
                      f"{n} rays, FP64 oracle BVH on {os.cpu_count()} host threads ({dt:.1f} s)"}


def run_reference(args, rank, world, local):
    if rank != 0:
        return
    sc, cam = workload()
    length = float(np.float32(0.05 * sc.extent))
    seed = WORKLOAD["seed"]
    S = oracle_scene(sc)
    budget = 10.0 * args.cpu_seconds / max(1, args.steps + args.warmup)  # seconds per step (2 min by default)
    n, dt = oracle_sample(S, sc, cam, length, seed, stride=4001)
    stride = max(1, int(4001 * dt / budget))
    times, count = [], 0
    for k in range(args.warmup + args.steps):
        n, dt = oracle_sample(S, sc, cam, length, seed, stride=stride, offset=k % stride)
        if k >= args.warmup:
            times.append(dt)
            count += n
    value = count / sum(times) / 1e6
    cb = {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"per step every {stride}th pixel (closest + 8 AO any-hit rays per hit), FP64 oracle"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="host cores"), "cpu_baseline": cb,
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- single-geometry workloads
ICOSPHERE = dict(workload="icosphere-512", mesh="icosphere level 3 (642 vertices, 1280 triangles, radius 1)",
                 width=512, height=512, camera="(0,0,3) looking down -z, 60 degree fov", query="closest hit")
SPHERES = dict(workload="spheres-1m", spheres=1_000_000, centres="U[-50,50]^3", radii="log-U[0.01,1]",
               rays=4_194_304, ray_origins="U[-50,50]^3", ray_directions="uniform on the sphere",
               queries="closest hit + any hit (tmax = inf)", seed=20260301)


def _setup_gpu(local, world):
    import torch

    from paper_2603_00292_gb300 import build as grt_build

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if int(os.environ.get("RANK", "0")) == 0:
        grt_build.build()
    if dist:
        dist.barrier()
    return dist


class StepTimer:
    """CUDA events around named parts of a step on one stream: mark(name) at the start
    of a part, mark(None) at the end of the step; durations in ms per part."""

    def __init__(self, stream, names):
        import torch

        self.stream = stream
        self.names = list(names)
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(self.names) + 1)]
        self.k = 0
        self.samples = {n: [] for n in self.names}

    def mark(self):
        self.ev[self.k].record(self.stream)
        self.k += 1

    def collect(self):
        self.ev[-1].synchronize()
        for i, n in enumerate(self.names):
            self.samples[n].append(self.ev[i].elapsed_time(self.ev[i + 1]))
        self.k = 0
        return sum(self.ev[i].elapsed_time(self.ev[i + 1]) for i in range(len(self.names)))

    def mean(self, name):
        return statistics.mean(self.samples[name])


def sah_cost(geom) -> float:
    """Surface-area cost of a built geometry's binary tree: the sum of the box areas of
    its internal nodes over the root's (leaf costs left out; one primitive per leaf)."""
    from paper_2603_00292_gb300.objects import read_device

    inf = geom.info()
    nd = read_device(inf.nodes, inf.nodeCount * 64, np.float32).reshape(-1, 16).astype(np.float64)
    lo = np.minimum(nd[:, [0, 4, 8]], nd[:, [2, 6, 10]])
    hi = np.maximum(nd[:, [1, 5, 9]], nd[:, [3, 7, 11]])
    ext = hi - lo
    area = ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 2] * ext[:, 0]
    return float(area.sum() / area[0]) if area[0] > 0 else 1.0


def roofline_entry(kernel, nbytes, ms, stats=None):
    """The roofline object of one kernel: algorithmic bytes per launch over its measured
    duration against the measured HBM copy peak; traffic = ncu DRAM bytes per launch of
    the kernel's current sources (else null)."""
    peaks, how = measured_peaks()
    achieved = nbytes / (ms / 1e3) / 1e9
    traffic = ncu_traffic(kernel)
    bound, counters = kernel_bound(kernel, peaks["hbm_gbs"])
    out = {"bound": bound, "kernel": kernel, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
           "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "peak_source": how, "traffic": traffic,
           "algorithmic_bytes_per_launch": int(nbytes), "launch_ms": round(ms, 4)}
    if traffic:
        out["dram_share_of_algorithmic"] = round(traffic / nbytes, 4)
    if counters:
        out["ncu_pct"] = counters
    if stats:
        out["per_ray"] = {k: round(v / max(1, stats["rays"]), 3) for k, v in stats.items() if k != "rays"}
    return out


def run_icosphere(args, rank, world, local):
    """The smallest instance of the plain method: one 1,280-triangle icosphere, 512x512
    primary rays from (0,0,3), closest hit. Step = LBVH build + camera rays + closest hit
    (+ FP64 refinement). The CPU baseline is the FP64 oracle's brute force on one core."""
    dist = _setup_gpu(local, world)
    import torch

    import paper_2603_00292_gb300 as grt
    import scenegen
    from paper_2603_00292_gb300.objects import Context, Geometry, device_tensor, new_hits, new_rays

    W, H = ICOSPHERE["width"], ICOSPHERE["height"]
    n = W * H
    mesh = scenegen.icosphere(3)
    cam = scenegen.look_down_z_camera([0, 0, 3], W, H)
    c = cam.packed()
    gcam = grt.camera(c[0:3], c[3:6], c[6:9])
    ctx = Context(local)
    verts, idx = device_tensor(mesh.vertices), device_tensor(mesh.indices)
    geom = Geometry(ctx, vertices=verts, indices=idx)
    rays, hits = new_rays(n), new_hits(n)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    T = StepTimer(stream, ["build", "raygen", "closest"])

    def step(timer):
        timer and timer.mark()
        geom.build(sh)
        timer and timer.mark()
        grt.grtGenerateCameraRays(ctx.handle, gcam, W, H, rays, sh)
        timer and timer.mark()
        grt.grtTraceClosest(ctx.handle, None, geom.handle, rays, n, hits, None, None, sh)
        timer and timer.mark()

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    l0 = grt.grtGetLaunchCount()
    if dist:
        dist.barrier()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        step(T)
        step_ms.append(T.collect())
    clk = clocks.stop()
    launches = grt.grtGetLaunchCount() - l0
    (total_s,) = max_over_ranks([sum(step_ms) / 1e3], dist)
    value = job_throughput(n * args.steps, world, total_s) / 1e6
    nhit = int((hits[:, 1].view(torch.int32) != -1).sum().item())
    cnt = grt.trace_options(flags=grt.GRT_TRACE_FLAG_COUNT)
    grt.grtGetTraceStatistics(ctx.handle, sh)
    grt.grtTraceClosest(ctx.handle, None, geom.handle, rays, n, new_hits(n), None, cnt, sh)
    st = grt.grtGetTraceStatistics(ctx.handle, sh)
    nbytes = n * (RAY_BYTES + HIT_BYTES) + NODE_BYTES * st["nodesVisited"] + TRI_BYTES * st["trianglesTested"]
    roofline = roofline_entry("traceKernel<closest, geometry> icosphere-512", nbytes, T.mean("closest"), st)

    # end to end: the mesh up from pinned host memory, the hit records back
    vh = torch.from_numpy(mesh.vertices).pin_memory()
    ih = torch.from_numpy(mesh.indices.view(np.int32)).pin_memory()
    hh = torch.empty((n, 5), dtype=torch.int32).pin_memory()
    e2e_ms = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for k in range(args.warmup + args.steps):
        flush.zero_()
        ev[0].record(stream)
        verts.copy_(vh, non_blocking=True)
        idx.copy_(ih, non_blocking=True)
        step(None)
        hh.copy_(hits, non_blocking=True)
        ev[1].record(stream)
        ev[1].synchronize()
        if k >= args.warmup:
            e2e_ms.append(ev[0].elapsed_time(ev[1]))
    (e2e_s,) = max_over_ranks([sum(e2e_ms) / 1e3], dist)
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(ICOSPHERE, rays_per_step=n, primary_hits=nhit, l2="flushed between steps",
                           parallelism=f"replicas{world}"),
            "trace_mrays_per_s": round(n / T.mean("closest") / 1e3, 1),
            "build": {"ms": round(T.mean("build"), 4), "prims": int(mesh.indices.shape[0]),
                      "mprims_per_s": round(mesh.indices.shape[0] / T.mean("build") / 1e3, 2)},
            "kernel_ms": {k: round(T.mean(k), 4) for k in T.names},
            "roofline": roofline,
            "e2e": {"value": round(job_throughput(n * args.steps, world, e2e_s) / 1e6, 2), "unit": UNIT,
                    "h2d_bytes_per_step": int(vh.numel() * 4 + ih.numel() * 4),
                    "d2h_bytes_per_step": int(hh.numel() * 4)},
            "gpu_launches": int(launches), "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_icosphere(mesh, c, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    geom.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


def cpu_icosphere(mesh, cam_packed, target_s: float):
    """The FP64 oracle's brute force (every ray against all 1,280 triangles) on one host
    core, over every k-th pixel of the 512x512 image."""
    import oracle

    W, H = ICOSPHERE["width"], ICOSPHERE["height"]
    rays = oracle.camera_rays(cam_packed, W, H)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(mesh.vertices, mesh.indices))

    def run(stride):
        r = rays[::stride]
        t0 = time.perf_counter()
        S.trace(r, bvh=False, threads=1)
        return r.shape[0], time.perf_counter() - t0

    m, dt = run(512)
    stride = max(1, int(512 * dt / max(target_s, 1e-3)))
    m, dt = run(stride)
    return {"value": round(m / dt / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"every {stride}th pixel of the 512x512 image ({m} rays), FP64 brute force over all 1,280 "
                      f"triangles on one host core ({dt:.1f} s)"}


def run_spheres(args, rank, world, local):
    """Custom primitives through the function table: 1 M spheres as an AABB-list
    geometry, 4,194,304 uniform random rays generated on the GPU, each traced as a
    closest-hit and an any-hit query. Step = LBVH build over the boxes + ray generation +
    closest hit (+ FP64 refinement) + any hit."""
    dist = _setup_gpu(local, world)
    import torch

    import paper_2603_00292_gb300 as grt
    import scenegen
    from paper_2603_00292_gb300.objects import Context, FuncTable, Geometry, device_tensor, new_hits, new_rays

    n, seed = SPHERES["rays"], SPHERES["seed"]
    sph = scenegen.spheres(SPHERES["spheres"], half=50.0, rmin=0.01, rmax=1.0, seed=seed, config=3)
    boxes = scenegen.sphere_aabbs(sph)
    ctx = Context(local)
    dsph, dbox = device_tensor(sph), device_tensor(boxes)
    geom = Geometry(ctx, boxes=dbox)
    table = FuncTable(ctx)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, dsph)
    rays, hc, ha = new_rays(n), new_hits(n), new_hits(n)
    lo, hi = [-50.0] * 3, [50.0] * 3
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    T = StepTimer(stream, ["build", "raygen", "closest", "any"])

    def step(timer):
        timer and timer.mark()
        geom.build(sh)
        timer and timer.mark()
        grt.grtGenerateUniformRays(ctx.handle, lo, hi, seed, n, rays, 0.0, float("inf"), sh)
        timer and timer.mark()
        grt.grtTraceClosest(ctx.handle, None, geom.handle, rays, n, hc, table.handle, None, sh)
        timer and timer.mark()
        grt.grtTraceAnyHit(ctx.handle, None, geom.handle, rays, n, ha, table.handle, None, sh)
        timer and timer.mark()

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    l0 = grt.grtGetLaunchCount()
    if dist:
        dist.barrier()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        step(T)
        step_ms.append(T.collect())
    clk = clocks.stop()
    launches = grt.grtGetLaunchCount() - l0
    (total_s,) = max_over_ranks([sum(step_ms) / 1e3], dist)
    value = job_throughput(2 * n * args.steps, world, total_s) / 1e6
    hits_c = int((hc[:, 1].view(torch.int32) != -1).sum().item())
    occl = int((ha[:, 1].view(torch.int32) != -1).sum().item())

    # any hit at tmax = 2.9 (about 70% occluded): a non-trivial occlusion query
    short = new_rays(n)
    grt.grtGenerateUniformRays(ctx.handle, lo, hi, seed, n, short, 0.0, 2.9, sh)
    hs = new_hits(n)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    short_ms = []
    for k in range(3 + 5):
        flush.zero_()
        e0.record(stream)
        grt.grtTraceAnyHit(ctx.handle, None, geom.handle, short, n, hs, table.handle, None, sh)
        e1.record(stream)
        e1.synchronize()
        if k >= 3:
            short_ms.append(e0.elapsed_time(e1))
    occl_short = int((hs[:, 1].view(torch.int32) != -1).sum().item())

    # the same geometry with quantised 64-byte nodes (GRT_BUILD_QUANTIZED_NODES) and with
    # 256-byte 8-wide nodes (GRT_BUILD_WIDE8_NODES): build, closest and any hit (tmax
    # infinite and 2.9), and how many hit records equal the 128-byte 4-wide nodes' (the
    # rest are equal-t ties)
    node_formats = {}
    for fname, fflag, fbytes in (("quantized_nodes", grt.GRT_BUILD_QUANTIZED_NODES, 64),
                                 ("wide8_nodes", grt.GRT_BUILD_WIDE8_NODES, 256)):
        node_formats[fname] = sphere_node_format(grt, ctx, table, dbox, fflag, fbytes, n, rays, short, hc, ha, hs,
                                                 flush, stream, sh)


    # algorithmic bytes per launch from counting passes: per ray the ray and the hit
    # record, per 4-wide node visit 112 B, per sphere test its leaf's primitive ID (4 B)
    # and its centre and radius (16 B)
    cnt = grt.trace_options(flags=grt.GRT_TRACE_FLAG_COUNT)
    grt.grtGetTraceStatistics(ctx.handle, sh)
    grt.grtTraceClosest(ctx.handle, None, geom.handle, rays, n, new_hits(n), table.handle, cnt, sh)
    st_c = grt.grtGetTraceStatistics(ctx.handle, sh)
    grt.grtTraceAnyHit(ctx.handle, None, geom.handle, rays, n, new_hits(n), table.handle, cnt, sh)
    st_a = grt.grtGetTraceStatistics(ctx.handle, sh)

    def nbytes(st):
        return n * (RAY_BYTES + HIT_BYTES) + NODE_BYTES * st["nodesVisited"] + 20 * st["customTested"]

    kern = {"closest": ("traceKernel<closest, geometry> spheres-1m", st_c),
            "any": ("traceKernel<any, geometry> spheres-1m", st_a)}
    dom = max(kern, key=lambda k: T.mean(k))
    roofline = roofline_entry(kern[dom][0], nbytes(kern[dom][1]), T.mean(dom), kern[dom][1])
    prims = SPHERES["spheres"]

    # end to end: spheres and boxes up from pinned host memory, both hit buffers back
    sh_h = torch.from_numpy(sph).pin_memory()
    bh = torch.from_numpy(boxes).pin_memory()
    hch = torch.empty((n, 5), dtype=torch.int32).pin_memory()
    hah = torch.empty((n, 5), dtype=torch.int32).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        e0.record(stream)
        dsph.copy_(sh_h, non_blocking=True)
        dbox.copy_(bh, non_blocking=True)
        step(None)
        hch.copy_(hc, non_blocking=True)
        hah.copy_(ha, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    (e2e_s,) = max_over_ranks([sum(e2e_ms) / 1e3], dist)
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(SPHERES, rays_per_step=2 * n, closest_hits=hits_c, occluded=occl,
                           l2="flushed between steps", parallelism=f"replicas{world}"),
            "trace_mrays_per_s": {"closest": round(n / T.mean("closest") / 1e3, 1),
                                  "any": round(n / T.mean("any") / 1e3, 1),
                                  "any_tmax_2.9": round(n / statistics.mean(short_ms) / 1e3, 1)},
            "occluded_tmax_2.9": occl_short,
            "node_formats": node_formats,
            "build": {"ms": round(T.mean("build"), 4), "prims": prims,
                      "mprims_per_s": round(prims / T.mean("build") / 1e3, 1)},
            "kernel_ms": {k: round(T.mean(k), 4) for k in T.names},
            "roofline": roofline,
            "e2e": {"value": round(job_throughput(2 * n * args.steps, world, e2e_s) / 1e6, 2), "unit": UNIT,
                    "h2d_bytes_per_step": int(sh_h.numel() * 4 + bh.numel() * 4),
                    "d2h_bytes_per_step": int(hch.numel() * 4 + hah.numel() * 4)},
            "gpu_launches": int(launches), "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_spheres(sph, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    table.close()
    geom.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


def sphere_node_format(grt, ctx, table, dbox, flag, node_bytes, n, rays, short, hc, ha, hs, flush, stream, sh):
    """The sphere geometry built with another node format (`flag`): build, closest and any
    hit (tmax infinite and 2.9) timed with CUDA events after an L2 flush (mean of 5 after
    3 warm-up runs), and how many hit records equal those of the 128-byte 4-wide nodes
    (hc, ha, hs; the rest are equal-t ties)."""
    import torch

    from paper_2603_00292_gb300.objects import Geometry, new_hits

    g = Geometry(ctx, boxes=dbox, build_flags=flag)
    qc, qa, qs = new_hits(n), new_hits(n), new_hits(n)
    runs = {"build": lambda: g.build(sh),
            "closest": lambda: grt.grtTraceClosest(ctx.handle, None, g.handle, rays, n, qc, table.handle, None, sh),
            "any": lambda: grt.grtTraceAnyHit(ctx.handle, None, g.handle, rays, n, qa, table.handle, None, sh),
            "any_tmax_2.9": lambda: grt.grtTraceAnyHit(ctx.handle, None, g.handle, short, n, qs, table.handle, None,
                                                       sh)}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = {}
    for name, fn in runs.items():
        vals = []
        for k in range(3 + 5):
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if k >= 3:
                vals.append(e0.elapsed_time(e1))
        ms[name] = statistics.mean(vals)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    out = {"node_bytes": node_bytes, "build_ms": round(ms["build"], 4), "closest_ms": round(ms["closest"], 4),
           "any_ms": round(ms["any"], 4), "any_tmax_2.9_ms": round(ms["any_tmax_2.9"], 4),
           "closest_mrays_per_s": round(n / ms["closest"] / 1e3, 1), "any_mrays_per_s": round(n / ms["any"] / 1e3, 1),
           "closest_records_equal": int((qc == hc).all(dim=1).sum().item()),
           "occluded_equal": int(((qa[:, 1] != -1) == (ha[:, 1] != -1)).sum().item()),
           "occluded_tmax_2.9_equal": int(((qs[:, 1] != -1) == (hs[:, 1] != -1)).sum().item())}
    g.close()
    return out


def cpu_spheres(sph, target_s: float):
    """The FP64 oracle (its own BVH over the spheres, closest + any hit) on the host
    cores over the first k rays of the workload's generator."""
    import oracle

    t0 = time.perf_counter()
    S = oracle.Scene()
    S.add_instance(S.add_spheres(sph))
    S.build()
    build_s = time.perf_counter() - t0

    def run(m):
        r = oracle.uniform_rays([-50.0] * 3, [50.0] * 3, SPHERES["seed"], m)
        t0 = time.perf_counter()
        S.trace(r)
        S.trace(r, any_hit=True)
        return 2 * m, time.perf_counter() - t0

    m, dt = run(20_000)
    m, dt = run(min(SPHERES["rays"], max(20_000, int(20_000 * target_s / max(dt, 1e-3)))))
    return {"value": round(m / dt / 1e6, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the first {m // 2} rays of the workload, closest + any hit ({m} queries), FP64 oracle BVH "
                      f"on {os.cpu_count()} host threads ({dt:.1f} s; its BVH build over the 1 M spheres took "
                      f"{build_s:.1f} s, not counted)"}


# ----------------------------------------------------------------------------- adjoint workload
ADJOINT = dict(workload="lambert-adjoint-1080p", mesh="icosphere level 3 (642 vertices, 1280 triangles)",
               width=1920, height=1080, camera="(0,0,3) looking down -z, 60 degree fov", shadow_rays=1,
               seed=20260301)


def adjoint_problem():
    import scenegen

    return scenegen.shading_problem(ADJOINT["width"], ADJOINT["height"], ADJOINT["seed"])


def run_adjoint(args, rank, world, local):
    """Differentiable Lambert shading at 1920x1080: forward (closest hit + shading with
    one shadow any-hit ray per lit pixel) against forward + adjoint backward, with the
    hit records stored or recomputed in the backward pass."""
    import torch

    import paper_2603_00292_gb300 as grt
    from paper_2603_00292_gb300 import build as grt_build
    from paper_2603_00292_gb300.objects import Context, Geometry, device_tensor, new_hits, new_rays

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    if rank == 0:
        grt_build.build()
    if dist:
        dist.barrier()
    P = adjoint_problem()
    W, H = ADJOINT["width"], ADJOINT["height"]
    n = W * H
    ctx = Context(local)
    pos, idx = device_tensor(P.mesh.vertices), device_tensor(P.mesh.indices)
    col, light = device_tensor(P.colours), device_tensor(P.light)
    rays = new_rays(n)
    c = P.camera.packed()
    grt.grtGenerateCameraRays(ctx.handle, grt.camera(c[0:3], c[3:6], c[6:9]), W, H, rays)
    geom = Geometry(ctx, vertices=pos, indices=idx).build()
    target = torch.rand((n, 3), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    hits = new_hits(n)
    img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    vis = torch.empty(n, dtype=torch.uint8, device="cuda")
    gimg = torch.empty_like(img)
    gc, gl, gp = torch.zeros_like(col), torch.zeros_like(light), torch.zeros_like(pos)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def forward(store: bool):
        grt.grtTraceClosest(ctx.handle, None, geom.handle, rays, n, hits, None, None, sh)
        grt.grtShadeLambert(ctx.handle, geom.handle, rays, hits, n, idx, pos, col, light, img,
                            vis if store else None, None, sh)

    def backward(store: bool, mark: bool):
        torch.sub(img, target, out=gimg).mul_(2.0)
        gc.zero_(), gl.zero_(), gp.zero_()
        if mark:
            ev[2].record(stream)
        grt.grtShadeLambertBackward(ctx.handle, geom.handle, rays, hits if store else None, vis if store else None,
                                    n, idx, pos, col, light, gimg, gc, gl, gp, None, sh)
        if mark:
            ev[3].record(stream)

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed(mode: str):
        for _ in range(args.warmup):
            forward(mode != "recompute")
            if mode != "forward":
                backward(mode == "store", False)
        torch.cuda.synchronize()
        step, bwd = [], []
        l0 = grt.grtGetLaunchCount()
        for _ in range(args.steps):
            flush.zero_()
            ev[0].record(stream)
            forward(mode != "recompute")
            if mode != "forward":
                backward(mode == "store", True)
            ev[1].record(stream)
            ev[1].synchronize()
            step.append(ev[0].elapsed_time(ev[1]))
            if mode != "forward":
                bwd.append(ev[2].elapsed_time(ev[3]))
        launches[mode] = grt.grtGetLaunchCount() - l0
        return statistics.mean(step), (statistics.mean(bwd) if bwd else None)

    clocks = ClockSampler(local)
    launches = {}
    if dist:
        dist.barrier()
    clocks.start()
    fwd_ms, _ = timed("forward")
    store_ms, bwd_store_ms = timed("store")
    rec_ms, bwd_rec_ms = timed("recompute")
    clk = clocks.stop()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    nhit = int((hits[:, 1].view(torch.int32) != -1).sum().item())
    fwd_ms, store_ms, rec_ms = max_over_ranks([fwd_ms, store_ms, rec_ms], dist)

    # backward (stored hits): the hit record of every pixel; the ray, visibility byte and
    # dL/dI of each hit pixel; the mesh tables (indices, positions, colours) read and the
    # colour and position gradients written once (a few tens of KB)
    tables = P.mesh.indices.nbytes + P.mesh.vertices.nbytes + P.colours.nbytes
    nbytes = n * HIT_BYTES + nhit * (RAY_BYTES + 1 + 12) + tables + 2 * P.mesh.vertices.nbytes
    roofline = roofline_entry("shadeBackwardKernel<false, true>", nbytes, bwd_store_ms)

    # end to end: parameters up from pinned host memory, image and gradients back
    ch = torch.from_numpy(P.colours).pin_memory()
    lh = torch.from_numpy(P.light).pin_memory()
    ph = torch.from_numpy(P.mesh.vertices).pin_memory()
    outs = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (img, gc, gl, gp)]
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        ev[0].record(stream)
        col.copy_(ch, non_blocking=True), light.copy_(lh, non_blocking=True), pos.copy_(ph, non_blocking=True)
        forward(True)
        backward(True, False)
        for o, t in zip(outs, (img, gc, gl, gp)):
            o.copy_(t, non_blocking=True)
        ev[1].record(stream)
        ev[1].synchronize()
        if k >= args.warmup:
            e2e.append(ev[0].elapsed_time(ev[1]))
    h2d = ch.numel() * 4 + lh.numel() * 4 + ph.numel() * 4
    d2h = sum(o.numel() * 4 for o in outs)
    line = {"metric": "adjoint fwd+bwd ms vs plain fwd ms, same GPU", "value": round(store_ms, 4), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(store_ms, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(ADJOINT, primary_hits=nhit, l2="flushed between steps", parallelism=f"replicas{world}"),
            "plain_forward_ms": round(fwd_ms, 4), "fwd_bwd_over_fwd": round(store_ms / fwd_ms, 3),
            "recompute_ms": round(rec_ms, 4), "backward_ms": {"stored": round(bwd_store_ms, 4),
                                                              "recompute": round(bwd_rec_ms, 4)},
            "stored_bytes_per_pixel": HIT_BYTES + 1, "roofline": roofline,
            "e2e": {"value": round(statistics.mean(e2e), 4), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches["store"]), "gpu_launches_by_mode": launches, "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_adjoint(P, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def cpu_adjoint(P, target_s: float):
    """The FP64 oracle's forward + analytic gradient on every k-th pixel, scaled to the
    whole image (the gradient is a sum over pixels); camera rays from the oracle."""
    import oracle

    rays = oracle.camera_rays(P.camera.packed(), ADJOINT["width"], ADJOINT["height"])
    v = P.mesh.vertices.astype(np.float64)
    c, l = P.colours.astype(np.float64), P.light.astype(np.float64)

    def run(stride):
        r = rays[::stride]
        tgt = np.zeros((r.shape[0], 3))
        t0 = time.perf_counter()
        oracle.lambert_forward(v, P.mesh.indices, c, l, r)
        oracle.lambert_gradient(v, P.mesh.indices, c, l, r, tgt)
        return time.perf_counter() - t0

    dt = run(2003)
    stride = max(1, int(2003 * dt / max(target_s, 1e-3)))
    dt = run(stride)
    return {"value": round(1e3 * dt * stride, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"every {stride}th pixel of the 1920x1080 image, FP64 forward + analytic gradient "
                      f"({dt:.1f} s), scaled by {stride}"}


# ----------------------------------------------------------------------------- batched workload
BATCHED = dict(workload="batched-soups-256", scenes=256, prims="log-U[1e3, 2e6] per scene",
               rays="log-U[4096, 2^20] per scene, half camera, half uniform random",
               clusters="8 Gaussian", edges="log-U[1e-3, 1e-1]", seed=20260301)


def _soup_worker(i: int):
    """One soup of the batched workload (host arrays), for a spawn-started pool."""
    import scenegen

    s = scenegen.soup_scene(i, seed=BATCHED["seed"])
    return (s.mesh.vertices, s.mesh.indices, s.camera.packed(), s.camera.width, s.camera.height, s.random_rays,
            float(np.max(s.hi - s.lo)))


def batched_soups(count: int):
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_soup_worker, range(count), chunksize=1)


def build_bytes_per_prim(bits: int) -> int:
    """Algorithmic DRAM bytes of building one triangle (LBVH): prep reads the indices
    and vertices (48) and writes a centroid and a fit counter (20); radix pass 0 reads
    the centroid and writes key and value, every pass reads the keys once for its
    histogram and reads and writes keys and values in its scatter; emission reads a key
    and writes a node word and two parent links (28 or 32); the fit reads the value,
    indices and vertices (52), writes the leaf record and its slot (52) and, per
    internal node, two parent links, two box writes and one box read (~80), plus the
    4-wide nodes: 128 bytes per internal node, written slot by slot."""
    kb, passes = (4, 4) if bits == 30 else (8, 8)
    sort = (16 + kb + 4) + (passes - 1) * kb + passes * 2 * (kb + 4)
    return 68 + sort + (kb + 24) + 52 + 52 + 80 + 128


def run_batched(args, rank, world, local):
    """256 uneven triangle soups, each with its own rays: every BVH build and closest-hit
    trace in one persistent launch (CUDA graph, autotuned options) against the same
    work as 256 sequential per-scene build + trace calls."""
    soups = batched_soups(min(args.scenes, BATCHED["scenes"]))  # before the first GPU call (spawned pool)
    import torch

    import paper_2603_00292_gb300 as grt
    from paper_2603_00292_gb300 import autotune
    from paper_2603_00292_gb300 import build as grt_build
    from paper_2603_00292_gb300.objects import Batch, Context, Geometry, device_tensor, empty_bytes, new_hits

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        grt_build.build()
    if dist:
        dist.barrier()
    ctx = Context(local)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    meshes, rays, hits_b, hits_s, geo_b, geo_s = [], [], [], [], [], []
    host = []
    total_prims = total_rays = 0
    # one build temporary for every geometry, sized for the largest
    big = max(range(len(soups)), key=lambda k: soups[k][1].shape[0])
    nbig = soups[big][1].shape[0]  # the size query reads only the counts (the addresses stand in)
    temp = empty_bytes(grt.grtGetGeometryBuildTemporaryBufferSize(
        ctx.handle, grt.triangle_mesh_input(256, 256, triangle_count=nbig, vertex_count=3 * nbig),
        grt.build_options()))
    for v, i, cam, W, H, rr, extent in soups:
        dv, di = device_tensor(v), device_tensor(i)
        R = W * H + rr.shape[0]
        r = torch.empty((R, 8), dtype=torch.float32, device="cuda")
        grt.grtGenerateCameraRays(ctx.handle, grt.camera(cam[0:3], cam[3:6], cam[6:9]), W, H, r, sh)
        r[W * H:].copy_(torch.from_numpy(rr))
        meshes.append((dv, di))
        rays.append(r)
        hits_b.append(new_hits(R))
        hits_s.append(new_hits(R))
        geo_b.append(Geometry(ctx, vertices=dv, indices=di, temp=temp))
        geo_s.append(Geometry(ctx, vertices=dv, indices=di, temp=temp))
        host.append((v, i, rr, W * H))
        total_prims += i.shape[0]
        total_rays += R
    scenes = list(zip(geo_b, rays, hits_b))
    torch.cuda.synchronize()

    tune_report = None
    if args.no_autotune:
        opts = dict(autotune.DEFAULTS)
    else:
        opts, tune_report = autotune.tune(ctx, scenes)
    B = Batch(ctx, scenes, grt.batch_options(graph=True, **opts))
    info = B.info()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def sequential():
        for g, r, h in zip(geo_s, rays, hits_s):
            g.build(sh)
            grt.grtTraceClosest(ctx.handle, None, g.handle, r, r.shape[0], h, None, None, sh)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        out = []
        l0 = grt.grtGetLaunchCount()
        for _ in range(args.steps):
            flush.zero_()
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            ev[1].synchronize()
            out.append(ev[0].elapsed_time(ev[1]))
        return out, grt.grtGetLaunchCount() - l0

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    clocks.start()
    b_ms, b_launches = timed(lambda: B.run(sh))
    if args.no_sequential:
        s_ms, s_launches = [float("nan")], 0
        for g, r, h in zip(geo_s, rays, hits_s):  # one untimed pass for the identity check
            g.build(sh)
            grt.grtTraceClosest(ctx.handle, None, g.handle, r, r.shape[0], h, None, None, sh)
    else:
        s_ms, s_launches = timed(sequential)
    clk = clocks.stop()
    assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
    identical = all(torch.equal(a, b) for a, b in zip(hits_b, hits_s))
    batched_ms, seq_ms = statistics.mean(b_ms), statistics.mean(s_ms)
    batched_ms, seq_ms = max_over_ranks([batched_ms, seq_ms], dist)

    # algorithmic bytes of one launch: the builds by formula, the traces from a
    # counting pass (nodes and triangles visited per ray) on the per-scene path
    cnt = grt.trace_options(flags=grt.GRT_TRACE_FLAG_COUNT)
    grt.grtGetTraceStatistics(ctx.handle, sh)
    for g, r, h in zip(geo_s, rays, hits_s):
        grt.grtTraceClosest(ctx.handle, None, g.handle, r, r.shape[0], h, None, cnt, sh)
    st = grt.grtGetTraceStatistics(ctx.handle, sh)
    trace_bytes = total_rays * (RAY_BYTES + HIT_BYTES) + NODE_BYTES * st["nodesVisited"] + TRI_BYTES * st["trianglesTested"]
    bits = [grt.grtGetBvhInfo(ctx.handle, geom=g.handle).mortonBits for g in geo_s]
    build_bytes = sum(build_bytes_per_prim(b) * m[1].shape[0] for b, m in zip(bits, meshes))
    nbytes = trace_bytes + build_bytes
    roofline = roofline_entry("batchKernel", nbytes, batched_ms)
    if len(soups) != BATCHED["scenes"]:
        # the record holds the full launch's bytes (scaled from a 16-soup capture): a smaller
        # case reports the captured 16-soup bytes where they are its own, else nothing
        t = (ncu_record("batchKernel") or {}).get("captured_dram_bytes") if len(soups) == 16 else None
        roofline["traffic"] = t
        roofline.pop("dram_share_of_algorithmic", None)
        if t:
            roofline["dram_share_of_algorithmic"] = round(t / nbytes, 4)
    roofline.update({"build_bytes": int(build_bytes), "trace_bytes": int(trace_bytes),
                     "per_ray": {"nodes": round(st["nodesVisited"] / max(1, st["rays"]), 2),
                                 "triangles": round(st["trianglesTested"] / max(1, st["rays"]), 2)}})

    # the same work with every soup built by clustering inside the linear BVH's subtrees
    # (the batch adds a clustering phase per scene), same launch options: batched against
    # sequential, hit records compared, and the mean surface-area cost of both trees
    clustered = None
    if not args.no_clustered:
        copt = grt.build_options(flags=grt.GRT_BUILD_CLUSTER_SUBTREES)
        ctemp = empty_bytes(grt.grtGetGeometryBuildTemporaryBufferSize(
            ctx.handle, grt.triangle_mesh_input(256, 256, triangle_count=nbig, vertex_count=3 * nbig), copt))
        geo_cb, geo_cs, hits_cb, hits_cs = [], [], [], []
        for (dv, di), r in zip(meshes, rays):
            geo_cb.append(Geometry(ctx, vertices=dv, indices=di, temp=ctemp, build_flags=grt.GRT_BUILD_CLUSTER_SUBTREES))
            geo_cs.append(Geometry(ctx, vertices=dv, indices=di, temp=ctemp, build_flags=grt.GRT_BUILD_CLUSTER_SUBTREES))
            hits_cb.append(new_hits(r.shape[0]))
            hits_cs.append(new_hits(r.shape[0]))
        BC = Batch(ctx, list(zip(geo_cb, rays, hits_cb)), grt.batch_options(graph=True, **opts))

        def sequential_clustered():
            for g, r, h in zip(geo_cs, rays, hits_cs):
                g.build(sh)
                grt.grtTraceClosest(ctx.handle, None, g.handle, r, r.shape[0], h, None, None, sh)

        cb_ms, cb_launches = timed(lambda: BC.run(sh))
        if args.no_sequential:
            sequential_clustered()
            cs_ms = [float("nan")]
        else:
            cs_ms, _ = timed(sequential_clustered)
        torch.cuda.synchronize()
        assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
        c_ms, cseq_ms = max_over_ranks([statistics.mean(cb_ms), statistics.mean(cs_ms)], dist)
        sah_l = [sah_cost(g) for g in geo_s]
        sah_c = [sah_cost(g) for g in geo_cs]
        clustered = {"build_flag": "GRT_BUILD_CLUSTER_SUBTREES", "ms": round(c_ms, 3),
                     "sequential_ms": None if math.isnan(cseq_ms) else round(cseq_ms, 3),
                     "speedup_vs_sequential": None if math.isnan(cseq_ms) else round(cseq_ms / c_ms, 3),
                     "mrays_per_s": round(total_rays / (c_ms / 1e3) / 1e6, 1),
                     "identical_to_sequential": bool(all(torch.equal(a, b) for a, b in zip(hits_cb, hits_cs))),
                     "sah_cost_mean": round(statistics.mean(sah_c), 3),
                     "lbvh_sah_cost_mean": round(statistics.mean(sah_l), 3),
                     "gpu_launches": int(cb_launches)}
        BC.close()
        for g in geo_cb + geo_cs:
            g.close()
        del ctemp, hits_cb, hits_cs

    # the linear BVH with quantised 64-byte nodes (GRT_BUILD_QUANTIZED_NODES), same
    # options: batched ms and how many hit records equal the 128-byte nodes' (the rest
    # are equal-t ties)
    quantized = None
    if not args.no_quantized:
        geo_q, hits_q = [], []
        for (dv, di), r in zip(meshes, rays):
            geo_q.append(Geometry(ctx, vertices=dv, indices=di, temp=temp, build_flags=grt.GRT_BUILD_QUANTIZED_NODES))
            hits_q.append(new_hits(r.shape[0]))
        BQ = Batch(ctx, list(zip(geo_q, rays, hits_q)), grt.batch_options(graph=True, **opts))
        q_ms, q_launches = timed(lambda: BQ.run(sh))
        torch.cuda.synchronize()
        assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
        (qms,) = max_over_ranks([statistics.mean(q_ms)], dist)
        equal = sum(int((a == b).all(dim=1).sum().item()) for a, b in zip(hits_q, hits_b))
        quantized = {"build_flag": "GRT_BUILD_QUANTIZED_NODES", "ms": round(qms, 3),
                     "mrays_per_s": round(total_rays / (qms / 1e3) / 1e6, 1), "records_equal": equal,
                     "records": int(total_rays), "gpu_launches": int(q_launches)}
        BQ.close()
        for g in geo_q:
            g.close()
        del hits_q

    # spatial splits (GRT_BUILD_SPLIT_TRIANGLES, one extra reference per triangle): the
    # per-scene path against the per-scene linear BVH above (hit records compared by
    # triangle ID, mean surface-area cost), and the batched launch of the split geometries
    # against the linear-BVH launch (its hits equal to the per-scene split path's)
    split = None
    if not args.no_split:
        sopt = grt.build_options(flags=grt.GRT_BUILD_SPLIT_TRIANGLES, split_factor=1.0)
        stemp = empty_bytes(grt.grtGetGeometryBuildTemporaryBufferSize(
            ctx.handle, grt.triangle_mesh_input(256, 256, triangle_count=nbig, vertex_count=3 * nbig), sopt))
        geo_p, hits_p = [], []
        for (dv, di), r in zip(meshes, rays):
            geo_p.append(Geometry(ctx, vertices=dv, indices=di, temp=stemp, build_flags=grt.GRT_BUILD_SPLIT_TRIANGLES,
                                  split_factor=1.0))
            hits_p.append(new_hits(r.shape[0]))

        def sequential_split():
            for g, r, h in zip(geo_p, rays, hits_p):
                g.build(sh)
                grt.grtTraceClosest(ctx.handle, None, g.handle, r, r.shape[0], h, None, None, sh)

        p_ms, p_launches = timed(sequential_split)
        # the same split geometries in one batched launch (its splitting phases), same options
        hits_pb = [new_hits(r.shape[0]) for r in rays]
        geo_pb = [Geometry(ctx, vertices=dv, indices=di, temp=stemp, build_flags=grt.GRT_BUILD_SPLIT_TRIANGLES,
                           split_factor=1.0) for (dv, di) in meshes]
        BP = Batch(ctx, list(zip(geo_pb, rays, hits_pb)), grt.batch_options(graph=True, **opts))
        pb_ms, pb_launches = timed(lambda: BP.run(sh))
        build_only, _ = timed(lambda: [g.build(sh) for g in geo_p])
        lbvh_build, _ = timed(lambda: [g.build(sh) for g in geo_s])
        torch.cuda.synchronize()
        assert grt.grtGetLastDeviceError(ctx.handle, sh) == grt.GRT_SUCCESS
        pms, pb, lb = max_over_ranks([statistics.mean(p_ms), statistics.mean(build_only), statistics.mean(lbvh_build)],
                                     dist)
        same = sum(int((a[:, 1] == b[:, 1]).sum().item()) for a, b in zip(hits_p, hits_s))
        (pbms,) = max_over_ranks([statistics.mean(pb_ms)], dist)
        batch_identical = bool(all(torch.equal(a, b) for a, b in zip(hits_pb, hits_p)))
        split = {"build_flag": "GRT_BUILD_SPLIT_TRIANGLES", "split_factor": 1.0, "path": "per-scene",
                 "sequential_ms": round(pms, 3),
                 "sequential_lbvh_ms": None if math.isnan(seq_ms) else round(seq_ms, 3),
                 "builds_ms": round(pb, 3), "lbvh_builds_ms": round(lb, 3),
                 "traces_ms": round(pms - pb, 3),
                 "lbvh_traces_ms": None if math.isnan(seq_ms) else round(seq_ms - lb, 3),
                 "sah_cost_mean": round(statistics.mean(sah_cost(g) for g in geo_p), 3),
                 "lbvh_sah_cost_mean": round(statistics.mean(sah_cost(g) for g in geo_s), 3),
                 "primitive_ids_equal": same, "records": int(total_rays), "gpu_launches": int(p_launches),
                 "batched_ms": round(pbms, 3), "batched_lbvh_ms": round(batched_ms, 3),
                 "batched_identical_to_per_scene": batch_identical, "batched_gpu_launches": int(pb_launches)}
        BP.close()
        for g in geo_p + geo_pb:
            g.close()
        del stemp, hits_p, hits_pb

    # end to end: meshes and rays up from pinned host memory, hit records back
    pin = [(torch.from_numpy(v).pin_memory(), torch.from_numpy(i.view(np.int32)).pin_memory(), r.cpu().pin_memory())
           for (v, i, _, _), r in zip(host, rays)]
    hits_h = [torch.empty(h.shape, dtype=h.dtype).pin_memory() for h in hits_b]
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        ev[0].record(stream)
        for (dv, di), r, (pv, pi, pr) in zip(meshes, rays, pin):
            dv.copy_(pv, non_blocking=True)
            di.copy_(pi, non_blocking=True)
            r.copy_(pr, non_blocking=True)
        B.run(sh)
        for hh, h in zip(hits_h, hits_b):
            hh.copy_(h, non_blocking=True)
        ev[1].record(stream)
        ev[1].synchronize()
        if k >= args.warmup:
            e2e.append(ev[0].elapsed_time(ev[1]))
    h2d = sum(pv.numel() * 4 + pi.numel() * 4 + pr.numel() * 4 for pv, pi, pr in pin)
    d2h = sum(h.numel() * 4 for h in hits_h)
    line = {"metric": f"batched build+trace of {len(soups)} uneven scenes: ms per launch vs {len(soups)} sequential "
                      "per-scene build+trace",
            "value": round(batched_ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(batched_ms, 3), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": dict(BATCHED, scenes=len(soups), total_prims=total_prims, total_rays=total_rays,
                           l2="flushed between steps", parallelism=f"replicas{world}"),
            "sequential_ms": None if math.isnan(seq_ms) else round(seq_ms, 3),
            "speedup_vs_sequential": None if math.isnan(seq_ms) else round(seq_ms / batched_ms, 3),
            "mrays_per_s": round(total_rays / (batched_ms / 1e3) / 1e6, 1),
            "mprims_per_s": round(total_prims / (batched_ms / 1e3) / 1e6, 1),
            "sequential_mrays_per_s": None if math.isnan(seq_ms) else round(total_rays / (seq_ms / 1e3) / 1e6, 1),
            "identical_to_sequential": bool(identical), "options": opts,
            "batch": {"items": info.itemCount, "small_scenes": info.smallScenes, "blocks": info.blocks,
                      "block_size": info.blockSize, "device_bytes": int(info.deviceBytes)},
            "autotune": None if tune_report is None else {k: tune_report[k] for k in tune_report if k != "tried"},
            "clustered": clustered,
            "quantized_nodes": quantized,
            "split_triangles": split,
            "roofline": roofline,
            "e2e": {"value": round(statistics.mean(e2e), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(b_launches), "sequential_gpu_launches": int(s_launches), "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_batched(host, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


def cpu_batched(host, target_s: float):
    """The FP64 oracle (its own BVH build + closest-hit trace) over the smallest scenes
    of the workload until about target_s seconds are spent."""
    import oracle

    order = sorted(range(len(host)), key=lambda k: host[k][1].shape[0])
    prims = rays = 0
    t0 = time.perf_counter()
    used = 0
    for k in order:
        v, i, rr, _ = host[k]
        S = oracle.Scene()
        S.add_instance(S.add_mesh(v, i))
        S.build()
        S.trace(rr)
        prims += i.shape[0]
        rays += rr.shape[0]
        used += 1
        if time.perf_counter() - t0 > target_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(rays / dt / 1e6, 4), "unit": "Mrays/s (build+trace)", "cores": os.cpu_count(),
            "kind": "oracle", "mprims_per_s": round(prims / dt / 1e6, 4),
            "sample": f"the {used} smallest scenes: FP64 BVH build + closest hit of their random rays "
                      f"({prims} triangles, {rays} rays, {dt:.1f} s)"}


def launch_command(args_list, gpus: int, port: int) -> list:
    """The torchrun command that runs this script as `gpus` ranks on this node (one
    process per GPU, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *args_list]


def spawn_ranks(args) -> int:
    """bench.py --gpus N (N > 1) started without torchrun: run itself under torchrun as N
    ranks and return its exit status (rank 0 prints the JSON line)."""
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    return subprocess.call(launch_command(sys.argv[1:], args.gpus, port))


def main():
    args = parse()
    if args.image:
        w, h = (int(x) for x in args.image.lower().split("x"))
        WORKLOAD.update(width=w, height=h)
    rank, world, local = dist_env()
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(spawn_ranks(args))
    if world != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but {world} ranks were launched")
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    elif args.workload == ADJOINT["workload"]:
        run_adjoint(args, rank, world, local)
    elif args.workload == BATCHED["workload"]:
        run_batched(args, rank, world, local)
    elif args.workload == ICOSPHERE["workload"]:
        run_icosphere(args, rank, world, local)
    elif args.workload == SPHERES["workload"]:
        run_spheres(args, rank, world, local)
    else:
        run_grt(args, rank, world, local)


if __name__ == "__main__":
    main()
