"""Parity at full benchmark sizes, in the launch configurations bench.py times.

The oracle traces every ray here, not a sample: the FP64 oracle BVH runs at a few
Mrays/s on the host cores, so the 2.1 M primary rays and ~1 M ambient-occlusion rays
of the terrain workload, the 4.2 M sphere rays and sampled rays of the batched soups
all finish in seconds.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import (Batch, FuncTable, Geometry, Scene, device_tensor, empty_bytes,
                                            hits_to_numpy, new_hits, new_rays, read_device)
from parity import NONE, compare_any, compare_closest
from test_gpu_build import check_bit_exact

pytestmark = pytest.mark.gpu

SEED = 20260301


def _no_device_error(gpu):
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


def test_terrain_ambient_occlusion_1080p(gpu):
    """64 terrain instances (131,072 triangles each), 1920x1080 primary rays, 8 AO rays
    of length 0.05 extent per hit: the benchmark's step, checked ray by ray."""
    W, H, spp = 1920, 1080, 8
    sc = scenegen.terrain_instances(64, 256, 0.2, SEED)
    cam = scenegen.overview_camera(sc, W, H)
    mesh = sc.meshes[0]
    length = float(np.float32(0.05 * sc.extent))
    verts, idx = device_tensor(mesh.vertices), device_tensor(mesh.indices)
    g = Geometry(gpu, vertices=verts, indices=idx).build()
    check_bit_exact(g, dict(vertices=mesh.vertices, indices=mesh.indices), 30)
    scene = Scene(gpu, [g.handle] * 64, device_tensor(sc.frames.packed())).build()
    rays = new_rays(W * H)
    c = cam.packed()
    grt.grtGenerateCameraRays(gpu.handle, grt.camera(c[0:3], c[3:6], c[6:9]), W, H, rays)
    hits = new_hits(W * H)
    grt.grtTraceClosest(gpu.handle, scene.handle, None, rays, W * H, hits)
    ao = torch.empty(W * H, dtype=torch.float32, device="cuda")
    grt.grtTraceAmbientOcclusion(gpu.handle, scene.handle, rays, hits, W * H, spp, SEED, length, ao)
    ao_rays = new_rays(W * H * spp)
    grt.grtGenerateAORays(gpu.handle, scene.handle, rays, hits, W * H, spp, SEED, length, ao_rays)
    torch.cuda.synchronize()
    _no_device_error(gpu)
    prim_rays = rays.cpu().numpy()
    ref_rays = oracle.camera_rays(c, W, H)
    assert np.array_equal(prim_rays[:, 7], ref_rays[:, 7])  # maxT = +inf
    assert np.abs(prim_rays[:, :7] - ref_rays[:, :7]).max() < 1e-6

    S = oracle.Scene()
    gi = S.add_mesh(mesh.vertices, mesh.indices)
    for f in sc.frames.packed():
        S.add_instance(gi, f)
    S.build()
    ref = S.trace(prim_rays)
    got = hits_to_numpy(hits)
    rep = compare_closest(got, ref, S, prim_rays, extent=sc.extent)
    rep.check()
    assert rep.matched > 100_000

    # AO rays: the GPU's against the oracle's wherever the primary hits agree
    same = (got[1] == ref.prim) & (got[0] == ref.inst) & (ref.prim != NONE)
    ref_ao = oracle.ao_rays(S, prim_rays, ref, spp, SEED, length)
    g_ao = ao_rays.cpu().numpy()
    sel = np.repeat(same, spp)
    assert np.abs(g_ao[sel, 0:3] - ref_ao[sel, 0:3]).max() < 1e-5 * sc.extent
    assert np.abs(g_ao[sel, 4:7] - ref_ao[sel, 4:7]).max() < 1e-5
    # occlusion of the oracle's AO rays: GPU any-hit against the oracle
    valid = ref_ao[:, 7] > 0
    occ = new_hits(int(valid.sum()))
    grt.grtTraceAnyHit(gpu.handle, scene.handle, None, device_tensor(ref_ao[valid]), int(valid.sum()), occ)
    ref_occ = S.trace(ref_ao[valid], any_hit=True)
    compare_any(hits_to_numpy(occ)[1], ref_occ, S, ref_ao[valid], extent=sc.extent).check()
    # the fused AO image equals any-hit over the GPU's own AO rays, and the oracle's
    # image up to the exempt rays
    occ_g = new_hits(W * H * spp)
    grt.grtTraceAnyHit(gpu.handle, scene.handle, None, ao_rays, W * H * spp, occ_g)
    counts = (hits_to_numpy(occ_g)[1] != NONE).reshape(W * H, spp).sum(axis=1)
    assert np.array_equal(ao.cpu().numpy(), (counts / spp).astype(np.float32))
    ref_counts = np.zeros(W * H, np.int64)
    np.add.at(ref_counts, np.nonzero(valid)[0] // spp, (ref_occ.prim != NONE).astype(np.int64))
    diff = np.abs(counts - ref_counts)[same]
    assert diff.sum() < max(3, 1e-4 * valid.sum()), (diff.sum(), valid.sum())
    _no_device_error(gpu)


def test_million_spheres_closest_and_any_hit(gpu):
    """1 M spheres (centres in [-50,50]^3, radii log-U[0.01,1]) through the function
    table, 4,194,304 uniform random rays generated on the GPU (checked against the
    oracle's generator), closest hit and any hit, every ray checked."""
    s = scenegen.spheres(1_000_000, half=50.0, rmin=0.01, rmax=1.0, seed=SEED, config=3)
    boxes = scenegen.sphere_aabbs(s)
    g = Geometry(gpu, boxes=device_tensor(boxes)).build()
    check_bit_exact(g, dict(boxes=boxes), 30)
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    n = 4_194_304
    # the rays come from the GPU generator as in bench.py; they equal the oracle's
    # generator (FP64 from the same splitmix64 numbers) within float32 rounding
    rd = new_rays(n)
    grt.grtGenerateUniformRays(gpu.handle, [-50.0] * 3, [50.0] * 3, SEED, n, rd)
    rays = rd.cpu().numpy()
    want = oracle.uniform_rays([-50.0] * 3, [50.0] * 3, SEED, n)
    assert np.abs(rays[:, 0:3] - want[:, 0:3]).max() <= 1e-5  # 50 x 2^-22: within two ulps of 50
    assert np.abs(rays[:, 4:7] - want[:, 4:7]).max() <= 1e-6
    assert np.array_equal(rays[:, [3, 7]], want[:, [3, 7]])
    hc, ha = new_hits(n), new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, g.handle, rd, n, hc, table.handle)
    grt.grtTraceAnyHit(gpu.handle, None, g.handle, rd, n, ha, table.handle)
    torch.cuda.synchronize()
    _no_device_error(gpu)
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    ref = S.trace(rays)
    rep = compare_closest(hits_to_numpy(hc), ref, S, rays, extent=100.0, has_spheres=True)
    rep.check()
    assert rep.matched > 100_000
    compare_any(hits_to_numpy(ha)[1], ref, S, rays, extent=100.0, has_spheres=True).check()
    # with tmax = +inf nearly every ray is occluded (mean free path ~2.9 in a box of
    # 100); at tmax = 2.9 about 70% are, so occlusion parity is not trivially met
    short = rays.copy()
    short[:, 7] = 2.9
    hs = new_hits(n)
    grt.grtTraceAnyHit(gpu.handle, None, g.handle, device_tensor(short), n, hs, table.handle)
    torch.cuda.synchronize()
    _no_device_error(gpu)
    ref_short = S.trace(short, any_hit=True)
    occluded = (ref_short.prim != NONE).mean()
    assert 0.3 < occluded < 0.85, occluded
    compare_any(hits_to_numpy(hs)[1], ref_short, S, short, extent=100.0, has_spheres=True).check()


def _soup_worker(i):
    s = scenegen.soup_scene(i, seed=SEED)
    cam = s.camera
    rays = np.concatenate([oracle.camera_rays(cam.packed(), cam.width, cam.height), s.random_rays])
    return s.mesh.vertices, s.mesh.indices, rays.astype(np.float32), float(np.max(s.hi - s.lo))


def test_batched_soups_full_size(gpu):
    """The 256-soup batch (67.8 M triangles, 51.7 M rays) in one graph-captured launch:
    hit records identical to 256 per-scene build+trace calls, BVHs of the smallest and
    the largest scene bit-exact, and the oracle on every scene: every ray of 16 seeded
    scenes, 100,000 sampled rays of the four picked scenes (smallest, median, largest
    30-bit and largest 63-bit) and 4,096 sampled rays of every other scene."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(16) as pool:
        soups = pool.map(_soup_worker, range(256), chunksize=1)
    nbig = max(s[1].shape[0] for s in soups)
    temp = empty_bytes(grt.grtGetGeometryBuildTemporaryBufferSize(
        gpu.handle, grt.triangle_mesh_input(256, 256, triangle_count=nbig, vertex_count=3 * nbig),
        grt.build_options()))
    scenes, singles = [], []
    for v, i, r, _ in soups:
        dv, di, dr = device_tensor(v), device_tensor(i), device_tensor(r)
        scenes.append((Geometry(gpu, vertices=dv, indices=di, temp=temp), dr, new_hits(r.shape[0])))
        singles.append((Geometry(gpu, vertices=dv, indices=di, temp=temp), new_hits(r.shape[0])))
    B = Batch(gpu, scenes, grt.batch_options(graph=True))
    B.run()
    for (gs, hs), (_, r, _) in zip(singles, scenes):
        gs.build()
        grt.grtTraceClosest(gpu.handle, None, gs.handle, r, r.shape[0], hs)
    torch.cuda.synchronize()
    _no_device_error(gpu)
    for (_, _, hb), (_, hs) in zip(scenes, singles):
        assert torch.equal(hb, hs)
    sizes = np.array([s[1].shape[0] for s in soups])
    order = np.argsort(sizes)
    big63 = int(order[-1])
    big30 = int(next(k for k in order[::-1] if sizes[k] <= (1 << 20)))
    picks = [int(order[0]), int(order[len(order) // 2]), big30, big63]
    for k in (picks[0], big63):  # the batched build itself, bit for bit
        v, i, _, _ = soups[k]
        g = scenes[k][0]
        bits = grt.grtGetBvhInfo(gpu.handle, geom=g.handle).mortonBits
        ref_g = Geometry(gpu, vertices=device_tensor(v), indices=device_tensor(i), morton_bits=bits).build()
        check_bit_exact(ref_g, dict(vertices=v, indices=i), bits)
        a, b = g.info(), ref_g.info()
        n = a.primCount
        assert np.array_equal(read_device(a.nodes, 64 * a.nodeCount, np.uint32),
                              read_device(b.nodes, 64 * b.nodeCount, np.uint32))
        assert np.array_equal(read_device(a.leaves, 48 * n, np.uint32), read_device(b.leaves, 48 * n, np.uint32))
        m = a.nodeCount  # 4-wide nodes: all but the unused last float4 of each
        assert np.array_equal(read_device(a.wideNodes, 128 * m, np.uint32).reshape(m, 32)[:, :28],
                              read_device(b.wideNodes, 128 * m, np.uint32).reshape(m, 32)[:, :28])
    # the oracle: every ray of 16 seeded scenes, 100,000 sampled rays of the four picked
    # above (unless they are among the 16) and 4,096 sampled rays of every other scene
    rng = np.random.default_rng(SEED)
    full = set(int(k) for k in rng.choice(256, size=16, replace=False))
    checked = 0
    for k in range(256):
        v, i, r, extent = soups[k]
        if k in full:
            cap = r.shape[0]
        elif k in picks:
            cap = 100_000
        else:
            cap = 4096
        take = np.arange(r.shape[0]) if cap >= r.shape[0] else np.sort(rng.choice(r.shape[0], cap, replace=False))
        S = oracle.Scene()
        S.add_instance(S.add_mesh(v, i))
        S.build()
        ref = S.trace(r[take])
        got = tuple(a[take] for a in hits_to_numpy(scenes[k][2]))
        compare_closest(got, ref, S, r[take], extent=extent).check()
        checked += take.size
    assert checked > 1_000_000
