"""GPU traversal vs the oracle: closest-hit and any-hit over a single geometry, a
two-level instanced scene and custom spheres; camera and ambient-occlusion rays;
edge cases (empty and single-primitive geometry, stack spill, stack overflow)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import (FuncTable, Geometry, Scene, device_tensor, hits_to_numpy, new_hits,
                                             new_rays)
from parity import NONE, check_any_hit_records, compare_any, compare_closest

pytestmark = pytest.mark.gpu


def _trace(ctx, rays_np, scene=None, geom=None, any_hit=False, table=None, opts=None):
    n = rays_np.shape[0]
    rays = device_tensor(rays_np)
    hits = new_hits(n)
    fn = grt.grtTraceAnyHit if any_hit else grt.grtTraceClosest
    fn(ctx.handle, scene, geom, rays, n, hits, table, opts)
    torch.cuda.synchronize()
    return hits_to_numpy(hits)


def _no_device_error(ctx):
    assert grt.grtGetLastDeviceError(ctx.handle) == grt.GRT_SUCCESS


# ------------------------------------------------------------------ one geometry
def test_icosphere_512_closest_hit(gpu):
    """The smallest scene at full size: 1,280 triangles, 512x512 camera rays,
    against FP64 brute force over every triangle."""
    m = scenegen.icosphere(3)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    cam = scenegen.look_down_z_camera([0, 0, 3], 512, 512)
    rays = oracle.camera_rays(cam.packed(), 512, 512)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(m.vertices, m.indices))
    ref = S.trace(rays, bvh=False)
    got = _trace(gpu, rays, geom=g.handle)
    rep = compare_closest(got, ref, S, rays, extent=2.0)
    rep.check()
    assert rep.matched > 70_000
    _no_device_error(gpu)


def test_camera_rays_match_oracle(gpu):
    for W, H, eye in [(512, 512, [0, 0, 3]), (333, 97, [1.5, -2, 7])]:
        cam = scenegen.look_down_z_camera(eye, W, H)
        ref = oracle.camera_rays(cam.packed(), W, H)
        out = new_rays(W * H)
        c = cam.packed()
        grt.grtGenerateCameraRays(gpu.handle, grt.camera(c[0:3], c[3:6], c[6:9]), W, H, out)
        got = out.cpu().numpy()
        assert np.array_equal(got[:, 0:4], ref[:, 0:4]) and np.all(np.isinf(got[:, 7]))
        assert np.abs(got[:, 4:7] - ref[:, 4:7]).max() < 1e-6


def test_random_rays_terrain_closest_and_any(gpu):
    m = scenegen.terrain(cells=64, amplitude=0.2)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    S = oracle.Scene()
    S.add_instance(S.add_mesh(m.vertices, m.indices))
    S.build()
    rays = scenegen.random_rays(50_000, [-1.2, -0.4, -1.2], [1.2, 0.4, 1.2], config=81)
    rays[::2, 7] = 0.3
    ref = S.trace(rays)
    got = _trace(gpu, rays, geom=g.handle)
    compare_closest(got, ref, S, rays, extent=2.0).check()
    anyg = _trace(gpu, rays, geom=g.handle, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=2.0).check()
    check_any_hit_records(anyg, S, rays, 2.0)
    _no_device_error(gpu)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_tiny_geometries(gpu, n):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [-1, 0.5, 0.2]], np.float32)
    idx = np.array([[0, 1, 2], [0, 1, 3], [3, 4, 5]], np.uint32)[:n]
    g = Geometry(gpu, vertices=device_tensor(v), indices=device_tensor(idx)).build()
    S = oracle.Scene()
    S.add_instance(S.add_mesh(v, idx.reshape(-1, 3)))
    rays = scenegen.random_rays(4000, [-1, -1, -1], [2, 2, 2], config=82)
    ref = S.trace(rays, bvh=False)
    got = _trace(gpu, rays, geom=g.handle)
    compare_closest(got, ref, S, rays, extent=2.0).check()
    if n == 0:
        assert np.all(got[1] == NONE) and np.all(got[0] == NONE) and np.all(np.isinf(got[2]))


def test_degenerate_rays(gpu):
    m = scenegen.icosphere(2)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    r = np.zeros((6, 8), np.float32)
    r[0] = [0, 0, 3, 0, 0, 0, -1, -1]          # maxT < minT: empty interval
    r[1] = [0, 0, 3, 5, 0, 0, -1, np.inf]      # minT past the sphere
    r[2] = [np.nan, 0, 3, 0, 0, 0, -1, np.inf]  # NaN origin
    r[3] = [0, 0, 3, 0, 0, 0, 0, np.inf]        # zero direction
    r[4] = [0, 0, 0, 0, 1, 0, 0, np.inf]        # from inside: hits the shell
    r[5] = [0, 2, 0, 0, 0, -1, 0, np.inf]       # axis-parallel
    got = _trace(gpu, r, geom=g.handle)
    assert got[1][0] == NONE and got[1][1] == NONE and got[1][2] == NONE and got[1][3] == NONE
    assert got[1][4] != NONE and got[1][5] != NONE
    _no_device_error(gpu)


def test_stack_spill_to_global_and_overflow(gpu):
    s = scenegen.spheres(30_000, half=10.0, rmin=0.01, rmax=0.3, config=83)
    boxes = device_tensor(scenegen.sphere_aabbs(s))
    g = Geometry(gpu, boxes=boxes).build()
    table = FuncTable(gpu)
    sd = device_tensor(s)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, sd)
    rays = scenegen.random_rays(20_000, [-10] * 3, [10] * 3, config=84)
    base = _trace(gpu, rays, geom=g.handle, table=table.handle)
    # one shared entry per thread: almost every push spills to the global stack
    spill = _trace(gpu, rays, geom=g.handle, table=table.handle,
                   opts=grt.trace_options(shared_depth=1, global_depth=128))
    for a, b in zip(base, spill):
        assert np.array_equal(a, b)
    _no_device_error(gpu)
    # caller-owned global stack buffer
    opts = grt.trace_options(shared_depth=2, global_depth=64)
    need = grt.grtGetTraceGlobalStackSize(gpu.handle, opts)
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    own = _trace(gpu, rays, geom=g.handle, table=table.handle,
                 opts=grt.trace_options(shared_depth=2, global_depth=64, global_stack=buf, global_stack_bytes=need))
    for a, b in zip(base, own):
        assert np.array_equal(a, b)
    # too small a stack: the overflow is reported, the kernel still finishes
    _trace(gpu, rays, geom=g.handle, table=table.handle, opts=grt.trace_options(shared_depth=1, global_depth=1))
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_ERROR_STACK_OVERFLOW
    _no_device_error(gpu)


# ------------------------------------------------------------------ custom primitives
def test_spheres_closest_and_any_hit(gpu):
    s = scenegen.spheres(20_000, half=10.0, rmin=0.01, rmax=0.5, config=85)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s))).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    rays = scenegen.random_rays(60_000, [-10] * 3, [10] * 3, config=86)
    rays[1::2, 7] = 2.5
    ref = S.trace(rays)
    got = _trace(gpu, rays, geom=g.handle, table=table.handle)
    rep = compare_closest(got, ref, S, rays, extent=20.0, has_spheres=True)
    rep.check()
    assert rep.matched > 5000
    anyg = _trace(gpu, rays, geom=g.handle, table=table.handle, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=20.0, has_spheres=True).check()
    # without a table entry custom primitives are never hit
    empty = FuncTable(gpu)
    none = _trace(gpu, rays, geom=g.handle, table=empty.handle)
    assert np.all(none[1] == NONE)


def test_function_table_layout(gpu):
    """Entry (rayType, geomType) at rayType * numGeomTypes + geomType."""
    s = scenegen.spheres(2000, half=5.0, config=87)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s)), geom_type=1).build()
    table = FuncTable(gpu, num_geom_types=2, num_ray_types=2)
    table.set(1, 1, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    rays = scenegen.random_rays(5000, [-5] * 3, [5] * 3, config=88)
    hit0 = _trace(gpu, rays, geom=g.handle, table=table.handle, opts=grt.trace_options(ray_type=0))
    hit1 = _trace(gpu, rays, geom=g.handle, table=table.handle, opts=grt.trace_options(ray_type=1))
    assert np.all(hit0[1] == NONE) and np.any(hit1[1] != NONE)


# ------------------------------------------------------------------ two levels
def _instanced(gpu, cells=32, count=12, with_spheres=False):
    mesh = scenegen.terrain(cells=cells, amplitude=0.2)
    fr = scenegen.random_frames(count, config=89)
    g = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    handles = [g.handle] * count
    S = oracle.Scene()
    gi = S.add_mesh(mesh.vertices, mesh.indices)
    for k in range(count):
        S.add_instance(gi, fr.packed()[k])
    keep = [g]
    table = None
    if with_spheres:
        s = scenegen.spheres(3000, half=1.0, rmin=0.01, rmax=0.2, config=90)
        gs = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s))).build()
        table = FuncTable(gpu)
        table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
        keep += [gs, table]
        handles.append(gs.handle)
        frames = np.concatenate([fr.packed(), np.array([[0, 0, 0.3826834, 0.9238795, 2, 1, 0.5, 1, 2, 3]],
                                                         np.float32)])
        S.add_instance(S.add_spheres(s), frames[-1])
    else:
        frames = fr.packed()
    sc = Scene(gpu, handles, device_tensor(frames)).build()
    keep.append(sc)
    S.build()
    return sc, S, fr, table, keep


def _aimed(n, targets, seed, spread=0.8):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-12, 12, (n, 3))
    t = targets[rng.integers(0, len(targets), n)] + rng.normal(0, spread, (n, 3))
    d = t - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = d
    r[:, 7] = np.inf
    return r


@pytest.mark.parametrize("with_spheres", [False, True])
def test_two_level_scene_closest_and_any(gpu, with_spheres):
    sc, S, fr, table, keep = _instanced(gpu, with_spheres=with_spheres)
    targets = np.concatenate([fr.translation.astype(np.float64), [[1, 2, 3]]])
    rays = _aimed(60_000, targets, 91)
    rays[::3, 7] = 6.0
    ref = S.trace(rays)
    tbl = table.handle if table else None
    got = _trace(gpu, rays, scene=sc.handle, table=tbl)
    rep = compare_closest(got, ref, S, rays, extent=25.0, has_spheres=with_spheres)
    rep.check()
    assert rep.matched > 10_000
    anyg = _trace(gpu, rays, scene=sc.handle, table=tbl, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=25.0, has_spheres=with_spheres).check()
    _no_device_error(gpu)


def test_instance_frames_and_world_boxes(gpu):
    sc, S, fr, table, keep = _instanced(gpu, count=7)
    info = sc.info()
    from paper_2603_00292_gb300.objects import read_device
    recs = read_device(info.leaves, 7 * 128, np.float32).reshape(7, 32)
    ids = recs.view(np.uint32)[:, 16]
    assert sorted(ids.tolist()) == list(range(7))
    mesh = scenegen.terrain(cells=32, amplitude=0.2)
    for row, i in zip(recs, ids):
        fwd, inv = S.instance_frames(int(i))
        # float32 inverse frame = the FP64 frame rounded
        assert np.array_equal(row[0:12].reshape(3, 4), inv.astype(np.float32))
        # the world box holds every transformed vertex
        w = mesh.vertices.astype(np.float64) @ fwd[:, :3].T + fwd[:, 3]
        assert np.all(row[20:23] <= w.min(axis=0)) and np.all(row[24:27] >= w.max(axis=0))


@pytest.mark.parametrize("count,cells", [(12, 32), (4500, 6)])
def test_scene_update_after_frames_moved(gpu, count, cells):
    """UPDATE of a scene after every instance frame changed in place: closest and any-hit
    traces equal the oracle's over the new frames. 12 instances take the one-block top
    level, 4,500 the grid launches."""
    mesh = scenegen.terrain(cells=cells, amplitude=0.2)
    g = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    fr0 = scenegen.random_frames(count, config=89)
    frames = device_tensor(fr0.packed())
    sc = Scene(gpu, [g.handle] * count, frames).build()
    fr1 = scenegen.random_frames(count, config=92)
    frames.copy_(torch.from_numpy(fr1.packed()))
    sc.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    S = oracle.Scene()
    gi = S.add_mesh(mesh.vertices, mesh.indices)
    for k in range(count):
        S.add_instance(gi, fr1.packed()[k])
    S.build()
    rays = _aimed(40_000, fr1.translation.astype(np.float64), 95)
    rays[::3, 7] = 6.0
    ref = S.trace(rays)
    got = _trace(gpu, rays, scene=sc.handle)
    rep = compare_closest(got, ref, S, rays, extent=25.0)
    rep.check()
    assert rep.matched > 10_000
    anyg = _trace(gpu, rays, scene=sc.handle, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=25.0).check()
    _no_device_error(gpu)
    sc.close()
    g.close()


# ------------------------------------------------------------------ ambient occlusion
def test_ambient_occlusion_rays_and_occlusion(gpu):
    sc, S, fr, table, keep = _instanced(gpu, cells=32, count=16)
    W, H, spp, seed = 192, 128, 8, 77
    from scenegen import InstancedScene
    mesh = scenegen.terrain(cells=32, amplitude=0.2)
    g = np.zeros(16, np.int32)
    blo, bhi = scenegen.world_bounds([mesh], g, fr)
    scn = InstancedScene([mesh], g, fr, blo, bhi)
    cam = scenegen.overview_camera(scn, W, H)
    prim_rays = oracle.camera_rays(cam.packed(), W, H)
    ref = S.trace(prim_rays)
    length = np.float32(0.05 * scn.extent)
    # GPU primary hits, then GPU AO rays; compare with the oracle's AO rays where hits agree
    rays_d = device_tensor(prim_rays)
    hits_d = new_hits(W * H)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, rays_d, W * H, hits_d)
    ao_d = new_rays(W * H * spp)
    grt.grtGenerateAORays(gpu.handle, sc.handle, rays_d, hits_d, W * H, spp, seed, float(length), ao_d)
    torch.cuda.synchronize()
    gh = hits_to_numpy(hits_d)
    same = (gh[1] == ref.prim) & (gh[0] == ref.inst) & (ref.prim != NONE)
    assert same.sum() >= 0.99 * (ref.prim != NONE).sum() and same.sum() > 200, (same.sum(), (ref.prim != NONE).sum())
    ao_ref = oracle.ao_rays(S, prim_rays, ref, spp, seed, float(length))
    ao_got = ao_d.cpu().numpy()
    sel = np.repeat(same, spp)
    d_o = np.abs(ao_got[sel, 0:3] - ao_ref[sel, 0:3]).max()
    d_d = np.abs(ao_got[sel, 4:7] - ao_ref[sel, 4:7]).max()
    assert d_o < 1e-5 * scn.extent and d_d < 1e-5, (d_o, d_d)
    miss = np.repeat(gh[1] == NONE, spp)
    assert np.all(ao_got[miss, 7] == -1)
    # occlusion of the oracle's AO rays, GPU any-hit vs oracle
    valid = ao_ref[:, 7] > 0
    occ = _trace(gpu, ao_ref[valid], scene=sc.handle, any_hit=True)
    ref_ao = S.trace(ao_ref[valid])
    rep = compare_any(occ[1], ref_ao, S, ao_ref[valid], extent=scn.extent)
    rep.check()
    # the fused kernel equals materialised rays + any-hit on the GPU, exactly
    ao_img = torch.empty(W * H, dtype=torch.float32, device="cuda")
    grt.grtTraceAmbientOcclusion(gpu.handle, sc.handle, rays_d, hits_d, W * H, spp, seed, float(length), ao_img)
    occ_all = _trace(gpu, ao_got, scene=sc.handle, any_hit=True)
    expect = (occ_all[1] != NONE).reshape(W * H, spp).sum(axis=1) / spp
    assert np.array_equal(ao_img.cpu().numpy(), expect.astype(np.float32))
    assert 0.0 < expect[gh[1] != NONE].mean() < 1.0
    _no_device_error(gpu)


# ------------------------------------------------------------------ instance and ray masks
def test_instance_and_ray_masks(gpu):
    """Sec. 7.5: an instance takes part only when its mask ANDed with the ray mask is
    nonzero (0 in either place means all bits). Closest and any hit against the oracle
    with the same effective masks, the fused AO kernel against any-hit on its own rays
    under the same mask, and the device-side entry point honouring the mask."""
    count = 12
    mesh = scenegen.terrain(cells=32, amplitude=0.2)
    fr = scenegen.random_frames(count, config=89)
    g = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    masks = [0, 1, 2, 3, 4, 6, 8, 1, 2, 0x10, 0x80000000, 5]
    sc = Scene(gpu, [g.handle] * count, device_tensor(fr.packed()), masks=masks).build()
    S = oracle.Scene()
    gi = S.add_mesh(mesh.vertices, mesh.indices)
    for k in range(count):
        S.add_instance(gi, fr.packed()[k])
        S.set_instance_mask(k, masks[k] if masks[k] else 0xFFFFFFFF)
    S.build()
    targets = fr.translation.astype(np.float64)
    rays = _aimed(40_000, targets, 93)
    rays[::4, 7] = 6.0
    for ray_mask in (0, 0x1, 0x6, 0x80000010, 0x40000000):
        effective = ray_mask if ray_mask else 0xFFFFFFFF
        opts = grt.trace_options(ray_mask=ray_mask)
        ref = S.trace(rays, ray_mask=effective)
        got = _trace(gpu, rays, scene=sc.handle, opts=opts)
        compare_closest(got, ref, S, rays, extent=25.0).check()
        anyg = _trace(gpu, rays, scene=sc.handle, any_hit=True, opts=opts)
        compare_any(anyg[1], ref, S, rays, extent=25.0).check()
        visible = {k for k in range(count) if (masks[k] if masks[k] else 0xFFFFFFFF) & effective}
        hit = got[1] != NONE
        assert set(np.unique(got[0][hit]).tolist()) <= visible
        if ray_mask == 0x40000000:  # only instance 0 (mask 0 = all bits) is visible
            assert visible == {0}
    _no_device_error(gpu)


def test_ambient_occlusion_with_a_ray_mask(gpu):
    sc, S, fr, table, keep = _instanced(gpu, cells=32, count=16)
    W, H, spp, seed = 160, 96, 8, 79
    from scenegen import InstancedScene
    mesh = scenegen.terrain(cells=32, amplitude=0.2)
    g = np.zeros(16, np.int32)
    blo, bhi = scenegen.world_bounds([mesh], g, fr)
    scn = InstancedScene([mesh], g, fr, blo, bhi)
    cam = scenegen.overview_camera(scn, W, H)
    masks = [1 << (k % 3) for k in range(16)]
    gm = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    scm = Scene(gpu, [gm.handle] * 16, device_tensor(fr.packed()), masks=masks).build()
    rays_d = device_tensor(oracle.camera_rays(cam.packed(), W, H))
    hits_d = new_hits(W * H)
    grt.grtTraceClosest(gpu.handle, scm.handle, None, rays_d, W * H, hits_d)
    length = float(np.float32(0.05 * scn.extent))
    ao_d = new_rays(W * H * spp)
    grt.grtGenerateAORays(gpu.handle, scm.handle, rays_d, hits_d, W * H, spp, seed, length, ao_d)
    opts = grt.trace_options(ray_mask=0x2)
    img = torch.empty(W * H, dtype=torch.float32, device="cuda")
    grt.grtTraceAmbientOcclusion(gpu.handle, scm.handle, rays_d, hits_d, W * H, spp, seed, length, img, opts)
    occ = _trace(gpu, ao_d.cpu().numpy(), scene=scm.handle, any_hit=True, opts=opts)
    expect = (occ[1] != NONE).reshape(W * H, spp).sum(axis=1) / spp
    assert np.array_equal(img.cpu().numpy(), expect.astype(np.float32))
    full = torch.empty_like(img)
    grt.grtTraceAmbientOcclusion(gpu.handle, scm.handle, rays_d, hits_d, W * H, spp, seed, length, full)
    assert (img <= full).all() and (img < full).any()  # fewer occluders under the mask
    _no_device_error(gpu)


# ------------------------------------------------------------------ intersection filters
def _bits(keep):
    w = np.zeros((keep.size + 31) // 32, np.uint32)
    idx = np.nonzero(keep)[0]
    np.bitwise_or.at(w, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return w


@pytest.mark.parametrize("two_level", [False, True])
def test_primitive_mask_filter(gpu, two_level):
    """Sec. 7.6: a filter rejects hits, for triangles and custom primitives alike; traversal
    goes on past them. The built-in primitive-mask filter against the oracle with the
    same filter; under another ray type (table row without a filter) nothing is rejected."""
    rng = np.random.default_rng(61)
    mesh = scenegen.terrain(cells=48, amplitude=0.2)
    sph = scenegen.spheres(2000, half=1.0, rmin=0.01, rmax=0.15, config=62)
    keep_t = rng.random(mesh.indices.shape[0]) < 0.55
    keep_s = rng.random(sph.shape[0]) < 0.5
    gt = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices), geom_type=0).build()
    gs = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(sph)), geom_type=1).build()
    table = FuncTable(gpu, num_geom_types=2, num_ray_types=2)
    table.set(0, 0, grt.GRT_INTERSECT_NONE, None, grt.GRT_FILTER_PRIMITIVE_MASK, device_tensor(_bits(keep_t)))
    table.set(1, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(sph), grt.GRT_FILTER_PRIMITIVE_MASK,
              device_tensor(_bits(keep_s)))
    table.set(1, 1, grt.GRT_INTERSECT_SPHERE, device_tensor(sph))  # ray type 1: no filter
    S = oracle.Scene()
    ot = S.add_mesh(mesh.vertices, mesh.indices)
    os_ = S.add_spheres(sph)
    U = oracle.Scene()  # unfiltered, for ray type 1
    ut = U.add_mesh(mesh.vertices, mesh.indices)
    us = U.add_spheres(sph)
    S.set_prim_filter(ot, _bits(keep_t))
    S.set_prim_filter(os_, _bits(keep_s))
    frame = np.array([0, 0, 0, 1, 1, 1, 1, 0, 0.4, 0], np.float32)
    rays = _aimed(50_000, np.array([[0.0, 0.0, 0.0], [0.0, 0.4, 0.0]]), 63, spread=0.6)
    rays[::3, 7] = 2.0
    if two_level:
        sc = Scene(gpu, [gt.handle, gs.handle], device_tensor(np.stack([np.array([0, 0, 0, 1, 1, 1, 1, 0, 0, 0],
                                                                                  np.float32), frame])))
        sc.build()
        for X, a, b in ((S, ot, os_), (U, ut, us)):
            X.add_instance(a)
            X.add_instance(b, frame)
        target = dict(scene=sc.handle)
    else:
        S.add_instance(ot)
        U.add_instance(ut)
        target = dict(geom=gt.handle)
    S.build()
    U.build()
    for ray_type, ref_scene in ((0, S), (1, U)):
        opts = grt.trace_options(ray_type=ray_type)
        ref = ref_scene.trace(rays)
        got = _trace(gpu, rays, table=table.handle, opts=opts, **target)
        compare_closest(got, ref, ref_scene, rays, extent=3.0, has_spheres=two_level).check()
        anyg = _trace(gpu, rays, any_hit=True, table=table.handle, opts=opts, **target)
        compare_any(anyg[1], ref, ref_scene, rays, extent=3.0, has_spheres=two_level).check()
        hit = got[1] != NONE
        assert hit.mean() > 0.05
        if ray_type == 0:  # no rejected primitive is ever reported
            tri = hit & (got[0] == 0)
            assert keep_t[got[1][tri]].all()
            if two_level:
                sp = hit & (got[0] == 1)
                assert sp.any() and keep_s[got[1][sp]].all()
    _no_device_error(gpu)


# ------------------------------------------------------------------ all hits (Sec. 7.5)
def _all_hits(gpu, rays_np, k, **kw):
    n = rays_np.shape[0]
    hits = new_hits(n * k)
    counts = torch.empty(n, dtype=torch.int32, device="cuda")
    grt.grtTraceAllHits(gpu.handle, kw.get("scene"), kw.get("geom"), device_tensor(rays_np), n, hits, k, counts,
                        kw.get("table"), kw.get("opts"))
    torch.cuda.synchronize()
    h = hits_to_numpy(hits)
    return tuple(a.reshape(n, k) for a in h), counts.cpu().numpy().astype(np.int64)


def _check_all_hits(got, cnt, ref, S, rays, k, extent):
    """Per ray the set of (instance, primitive) equals the oracle's; matched t within
    1e-5 relative, u, v within 1e-5. A ray may differ only where it grazes an edge
    (margin below 1e-6), and such rays must stay below 1e-4 of all (at least 3 allowed)."""
    gi, gp, gt, gu, gv = got
    ri, rp, rt, ru, rv, rc = ref
    bad = 0
    for r in range(rays.shape[0]):
        m = min(cnt[r], k)
        a = sorted(zip(gi[r, :m].tolist(), gp[r, :m].tolist()))
        b = sorted(zip(ri[r, :min(rc[r], k)].tolist(), rp[r, :min(rc[r], k)].tolist()))
        if cnt[r] != rc[r] or (cnt[r] <= k and a != b):
            assert S.min_edge_margin(rays[r]) < 1e-6, (r, a, b)
            bad += 1
            continue
        if cnt[r] > k:  # truncated: the test keeps k above the largest count
            continue
        ref_t = {(i, p): (t, uu, vv) for i, p, t, uu, vv in zip(ri[r, :m], rp[r, :m], rt[r, :m], ru[r, :m], rv[r, :m])}
        for j in range(m):
            t, uu, vv = ref_t[(gi[r, j], gp[r, j])]
            assert abs(gt[r, j] - t) <= 1e-5 * max(abs(t), 1e-3 * extent), (r, gt[r, j], t)
            assert abs(gu[r, j] - uu) <= 1e-5 and abs(gv[r, j] - vv) <= 1e-5
    assert bad <= max(3, 1e-4 * rays.shape[0]), bad


def test_all_hits_two_level_scene(gpu):
    sc, S, fr, table, keep = _instanced(gpu, cells=32, count=12)
    rays = _aimed(20_000, fr.translation.astype(np.float64), 88)
    rays[::2, 7] = 8.0
    k = 12
    got, cnt = _all_hits(gpu, rays, k, scene=sc.handle)
    ref = S.all_hits(rays, k)
    assert (ref[5] >= 2).sum() > 200 and ref[5].max() <= k
    _check_all_hits(got, cnt, ref, S, rays, k, extent=25.0)
    # counts agree with any-hit, and the nearest stored hit is the closest hit
    anyg = _trace(gpu, rays, scene=sc.handle, any_hit=True)
    assert np.array_equal(cnt > 0, anyg[1] != NONE)
    close = _trace(gpu, rays, scene=sc.handle)
    hit = cnt > 0
    tmin = np.where(np.arange(k)[None, :] < cnt[:, None], got[2], np.inf).min(axis=1)
    assert np.array_equal(tmin[hit], close[2][hit])
    # truncation: two slots per ray, the count still complete
    got2, cnt2 = _all_hits(gpu, rays, 2, scene=sc.handle)
    assert np.array_equal(cnt2, cnt)
    assert np.array_equal(got2[1], got[1][:, :2]) and np.array_equal(got2[2].view(np.uint32), got[2][:, :2].view(np.uint32))
    _no_device_error(gpu)


def test_all_hits_with_masks_filters_and_spheres(gpu):
    rng = np.random.default_rng(64)
    mesh = scenegen.terrain(cells=32, amplitude=0.3)
    sph = scenegen.spheres(1500, half=1.0, rmin=0.01, rmax=0.15, config=65)
    keep_s = rng.random(sph.shape[0]) < 0.6
    gt = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices), geom_type=0).build()
    gs = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(sph)), geom_type=1).build()
    table = FuncTable(gpu, num_geom_types=2, num_ray_types=1)
    table.set(1, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(sph), grt.GRT_FILTER_PRIMITIVE_MASK,
              device_tensor(_bits(keep_s)))
    frames = np.array([[0, 0, 0, 1, 1, 1, 1, 0, 0, 0], [0, 0, 0, 1, 1, 1, 1, 0, 0.3, 0],
                       [0, 0.3826834, 0, 0.9238795, 1, 1, 1, 0, -0.2, 0]], np.float32)
    masks = [1, 2, 4]
    sc = Scene(gpu, [gt.handle, gs.handle, gt.handle], device_tensor(frames), masks=masks).build()
    S = oracle.Scene()
    ot, os_ = S.add_mesh(mesh.vertices, mesh.indices), S.add_spheres(sph)
    S.set_prim_filter(os_, _bits(keep_s))
    for i, (g_, f) in enumerate(zip((ot, os_, ot), frames)):
        S.add_instance(g_, f)
        S.set_instance_mask(i, masks[i])
    S.build()
    rays = _aimed(15_000, np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 0.0]]), 66, spread=0.5)
    k = 16
    for ray_mask in (0x3, 0x6, 0x7):
        got, cnt = _all_hits(gpu, rays, k, scene=sc.handle, table=table.handle,
                             opts=grt.trace_options(ray_mask=ray_mask))
        ref = S.all_hits(rays, k, ray_mask=ray_mask)
        _check_all_hits(got, cnt, ref, S, rays, k, extent=3.0)
        assert (cnt >= 2).sum() > 100
    _no_device_error(gpu)


def test_all_hits_edge_cases(gpu):
    empty = Geometry(gpu, vertices=device_tensor(np.zeros((3, 3), np.float32)),
                     indices=device_tensor(np.zeros((0, 3), np.uint32))).build()
    rays = _aimed(100, np.zeros((1, 3)), 87)
    got, cnt = _all_hits(gpu, rays, 3, geom=empty.handle)
    assert (cnt == 0).all() and (got[1] == NONE).all()
    with pytest.raises(grt.GrtError):
        grt.grtTraceAllHits(gpu.handle, None, empty.handle, device_tensor(rays), 100, new_hits(100), 0,
                            torch.empty(100, dtype=torch.int32, device="cuda"))
    grt.grtTraceAllHits(gpu.handle, None, empty.handle, None, 0, None, 4, None)  # no rays: nothing to do
    _no_device_error(gpu)


@pytest.mark.parametrize("count", [1, 255, 257, 100_003])
def test_uniform_rays_match_oracle(gpu, count):
    """grtGenerateUniformRays against the oracle's FP64 generator from the same
    splitmix64 numbers: origins within float32 rounding of the box, directions within
    1e-6, range ends exact; an off-centre, non-cubic box."""
    lo, hi = [-3.0, 10.0, -0.5], [5.0, 11.0, 0.25]
    rays = new_rays(count)
    grt.grtGenerateUniformRays(gpu.handle, lo, hi, 1234567, count, rays, 0.125, 7.5)
    torch.cuda.synchronize()
    got = rays.cpu().numpy()
    want = oracle.uniform_rays(lo, hi, 1234567, count, 0.125, 7.5)
    assert np.abs(got[:, 0:3] - want[:, 0:3]).max() <= 2.5e-6  # two ulps of 11
    assert np.abs(got[:, 4:7] - want[:, 4:7]).max() <= 1e-6
    assert np.all(got[:, 3] == np.float32(0.125)) and np.all(got[:, 7] == np.float32(7.5))
    assert np.all(got[:, 0:3] >= np.float32(lo)) and np.all(got[:, 0:3] <= np.float32(hi))
    # rejected: a box with hi < lo, a misaligned ray buffer
    with pytest.raises(grt.GrtError):
        grt.grtGenerateUniformRays(gpu.handle, hi, lo, 1, count, rays)
    flat = torch.empty(8 * count + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(grt.GrtError):
        grt.grtGenerateUniformRays(gpu.handle, lo, hi, 1, count, flat[1:])
