"""GPU 8-wide nodes (GRT_BUILD_WIDE8_NODES) against the oracle (oracle.wide8_nodes of its
own binary tree): every node bit for bit for the linear BVH (single-block and grid
builds, 30- and 63-bit codes), the clustering builds, refits and the batched launch;
traces through 8-wide geometries and scenes (8-wide on every level; 4-wide scenes over
8-wide, quantised and 4-wide instances) against the oracle's hits; ambient occlusion
through an 8-wide scene against the 4-wide one; an 8-wide scene rejecting a 4-wide
instance; device targets and flag validation."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import (FuncTable, Geometry, Scene, device_tensor, hits_to_numpy, new_hits,
                                            read_device)
from parity import compare_any, compare_closest
from test_gpu_build import _case, _oracle_for, check_tree, refit_reference

pytestmark = pytest.mark.gpu

W8 = grt.GRT_BUILD_WIDE8_NODES


def _ok(gpu):
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


def _ref(case, bits, method=grt.GRT_BUILD_PREFER_FAST):
    lo, hi, cen = _oracle_for(case)
    b = 10 if bits == 30 else 21
    if method == grt.GRT_BUILD_CLUSTER_SUBTREES:
        return oracle.subtree_cluster(lo, hi, cen, b, grt.CLUSTER_CAP)
    if method == grt.GRT_BUILD_PREFER_BALANCED:
        return oracle.ploc(lo, hi, cen, b, 8)
    return oracle.lbvh(lo, hi, cen, b)


def check_wide8(info, ref):
    """The 8-wide nodes traversal reads equal the oracle's collapse of its own binary tree,
    bit for bit: every slot box, child word and zero row."""
    assert info.wide8Nodes, "no 8-wide nodes"
    lo, hi, child = oracle.wide8_nodes(ref)
    m = info.nodeCount
    assert lo.shape[0] == m
    got = read_device(info.wide8Nodes, m * 256, np.float32).reshape(m, 16, 4)
    want = np.zeros((m, 16, 4), np.float32)
    for a in range(3):
        for h in range(2):
            want[:, 4 * a + h] = lo[:, 4 * h:4 * h + 4, a]
            want[:, 4 * a + 2 + h] = hi[:, 4 * h:4 * h + 4, a]
    want[:, 12] = child[:, 0:4].view(np.float32)
    want[:, 13] = child[:, 4:8].view(np.float32)
    gw, ww = got.view(np.uint32), want.view(np.uint32)
    bad = np.nonzero((gw != ww).reshape(m, -1).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {m} nodes differ, first {bad[:5]}"


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "spheres", "dupes", "dupes_small", "n1", "n2", "n3",
                                  "n17", "n2048", "n2049", "n4097"])
@pytest.mark.parametrize("bits", [30, 63])
def test_wide8_nodes_match_oracle_bit_exact(gpu, name, bits):
    case = _case(name)
    dev = {k: device_tensor(v) for k, v in case.items()}
    g = Geometry(gpu, morton_bits=bits, build_flags=W8, **dev).build()
    torch.cuda.synchronize()
    info = g.info()
    ref = _ref(case, bits)
    check_tree(info, ref, case)  # the rest of the build is unchanged by the flag
    check_wide8(info, ref)
    _ok(gpu)
    g.close()


@pytest.mark.parametrize("method", [grt.GRT_BUILD_PREFER_BALANCED, grt.GRT_BUILD_CLUSTER_SUBTREES])
def test_wide8_nodes_of_clustering_builds(gpu, method):
    for name in ("terrain", "spheres"):
        case = _case(name)
        dev = {k: device_tensor(v) for k, v in case.items()}
        g = Geometry(gpu, build_flags=method | W8, **dev).build()
        torch.cuda.synchronize()
        check_wide8(g.info(), _ref(case, 30, method))
        g.close()
    _ok(gpu)


def test_wide8_nodes_after_refit(gpu):
    from test_gpu_build import check_refit_traces

    m = scenegen.terrain(cells=70, amplitude=0.2)
    case = dict(vertices=m.vertices.copy(), indices=m.indices)
    dv, di = device_tensor(case["vertices"]), device_tensor(m.indices)
    g = Geometry(gpu, vertices=dv, indices=di, build_flags=W8).build()
    ref = _ref(case, 30)
    rng = np.random.default_rng(18)
    moved = (case["vertices"] + rng.normal(0, 0.01, case["vertices"].shape)).astype(np.float32)
    dv.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    case_m = dict(vertices=moved, indices=m.indices)
    check_wide8(g.info(), refit_reference(ref, case_m))
    check_refit_traces(gpu, g, case_m, seed=19)
    _ok(gpu)
    g.close()


def _terrain_scene_rays(k, n, seed):
    from test_gpu_trace import _aimed

    fr = scenegen.random_frames(k, config=seed)
    rays = _aimed(n, fr.translation.astype(np.float64), seed + 1)
    rays[::3, 7] = 5.0
    return fr, rays


def _oracle_terrain_scene(mesh, fr, k):
    T = oracle.Scene()
    gi = T.add_mesh(mesh.vertices, mesh.indices)
    for j in range(k):
        T.add_instance(gi, fr.packed()[j])
    T.build()
    return T


def test_traces_through_wide8_nodes(gpu):
    """Closest and any hit against the oracle's hits: spheres through an 8-wide geometry
    (tmax infinite and short); a two-level scene with an 8-wide top level over 8-wide
    terrain instances, whose closest hits equal those of the all-4-wide scene up to
    equal-t ties; and a 4-wide scene whose instances alternate between 8-wide (walked
    through their 4-wide nodes), quantised and 4-wide copies of the terrain."""
    s = scenegen.spheres(40_000, half=20.0, rmin=0.01, rmax=0.6, config=105)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s)), build_flags=W8).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    rays = scenegen.random_rays(60_000, [-20] * 3, [20] * 3, config=106)
    rays[1::2, 7] = 2.5
    ref = S.trace(rays)
    n = rays.shape[0]
    hc, ha = new_hits(n), new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, g.handle, device_tensor(rays), n, hc, table.handle)
    grt.grtTraceAnyHit(gpu.handle, None, g.handle, device_tensor(rays), n, ha, table.handle)
    torch.cuda.synchronize()
    rep = compare_closest(hits_to_numpy(hc), ref, S, rays, extent=40.0, has_spheres=True)
    rep.check()
    assert rep.matched > 10_000
    compare_any(hits_to_numpy(ha)[1], ref, S, rays, extent=40.0, has_spheres=True).check()

    mesh = scenegen.terrain(cells=48, amplitude=0.2)
    v, i = device_tensor(mesh.vertices), device_tensor(mesh.indices)
    g8 = Geometry(gpu, vertices=v, indices=i, build_flags=W8).build()
    gq = Geometry(gpu, vertices=v, indices=i, build_flags=grt.GRT_BUILD_QUANTIZED_NODES).build()
    g4 = Geometry(gpu, vertices=v, indices=i).build()
    k = 12
    fr, rays = _terrain_scene_rays(k, 60_000, 107)
    s8 = Scene(gpu, [g8.handle] * k, device_tensor(fr.packed()), build_flags=W8).build()
    sm = Scene(gpu, [(g8, gq, g4)[j % 3].handle for j in range(k)], device_tensor(fr.packed())).build()
    s4 = Scene(gpu, [g4.handle] * k, device_tensor(fr.packed())).build()
    T = _oracle_terrain_scene(mesh, fr, k)
    ref = T.trace(rays)
    n = rays.shape[0]
    dr = device_tensor(rays)
    h4 = new_hits(n)
    grt.grtTraceClosest(gpu.handle, s4.handle, None, dr, n, h4)
    torch.cuda.synchronize()
    w4 = hits_to_numpy(h4)
    for sc in (s8, sm):
        hc, ha = new_hits(n), new_hits(n)
        grt.grtTraceClosest(gpu.handle, sc.handle, None, dr, n, hc)
        grt.grtTraceAnyHit(gpu.handle, sc.handle, None, dr, n, ha)
        torch.cuda.synchronize()
        got = hits_to_numpy(hc)
        rep = compare_closest(got, ref, T, rays, extent=25.0)
        rep.check()
        assert rep.matched > 15_000
        compare_any(hits_to_numpy(ha)[1], ref, T, rays, extent=25.0).check()
        same = (got[0] == w4[0]) & (got[1] == w4[1])
        assert (~same).sum() <= max(3, 1e-4 * n)
        for j in (2, 3, 4):
            assert np.array_equal(got[j][same].view(np.uint32), w4[j][same].view(np.uint32))
    _ok(gpu)


def test_ambient_occlusion_through_an_8wide_scene(gpu):
    """The fused ambient-occlusion kernel over an all-8-wide terrain scene gives the image
    of the same scene on 4-wide nodes, except where the primary hits differ (equal-t
    ties)."""
    mesh = scenegen.terrain(cells=40, amplitude=0.2)
    v, i = device_tensor(mesh.vertices), device_tensor(mesh.indices)
    g8 = Geometry(gpu, vertices=v, indices=i, build_flags=W8).build()
    g4 = Geometry(gpu, vertices=v, indices=i).build()
    k = 10
    fr = scenegen.random_frames(k, config=111, scale_lo=1.5)
    s8 = Scene(gpu, [g8.handle] * k, device_tensor(fr.packed()), build_flags=W8).build()
    s4 = Scene(gpu, [g4.handle] * k, device_tensor(fr.packed())).build()
    W, H, spp = 320, 180, 8
    cam = scenegen.look_at_camera([0, 16, 22], [0, 0, 0], W, H)
    cr = torch.empty((W * H, 8), dtype=torch.float32, device="cuda")
    c = cam.packed()
    grt.grtGenerateCameraRays(gpu.handle, grt.camera(c[0:3], c[3:6], c[6:9]), W, H, cr)
    out = []
    for sc in (s8, s4):
        hits = new_hits(W * H)
        grt.grtTraceClosest(gpu.handle, sc.handle, None, cr, W * H, hits)
        ao = torch.empty(W * H, dtype=torch.float32, device="cuda")
        grt.grtTraceAmbientOcclusion(gpu.handle, sc.handle, cr, hits, W * H, spp, 5, 1.5, ao)
        torch.cuda.synchronize()
        out.append((hits, ao))
    (h8, a8), (h4, a4) = out
    same_hit = (h8[:, 0] == h4[:, 0]) & (h8[:, 1] == h4[:, 1])
    assert int((same_hit & (h8[:, 1] != -1)).sum()) > 500
    assert float(((a8 == a4) | ~same_hit).float().mean()) >= 0.999
    _ok(gpu)


def test_8wide_scene_rejects_a_4wide_instance(gpu):
    """An 8-wide scene instancing a geometry without 8-wide nodes latches
    GRT_ERROR_INVALID_PARAMETER (read on the host) and leaves that instance empty; the
    context stays usable."""
    m = scenegen.icosphere(2)
    v, i = device_tensor(m.vertices), device_tensor(m.indices)
    g8 = Geometry(gpu, vertices=v, indices=i, build_flags=W8).build()
    g4 = Geometry(gpu, vertices=v, indices=i).build()
    frames = np.array([[0, 0, 0, 1, 1, 1, 1, 0, 0, 0], [0, 0, 0, 1, 1, 1, 1, 5, 0, 0]], np.float32)
    sc = Scene(gpu, [g8.handle, g4.handle], device_tensor(frames), build_flags=W8).build()
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_ERROR_INVALID_PARAMETER
    rays = np.zeros((2, 8), np.float32)
    rays[:, 2], rays[:, 6], rays[:, 7] = 5.0, -1.0, np.inf
    rays[1, 0] = 5.0
    h = new_hits(2)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, device_tensor(rays), 2, h)
    torch.cuda.synchronize()
    got = hits_to_numpy(h)
    assert got[0][0] == 0 and got[1][0] != oracle.NONE  # the 8-wide instance is hit
    assert got[1][1] == oracle.NONE  # the 4-wide one is empty
    _ok(gpu)


def test_batched_launch_with_wide8_geometries(gpu):
    """The batched launch builds 8-wide geometries (one-block and phased scenes, 30- and
    63-bit codes, linear BVH and subtree clustering) exactly as grtBuildGeometry does,
    8-wide nodes included, and its hit records equal the per-scene traces (through the
    8-wide nodes there)."""
    from test_gpu_batch import _assert_identical, _run, _workload

    work = _workload(12, nmax=120_000, rmax=20_000)
    flags = lambda k: W8 | (grt.GRT_BUILD_CLUSTER_SUBTREES if k % 4 == 1 else 0)
    B, batched, single = _run(gpu, work, grt.batch_options(), morton_bits=lambda k: 63 if k % 5 == 3 else 0,
                              build_flags=flags)
    _assert_identical(batched, single)
    for (gb, _, _), (gs, _) in zip(batched, single):
        i1, i2 = gb.info(), gs.info()
        m = i1.nodeCount
        assert np.array_equal(read_device(i1.wide8Nodes, m * 256, np.uint32),
                              read_device(i2.wide8Nodes, m * 256, np.uint32))
    s, _ = work[0]
    lo, hi, cen = oracle.triangle_aabbs(s.mesh.vertices, s.mesh.indices)
    info = batched[0][0].info()
    check_wide8(info, oracle.lbvh(lo, hi, cen, 10 if info.mortonBits == 30 else 21))
    B.close()


def test_device_target_and_flag_validation(gpu):
    m = scenegen.icosphere(2)
    v, i = device_tensor(m.vertices), device_tensor(m.indices)
    g8 = Geometry(gpu, vertices=v, indices=i, build_flags=W8).build()
    t8 = grt.grtGetDeviceTarget(gpu.handle, geom=g8.handle)
    assert t8.nodeFormat == 2 and t8.nodes == g8.info().wide8Nodes
    with pytest.raises(grt.GrtError):  # one node format per geometry
        Geometry(gpu, vertices=v, indices=i, build_flags=W8 | grt.GRT_BUILD_QUANTIZED_NODES)
    with pytest.raises(grt.GrtError):  # a build must repeat the creation's flag
        grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, g8.input, grt.build_options(), g8.temp, None,
                             g8.handle)
    fr = scenegen.random_frames(3, config=4)
    sc = Scene(gpu, [g8.handle] * 3, device_tensor(fr.packed()), build_flags=W8).build()
    assert sc.info().wide8Nodes
    with pytest.raises(grt.GrtError):
        grt.grtBuildScene(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, sc.input, grt.build_options(), sc.temp, None,
                          sc.handle)
    _ok(gpu)
