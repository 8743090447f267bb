"""GPU clustering build (PLOC: GRT_BUILD_PREFER_BALANCED, search radius 8, and
GRT_BUILD_PREFER_HIGH_QUALITY, radius 32) vs the oracle's sequential clustering:
topology, node numbering, parent links, boxes, 4-wide nodes and leaves bit-exact; traces
over the resulting trees (one level and instanced) vs the oracle's hits; refit; repeated
(graph-replayed) builds; flag validation."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import Geometry, device_tensor, hits_to_numpy, new_hits
from parity import check_any_hit_records, compare_any, compare_closest
from test_gpu_build import _case, _oracle_for, _read, check_bit_exact, check_refit_traces, check_tree, refit_reference

pytestmark = pytest.mark.gpu

FLAG = {8: grt.GRT_BUILD_PREFER_BALANCED, 32: grt.GRT_BUILD_PREFER_HIGH_QUALITY}


def _geometry(gpu, case, bits, radius):
    dev = {k: device_tensor(v) for k, v in case.items()}
    return Geometry(gpu, morton_bits=bits, build_flags=FLAG[radius], **dev).build()


def _no_device_error(ctx):
    assert grt.grtGetLastDeviceError(ctx.handle) == grt.GRT_SUCCESS


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "spheres", "dupes", "n1", "n2", "n3", "n17",
                                  "n257", "n4097"])
@pytest.mark.parametrize("radius", [8, 32])
def test_clustering_build_matches_oracle_bit_exact(gpu, name, radius):
    case = _case(name)
    g = _geometry(gpu, case, 30, radius)
    check_bit_exact(g, case, 30, radius)
    _no_device_error(gpu)
    g.close()


@pytest.mark.parametrize("name", ["terrain", "spheres"])
def test_clustering_build_63_bit_codes(gpu, name):
    case = _case(name)
    g = _geometry(gpu, case, 63, 8)
    check_bit_exact(g, case, 63, 8)
    _no_device_error(gpu)
    g.close()


def test_clustering_build_full_terrain_many_blocks(gpu):
    """The 131,072-triangle terrain of the instanced workload: hundreds of tiles spread
    over every block of the persistent launch, dozens of iterations."""
    m = scenegen.terrain(cells=256, amplitude=0.2)
    case = dict(vertices=m.vertices, indices=m.indices)
    for radius in (8, 32):
        g = _geometry(gpu, case, 30, radius)
        check_bit_exact(g, case, 30, radius)
        _no_device_error(gpu)
        g.close()


def test_clustering_build_equal_boxes(gpu):
    """Thousands of identical boxes: every candidate ties on area, the pair hash decides."""
    b = np.tile(np.array([[0, 0, 0, 1, 1, 1]], np.float32), (5000, 1))
    case = dict(boxes=b)
    g = _geometry(gpu, case, 30, 8)
    check_bit_exact(g, case, 30, 8)
    _no_device_error(gpu)
    g.close()


def test_clustering_cost_below_linear(gpu):
    """Surface-area cost of the GPU trees (from their own node boxes) on the terrain."""
    m = scenegen.terrain(cells=128, amplitude=0.2)
    dev = dict(vertices=device_tensor(m.vertices), indices=device_tensor(m.indices))
    costs = {}
    for flags in (grt.GRT_BUILD_PREFER_FAST, grt.GRT_BUILD_PREFER_BALANCED, grt.GRT_BUILD_PREFER_HIGH_QUALITY):
        g = Geometry(gpu, build_flags=flags, **dev).build()
        torch.cuda.synchronize()
        info = g.info()
        nodes = _read(info.nodes, info.nodeCount * 64, np.float32).reshape(-1, 16)
        lo = np.minimum(nodes[:, [0, 4, 8]], nodes[:, [2, 6, 10]])
        hi = np.maximum(nodes[:, [1, 5, 9]], nodes[:, [3, 7, 11]])
        costs[flags] = oracle.sah_cost(lo, hi)
        g.close()
    assert costs[1] < 0.85 * costs[0] and costs[2] < 0.85 * costs[0], costs


def _trace(ctx, rays_np, geom, any_hit=False):
    n = rays_np.shape[0]
    rays = device_tensor(rays_np)
    hits = new_hits(n)
    (grt.grtTraceAnyHit if any_hit else grt.grtTraceClosest)(ctx.handle, None, geom, rays, n, hits, None, None)
    torch.cuda.synchronize()
    return hits_to_numpy(hits)


@pytest.mark.parametrize("radius", [8, 32])
def test_trace_over_clustering_tree(gpu, radius):
    m = scenegen.terrain(cells=64, amplitude=0.2)
    g = _geometry(gpu, dict(vertices=m.vertices, indices=m.indices), 30, radius)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(m.vertices, m.indices))
    S.build()
    rays = scenegen.random_rays(50_000, [-1.2, -0.4, -1.2], [1.2, 0.4, 1.2], config=81)
    rays[::2, 7] = 0.3
    ref = S.trace(rays)
    got = _trace(gpu, rays, g.handle)
    compare_closest(got, ref, S, rays, extent=2.0).check()
    anyg = _trace(gpu, rays, g.handle, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=2.0).check()
    check_any_hit_records(anyg, S, rays, 2.0)
    _no_device_error(gpu)


def test_trace_spheres_over_clustering_tree(gpu):
    from paper_2603_00292_gb300.objects import FuncTable

    s = scenegen.spheres(20_000, half=10.0, rmin=0.01, rmax=0.5, config=85)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s)),
                 build_flags=grt.GRT_BUILD_PREFER_BALANCED).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    rays = scenegen.random_rays(40_000, [-10] * 3, [10] * 3, config=86)
    ref = S.trace(rays)
    n = rays.shape[0]
    hits = new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, g.handle, device_tensor(rays), n, hits, table.handle, None)
    torch.cuda.synchronize()
    compare_closest(hits_to_numpy(hits), ref, S, rays, extent=20.0, has_spheres=True).check()
    _no_device_error(gpu)


def test_refit_of_clustering_tree(gpu):
    """UPDATE of a clustered tree keeps its topology: both child boxes of every node,
    parent links, leaves and 4-wide nodes equal the oracle's fit of the kept clustering
    over the moved vertices, and closest hits traced afterwards equal the oracle's."""
    m = scenegen.terrain(cells=48, amplitude=0.2)
    v = device_tensor(m.vertices)
    g = Geometry(gpu, vertices=v, indices=device_tensor(m.indices), morton_bits=30,
                 build_flags=grt.GRT_BUILD_PREFER_BALANCED).build()
    moved = m.vertices.copy()
    moved[:, 1] *= 2.5
    v.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    lo, hi, cen = oracle.triangle_aabbs(m.vertices, m.indices)
    ref = oracle.ploc(lo, hi, cen, 10, 8)  # topology of the first build
    case = dict(vertices=moved, indices=m.indices)
    check_tree(g.info(), refit_reference(ref, case), case)
    check_refit_traces(gpu, g, case, seed=48)
    _no_device_error(gpu)
    g.close()


def test_repeated_builds_replay_and_follow_new_vertices(gpu):
    """The second and later BUILDs replay a captured graph of the same launches; moving
    the vertices in place gives the clustering of the new positions."""
    m = scenegen.terrain(cells=72, amplitude=0.2)
    v = device_tensor(m.vertices)
    idx = device_tensor(m.indices)
    g = Geometry(gpu, vertices=v, indices=idx, build_flags=grt.GRT_BUILD_PREFER_BALANCED).build()
    check_bit_exact(g, dict(vertices=m.vertices, indices=m.indices), 30, 8)
    g.build()
    check_bit_exact(g, dict(vertices=m.vertices, indices=m.indices), 30, 8)
    moved = m.vertices.copy()
    moved[:, 1] = -moved[:, 1] + 0.05 * np.cos(3 * moved[:, 0])
    v.copy_(torch.from_numpy(moved))
    g.build()
    check_bit_exact(g, dict(vertices=moved, indices=m.indices), 30, 8)
    _no_device_error(gpu)
    g.close()


def test_flag_validation(gpu):
    m = scenegen.icosphere(2)
    dev = dict(vertices=device_tensor(m.vertices), indices=device_tensor(m.indices))
    g = Geometry(gpu, build_flags=grt.GRT_BUILD_PREFER_BALANCED, **dev)
    # building with another flag than the geometry was created with
    with pytest.raises(grt.GrtError) as e:
        grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, g.input, grt.build_options(0, 0), g.temp,
                             None, g.handle)
    assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    with pytest.raises(grt.GrtError) as e:
        grt.grtGetGeometryBuildTemporaryBufferSize(gpu.handle, g.input, grt.build_options(0, 4))
    assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    fast = grt.grtGetGeometryBuildTemporaryBufferSize(gpu.handle, g.input, grt.build_options(0, 0))
    bal = grt.grtGetGeometryBuildTemporaryBufferSize(gpu.handle, g.input, grt.build_options(0, 1))
    sub = grt.grtGetGeometryBuildTemporaryBufferSize(gpu.handle, g.input,
                                                     grt.build_options(0, grt.GRT_BUILD_CLUSTER_SUBTREES))
    assert bal >= fast + 68 * m.indices.shape[0] and sub >= fast + 64 * m.indices.shape[0]
    g.close()


def test_two_level_scene_over_clustering_trees(gpu):
    """Instances of two clustered bottom levels (radius 8 and 32) under random SRT frames
    (the top level stays a linear BVH): closest and any hit against the oracle."""
    from paper_2603_00292_gb300.objects import Scene
    from test_gpu_trace import _aimed

    mesh = scenegen.terrain(cells=40, amplitude=0.2)
    dev = dict(vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices))
    g8 = Geometry(gpu, build_flags=grt.GRT_BUILD_PREFER_BALANCED, **dev).build()
    g32 = Geometry(gpu, build_flags=grt.GRT_BUILD_PREFER_HIGH_QUALITY, **dev).build()
    count = 10
    fr = scenegen.random_frames(count, config=89)
    handles = [g8.handle if k % 2 == 0 else g32.handle for k in range(count)]
    sc = Scene(gpu, handles, device_tensor(fr.packed())).build()
    S = oracle.Scene()
    gi = S.add_mesh(mesh.vertices, mesh.indices)
    for k in range(count):
        S.add_instance(gi, fr.packed()[k])
    S.build()
    rays = _aimed(40_000, fr.translation.astype(np.float64), 93)
    rays[::3, 7] = 6.0
    ref = S.trace(rays)
    n = rays.shape[0]
    hits = new_hits(n)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, device_tensor(rays), n, hits)
    torch.cuda.synchronize()
    rep = compare_closest(hits_to_numpy(hits), ref, S, rays, extent=25.0)
    rep.check()
    assert rep.matched > 10_000
    anyh = new_hits(n)
    grt.grtTraceAnyHit(gpu.handle, sc.handle, None, device_tensor(rays), n, anyh)
    torch.cuda.synchronize()
    compare_any(hits_to_numpy(anyh)[1], ref, S, rays, extent=25.0).check()
    _no_device_error(gpu)
    for obj in (sc, g8, g32):
        obj.close()
