"""Batched build + trace of many uneven triangle soups in one persistent launch.

Every geometry the batch builds must be bit-identical to grtBuildGeometry on the same
input (nodes, leaves, parents: the same Morton codes, stable sort and Karras topology),
every hit record identical to grtTraceClosest, and the hits must match the FP64 oracle
within the stated tolerances on sampled scenes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import Batch, Geometry, device_tensor, hits_to_numpy, new_hits, read_device
from parity import compare_closest

pytestmark = pytest.mark.gpu


def _soup_rays(s):
    cam = s.camera
    cam_rays = oracle.camera_rays(cam.packed(), cam.width, cam.height)
    return np.concatenate([cam_rays, s.random_rays]).astype(np.float32)


def _workload(count, nmax, rmax, seed=scenegen.MASTER_SEED):
    out = []
    for i in range(count):
        s = scenegen.soup_scene(i, seed=seed, nmin=100, nmax=nmax, rmin=256, rmax=rmax)
        out.append((s, _soup_rays(s)))
    return out


def _bvh_arrays(g):
    info = g.info()
    n = info.leafCount
    nodes = read_device(info.nodes, 64 * info.nodeCount, np.uint32)
    leaves = read_device(info.leaves, 48 * n, np.uint32)
    # a one-primitive hierarchy has no parent links (its leaf sits in node 0)
    parents = read_device(info.parents, 4 * (2 * n - 1), np.uint32) if n >= 2 else np.zeros(0, np.uint32)
    m = info.nodeCount  # 4-wide nodes without their unused last float4
    wide = read_device(info.wideNodes, 128 * m, np.uint32).reshape(m, 32)[:, :28]
    return nodes, leaves, parents, wide


def _run(gpu, work, opts, morton_bits=None, build_flags=None, split_factor=None):
    """The batch over `work`, and the same scenes built and traced one by one (each
    geometry of both created with build_flags(k), default the linear BVH, and
    split_factor(k))."""
    batched, single = [], []
    for k, (s, rays) in enumerate(work):
        bits = 0 if morton_bits is None else morton_bits(k)
        flags = 0 if build_flags is None else build_flags(k)
        f = 0.0 if split_factor is None else split_factor(k)
        v, i = device_tensor(s.mesh.vertices), device_tensor(s.mesh.indices)
        r = device_tensor(rays)
        batched.append((Geometry(gpu, vertices=v, indices=i, morton_bits=bits, build_flags=flags, split_factor=f), r,
                        new_hits(rays.shape[0])))
        g = Geometry(gpu, vertices=v, indices=i, morton_bits=bits, build_flags=flags, split_factor=f).build()
        h = new_hits(rays.shape[0])
        grt.grtTraceClosest(gpu.handle, None, g.handle, r, rays.shape[0], h)
        single.append((g, h))
    B = Batch(gpu, batched, opts)
    B.run()
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    return B, batched, single


def _assert_identical(batched, single):
    for (gb, _, hb), (gs, hs) in zip(batched, single):
        for a, b in zip(_bvh_arrays(gb), _bvh_arrays(gs)):
            assert np.array_equal(a, b)
        assert torch.equal(hb, hs)


def test_batch_matches_per_scene_builds_and_traces(gpu):
    """Small scenes (one block), 30-bit and forced 63-bit multi-item scenes."""
    work = _workload(24, nmax=120_000, rmax=30_000)
    B, batched, single = _run(gpu, work, grt.batch_options(), morton_bits=lambda k: 63 if k % 5 == 3 else 0)
    info = B.info()
    assert info.sceneCount == 24 and 0 < info.smallScenes < 24
    _assert_identical(batched, single)


@pytest.mark.parametrize("opts", [
    dict(block_size=64, shared_depth=8, compact=0.25, small_scene_prims=2000, sort_chunk_tiles=1, build_chunk=1024,
         trace_chunk=512),
    dict(block_size=256, shared_depth=32, compact=0.75, small_scene_prims=50_000, sort_chunk_tiles=32,
         build_chunk=100_000, trace_chunk=100_000, graph=True),
])
def test_batch_options_do_not_change_results(gpu, opts):
    work = _workload(10, nmax=60_000, rmax=8_000)
    B, batched, single = _run(gpu, work, grt.batch_options(**opts))
    _assert_identical(batched, single)
    if opts.get("graph"):  # a replay of the captured graph gives the same records
        before = [h.clone() for _, _, h in batched]
        for _, _, h in batched:
            h.fill_(-1)
        B.run()
        torch.cuda.synchronize()
        assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
        for a, (_, _, h) in zip(before, batched):
            assert torch.equal(a, h)


def test_batch_hits_match_oracle_on_sampled_scenes(gpu):
    work = _workload(6, nmax=40_000, rmax=6_000, seed=scenegen.MASTER_SEED + 7)
    B, batched, _ = _run(gpu, work, grt.batch_options(graph=True))
    for (s, rays), (g, r, h) in zip(work, batched):
        S = oracle.Scene()
        S.add_instance(S.add_mesh(s.mesh.vertices, s.mesh.indices))
        S.build()
        take = np.arange(0, rays.shape[0], max(1, rays.shape[0] // 1500))
        ref = S.trace(rays[take])
        got = tuple(a[take] for a in hits_to_numpy(h))
        extent = float(np.max(s.hi - s.lo))
        compare_closest(got, ref, S, rays[take], extent=extent).check()
        assert (got[1] != 0xFFFFFFFF).sum() > 0


def test_batch_edge_cases(gpu):
    """A one-triangle scene, a scene with no rays, and a scene whose rays all miss."""
    tri = scenegen.Mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.uint32))
    s = scenegen.soup_scene(0, nmin=3000, nmax=3000, rmin=600, rmax=600)
    away = np.tile(np.array([[0, 0, 5, 0, 0, 0, 1, np.inf]], np.float32), (100, 1))
    cases = [(tri, scenegen.random_rays(64, np.array([-1.0] * 3), np.array([1.0] * 3), 3, 1)),
             (s.mesh, np.zeros((0, 8), np.float32)), (s.mesh, away)]
    work = []
    for mesh, rays in cases:
        class _S:
            pass
        x = _S()
        x.mesh = mesh
        work.append((x, rays.astype(np.float32)))
    B, batched, single = _run(gpu, work, grt.batch_options())
    _assert_identical(batched, single)
    assert (hits_to_numpy(batched[2][2])[1] == 0xFFFFFFFF).all()


def test_expired_wait_latches_timeout_and_the_context_stays_usable(gpu):
    """A work item planned to wait for a completion that never comes: its wait runs out
    after wait_limit_ms, the launch latches GRT_ERROR_TIMEOUT and drains (every later item
    skips its work), and the same context then runs a normal batch correctly."""
    work = _workload(6, nmax=40_000, rmax=4_000)
    scenes = []
    for s, rays in work:
        v, i = device_tensor(s.mesh.vertices), device_tensor(s.mesh.indices)
        scenes.append((Geometry(gpu, vertices=v, indices=i), device_tensor(rays), new_hits(rays.shape[0])))
    stalled = Batch(gpu, scenes, grt.batch_options(wait_limit_ms=100, test_expire_wait=True))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    stalled.run()
    t1.record()
    t1.synchronize()
    assert 90.0 <= t0.elapsed_time(t1) < 5000.0  # the wait ran out, and the launch ended
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_ERROR_TIMEOUT
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS  # read and cleared
    stalled.close()
    B, batched, single = _run(gpu, work, grt.batch_options())
    _assert_identical(batched, single)


def test_batch_with_subtree_clustered_scenes(gpu):
    """Every other geometry created with GRT_BUILD_CLUSTER_SUBTREES (small and
    multi-item, 30- and 63-bit codes): the batch builds those by the clustering phases
    and the rest as linear BVHs; every geometry and hit record identical to the
    per-scene build and trace with the same flag, and the clustered per-scene builds
    bit-exact against the oracle."""
    from test_gpu_build import check_bit_exact

    work = _workload(20, nmax=120_000, rmax=30_000, seed=scenegen.MASTER_SEED + 5)
    cl = grt.GRT_BUILD_CLUSTER_SUBTREES
    B, batched, single = _run(gpu, work, grt.batch_options(), morton_bits=lambda k: 63 if k % 7 == 2 else 0,
                              build_flags=lambda k: cl if k % 2 == 0 else 0)
    info = B.info()
    assert info.sceneCount == 20 and info.smallScenes < 10  # clustered scenes never take the one-block path
    _assert_identical(batched, single)
    sizes = [w[0].mesh.indices.shape[0] for w in work]
    clustered = [k for k in range(20) if k % 2 == 0]
    for k in (min(clustered, key=lambda k: sizes[k]), max(clustered, key=lambda k: sizes[k]), 2):
        s = work[k][0]
        bits = grt.grtGetBvhInfo(gpu.handle, geom=single[k][0].handle).mortonBits
        check_bit_exact(single[k][0], dict(vertices=s.mesh.vertices, indices=s.mesh.indices), bits, subtree=True)
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    B.close()


@pytest.mark.parametrize("opts", [dict(), dict(block_size=64, build_chunk=1024, small_scene_prims=2000)])
def test_batch_with_split_scenes(gpu, opts):
    """Geometries with split triangles (factors 1, 0.5, 0.1) among plain ones, some also
    subtree-clustered, 8-wide or with 63-bit codes: the batch runs their splitting
    phases (chunk scans over several rounds with the small chunks) and builds and traces
    them exactly as grtBuildGeometry and grtTraceClosest do; the largest split scene
    bit-exact against the oracle's split and build."""
    from test_gpu_build import check_bit_exact

    work = _workload(14, nmax=120_000, rmax=20_000, seed=scenegen.MASTER_SEED + 9)
    sp = grt.GRT_BUILD_SPLIT_TRIANGLES
    flags = lambda k: ((sp if k % 3 != 2 else 0) | (grt.GRT_BUILD_CLUSTER_SUBTREES if k % 4 == 1 else 0) |
                       (grt.GRT_BUILD_WIDE8_NODES if k % 5 == 3 else 0))
    B, batched, single = _run(gpu, work, grt.batch_options(**opts), morton_bits=lambda k: 63 if k % 6 == 4 else 0,
                              build_flags=flags, split_factor=lambda k: (1.0, 0.5, 0.1)[k % 3])
    _assert_identical(batched, single)
    split = [k for k in range(14) if flags(k) & sp and not flags(k) & grt.GRT_BUILD_CLUSTER_SUBTREES]
    k = max(split, key=lambda k: work[k][0].mesh.indices.shape[0])
    s = work[k][0]
    info = grt.grtGetBvhInfo(gpu.handle, geom=batched[k][0].handle)
    n = s.mesh.indices.shape[0]
    ref = oracle.split_triangles(s.mesh.vertices, s.mesh.indices, oracle.split_budget(n, (1.0, 0.5, 0.1)[k % 3]))
    assert info.leafCount == ref[0].shape[0]
    check_bit_exact(single[k][0], dict(vertices=s.mesh.vertices, indices=s.mesh.indices), info.mortonBits, split=ref)
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    B.close()
