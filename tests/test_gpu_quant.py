"""GPU quantised 4-wide nodes (GRT_BUILD_QUANTIZED_NODES) against the oracle
(oracle.quantized_wide_nodes of its own wide nodes): every node word bit for bit, for the
linear BVH (single-block and grid builds, 30- and 63-bit codes), the clustering builds,
refits and the batched launch; traces through quantised geometries, alone and as
instances beside 128-byte ones, against the oracle's hits; the device-side target; flag
validation."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import (FuncTable, Geometry, Scene, device_tensor, hits_to_numpy,
                                            new_hits, read_device)
from parity import compare_any, compare_closest
from test_gpu_build import _case, _oracle_for, check_tree, refit_reference

pytestmark = pytest.mark.gpu

Q = grt.GRT_BUILD_QUANTIZED_NODES


def _ok(gpu):
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


def _geometry(gpu, case, bits=0, method=grt.GRT_BUILD_PREFER_FAST):
    dev = {k: device_tensor(v) for k, v in case.items()}
    return Geometry(gpu, morton_bits=bits, build_flags=method | Q, **dev).build()


def _oracle_ref(case, bits, method):
    lo, hi, cen = _oracle_for(case)
    b = 10 if bits == 30 else 21
    if method == grt.GRT_BUILD_CLUSTER_SUBTREES:
        return oracle.subtree_cluster(lo, hi, cen, b, grt.CLUSTER_CAP)
    if method == grt.GRT_BUILD_PREFER_BALANCED:
        return oracle.ploc(lo, hi, cen, b, 8)
    return oracle.lbvh(lo, hi, cen, b)


def check_quant(info, ref):
    """The quantised nodes the traversal reads equal the oracle's quantisation of its own
    4-wide nodes, word for word."""
    assert info.quantNodes, "no quantised nodes"
    want = oracle.quantized_wide_nodes(*oracle.wide_nodes(ref))
    m = info.nodeCount
    assert want.shape[0] == m
    got = read_device(info.quantNodes, m * 64, np.uint32).reshape(m, 16)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {m} nodes differ, first {bad[:5]}: {got[bad[0]]} vs {want[bad[0]]}"


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "spheres", "dupes", "dupes_small", "n1", "n2", "n3",
                                  "n17", "n2048", "n2049", "n4097"])
@pytest.mark.parametrize("bits", [30, 63])
def test_quantized_nodes_match_oracle_bit_exact(gpu, name, bits):
    case = _case(name)
    g = _geometry(gpu, case, bits)
    torch.cuda.synchronize()
    info = g.info()
    ref = _oracle_ref(case, bits, grt.GRT_BUILD_PREFER_FAST)
    check_tree(info, ref, case)  # the rest of the build is unchanged by the flag
    check_quant(info, ref)
    _ok(gpu)
    g.close()


@pytest.mark.parametrize("method", [grt.GRT_BUILD_PREFER_BALANCED, grt.GRT_BUILD_CLUSTER_SUBTREES])
@pytest.mark.parametrize("name", ["terrain", "spheres", "n513"])
def test_quantized_nodes_of_clustering_builds(gpu, name, method):
    case = _case(name)
    g = _geometry(gpu, case, 30, method)
    torch.cuda.synchronize()
    info = g.info()
    check_quant(info, _oracle_ref(case, 30, method))
    _ok(gpu)
    g.close()


def test_quantized_nodes_after_refit(gpu):
    """UPDATE after the vertices moved writes the quantised nodes of the refitted tree,
    and traces through them find the oracle's hits on the moved mesh."""
    from test_gpu_build import check_refit_traces

    m = scenegen.terrain(cells=70, amplitude=0.2)
    case = dict(vertices=m.vertices.copy(), indices=m.indices)
    dv, di = device_tensor(case["vertices"]), device_tensor(m.indices)
    g = Geometry(gpu, vertices=dv, indices=di, build_flags=Q).build()
    ref = _oracle_ref(case, 30, grt.GRT_BUILD_PREFER_FAST)
    rng = np.random.default_rng(8)
    moved = (case["vertices"] + rng.normal(0, 0.01, case["vertices"].shape)).astype(np.float32)
    dv.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    case_m = dict(vertices=moved, indices=m.indices)
    check_quant(g.info(), refit_reference(ref, case_m))
    check_refit_traces(gpu, g, case_m, seed=12)
    _ok(gpu)
    g.close()


def test_traces_through_quantized_nodes(gpu):
    """Closest and any hit through quantised nodes against the oracle's hits: a million-
    sphere-style AABB list (random rays, tmax infinite and short), and a two-level scene
    whose instances alternate between a quantised and a 128-byte copy of one terrain
    (per-level node format inside one walk); the scene's hits also agree with the same
    scene over 128-byte nodes only, up to equal-t ties."""
    s = scenegen.spheres(40_000, half=20.0, rmin=0.01, rmax=0.6, config=95)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s)), build_flags=Q).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    rays = scenegen.random_rays(60_000, [-20] * 3, [20] * 3, config=96)
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

    from test_gpu_trace import _aimed

    mesh = scenegen.terrain(cells=48, amplitude=0.2)
    v, i = device_tensor(mesh.vertices), device_tensor(mesh.indices)
    gq = Geometry(gpu, vertices=v, indices=i, build_flags=Q).build()
    gw = Geometry(gpu, vertices=v, indices=i).build()
    fr = scenegen.random_frames(12, config=97)
    handles = [gq.handle if k % 2 == 0 else gw.handle for k in range(12)]
    sc = Scene(gpu, handles, device_tensor(fr.packed())).build()
    sw = Scene(gpu, [gw.handle] * 12, device_tensor(fr.packed())).build()
    T = oracle.Scene()
    gi = T.add_mesh(mesh.vertices, mesh.indices)
    for k in range(12):
        T.add_instance(gi, fr.packed()[k])
    T.build()
    rays = _aimed(60_000, fr.translation.astype(np.float64), 98)
    rays[::3, 7] = 5.0
    ref = T.trace(rays)
    n = rays.shape[0]
    hc, ha, hw = new_hits(n), new_hits(n), new_hits(n)
    dr = device_tensor(rays)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, dr, n, hc)
    grt.grtTraceAnyHit(gpu.handle, sc.handle, None, dr, n, ha)
    grt.grtTraceClosest(gpu.handle, sw.handle, None, dr, n, hw)
    torch.cuda.synchronize()
    got = hits_to_numpy(hc)
    rep = compare_closest(got, ref, T, rays, extent=25.0)
    rep.check()
    assert rep.matched > 15_000
    compare_any(hits_to_numpy(ha)[1], ref, T, rays, extent=25.0).check()
    wide = hits_to_numpy(hw)
    same = (got[0] == wide[0]) & (got[1] == wide[1])
    assert (~same).sum() <= max(3, 1e-4 * n)
    for k in (2, 3, 4):  # the FP64-refined t, u, v of the same hit are identical
        assert np.array_equal(got[k][same].view(np.uint32), wide[k][same].view(np.uint32))
    _ok(gpu)


def test_batched_launch_with_quantized_geometries(gpu):
    """The batched launch builds quantised geometries (one-block scenes and phased ones,
    30- and 63-bit codes, linear BVH and subtree clustering) exactly as grtBuildGeometry
    does, quantised nodes included, and its hit records equal the per-scene traces."""
    from test_gpu_batch import _assert_identical, _run, _workload

    work = _workload(16, nmax=120_000, rmax=20_000)
    flags = lambda k: Q | (grt.GRT_BUILD_CLUSTER_SUBTREES if k % 4 == 1 else 0)
    B, batched, single = _run(gpu, work, grt.batch_options(), morton_bits=lambda k: 63 if k % 5 == 3 else 0,
                              build_flags=flags)
    _assert_identical(batched, single)
    for (gb, _, _), (gs, _) in zip(batched, single):
        i1, i2 = gb.info(), gs.info()
        m = i1.nodeCount
        assert i1.quantNodes and i2.quantNodes
        assert np.array_equal(read_device(i1.quantNodes, m * 64, np.uint32),
                              read_device(i2.quantNodes, m * 64, np.uint32))
    # one soup against the oracle's quantisation of its own tree
    s, _ = work[0]
    lo, hi, cen = oracle.triangle_aabbs(s.mesh.vertices, s.mesh.indices)
    info = batched[0][0].info()
    check_quant(info, oracle.lbvh(lo, hi, cen, 10 if info.mortonBits == 30 else 21))
    B.close()


def test_device_target_and_flag_validation(gpu):
    m = scenegen.icosphere(2)
    v, i = device_tensor(m.vertices), device_tensor(m.indices)
    gq = Geometry(gpu, vertices=v, indices=i, build_flags=Q).build()
    gw = Geometry(gpu, vertices=v, indices=i).build()
    tq = grt.grtGetDeviceTarget(gpu.handle, geom=gq.handle)
    tw = grt.grtGetDeviceTarget(gpu.handle, geom=gw.handle)
    assert tq.nodeFormat == 1 and tq.nodes == gq.info().quantNodes
    assert tw.nodeFormat == 0 and tw.nodes == gw.info().wideNodes and not gw.info().quantNodes
    # a build of either geometry with the other's flag is rejected
    with pytest.raises(grt.GrtError):
        grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, gq.input, grt.build_options(), gq.temp, None,
                             gq.handle)
    with pytest.raises(grt.GrtError):
        grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, gw.input, grt.build_options(flags=Q), gw.temp,
                             None, gw.handle)
    with pytest.raises(grt.GrtError):  # an unknown method bit
        Geometry(gpu, vertices=v, indices=i, build_flags=Q | 4)
    # an empty quantised geometry builds and traces to misses
    ge = Geometry(gpu, vertices=v, indices=device_tensor(np.zeros((0, 3), np.uint32)), build_flags=Q).build()
    rays = device_tensor(scenegen.random_rays(64, [-1] * 3, [1] * 3, config=3))
    h = new_hits(64)
    grt.grtTraceClosest(gpu.handle, None, ge.handle, rays, 64, h)
    torch.cuda.synchronize()
    assert (hits_to_numpy(h)[1] == oracle.NONE).all()
    _ok(gpu)
