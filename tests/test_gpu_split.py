"""GPU spatial splits of triangles (GRT_BUILD_SPLIT_TRIANGLES; the paper's high-quality
option, Sec. 8) vs the oracle: the references (boxes, triangles, owners) and the whole
build over them (Morton codes, sort, topology, boxes, parent links, leaf records, 4-wide,
8-wide and quantised nodes) bit-exact for the linear BVH and both clustering builds;
closest and any hits through split geometries, one level and instanced, vs the oracle's
hits on the unsplit mesh; primitive-to-leaf map; rejections (UPDATE, all hits, AABB lists,
factors out of range). The batched launch with split geometries: tests/test_gpu_batch.py."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import Geometry, Scene, device_tensor, hits_to_numpy, new_hits, read_device
from parity import check_any_hit_records, compare_any, compare_closest
from test_gpu_build import _read, check_bit_exact

pytestmark = pytest.mark.gpu

SPLIT = grt.GRT_BUILD_SPLIT_TRIANGLES
METHODS = {"lbvh": (grt.GRT_BUILD_PREFER_FAST, 0, False), "ploc8": (grt.GRT_BUILD_PREFER_BALANCED, 8, False),
           "subtree": (grt.GRT_BUILD_CLUSTER_SUBTREES, 0, True)}


def _ok(gpu):
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


def _soup(n, seed, big=0.4):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (n, 1, 3))
    size = np.exp(rng.uniform(np.log(1e-3), np.log(big), (n, 1, 1)))
    v = (c + size * rng.normal(size=(n, 3, 3))).astype(np.float32).reshape(-1, 3)
    return dict(vertices=v, indices=np.arange(3 * n, dtype=np.uint32).reshape(n, 3))


def _case(name):
    if name == "icosphere":
        m = scenegen.icosphere(3)
    elif name == "terrain":
        m = scenegen.terrain(cells=64, amplitude=0.2)
    elif name == "flat":  # zero extent on y, vertices on grid lines
        m = scenegen.terrain(cells=32, amplitude=0.0)
    elif name == "soup":
        return _soup(3000, 5)
    elif name == "soup_big":  # several sort tiles and split blocks
        return _soup(60_000, 6, big=0.2)
    elif name.startswith("tri"):
        return _soup(int(name[3:]), int(name[3:]) + 100, big=1.0)
    else:
        raise KeyError(name)
    return dict(vertices=m.vertices, indices=m.indices)


def _split_ref(case, factor):
    n = case["indices"].shape[0]
    return oracle.split_triangles(case["vertices"], case["indices"], oracle.split_budget(n, factor))


def _geometry(gpu, case, flags, factor=0.0):
    dev = {k: device_tensor(v) for k, v in case.items()}
    return Geometry(gpu, build_flags=flags | SPLIT, split_factor=factor, **dev).build()


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "soup", "tri1", "tri2", "tri17"])
@pytest.mark.parametrize("method", ["lbvh", "ploc8", "subtree"])
def test_split_build_matches_oracle_bit_exact(gpu, name, method):
    case = _case(name)
    flags, radius, subtree = METHODS[method]
    g = _geometry(gpu, case, flags)
    split = _split_ref(case, 0.0)
    info = g.info()
    assert info.leafCount == split[0].shape[0] == info.primCount + oracle.split_budget(info.primCount, 0.0)
    check_bit_exact(g, case, 30, radius, subtree, split=split)
    _ok(gpu)
    g.close()


@pytest.mark.parametrize("factor", [0.1, 1.0])
def test_split_factors_and_many_blocks(gpu, factor):
    """60,000 triangles: 235 blocks of the splitting launches, many sort tiles."""
    case = _case("soup_big")
    g = _geometry(gpu, case, grt.GRT_BUILD_PREFER_FAST, factor)
    check_bit_exact(g, case, 30, split=_split_ref(case, factor))
    _ok(gpu)
    g.close()


def test_split_primitive_to_leaf_map_names_the_owner(gpu):
    case = _case("soup")
    g = _geometry(gpu, case, grt.GRT_BUILD_PREFER_FAST)
    lo, hi, prim, owner, _ = _split_ref(case, 0.0)
    ref = oracle.lbvh(lo, hi, oracle.box_centroids(np.concatenate([lo, hi], axis=1)), 10)
    pos = np.empty_like(ref["order"])
    pos[ref["order"]] = np.arange(ref["order"].shape[0], dtype=pos.dtype)  # reference -> sorted leaf
    t = grt.grtGetDeviceTarget(gpu.handle, geom=g.handle)
    assert t.nodeFormat == 0x100 and t.primCount == case["indices"].shape[0]
    got = read_device(t.primToLeaf, 4 * t.primCount, np.uint32)
    assert np.array_equal(got, pos[np.flatnonzero(owner)])
    _ok(gpu)


def test_split_node_formats(gpu):
    """8-wide and quantised nodes of a split build equal the oracle's collapse and
    quantisation of its tree over the references."""
    from test_gpu_quant import check_quant
    from test_gpu_wide8 import check_wide8

    case = _case("soup")
    lo, hi, prim, owner, _ = _split_ref(case, 0.0)
    ref = oracle.lbvh(lo, hi, oracle.box_centroids(np.concatenate([lo, hi], axis=1)), 10)
    g8 = _geometry(gpu, case, grt.GRT_BUILD_WIDE8_NODES)
    torch.cuda.synchronize()
    check_wide8(g8.info(), ref)
    gq = _geometry(gpu, case, grt.GRT_BUILD_QUANTIZED_NODES)
    torch.cuda.synchronize()
    check_quant(gq.info(), ref)
    _ok(gpu)


def _trace(ctx, rays_np, scene=None, geom=None, any_hit=False):
    n = rays_np.shape[0]
    hits = new_hits(n)
    (grt.grtTraceAnyHit if any_hit else grt.grtTraceClosest)(ctx.handle, scene, geom, device_tensor(rays_np), n, hits,
                                                             None, None)
    torch.cuda.synchronize()
    return hits_to_numpy(hits)


@pytest.mark.parametrize("flags", [grt.GRT_BUILD_PREFER_FAST, grt.GRT_BUILD_PREFER_BALANCED,
                                   grt.GRT_BUILD_WIDE8_NODES, grt.GRT_BUILD_QUANTIZED_NODES])
def test_traces_through_split_geometry(gpu, flags):
    """Closest and any hits of rays through a split soup (every triangle met once per
    reference the ray reaches) equal the oracle's hits on the unsplit mesh."""
    case = _soup(20_000, 9, big=0.6)
    g = _geometry(gpu, case, flags, 1.0)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(case["vertices"], case["indices"]))
    S.build()
    rays = scenegen.random_rays(40_000, [-1.5] * 3, [1.5] * 3, config=93)
    rays[::3, 7] = 0.2
    ref = S.trace(rays)
    compare_closest(_trace(gpu, rays, geom=g.handle), ref, S, rays, extent=3.0).check()
    anyg = _trace(gpu, rays, geom=g.handle, any_hit=True)
    compare_any(anyg[1], ref, S, rays, extent=3.0).check()
    check_any_hit_records(anyg, S, rays, 3.0)
    _ok(gpu)


def test_traces_through_instances_of_a_split_geometry(gpu):
    """A two-level scene (4-wide and 8-wide top levels) over instances of split terrain and
    soup geometries under SRT frames vs the oracle's two-level hits."""
    from test_gpu_trace import _aimed

    soup = _soup(5000, 12, big=0.5)
    terr = scenegen.terrain(cells=48, amplitude=0.3)
    k = 10
    fr = scenegen.random_frames(k, config=94)
    T = oracle.Scene()
    gs = T.add_mesh(soup["vertices"], soup["indices"])
    gt = T.add_mesh(terr.vertices, terr.indices)
    for j in range(k):
        T.add_instance(gs if j % 2 else gt, fr.packed()[j])
    T.build()
    rays = _aimed(30_000, fr.translation.astype(np.float64), 95)
    rays[::4, 7] = 3.0
    ref = T.trace(rays)
    for w8 in (0, grt.GRT_BUILD_WIDE8_NODES):
        a = _geometry(gpu, soup, w8)
        b = _geometry(gpu, dict(vertices=terr.vertices, indices=terr.indices), w8)
        sc = Scene(gpu, [(a if j % 2 else b).handle for j in range(k)], device_tensor(fr.packed()),
                   build_flags=w8).build()
        compare_closest(_trace(gpu, rays, scene=sc.handle), ref, T, rays, extent=8.0).check()
        compare_any(_trace(gpu, rays, scene=sc.handle, any_hit=True)[1], ref, T, rays, extent=8.0).check()
        _ok(gpu)


def test_split_lowers_the_tree_cost(gpu):
    """Surface-area cost of the GPU trees (from their own node boxes) over a soup of long
    triangles: lower with the references than with whole triangles."""
    rng = np.random.default_rng(13)
    n = 20_000
    a = rng.uniform(-1, 1, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = np.stack([a, a + 0.5 * d, a + 0.5 * d + 0.01 * rng.normal(size=(n, 3))], 1).astype(np.float32).reshape(-1, 3)
    dev = dict(vertices=device_tensor(v), indices=device_tensor(np.arange(3 * n, dtype=np.uint32).reshape(n, 3)))
    costs = []
    for flags in (0, SPLIT):
        g = Geometry(gpu, build_flags=flags, split_factor=1.0 if flags else 0.0, **dev).build()
        torch.cuda.synchronize()
        info = g.info()
        nodes = _read(info.nodes, info.nodeCount * 64, np.float32).reshape(-1, 16)
        lo = np.minimum(nodes[:, [0, 4, 8]], nodes[:, [2, 6, 10]])
        hi = np.maximum(nodes[:, [1, 5, 9]], nodes[:, [3, 7, 11]])
        costs.append(oracle.sah_cost(lo, hi))
        g.close()
    assert costs[1] < 0.95 * costs[0], costs


def test_repeated_builds_and_new_vertices(gpu):
    """A second BUILD (a replay of the captured launch sequence) gives the same tree; new
    vertex data in the same buffer is split again."""
    case = _case("soup")
    dev = {k: device_tensor(v) for k, v in case.items()}
    g = Geometry(gpu, build_flags=SPLIT, **dev).build().build()
    check_bit_exact(g, case, 30, split=_split_ref(case, 0.0))
    moved = dict(case, vertices=(case["vertices"] * np.float32(1.5) + np.float32(0.25)).astype(np.float32))
    dev["vertices"].copy_(device_tensor(moved["vertices"]))
    g.build()
    check_bit_exact(g, moved, 30, split=_split_ref(moved, 0.0))
    _ok(gpu)


def test_split_rejections(gpu):
    case = _case("soup")
    v, i = device_tensor(case["vertices"]), device_tensor(case["indices"])
    g = Geometry(gpu, vertices=v, indices=i, build_flags=SPLIT).build()
    with pytest.raises(grt.GrtError) as e:  # refit of a split geometry
        g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    for factor in (-0.5, 1.5, float("nan")):
        with pytest.raises(grt.GrtError):
            Geometry(gpu, vertices=v, indices=i, build_flags=SPLIT, split_factor=factor)
    with pytest.raises(grt.GrtError):  # boxes cannot be split
        Geometry(gpu, boxes=device_tensor(np.array([[0, 0, 0, 1, 1, 1]], np.float32)), build_flags=SPLIT)
    for opts in (grt.build_options(), grt.build_options(flags=SPLIT, split_factor=0.25)):  # must repeat the creation's
        with pytest.raises(grt.GrtError):
            grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, g.input, opts, g.temp, None, g.handle)
    # the factor 0 of the creation is 0.5: naming it explicitly is the same build
    grt.grtBuildGeometry(gpu.handle, grt.GRT_BUILD_OPERATION_BUILD, g.input, grt.build_options(flags=SPLIT, split_factor=0.5),
                         g.temp, None, g.handle)
    rays = device_tensor(scenegen.random_rays(64, [-1] * 3, [1] * 3, config=96))
    with pytest.raises(grt.GrtError) as e:  # each triangle would be met once per reference
        grt.grtTraceAllHits(gpu.handle, None, g.handle, rays, 64, new_hits(64 * 4), 4,
                            torch.zeros(64, dtype=torch.int32, device="cuda"))
    assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    _ok(gpu)


def test_all_hits_skip_split_instances(gpu):
    """All hits through a scene with a split and an unsplit instance of the same mesh:
    the split one is skipped (GRT_ERROR_INVALID_PARAMETER latched), the other reported as
    by the oracle."""
    m = scenegen.icosphere(2)
    v, i = device_tensor(m.vertices), device_tensor(m.indices)
    gs = Geometry(gpu, vertices=v, indices=i, build_flags=SPLIT).build()
    gp = Geometry(gpu, vertices=v, indices=i).build()
    frames = np.array([[0, 0, 0, 1, 1, 1, 1, 0, 0, 0], [0, 0, 0, 1, 1, 1, 1, 5, 0, 0]], np.float32)
    sc = Scene(gpu, [gs.handle, gp.handle], device_tensor(frames)).build()
    rays = np.zeros((2, 8), np.float32)
    rays[:, 0], rays[:, 1], rays[:, 2], rays[:, 6], rays[:, 7] = 0.1, 0.13, 5.0, -1.0, np.inf  # off every vertex
    rays[1, 0] = 5.1
    hits = new_hits(2 * 8)
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    grt.grtTraceAllHits(gpu.handle, sc.handle, None, device_tensor(rays), 2, hits, 8, counts)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_ERROR_INVALID_PARAMETER
    c = counts.cpu().numpy()
    assert c[0] == 0 and c[1] == 2  # the sphere at x = 5 is entered and left
    got = hits_to_numpy(hits)
    assert np.all(got[0][8:10] == 1)
