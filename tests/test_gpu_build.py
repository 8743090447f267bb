"""GPU LBVH build vs the oracle: Morton codes, sort order, topology, parent links,
boxes and leaf records must be bit-exact (CUDA path called through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import Geometry, device_tensor, empty_bytes, read_device

pytestmark = pytest.mark.gpu

LEAF = 0x80000000


def _read(ptr: int, nbytes: int, dtype) -> np.ndarray:
    return read_device(ptr, nbytes, dtype)


def _tensor_bytes(t: torch.Tensor, offset: int, nbytes: int, dtype) -> np.ndarray:
    return t[offset:offset + nbytes].cpu().numpy().view(dtype).copy()


def _case(name):
    if name == "icosphere":
        m = scenegen.icosphere(3)
        return dict(vertices=m.vertices, indices=m.indices)
    if name == "terrain":
        m = scenegen.terrain(cells=90, amplitude=0.2)
        return dict(vertices=m.vertices, indices=m.indices)
    if name == "flat":  # many identical y, exercises zero extent
        m = scenegen.terrain(cells=40, amplitude=0.0)
        return dict(vertices=m.vertices, indices=m.indices)
    if name == "spheres":
        s = scenegen.spheres(50_003, half=20.0, config=91)
        return dict(boxes=scenegen.sphere_aabbs(s))
    if name in ("dupes", "dupes_small"):  # many primitives sharing one centroid -> equal Morton codes
        rng = np.random.default_rng(4)
        c = rng.integers(0, 4, (9000 if name == "dupes" else 3000, 3)).astype(np.float32)
        b = np.concatenate([c - 0.25, c + 0.25], axis=1).astype(np.float32)
        return dict(boxes=b)
    if name.startswith("n"):
        n = int(name[1:])
        rng = np.random.default_rng(n)
        c = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
        return dict(boxes=np.concatenate([c - 0.1, c + 0.1], axis=1).astype(np.float32))
    raise KeyError(name)


def _oracle_for(case):
    if "boxes" in case:
        b = case["boxes"]
        lo, hi = b[:, :3].copy(), b[:, 3:].copy()
        c = oracle.box_centroids(b)
    else:
        lo, hi, c = oracle.triangle_aabbs(case["vertices"], case["indices"])
    return lo, hi, c


def check_wide(info, ref):
    """The 4-wide nodes the traversal reads equal the oracle's collapse of its own binary
    LBVH (oracle.wide_nodes), bit for bit: slot boxes and child words."""
    lo, hi, child = oracle.wide_nodes(ref)
    m = info.nodeCount
    assert lo.shape[0] == m
    w = _read(info.wideNodes, m * 128, np.float32).reshape(m, 32)
    assert np.array_equal(w[:, 24:28].view(np.uint32), child), "wide children"
    assert np.array_equal(np.stack([w[:, 0:4], w[:, 8:12], w[:, 16:20]], axis=2), lo), "wide lo"
    assert np.array_equal(np.stack([w[:, 4:8], w[:, 12:16], w[:, 20:24]], axis=2), hi), "wide hi"


def check_bit_exact(g, case, bits, radius: int = 0, subtree: bool = False, split=None):
    """The built geometry `g` of `case` equals the oracle's build bit for bit (the LBVH,
    with radius > 0 the clustering build of that search radius, with subtree the
    clustering inside the LBVH's subtrees): sorted Morton codes and order (from the build
    temporary), topology, child boxes, parent links and leaf records. With `split` (the
    oracle's split_triangles result) the build runs over its references."""
    torch.cuda.synchronize()
    info = g.info()
    n = info.leafCount
    if split is None:
        lo, hi, cen = _oracle_for(case)
    else:
        lo, hi = split[0], split[1]
        cen = oracle.box_centroids(np.concatenate([lo, hi], axis=1))
    if subtree:
        ref = oracle.subtree_cluster(lo, hi, cen, 10 if bits == 30 else 21, grt.CLUSTER_CAP)
    elif radius:
        ref = oracle.ploc(lo, hi, cen, 10 if bits == 30 else 21, radius)
    else:
        ref = oracle.lbvh(lo, hi, cen, 10 if bits == 30 else 21)
    assert info.mortonBits == bits
    koff, voff, boff = grt.grtGetBuildTemporaryLayout(n, bits)
    kdt = np.uint32 if bits == 30 else np.uint64
    keys = _tensor_bytes(g.temp, koff, n * (4 if bits == 30 else 8), kdt)
    order = _tensor_bytes(g.temp, voff, n * 4, np.uint32)
    assert np.array_equal(keys.astype(np.uint64), ref["sorted_codes"]), "Morton codes / sort"
    assert np.array_equal(order, ref["order"]), "stable sort order"
    check_tree(info, ref, case, None if split is None else split[2])


def check_tree(info, ref, case, prim_of=None):
    """The geometry's binary nodes (both child boxes and child words), parent links,
    4-wide nodes and leaf records equal those of the oracle build `ref` of `case`, bit
    for bit. Triangle leaves hold the sorted triangles' vertices, the primitive ID and
    the L1 norms |v1 - v0|_1 and |v2 - v0|_1 (summed x, y, z in float32). prim_of maps
    the build's items to triangles (split references), identity by default."""
    n = info.leafCount
    lo, hi = ref["leaf_lo"], ref["leaf_hi"]
    nodes = _read(info.nodes, info.nodeCount * 64, np.float32).reshape(-1, 16)
    children = nodes.view(np.uint32)[:, 12:14]
    check_wide(info, ref)
    if n == 1:
        assert children.tolist() == [[LEAF, LEAF]]
        assert np.array_equal(nodes[0, [0, 4, 8]], lo[0]) and np.array_equal(nodes[0, [1, 5, 9]], hi[0])
    else:
        cl = ref["childL"].view(np.uint32)
        cr = ref["childR"].view(np.uint32)
        assert np.array_equal(children[:, 0], cl) and np.array_equal(children[:, 1], cr), "topology"

        def child_box(c):
            c = np.asarray(c, np.uint32)
            leaf = (c & LEAF) != 0
            idx = (c & 0x7FFFFFFF).astype(np.int64)
            blo = np.where(leaf[:, None], lo[np.minimum(idx, n - 1)], ref["node_lo"][np.minimum(idx, n - 2)])
            bhi = np.where(leaf[:, None], hi[np.minimum(idx, n - 1)], ref["node_hi"][np.minimum(idx, n - 2)])
            return blo, bhi

        l0, h0 = child_box(cl)
        l1, h1 = child_box(cr)
        # node rows: x = (c0.lo, c0.hi, c1.lo, c1.hi) at 0..3, y at 4..7, z at 8..11
        assert np.array_equal(nodes[:, [0, 4, 8]], l0) and np.array_equal(nodes[:, [1, 5, 9]], h0), "left boxes"
        assert np.array_equal(nodes[:, [2, 6, 10]], l1) and np.array_equal(nodes[:, [3, 7, 11]], h1), "right boxes"
        # parent links: (parent << 1 | side), root marked invalid
        par = _read(info.parents, (2 * n - 1) * 4, np.uint32)
        assert par[0] == 0xFFFFFFFF
        k = np.arange(n - 1, dtype=np.uint64)
        for side, c in enumerate((cl, cr)):
            c = c.astype(np.uint64)
            slot = np.where(c & LEAF, n - 1 + (c & 0x7FFFFFFF), c).astype(np.int64)
            assert np.array_equal(par[slot].astype(np.uint64), (k << 1) | side), "parent links"
    if "indices" in case:
        rec = _read(info.leaves, n * 48, np.float32).reshape(n, 12)
        prim = rec[:, 3].view(np.uint32)
        tri = ref["order"] if prim_of is None else prim_of[ref["order"]]
        assert np.array_equal(prim, tri)
        v = case["vertices"][case["indices"][tri]]  # (n,3,3)
        assert np.array_equal(rec[:, 0:3], v[:, 0]) and np.array_equal(rec[:, 4:7], v[:, 1])
        assert np.array_equal(rec[:, 8:11], v[:, 2])
        for j, col in ((1, 7), (2, 11)):
            d = np.abs(v[:, j] - v[:, 0])
            assert np.array_equal(rec[:, col], (d[:, 0] + d[:, 1]) + d[:, 2]), "leaf edge norms"
    else:
        ids = _read(info.leaves, n * 4, np.uint32)
        assert np.array_equal(ids, ref["order"])


def refit_reference(ref, case):
    """The oracle build `ref` with its topology and order kept and every box fitted again
    over the primitives of `case` (the moved vertices or boxes)."""
    lo, hi, _ = _oracle_for(case)
    slo = np.ascontiguousarray(lo[ref["order"]])
    shi = np.ascontiguousarray(hi[ref["order"]])
    nlo, nhi = oracle.fit(ref["childL"], ref["childR"], slo, shi)
    return dict(ref, leaf_lo=slo, leaf_hi=shi, node_lo=nlo, node_hi=nhi)


def check_refit_traces(gpu, g, case, seed):
    """Closest hits traced through the refitted geometry equal the oracle's hits on the
    moved primitives (rays from above the terrain's box, aimed down at it)."""
    from paper_2603_00292_gb300.objects import hits_to_numpy, new_hits
    from parity import compare_closest

    v = case["vertices"]
    lo, hi = v.min(axis=0).astype(np.float64), v.max(axis=0).astype(np.float64)
    rng = np.random.default_rng(seed)
    n = 20_000
    org = np.stack([rng.uniform(lo[0], hi[0], n), np.full(n, hi[1] + 1.0), rng.uniform(lo[2], hi[2], n)], axis=1)
    tgt = np.stack([rng.uniform(lo[0], hi[0], n), rng.uniform(lo[1], hi[1], n), rng.uniform(lo[2], hi[2], n)], axis=1)
    d = tgt - org
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3], rays[:, 4:7], rays[:, 7] = org, d, np.inf
    S = oracle.Scene()
    S.add_instance(S.add_mesh(v, case["indices"]))
    S.build()
    ref = S.trace(rays)
    hits = new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, g.handle, device_tensor(rays), n, hits)
    torch.cuda.synchronize()
    rep = compare_closest(hits_to_numpy(hits), ref, S, rays, extent=float(np.max(hi - lo)))
    rep.check()
    assert rep.matched > n // 2, rep.summary()


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "spheres", "dupes", "dupes_small", "n1", "n2", "n3",
                                  "n17", "n513", "n1025", "n2048", "n2049", "n4096", "n4097"])
@pytest.mark.parametrize("bits", [30, 63])
def test_build_matches_oracle_bit_exact(gpu, name, bits):
    case = _case(name)
    dev = {k: device_tensor(v) for k, v in case.items()}
    g = Geometry(gpu, morton_bits=bits, **dev).build()
    check_bit_exact(g, case, bits)
    g.close()


def test_rebuild_is_deterministic(gpu):
    case = _case("spheres")
    b = device_tensor(case["boxes"])
    g1 = Geometry(gpu, boxes=b, morton_bits=30).build()
    g2 = Geometry(gpu, boxes=b, morton_bits=30).build()
    torch.cuda.synchronize()
    i1, i2 = g1.info(), g2.info()
    a = _read(i1.nodes, i1.nodeCount * 64, np.uint8)
    c = _read(i2.nodes, i2.nodeCount * 64, np.uint8)
    assert np.array_equal(a, c)


@pytest.mark.parametrize("cells", [32, 80])
def test_refit_after_moving_vertices(gpu, cells):
    """UPDATE keeps the topology and fits every box again from the moved vertices: both
    child boxes of every binary node, the parent links, the triangle leaves (moved
    vertices and edge norms) and the 4-wide nodes equal the oracle's fit of the kept
    tree, bit for bit; closest hits traced afterwards equal the oracle's on the moved
    mesh. 32 cells (2,048 triangles) stay under the one-block build size, 80 cells
    (12,800) take the grid launches."""
    m = scenegen.terrain(cells=cells, amplitude=0.2)
    v = device_tensor(m.vertices)
    g = Geometry(gpu, vertices=v, indices=device_tensor(m.indices), morton_bits=30).build()
    moved = m.vertices.copy()
    moved[:, 1] *= 3.0
    moved[:, 0] += 0.01 * np.sin(np.arange(len(moved)))
    v.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    lo, hi, cen = oracle.triangle_aabbs(m.vertices, m.indices)
    ref = oracle.lbvh(lo, hi, cen, 10)  # the topology of the first build
    case = dict(vertices=moved, indices=m.indices)
    check_tree(g.info(), refit_reference(ref, case), case)
    check_refit_traces(gpu, g, case, seed=cells)
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    g.close()


def test_refit_of_aabb_list(gpu):
    """UPDATE of an AABB-list geometry after its boxes moved: node boxes and 4-wide nodes
    against the oracle's fit of the kept tree."""
    case = _case("n4097")
    b = device_tensor(case["boxes"])
    g = Geometry(gpu, boxes=b, morton_bits=30).build()
    rng = np.random.default_rng(5)
    moved = case["boxes"] + np.repeat(rng.uniform(-0.3, 0.3, (case["boxes"].shape[0], 3)), 2, axis=0).reshape(-1, 6)
    moved = moved.astype(np.float32)
    b.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    lo, hi, cen = _oracle_for(case)
    ref = oracle.lbvh(lo, hi, cen, 10)
    moved_case = dict(boxes=moved)
    check_tree(g.info(), refit_reference(ref, moved_case), moved_case)
    g.close()


@pytest.mark.parametrize("n", [0, 1, 5, 4096, 4097, 100_003, 1_000_003])
@pytest.mark.parametrize("key_bits", [32, 64])
def test_radix_sort_is_stable(gpu, n, key_bits):
    rng = np.random.default_rng(n + key_bits)
    hi = 1 << (20 if n > 1000 else 3)
    keys = rng.integers(0, hi, n, dtype=np.uint64)
    if key_bits == 64:
        keys = keys | (rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(60))
    kd = np.uint32 if key_bits == 32 else np.uint64
    k = device_tensor(keys.astype(kd).view(np.int32 if key_bits == 32 else np.int64))
    v = device_tensor(np.arange(n, dtype=np.int32))
    temp = empty_bytes(grt.grtSortTemporaryBufferSize(n, key_bits))
    grt.grtSortPairs(gpu.handle, k, v, n, key_bits, 62 if key_bits == 64 else 32, temp)
    torch.cuda.synchronize()
    order = np.argsort(keys.astype(kd), kind="stable")
    assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))
    assert np.array_equal(k.cpu().numpy().view(kd), keys.astype(kd)[order])
