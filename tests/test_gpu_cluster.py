"""GPU clustering inside the linear BVH's subtrees (GRT_BUILD_CLUSTER_SUBTREES) vs the
oracle (oracle.subtree_cluster): topology, numbering, parent links, boxes, 4-wide nodes
and leaves bit for bit on inputs that exercise one- and two-leaf lists, equal Morton
codes, zero extent, 63-bit codes and hundreds of thousands of primitives across many
blocks; traces over the clustered trees against the oracle's hits; refit and replayed
builds after the vertices moved."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import FuncTable, Geometry, Scene, device_tensor, hits_to_numpy, new_hits
from parity import compare_any, compare_closest
from test_gpu_build import _case, check_bit_exact, check_refit_traces, check_tree, refit_reference

pytestmark = pytest.mark.gpu

FLAG = grt.GRT_BUILD_CLUSTER_SUBTREES


def _geometry(gpu, case, bits):
    dev = {k: device_tensor(v) for k, v in case.items()}
    return Geometry(gpu, morton_bits=bits, build_flags=FLAG, **dev).build()


def _ok(gpu):
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


@pytest.mark.parametrize("name", ["icosphere", "terrain", "flat", "spheres", "dupes", "dupes_small", "n2", "n3",
                                  "n17", "n513", "n4097"])
@pytest.mark.parametrize("bits", [30, 63])
def test_subtree_clustering_matches_oracle_bit_exact(gpu, name, bits):
    case = _case(name)
    g = _geometry(gpu, case, bits)
    check_bit_exact(g, case, bits, subtree=True)
    _ok(gpu)
    g.close()


def test_subtree_clustering_large_inputs(gpu):
    """The 131,072-triangle terrain and a 300,000-triangle clustered soup (many blocks,
    deep LBVH subtrees), and 5,000 identical boxes (every distance ties)."""
    m = scenegen.terrain(cells=256, amplitude=0.2)
    soup = scenegen.soup_scene(5, seed=3, nmin=300_000, nmax=300_000).mesh
    for case in (dict(vertices=m.vertices, indices=m.indices), dict(vertices=soup.vertices, indices=soup.indices),
                 dict(boxes=np.tile(np.array([[0, 0, 0, 1, 1, 1]], np.float32), (5000, 1)))):
        g = _geometry(gpu, case, 30)
        check_bit_exact(g, case, 30, subtree=True)
        _ok(gpu)
        g.close()


def test_traces_over_clustered_trees(gpu):
    """Closest and any hit through clustered bottom levels, one level (spheres) and two
    levels (terrain instances), against the oracle's hits."""
    s = scenegen.spheres(20_000, half=10.0, rmin=0.01, rmax=0.5, config=85)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s)), build_flags=FLAG).build()
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
    from test_gpu_trace import _aimed

    mesh = scenegen.terrain(cells=40, amplitude=0.2)
    gt = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices),
                  build_flags=FLAG).build()
    fr = scenegen.random_frames(10, config=89)
    sc = Scene(gpu, [gt.handle] * 10, device_tensor(fr.packed())).build()
    T = oracle.Scene()
    gi = T.add_mesh(mesh.vertices, mesh.indices)
    for k in range(10):
        T.add_instance(gi, fr.packed()[k])
    T.build()
    rays = _aimed(40_000, fr.translation.astype(np.float64), 93)
    rays[::3, 7] = 6.0
    ref = T.trace(rays)
    hits, anyh = new_hits(n), new_hits(n)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, device_tensor(rays), n, hits)
    grt.grtTraceAnyHit(gpu.handle, sc.handle, None, device_tensor(rays), n, anyh)
    torch.cuda.synchronize()
    rep = compare_closest(hits_to_numpy(hits), ref, T, rays, extent=25.0)
    rep.check()
    assert rep.matched > 10_000
    compare_any(hits_to_numpy(anyh)[1], ref, T, rays, extent=25.0).check()
    _ok(gpu)


def test_refit_and_replayed_builds(gpu):
    """UPDATE keeps the clustered topology and refits every box; a second BUILD replays
    the captured launches and follows moved vertices to the new clustering."""
    m = scenegen.terrain(cells=48, amplitude=0.2)
    v = device_tensor(m.vertices)
    g = Geometry(gpu, vertices=v, indices=device_tensor(m.indices), morton_bits=30, build_flags=FLAG).build()
    check_bit_exact(g, dict(vertices=m.vertices, indices=m.indices), 30, subtree=True)
    moved = m.vertices.copy()
    moved[:, 1] *= 2.5
    v.copy_(torch.from_numpy(moved))
    g.build(op=grt.GRT_BUILD_OPERATION_UPDATE)
    torch.cuda.synchronize()
    lo, hi, cen = oracle.triangle_aabbs(m.vertices, m.indices)
    ref = oracle.subtree_cluster(lo, hi, cen, 10, grt.CLUSTER_CAP)
    case = dict(vertices=moved, indices=m.indices)
    check_tree(g.info(), refit_reference(ref, case), case)
    check_refit_traces(gpu, g, case, seed=49)
    g.build()  # a fresh build of the moved vertices (replayed graph)
    check_bit_exact(g, case, 30, subtree=True)
    moved2 = m.vertices.copy()
    moved2[:, 0] = -moved2[:, 0]
    v.copy_(torch.from_numpy(moved2))
    g.build()
    check_bit_exact(g, dict(vertices=moved2, indices=m.indices), 30, subtree=True)
    _ok(gpu)
    g.close()
