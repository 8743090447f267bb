"""Pins for the oracle's ray queries and ray generation (CPU only).

Closed forms (analytic sphere, the flat plane y=0, exact pixel coverage of an
axis-aligned quad), the paper's plane/edge triangle test against Moller-Trumbore,
brute force against the oracle's own BVH, instancing identities, and the
cosine-weighted hemisphere's known moments."""
import math

import numpy as np
import pytest

import oracle
import scenegen

NONE = oracle.NONE


def _rays(o, d, tmin=0.0, tmax=np.inf):
    o = np.atleast_2d(np.asarray(o, np.float64))
    d = np.atleast_2d(np.asarray(d, np.float64))
    n = max(o.shape[0], d.shape[0])
    r = np.empty((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


# ---------------------------------------------------------------- triangle formulas
def test_mt_agrees_with_paper_plane_edge_form():
    rng = np.random.default_rng(3)
    agree = 0
    for _ in range(3000):
        tri = rng.uniform(-1, 1, 9).astype(np.float32)
        o = rng.uniform(-3, 3, 3)
        target = tri.reshape(3, 3).astype(np.float64).mean(0) + rng.normal(0, 0.4, 3)
        d = target - o
        ray = _rays(o, d / np.linalg.norm(d))[0]
        h1, t1, u1, v1 = oracle.mt_test(ray, tri)
        h2, t2, u2, v2 = oracle.plane_edge_test(ray, tri)
        if h1 != h2:
            # only allowed within rounding of an edge
            assert min(u2, v2, 1 - u2 - v2) > -1e-12 and min(u2, v2, 1 - u2 - v2) < 1e-12
            continue
        if h1:
            agree += 1
            assert abs(t1 - t2) <= 1e-12 * max(1.0, abs(t2))
            assert abs(u1 - u2) <= 1e-12 and abs(v1 - v2) <= 1e-12
    assert agree > 500


def test_triangle_is_double_sided_with_inclusive_edges():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    for dz in (-1.0, 1.0):
        h, t, u, v = oracle.mt_test(_rays([0.25, 0.25, -dz], [0, 0, dz])[0], tri)
        assert h and t == 1.0 and u == 0.25 and v == 0.25
    # exactly on a vertex and on an edge: still a hit (edges inclusive)
    assert oracle.mt_test(_rays([0, 0, 1], [0, 0, -1])[0], tri)[0]
    assert oracle.mt_test(_rays([0.5, 0.5, 1], [0, 0, -1])[0], tri)[0]
    assert not oracle.mt_test(_rays([0.5, 0.51, 1], [0, 0, -1])[0], tri)[0]
    # t range inclusive at both ends, exclusive outside
    assert oracle.mt_test(_rays([0.2, 0.2, 1], [0, 0, -1], 1.0, 1.0)[0], tri)[0]
    assert not oracle.mt_test(_rays([0.2, 0.2, 1], [0, 0, -1], 0.0, 0.999)[0], tri)[0]
    # parallel ray misses
    assert not oracle.mt_test(_rays([0.2, 0.2, 0], [1, 0, 0])[0], tri)[0]


# ---------------------------------------------------------------- closed forms
def test_sphere_closed_form():
    rng = np.random.default_rng(5)
    sph = np.array([[1.0, -2.0, 0.5, 0.75]], np.float32)
    S = oracle.Scene()
    S.add_instance(S.add_spheres(sph))
    c = sph[0, :3].astype(np.float64)
    r = float(sph[0, 3])
    o = rng.uniform(-5, 5, (2000, 3))
    d = scenegen.unit_vectors(11, 2000)
    rays = _rays(o, d)
    h = S.trace(rays, bvh=False)
    o32 = rays[:, :3].astype(np.float64)
    d32 = rays[:, 4:7].astype(np.float64)
    # perpendicular distance from the centre to the ray's line decides hit vs miss
    f = c - o32
    along = np.einsum("ij,ij->i", f, d32) / np.einsum("ij,ij->i", d32, d32)
    perp = np.linalg.norm(f - along[:, None] * d32, axis=1)
    inside = np.linalg.norm(f, axis=1) < r
    expect_hit = inside | ((perp < r) & (along > 0))
    margin = np.abs(perp - r) > 1e-9
    assert np.array_equal((h.prim != NONE)[margin], expect_hit[margin])
    hit = h.prim != NONE
    p = o32[hit] + h.t[hit, None] * d32[hit]
    assert np.allclose(np.linalg.norm(p - c, axis=1), r, rtol=0, atol=1e-9)
    # from outside the near root is taken, from inside the far one
    assert np.all((np.einsum("ij,ij->i", p - c, d32[hit]) <= 1e-9) == ~inside[hit])


def test_flat_terrain_is_the_plane_y0():
    mesh = scenegen.terrain(cells=16, amplitude=0.0)
    assert np.all(mesh.vertices[:, 1] == 0)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(mesh.vertices, mesh.indices))
    rng = np.random.default_rng(9)
    o = np.column_stack([rng.uniform(-0.9, 0.9, 3000), rng.uniform(0.5, 2, 3000), rng.uniform(-0.9, 0.9, 3000)])
    target = np.column_stack([rng.uniform(-0.95, 0.95, 3000), np.zeros(3000), rng.uniform(-0.95, 0.95, 3000)])
    d = target - o
    rays = _rays(o, d / np.linalg.norm(d, axis=1, keepdims=True))
    h = S.trace(rays, bvh=False)
    o32 = rays[:, :3].astype(np.float64)
    d32 = rays[:, 4:7].astype(np.float64)
    t = -o32[:, 1] / d32[:, 1]
    p = o32 + t[:, None] * d32
    assert np.all(h.prim != NONE)
    assert np.allclose(h.t, t, rtol=1e-12, atol=0)
    # the triangle: cell from floor(), then the side of the diagonal (i,j)-(i+1,j+1)
    gx = (p[:, 0] + 1) * 8
    gz = (p[:, 2] + 1) * 8
    i = np.floor(gx).astype(int)
    j = np.floor(gz).astype(int)
    fx, fz = gx - i, gz - j
    tri = 2 * (j * 16 + i) + (fz > fx).astype(int)
    clear = (np.abs(fx - fz) > 1e-9) & (np.minimum.reduce([fx, fz, 1 - fx, 1 - fz]) > 1e-9)
    assert np.array_equal(h.prim[clear].astype(int), tri[clear])


def test_quad_pixel_coverage_through_the_camera():
    W, H = 64, 48
    cam = scenegen.look_down_z_camera([0, 0, 3], W, H)
    rays = oracle.camera_rays(cam.packed(), W, H)
    z0 = 1.0
    dist = 3.0 - z0
    th = math.tan(math.radians(30))
    aspect = W / H
    # choose quad edges half-way between pixel centres so no centre lies on an edge
    def film_x(x):
        return (2 * (x + 0.5) / W - 1) * aspect * th

    def film_y(y):
        return (1 - 2 * (y + 0.5) / H) * th

    x0 = 0.5 * (film_x(10) + film_x(11)) * dist
    x1 = 0.5 * (film_x(40) + film_x(41)) * dist
    y1 = 0.5 * (film_y(5) + film_y(6)) * dist
    y0 = 0.5 * (film_y(30) + film_y(31)) * dist
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0]], np.float32)
    idx = np.array([[0, 1, 2], [0, 2, 3]], np.uint32)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(v, idx))
    h = S.trace(rays, bvh=False)
    got = (h.prim != NONE).reshape(H, W)
    want = np.zeros((H, W), bool)
    want[6:31, 11:41] = True
    assert np.array_equal(got, want)
    assert np.allclose(h.t[want.ravel()], dist / -rays[want.ravel(), 6].astype(np.float64), rtol=1e-12)


def test_icosphere_hits_lie_between_inradius_and_radius():
    mesh = scenegen.icosphere(3)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(mesh.vertices, mesh.indices))
    cam = scenegen.look_down_z_camera([0, 0, 3], 128, 128)
    rays = oracle.camera_rays(cam.packed(), 128, 128)
    h = S.trace(rays, bvh=False)
    hit = h.prim != NONE
    p = rays[hit, :3].astype(np.float64) + h.t[hit, None] * rays[hit, 4:7].astype(np.float64)
    r = np.linalg.norm(p, axis=1)
    v = mesh.vertices.astype(np.float64)
    i = mesh.indices
    n = np.cross(v[i[:, 1]] - v[i[:, 0]], v[i[:, 2]] - v[i[:, 0]])
    r_in = np.min(np.abs(np.einsum("ij,ij->i", n / np.linalg.norm(n, axis=1, keepdims=True), v[i[:, 0]])))
    assert r.min() >= r_in - 1e-7 and r.max() <= 1 + 1e-7
    # the centre pixel of an even image sees the sphere; a corner pixel does not
    assert hit.reshape(128, 128)[64, 64] and not hit.reshape(128, 128)[0, 0]


# ---------------------------------------------------------------- BVH vs brute force
def _aimed_rays(n, targets, seed):
    """Rays from random origins in [-12,12]^3 toward random points near `targets`."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(-12, 12, (n, 3))
    tgt = targets[rng.integers(0, len(targets), n)] + rng.normal(0, 0.8, (n, 3))
    d = tgt - o
    return _rays(o, d / np.linalg.norm(d, axis=1, keepdims=True))


def _small_instanced_scene():
    mesh = scenegen.terrain(cells=24, amplitude=0.2)
    fr = scenegen.random_frames(6, config=99)
    S = oracle.Scene()
    g = S.add_mesh(mesh.vertices, mesh.indices)
    for k in range(6):
        S.add_instance(g, fr.packed()[k])
    return S, mesh, fr


@pytest.mark.parametrize("any_hit", [False, True])
def test_bvh_equals_brute_force(any_hit):
    S, mesh, fr = _small_instanced_scene()
    sph = scenegen.spheres(500, half=8.0, config=98)
    S.add_instance(S.add_spheres(sph))
    S.build()
    rays = _aimed_rays(6000, fr.translation.astype(np.float64), 97)
    rays[:, 7] = np.where(np.arange(6000) % 2 == 0, np.inf, 4.0)
    a = S.trace(rays, any_hit=any_hit, bvh=False)
    b = S.trace(rays, any_hit=any_hit, bvh=True)
    assert np.array_equal(a.prim != NONE, b.prim != NONE)
    assert (a.prim != NONE).mean() > 0.1
    if not any_hit:
        assert np.array_equal(a.prim, b.prim) and np.array_equal(a.inst, b.inst)
        assert np.array_equal(a.t, b.t)


@pytest.mark.parametrize("bvh", [False, True])
def test_instance_masks_equal_a_scene_of_the_visible_instances(bvh):
    """Sec. 7.5: an instance takes part only when its mask ANDed with the ray mask is
    nonzero. So a masked trace equals a trace of a scene that holds only the visible
    instances (instance IDs mapped back), and a ray mask that no instance shares hits
    nothing."""
    S, mesh, fr = _small_instanced_scene()
    masks = [0x1, 0x2, 0x3, 0x4, 0x5, 0x8]
    for k, m in enumerate(masks):
        S.set_instance_mask(k, m)
    S.build()
    rays = _aimed_rays(5000, fr.translation.astype(np.float64), 95)
    for ray_mask in (0x1, 0x6, 0xFFFFFFFF):
        visible = [k for k, m in enumerate(masks) if m & ray_mask]
        V = oracle.Scene()
        g = V.add_mesh(mesh.vertices, mesh.indices)
        for k in visible:
            V.add_instance(g, fr.packed()[k])
        V.build()
        for any_hit in (False, True):
            a = S.trace(rays, any_hit=any_hit, bvh=bvh, ray_mask=ray_mask)
            b = V.trace(rays, any_hit=any_hit, bvh=bvh)
            assert np.array_equal(a.prim != NONE, b.prim != NONE)
            if not any_hit:
                hit = b.prim != NONE
                assert np.array_equal(a.inst[hit], np.asarray(visible, np.uint32)[b.inst[hit]])
                assert np.array_equal(a.prim, b.prim) and np.array_equal(a.t, b.t)
        assert (a.prim != NONE).mean() > 0.02
    none = S.trace(rays, bvh=bvh, ray_mask=0x10)
    assert (none.prim == NONE).all()


@pytest.mark.parametrize("bvh", [False, True])
def test_primitive_filter_equals_removing_the_rejected_primitives(bvh):
    """Sec. 7.6's intersection filter, as a primitive mask: tracing with hits on the
    masked-out primitives rejected equals tracing a geometry without those primitives
    (IDs mapped back), for triangles and for spheres."""
    rng = np.random.default_rng(94)
    mesh = scenegen.terrain(cells=24, amplitude=0.2)
    sph = scenegen.spheres(400, half=1.0, rmin=0.02, rmax=0.2, config=93)
    keep_t = rng.random(mesh.indices.shape[0]) < 0.6
    keep_s = rng.random(sph.shape[0]) < 0.5

    def bits(keep):
        w = np.zeros((keep.size + 31) // 32, np.uint32)
        for i in np.nonzero(keep)[0]:
            w[i >> 5] |= np.uint32(1) << np.uint32(i & 31)
        return w

    S = oracle.Scene()
    gt = S.add_mesh(mesh.vertices, mesh.indices)
    gs = S.add_spheres(sph)
    S.set_prim_filter(gt, bits(keep_t))
    S.set_prim_filter(gs, bits(keep_s))
    S.add_instance(gt)
    S.add_instance(gs, np.array([0, 0, 0, 1, 1, 1, 1, 0, 0.5, 0], np.float32))
    S.build()
    R = oracle.Scene()
    R.add_instance(R.add_mesh(mesh.vertices, mesh.indices[keep_t]))
    R.add_instance(R.add_spheres(sph[keep_s]), np.array([0, 0, 0, 1, 1, 1, 1, 0, 0.5, 0], np.float32))
    R.build()
    rays = _aimed_rays(5000, np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.0]]), 92)
    ids = [np.nonzero(keep_t)[0], np.nonzero(keep_s)[0]]
    for any_hit in (False, True):
        a = S.trace(rays, any_hit=any_hit, bvh=bvh)
        b = R.trace(rays, any_hit=any_hit, bvh=bvh)
        assert np.array_equal(a.prim != NONE, b.prim != NONE)
        if not any_hit:
            hit = b.prim != NONE
            mapped = np.array([ids[i][p] for i, p in zip(b.inst[hit], b.prim[hit])], np.uint32)
            assert np.array_equal(a.inst, b.inst) and np.array_equal(a.prim[hit], mapped)
            assert np.array_equal(a.t, b.t)
            assert hit.mean() > 0.05
    # a filtered primitive is no hit for the single-primitive query either
    rej = int(np.nonzero(~keep_t)[0][0])
    assert not S.intersect_prim(rays[0], 0, rej)[0]


def test_any_hit_equals_closest_within_max_t():
    S, mesh, fr = _small_instanced_scene()
    S.build()
    rays = _aimed_rays(4000, fr.translation.astype(np.float64), 96)
    c = S.trace(rays, any_hit=False)  # maxT = +inf
    rays[:, 7] = 14.0
    a = S.trace(rays, any_hit=True)
    assert np.array_equal(a.prim != NONE, c.t <= 14.0)
    assert 0.05 < (c.t <= 14.0).mean() < (c.prim != NONE).mean()


def test_instancing_matches_world_space_triangles():
    """Two levels: tracing object-space BLAS under SRT frames equals tracing the
    instanced triangles placed in world space (float64, computed independently)."""
    S, mesh, fr = _small_instanced_scene()
    R = scenegen.quat_to_matrix64(fr.rotation)
    world_v = []
    world_i = []
    for k in range(6):
        w = (mesh.vertices.astype(np.float64) * fr.scale[k].astype(np.float64)) @ R[k].T + fr.translation[k]
        world_v.append(w)
        world_i.append(mesh.indices.astype(np.int64) + k * mesh.vertices.shape[0])
    W = oracle.Scene()
    W.add_instance(W.add_mesh(np.concatenate(world_v).astype(np.float32), np.concatenate(world_i).astype(np.uint32)))
    rays = _aimed_rays(4000, fr.translation.astype(np.float64), 95)
    a = S.trace(rays, bvh=False)
    b = W.trace(rays, bvh=False)
    hit = a.prim != NONE
    assert hit.mean() > 0.05
    ntri = mesh.num_triangles
    same = (a.prim.astype(np.int64) + a.inst.astype(np.int64) * ntri == b.prim.astype(np.int64)) | ~hit
    # world vertices were rounded to float32, so only near-edge rays may differ
    assert same.mean() > 0.995
    both = hit & (b.prim != NONE) & same
    assert np.allclose(a.t[both], b.t[both], rtol=1e-5)


def test_identity_and_translation_frames():
    mesh = scenegen.icosphere(2)
    rays = scenegen.random_rays(3000, [-3, -3, -3], [3, 3, 3], config=94)
    D = oracle.Scene()
    D.add_instance(D.add_mesh(mesh.vertices, mesh.indices))
    I = oracle.Scene()
    I.add_instance(I.add_mesh(mesh.vertices, mesh.indices), np.array([0, 0, 0, 1, 1, 1, 1, 0, 0, 0], np.float32))
    a, b = D.trace(rays), I.trace(rays)
    assert np.array_equal(a.prim, b.prim) and np.array_equal(a.t, b.t)
    # translation by (1,2,3) equals shifting the ray origins by -(1,2,3) (exact in float32 here)
    T = oracle.Scene()
    T.add_instance(T.add_mesh(mesh.vertices, mesh.indices), np.array([0, 0, 0, 1, 1, 1, 1, 1, 2, 3], np.float32))
    shifted = rays.copy()
    shifted[:, 0:3] -= np.array([1, 2, 3], np.float32)
    c = T.trace(rays)
    d = D.trace(shifted)
    ok = np.abs(rays[:, 0:3] - np.round(rays[:, 0:3] * 1024) / 1024).max(axis=1) >= 0  # all rays
    assert np.array_equal(c.prim[ok], d.prim[ok])
    # uniform scale 2 with an unnormalised direction keeps t: the ray (o, d) against the
    # sphere scaled by 2 hits where (o/2, d/2) hits the unit-scale sphere, at the same t
    S2 = oracle.Scene()
    S2.add_instance(S2.add_mesh(mesh.vertices, mesh.indices), np.array([0, 0, 0, 1, 2, 2, 2, 0, 0, 0], np.float32))
    half = rays.copy()
    half[:, 0:3] *= 0.5
    half[:, 4:7] *= 0.5
    e, f = S2.trace(rays), D.trace(half)
    assert np.array_equal(e.prim, f.prim)
    hit = e.prim != NONE
    assert np.allclose(e.t[hit], f.t[hit], rtol=1e-12)


# ---------------------------------------------------------------- ray generation
def test_camera_closed_form():
    cam = scenegen.look_down_z_camera([0, 0, 3], 3, 3)
    rays = oracle.camera_rays(cam.packed(), 3, 3)
    # centre pixel of an odd image looks straight down -z
    assert np.allclose(rays[4, 4:7], [0, 0, -1], atol=1e-7)
    th = math.tan(math.radians(30))
    # top-left pixel centre u=v=1/6: film point (-(2/3) th, (2/3) th, -1)
    d = np.array([-(2 / 3) * th, (2 / 3) * th, -1.0])
    assert np.allclose(rays[0, 4:7], d / np.linalg.norm(d), atol=1e-7)
    assert np.all(rays[:, 3] == 0) and np.all(np.isinf(rays[:, 7]))
    assert np.allclose(rays[:, 0:3], [0, 0, 3])


def test_splitmix64_published_outputs(golden_dir):
    vals = [int(l, 16) for l in open(f"{golden_dir}/splitmix64_seed0.txt") if l.startswith("0x")]
    # xi keeps the top 24 bits of the generator's output at counters 0 and 1
    assert oracle.xi(0, 0, 0, 0) == (vals[0] >> 40) / 2.0 ** 24
    assert oracle.xi(0, 0, 0, 1) == (vals[1] >> 40) / 2.0 ** 24
    assert int(scenegen.u64(0, 2)[0]) == vals[0] and int(scenegen.u64(0, 2)[1]) == vals[1]


def test_cosine_hemisphere_moments():
    n = 20000
    xs = np.array([oracle.sample_hemisphere(a, b) for a, b in zip(scenegen.uniform(1, n), scenegen.uniform(2, n))])
    assert np.allclose(np.linalg.norm(xs, axis=1), 1, atol=1e-12)
    assert xs[:, 1].min() >= 0
    # cos-weighted: E[cos] = 2/3, E[cos^2] = 1/2, P(cos > 1/2) = 3/4
    assert abs(xs[:, 1].mean() - 2 / 3) < 0.01
    assert abs((xs[:, 1] ** 2).mean() - 0.5) < 0.01
    assert abs((xs[:, 1] > 0.5).mean() - 0.75) < 0.01
    assert np.allclose(oracle.sample_hemisphere(0.0, 0.0), [0, 1, 0])
    assert np.allclose(oracle.sample_hemisphere(0.25, 1.0), [0, 0, 1], atol=1e-15)


def test_ao_rays_on_the_flat_plane():
    mesh = scenegen.terrain(cells=8, amplitude=0.0)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(mesh.vertices, mesh.indices))
    prim = scenegen.random_rays(200, [-0.5, 1, -0.5], [0.5, 2, 0.5], config=93)
    prim[:, 4:7] = np.array([0.1, -1, 0.05], np.float32) / np.float32(np.linalg.norm([0.1, -1, 0.05]))
    h = S.trace(prim)
    assert np.all(h.prim != NONE)
    ao = oracle.ao_rays(S, prim, h, 8, 1234, 0.25)
    assert np.allclose(ao[:, 1], 1e-4, atol=1e-7)  # origin p + 1e-4 n with n = +y
    assert np.all(ao[:, 5] >= 0)  # hemisphere about +y
    assert np.allclose(np.linalg.norm(ao[:, 4:7].astype(np.float64), axis=1), 1, atol=1e-6)
    assert np.all(ao[:, 7] == np.float32(0.25)) and np.all(ao[:, 3] == 0)
    # the plane never occludes rays leaving it upward
    assert np.all(S.trace(ao, any_hit=True).prim == NONE)
    # seen from below, the normal flips to -y
    prim[:, 1] = -prim[:, 1]
    prim[:, 5] = -prim[:, 5]
    h = S.trace(prim)
    ao = oracle.ao_rays(S, prim, h, 4, 1234, 0.25)
    assert np.allclose(ao[:, 1], -1e-4, atol=1e-7) and np.all(ao[:, 5] <= 0)


# ---------------------------------------------------------------- all hits (Sec. 7.5)
@pytest.mark.parametrize("bvh", [False, True])
def test_all_hits_agree_with_closest_and_any_hit(bvh):
    S, mesh, fr = _small_instanced_scene()
    S.build()
    rays = _aimed_rays(3000, fr.translation.astype(np.float64), 91)
    rays[1::2, 7] = 9.0
    inst, prim, t, u, v, cnt = S.all_hits(rays, 16, bvh=bvh)
    c = S.trace(rays)
    a = S.trace(rays, any_hit=True)
    assert np.array_equal(cnt > 0, a.prim != NONE)
    hit = cnt > 0
    # the first hit in (t, instance, primitive) order is the closest hit (same tie rule)
    assert np.array_equal(inst[hit, 0], c.inst[hit]) and np.array_equal(prim[hit, 0], c.prim[hit])
    assert np.array_equal(t[hit, 0], c.t[hit])
    # sorted, within [minT, maxT], misses after the last hit
    k = np.minimum(cnt, 16)
    col = np.arange(16)[None, :]
    valid = col < k[:, None]
    assert np.all(np.diff(np.where(valid, t, 1e300), axis=1) >= 0)
    assert np.all(t[valid] <= np.repeat(rays[:, 7:8], 16, axis=1)[valid])
    assert np.all(prim[~valid] == NONE)
    assert (cnt >= 2).mean() > 0.01 and cnt.max() >= 3  # some rays cross several surfaces
    if bvh:
        b = S.all_hits(rays, 16, bvh=False)
        assert np.array_equal(b[5], cnt) and np.array_equal(b[1], prim) and np.array_equal(b[2], t)


def test_all_hits_through_a_closed_sphere_mesh():
    """A ray from outside through the centre of a closed convex mesh crosses it exactly
    twice (away from edges and vertices), once on each side of the centre."""
    mesh = scenegen.icosphere(3)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(mesh.vertices, mesh.indices))
    S.build()
    rng = np.random.default_rng(90)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = -5.0 * d
    rays = _rays(o, d)
    inst, prim, t, u, v, cnt = S.all_hits(rays, 8)
    clean = np.array([S.min_edge_margin(r) > 1e-6 for r in rays])
    assert clean.mean() > 0.9
    assert np.all(cnt[clean] == 2)
    assert np.all(t[clean, 0] < 5.0) and np.all(t[clean, 1] > 5.0)
    # the two crossings are at distance between the inradius and 1 from the centre
    assert np.all(np.abs(t[clean, :2] - 5.0) <= 1.0 + 1e-9)
    assert np.all(np.abs(t[clean, :2] - 5.0) >= 0.98)


# ---------------------------------------------------------------- comparator helpers
def _down_ray(x, y, z=1.0, tmax=np.inf):
    r = np.zeros(8, np.float32)
    r[0:3] = (x, y, z)
    r[4:7] = (0, 0, -1)
    r[7] = tmax
    return r


def test_min_edge_margin_closed_forms():
    """The right triangle (0,0,0), (1,0,0), (0,1,0) hit straight down at (x, y): the
    plane point's barycentrics are u = x, v = y, so the margin is |min(x, y, 1-x-y)|,
    inside or outside the triangle; a plane crossing beyond maxT does not count; an
    instance translation moves the triangle with it."""
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    S = oracle.Scene()
    g = S.add_mesh(tri, np.array([[0, 1, 2]], np.uint32))
    S.add_instance(g)
    assert S.min_edge_margin(_down_ray(0.25, 0.25)) == 0.25
    assert S.min_edge_margin(_down_ray(0.125, 0.5)) == 0.125
    assert S.min_edge_margin(_down_ray(0.5, 0.0)) == 0.0  # on the edge v = 0
    assert S.min_edge_margin(_down_ray(0.5, 0.5)) == 0.0  # on the hypotenuse
    assert S.min_edge_margin(_down_ray(0.0, 0.0)) == 0.0  # on a vertex
    assert abs(S.min_edge_margin(_down_ray(0.75, 0.5)) - 0.25) < 1e-15  # outside: 1-u-v = -0.25
    assert S.min_edge_margin(_down_ray(0.25, 0.25, tmax=0.5)) == np.inf  # plane at t = 1 > maxT
    T = oracle.Scene()
    T.add_instance(T.add_mesh(tri, np.array([[0, 1, 2]], np.uint32)), [0, 0, 0, 1, 1, 1, 1, 5, 0, 0])
    assert T.min_edge_margin(_down_ray(5.25, 0.125)) == 0.125
    assert T.min_edge_margin(_down_ray(5.5, 0.0)) == 0.0


def test_min_sphere_margin_closed_forms():
    """The unit sphere at the origin and a ray along +z at lateral offset b from (0, b, -5):
    the closest approach is at t = 5, the line's distance to the centre is b, and the
    margin is |1 - b^2| / (b^2 + 25 + 1). Tangent rays give 0; a sphere behind the origin
    does not count; under a uniform scale 2 the tangent offset is 2."""
    S = oracle.Scene()
    S.add_instance(S.add_spheres(np.array([[0, 0, 0, 1]], np.float32)))

    def ray(b, dz=1.0, scale=1.0):
        r = np.zeros(8, np.float32)
        r[0:3] = (0, b, -5 * scale)
        r[4:7] = (0, 0, dz)
        r[7] = np.inf
        return r

    assert S.min_sphere_margin(ray(1.0)) == 0.0
    assert abs(S.min_sphere_margin(ray(0.0)) - 1 / 26) < 1e-15
    assert abs(S.min_sphere_margin(ray(0.5)) - 0.75 / 26.25) < 1e-15
    assert abs(S.min_sphere_margin(ray(2.0)) - 3 / 30) < 1e-15  # a miss still has a margin
    assert S.min_sphere_margin(ray(0.0, dz=-1.0)) == np.inf  # the sphere lies behind
    T = oracle.Scene()
    T.add_instance(T.add_spheres(np.array([[0, 0, 0, 1]], np.float32)), [0, 0, 0, 1, 2, 2, 2, 0, 0, 0])
    assert T.min_sphere_margin(ray(2.0, scale=2.0)) == 0.0
    assert abs(T.min_sphere_margin(ray(0.0, scale=2.0)) - 1 / 26) < 1e-15


def test_ao_frame_of_a_tilted_triangle():
    """AO rays off the triangle v0 = (1,1,1), v1 = v0 + (3,0,4), v2 = v0 + (0,2,0), hit
    from the side its normal (-0.8, 0, 0.6) faces: tangent = (v1 - v0)/5 = (0.6, 0, 0.8),
    bitangent = n x tangent = (0, 1, 0), so a hemisphere sample (x, y, z) becomes the
    direction (0.6x - 0.8y, z, 0.8x + 0.6y); the origin is the hit point + 1e-4 n."""
    v0 = np.array([1, 1, 1], np.float64)
    tri = np.array([v0, v0 + [3, 0, 4], v0 + [0, 2, 0]], np.float32)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(tri, np.array([[0, 1, 2]], np.uint32)))
    n = np.array([-0.8, 0.0, 0.6])
    p = v0 + 0.25 * np.array([3, 0, 4]) + 0.25 * np.array([0, 2, 0])
    prim = np.zeros((1, 8), np.float32)
    prim[0, 0:3] = p + 2.0 * n
    prim[0, 4:7] = -n
    prim[0, 7] = np.inf
    h = S.trace(prim, bvh=False)
    assert h.prim[0] == 0 and abs(h.t[0] - 2.0) < 1e-6
    spp, seed = 6, 99
    ao = oracle.ao_rays(S, prim, h, spp, seed, 0.5)
    hit = prim[0, 0:3].astype(np.float64) + h.t[0] * prim[0, 4:7].astype(np.float64)
    for s in range(spp):
        x, y, z = oracle.sample_hemisphere(oracle.xi(seed, 0, s, 0), oracle.xi(seed, 0, s, 1))
        want = np.array([0.6 * x - 0.8 * y, z, 0.8 * x + 0.6 * y])
        assert np.allclose(ao[s, 4:7], want, atol=1e-6), (s, ao[s, 4:7], want)
        assert np.allclose(ao[s, 0:3], hit + 1e-4 * n, atol=1e-6)
        assert ao[s, 3] == 0 and ao[s, 7] == np.float32(0.5)


def test_uniform_rays_distribution():
    """The oracle's uniform rays: unit directions whose moments are those of the uniform
    distribution on the sphere (mean 0, E[d_i^2] = 1/3, E[d_i d_j] = 0, z uniform in
    [-1, 1] by Archimedes' theorem, every octant 1/8), origins uniform in the box (mean
    the centre, variance (hi - lo)^2 / 12), all in range; different seeds differ, equal
    seeds repeat."""
    n = 200_000
    lo, hi = np.array([-3.0, 10.0, -0.5]), np.array([5.0, 11.0, 0.25])
    r = oracle.uniform_rays(lo, hi, 99, n, 0.0, 4.0).astype(np.float64)
    d, o = r[:, 4:7], r[:, 0:3]
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    assert np.abs(d.mean(axis=0)).max() < 0.01
    assert np.abs((d ** 2).mean(axis=0) - 1 / 3).max() < 0.01
    c = d.T @ d / n
    assert abs(c[0, 1]) < 0.01 and abs(c[0, 2]) < 0.01 and abs(c[1, 2]) < 0.01
    hist = np.histogram(d[:, 2], bins=10, range=(-1, 1))[0] / n
    assert np.abs(hist - 0.1).max() < 0.005
    octant = (d[:, 0] > 0) * 4 + (d[:, 1] > 0) * 2 + (d[:, 2] > 0)
    assert np.abs(np.bincount(octant, minlength=8) / n - 0.125).max() < 0.005
    assert np.all(o >= lo) and np.all(o <= hi)
    assert np.abs(o.mean(axis=0) - 0.5 * (lo + hi)).max() < 0.01 * (hi - lo).max()
    assert np.abs(o.var(axis=0) / ((hi - lo) ** 2 / 12) - 1).max() < 0.02
    assert np.all(r[:, 3] == 0.0) and np.all(r[:, 7] == 4.0)
    assert np.array_equal(r, oracle.uniform_rays(lo, hi, 99, n, 0.0, 4.0))
    assert not np.array_equal(r[:100], oracle.uniform_rays(lo, hi, 100, 100, 0.0, 4.0))


# ---------------------------------------------------------------- discs (a custom primitive for user code)
def _disc_rows(c, r, n):
    d = np.zeros((len(c), 8), np.float32)
    d[:, 0:3], d[:, 3], d[:, 4:7] = c, r, n
    return d


def test_disc_closed_forms():
    """The unit disc at the origin facing +z, hit straight down from (x, y, 5): t = 5 iff
    x^2 + y^2 <= 1 (rim included); a tilted disc (normal (0, 0.6, 0.8), radius 0.5) hit
    along its normal through points 0.49 and 0.51 from its centre; parallel rays and
    planes behind the origin miss; the rim margin is 0 on the rim, 1 at the centre; a
    uniform scale 2 doubles the world radius."""
    S = oracle.Scene()
    S.add_instance(S.add_discs(_disc_rows([[0, 0, 0]], [1.0], [[0, 0, 1]])))
    def down(x, y, tmax=np.inf):
        r = np.zeros((1, 8), np.float32)
        r[0, 0:3], r[0, 4:7], r[0, 7] = (x, y, 5), (0, 0, -1), tmax
        return r
    for x, y, hit in ((0.0, 0.0, True), (0.0, 1.0, True), (0.6, 0.81, False), (-1.0, 0.0, True), (0.9, 0.5, False)):
        h = S.trace(down(x, y), bvh=False)
        assert (h.prim[0] != NONE) == hit, (x, y)
        if hit:
            assert h.t[0] == 5.0 and h.u[0] == 0.0 and h.v[0] == 0.0
    assert S.trace(down(0, 0, tmax=4.5), bvh=False).prim[0] == NONE
    assert S.min_disc_margin(down(0.0, 1.0)[0]) == 0.0 and S.min_disc_margin(down(0, 0)[0]) == 1.0
    side = np.zeros((1, 8), np.float32)
    side[0, 0:3], side[0, 4:7], side[0, 7] = (-3, 0, 0), (1, 0, 0), np.inf
    assert S.trace(side, bvh=False).prim[0] == NONE and S.min_disc_margin(side[0]) == 0.0
    up = down(0, 0)
    up[0, 6] = 1.0  # pointing away from the plane
    assert S.trace(up, bvh=False).prim[0] == NONE
    c, n = np.array([1.0, 2.0, 3.0]), np.array([0.0, 0.6, 0.8])
    T = oracle.Scene()
    T.add_instance(T.add_discs(_disc_rows([c], [0.5], [n])))
    inplane = np.array([1.0, 0.0, 0.0])
    for off, hit in ((0.49, True), (0.51, False)):
        r = np.zeros((1, 8), np.float32)
        r[0, 0:3], r[0, 4:7], r[0, 7] = c + off * inplane + 3 * n, -n, np.inf
        h = T.trace(r, bvh=False)
        assert (h.prim[0] != NONE) == hit
        if hit:
            assert abs(h.t[0] - 3.0) < 1e-6
    U = oracle.Scene()
    U.add_instance(U.add_discs(_disc_rows([[0, 0, 0]], [1.0], [[0, 0, 1]])), [0, 0, 0, 1, 2, 2, 2, 0, 0, 0])
    assert U.trace(down(1.9, 0.0), bvh=False).prim[0] == 0 and U.trace(down(2.1, 0.0), bvh=False).prim[0] == NONE


def test_disc_bvh_equals_brute_force():
    """Random discs of random orientation: the oracle BVH (disc boxes c +- r sqrt(1 - n_a^2))
    finds the same closest hits as brute force, for a plain geometry and instances."""
    rng = np.random.default_rng(5)
    m = 3000
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d = _disc_rows(rng.uniform(-5, 5, (m, 3)), rng.uniform(0.05, 0.6, m), n)
    S = oracle.Scene()
    g = S.add_discs(d)
    S.add_instance(g)
    S.add_instance(g, [0.2, 0.1, 0.3, 0.92, 1.5, 0.7, 1.2, 3, -2, 1])
    S.build()
    rays = scenegen.random_rays(20_000, [-6] * 3, [6] * 3, config=97)
    a, b = S.trace(rays, bvh=True), S.trace(rays, bvh=False)
    assert (a.prim != NONE).sum() > 5000
    assert np.array_equal(a.prim, b.prim) and np.array_equal(a.inst, b.inst) and np.array_equal(a.t, b.t)
