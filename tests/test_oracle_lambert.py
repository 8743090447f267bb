"""Pins for the oracle's Lambertian shading and its gradient (CPU only): FP64 central
differences against the analytic gradient on a small render, Euler's identity for the
light (the image is homogeneous of degree 1 in an unnormalised light where lit), and
a closed form for the colour gradient of a one-triangle scene."""
import math

import numpy as np

import oracle
import scenegen


def _setup(level=1, W=48, H=36, seed=3):
    mesh = scenegen.icosphere(level)
    rng = np.random.default_rng(seed)
    cols = rng.uniform(0, 1, (mesh.vertices.shape[0], 3))
    light = np.array([1.0, 1.0, 1.0]) / math.sqrt(3)
    cam = scenegen.look_down_z_camera([0, 0, 3], W, H)
    rays = oracle.camera_rays(cam.packed(), W, H)
    verts = mesh.vertices.astype(np.float64)
    # target: perturbed colours and a light rotated by a few degrees
    tcols = cols + rng.uniform(-0.1, 0.1, cols.shape)
    axis = np.cross(light, [0, 1.0, 0])
    axis /= np.linalg.norm(axis)
    ang = math.radians(4.0)
    tlight = light * math.cos(ang) + np.cross(axis, light) * math.sin(ang)
    target = oracle.lambert_forward(verts, mesh.indices, tcols, tlight, rays).image
    return mesh, verts, cols, light, rays, target


def test_forward_is_shaded_hits_only():
    mesh, verts, cols, light, rays, target = _setup()
    R = oracle.lambert_forward(verts, mesh.indices, cols, light, rays)
    miss = R.prim < 0
    assert miss.any() and (~miss).any()
    assert np.all(R.image[miss] == 0)
    # a convex sphere never shadows a lit point
    lit = (R.prim >= 0) & (R.sign > 0)
    assert np.all(R.vis[lit] == 1)
    assert np.all(R.image[(R.prim >= 0) & (R.sign <= 0)] == 0)
    assert np.all(R.image >= 0) and np.all(R.image <= 1)


def test_gradient_matches_central_differences():
    mesh, verts, cols, light, rays, target = _setup()
    loss, dc, dl, dp = oracle.lambert_gradient(verts, mesh.indices, cols, light, rays, target)
    nv = verts.shape[0]
    analytic = np.concatenate([dc.ravel(), dl, dp.ravel()])
    params = np.nonzero(analytic != 0)[0]
    assert params.size > 60
    fd, masked, count = oracle.lambert_fd(verts, mesh.indices, cols, light, rays, target, params, 1e-4)
    g = analytic[params] - masked
    scale = max(np.abs(fd).max(), 1e-30)
    err = np.abs(g - fd)
    ok = err <= 1e-3 * np.maximum(np.abs(fd), 1e-6 * scale)
    assert ok.mean() == 1.0, (params[~ok][:5], g[~ok][:5], fd[~ok][:5])
    # the three kinds of parameters are all exercised
    assert (params < 3 * nv).any() and ((params >= 3 * nv) & (params < 3 * nv + 3)).any() and (params >= 3 * nv + 3).any()


def test_light_gradient_euler_identity():
    mesh, verts, cols, light, rays, target = _setup(level=2, seed=5)
    loss, dc, dl, dp = oracle.lambert_gradient(verts, mesh.indices, cols, light, rays, target)
    R = oracle.lambert_forward(verts, mesh.indices, cols, light, rays)
    # I is homogeneous of degree 1 in l (max(0, n.l) with l unnormalised), so
    # l . dL/dl = sum 2 (I - I*) . I
    lhs = float(np.dot(light, dl))
    rhs = float(np.sum(2 * (R.image - target) * R.image))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))


def test_colour_gradient_closed_form_one_triangle():
    v = np.array([[-1.0, -0.8, 0.0], [1.2, -0.6, 0.0], [0.1, 1.1, 0.0]])
    idx = np.array([[0, 1, 2]], np.uint32)
    cols = np.array([[0.2, 0.5, 0.9], [0.7, 0.1, 0.4], [0.3, 0.8, 0.6]])
    tcols = cols + np.array([[0.05, -0.02, 0.03], [-0.04, 0.06, 0.01], [0.02, 0.02, -0.05]])
    light = np.array([0.3, 0.2, 0.9])
    cam = scenegen.look_down_z_camera([0, 0, 3], 40, 30)
    rays = oracle.camera_rays(cam.packed(), 40, 30)
    target = oracle.lambert_forward(v, idx, tcols, light, rays).image
    loss, dc, dl, dp = oracle.lambert_gradient(v, idx, cols, light, rays, target)
    R = oracle.lambert_forward(v, idx, cols, light, rays)
    # the triangle faces +z toward the camera: s = n . l = l_z everywhere it is hit
    hit = R.prim >= 0
    u, w = R.tuv[hit, 1], R.tuv[hit, 2]
    B = np.stack([1 - u - w, u, w], axis=1)           # barycentric weights per pixel
    s = light[2]
    G = (s * s) * (B.T @ B)                             # sum_p s^2 w w^T
    expect = 2 * G @ (cols - tcols)                    # I - I* = s W (c - c*)
    assert np.allclose(dc, expect, rtol=1e-10, atol=1e-12)


def test_shadow_closed_form_occluder_above_ground():
    """A ground quad in the plane y = 0 (facing +y) and a small square occluder in the
    plane y = 1 over x, z in [-0.5, 0.5], light straight up (0, 1, 0), camera rays straight
    down. Under the occluder the shadow ray meets it (V = 0, I = 0); elsewhere on the
    ground I = (n . l) c = c exactly, with c the barycentric blend of the ground colours;
    the occluder itself is lit from above but is seen from above, facing the ray: V = 1."""
    g = [[-3, 0, -3], [3, 0, -3], [3, 0, 3], [-3, 0, 3]]
    o = [[-0.5, 1, -0.5], [0.5, 1, -0.5], [0.5, 1, 0.5], [-0.5, 1, 0.5]]
    v = np.array(g + o, np.float64)
    idx = np.array([[0, 2, 1], [0, 3, 2], [4, 6, 5], [4, 7, 6]], np.uint32)
    cols = np.tile(np.array([[0.25, 0.5, 0.75]]), (8, 1))  # uniform: c(u, v) is exact
    light = np.array([0.0, 1.0, 0.0])
    xs = np.array([-2.0, -0.8, -0.3, 0.0, 0.2, 0.45, 0.7, 1.9])
    rays = np.zeros((xs.size * xs.size, 8), np.float32)
    X, Z = np.meshgrid(xs, xs)
    rays[:, 0], rays[:, 1], rays[:, 2] = X.ravel(), 5.0, Z.ravel()
    rays[:, 5] = -1.0
    rays[:, 7] = np.inf
    R = oracle.lambert_forward(v, idx, cols, light, rays)
    under = (np.abs(X.ravel()) < 0.5) & (np.abs(Z.ravel()) < 0.5)
    assert np.all(R.prim[under] >= 2)  # the camera ray meets the occluder first
    assert np.all(R.vis[under] == 1) and np.allclose(R.image[under], cols[0], rtol=0, atol=1e-15)
    # move the occluder out of the camera's way (camera rays start below it) but keep it
    # between the ground and the light
    rays2 = rays.copy()
    rays2[:, 1] = 0.5
    R2 = oracle.lambert_forward(v, idx, cols, light, rays2)
    assert np.all(R2.prim <= 1)  # only the ground is hit
    assert np.all(R2.vis[under] == 0) and np.all(R2.image[under] == 0)
    assert np.all(R2.vis[~under] == 1) and np.allclose(R2.image[~under], cols[0], rtol=0, atol=1e-15)


def test_gradient_term_l1_norms():
    """The per-parameter L1 norms of the gradient's per-pixel terms: at least |gradient|
    (triangle inequality), equal to it for a single pixel, zero where the render meets
    its target (every term carries the residual I - I*), and linear in a common scale of
    the residual; the light's norm is the sum of the per-pixel |terms| of each pixel."""
    mesh, verts, cols, light, rays, target = _setup()
    _, dc, dl, dp = oracle.lambert_gradient(verts, mesh.indices, cols, light, rays, target)
    ac, al, ap = oracle.lambert_gradient_l1(verts, mesh.indices, cols, light, rays, target)
    for g, a in ((dc, ac), (dl, al), (dp, ap)):
        assert np.all(a >= np.abs(g) - 1e-12 * (1 + np.abs(g)))
    assert (ap > 10 * np.abs(dp)).any()  # some position gradients cancel strongly
    R = oracle.lambert_forward(verts, mesh.indices, cols, light, rays)
    p = int(np.nonzero((R.prim >= 0) & (R.sign > 0))[0][0])
    one = rays[p:p + 1]
    _, dc1, dl1, dp1 = oracle.lambert_gradient(verts, mesh.indices, cols, light, one, target[p:p + 1])
    ac1, al1, ap1 = oracle.lambert_gradient_l1(verts, mesh.indices, cols, light, one, target[p:p + 1])
    assert np.array_equal(ac1, np.abs(dc1)) and np.array_equal(al1, np.abs(dl1)) and np.array_equal(ap1, np.abs(dp1))
    z = oracle.lambert_gradient_l1(verts, mesh.indices, cols, light, rays, R.image)
    assert all(not a.any() for a in z)
    # residual scaled by 2 about the render: every term doubles
    t2 = R.image + 2.0 * (target - R.image)
    ac2, al2, ap2 = oracle.lambert_gradient_l1(verts, mesh.indices, cols, light, rays, t2)
    assert np.allclose(ac2, 2 * ac, rtol=1e-12) and np.allclose(ap2, 2 * ap, rtol=1e-12)
    assert np.allclose(al2, 2 * al, rtol=1e-12)


# ---------------------------------------------------------------- two-level scenes
def _two_level(light=(0.0, 1.0, 0.0), W=64, H=48, second=True):
    """An icosphere (scale 0.7, rotated) above a 8x8 ground quad at y = -1.2, optionally a
    second icosphere instance of the same mesh; camera from (0, 1, 5) toward the origin."""
    ico = scenegen.icosphere(2)
    ground = np.array([[-4, 0, -4], [4, 0, -4], [4, 0, 4], [-4, 0, 4]], np.float32)
    nv = ico.vertices.shape[0]
    verts = np.concatenate([ico.vertices, ground]).astype(np.float32)
    idx = np.concatenate([ico.indices, np.array([[0, 2, 1], [0, 3, 2]], np.uint32) + nv]).astype(np.uint32)
    nt = ico.indices.shape[0]
    frames = [[0.1, 0.2, 0.0, 0.97, 0.7, 0.7, 0.7, 0.0, 0.2, 0.0], [0, 0, 0, 1, 1, 1, 1, 0, -1.2, 0]]
    offs, cnts = [0, nt], [nt, 2]
    if second:
        frames.append([0.0, 0.6, 0.3, 0.74, 0.5, 0.4, 0.45, 1.6, -0.3, 0.8])
        offs.append(0), cnts.append(nt)
    rng = np.random.default_rng(8)
    cols = rng.uniform(0.2, 1.0, verts.shape)
    l = np.array(light, np.float64)
    l /= np.linalg.norm(l)
    cam = scenegen.look_at_camera([0, 1.0, 5.0], [0, -0.4, 0], W, H)
    rays = oracle.camera_rays(cam.packed(), W, H)
    return oracle.LambertScene(verts, idx, offs, cnts, np.array(frames, np.float32)), verts, idx, cols, l, rays


def test_scene_identity_frame_equals_plain_oracle():
    mesh, verts, cols, light, rays, target = _setup()
    L = oracle.LambertScene(verts, mesh.indices, [0], [mesh.indices.shape[0]], [[0, 0, 0, 1, 1, 1, 1, 0, 0, 0]])
    a = L.forward(cols, light, rays)
    b = oracle.lambert_forward(verts, mesh.indices, cols, light, rays)
    assert np.array_equal(a.image, b.image) and np.array_equal(a.iprim, b.prim) and np.all(a.inst[b.prim >= 0] == 0)
    ga, gb = L.gradient(cols, light, rays, target), oracle.lambert_gradient(verts, mesh.indices, cols, light, rays,
                                                                              target)
    for x, y in zip(ga, gb):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_scene_shadow_cast_by_another_instance():
    """Light straight up: a ground point whose vertical line passes within 0.9 x the
    sphere's world radius of its centre is in shadow (the level-2 icosphere contains the
    ball of radius 0.9), one farther than the radius is lit."""
    L, verts, idx, cols, l, rays = _two_level(second=False)
    R = L.forward(cols, l, rays)
    on_ground = R.inst == 1
    assert on_ground.sum() > 500
    t = R.tuv[:, 0]
    p = rays[:, 0:3].astype(np.float64) + t[:, None] * rays[:, 4:7].astype(np.float64)
    centre, radius = np.array([0.0, 0.2, 0.0]), 0.7
    horiz = np.hypot(p[:, 0] - centre[0], p[:, 2] - centre[2])
    inside, outside = on_ground & (horiz < 0.9 * radius), on_ground & (horiz > radius)
    assert inside.sum() > 20 and outside.sum() > 100
    assert np.all(R.vis[inside] == 0) and np.all(R.image[inside] == 0)
    assert np.all(R.vis[outside] == 1) and np.all(R.image[outside].max(axis=1) > 0)


def test_scene_gradient_matches_central_differences():
    """Object-space positions and colours of the shared mesh (two icosphere instances
    under scaled, rotated frames, and the ground): FP64 central differences (h = 1e-6)
    of the loss, recomputed from the perturbed object mesh, against the analytic gradient
    mapped back through each frame. Parameters whose perturbation changes any pixel's
    hit, visibility or sign of n.l are skipped."""
    L, verts, idx, cols, l, rays = _two_level(light=(0.3, 1.0, 0.4))
    tcols = cols + np.random.default_rng(9).uniform(-0.1, 0.1, cols.shape)
    frames = np.array([[0.1, 0.2, 0.0, 0.97, 0.7, 0.7, 0.7, 0.0, 0.2, 0.0], [0, 0, 0, 1, 1, 1, 1, 0, -1.2, 0],
                       [0.0, 0.6, 0.3, 0.74, 0.5, 0.4, 0.45, 1.6, -0.3, 0.8]], np.float32)
    nt = idx.shape[0] - 2
    target = L.forward(tcols, l, rays).image
    _, dc, dl, dp = L.gradient(cols, l, rays, target)

    def loss_state(v, c):
        S = oracle.LambertScene(v, idx, [0, nt, 0], [nt, 2, nt], frames)
        R = S.forward(c, l, rays)
        return ((R.image - target) ** 2).sum(), np.stack([R.prim, R.vis, R.sign])

    rng = np.random.default_rng(10)
    used = np.unique(idx[:nt])
    checked = 0
    for vtx in rng.choice(used, 24, replace=False):
        for a in range(3):
            h = 1e-6
            vp, vm = verts.astype(np.float64), verts.astype(np.float64)
            vp[vtx, a] += h
            vm[vtx, a] -= h
            (lp, sp), (lm, sm) = loss_state(vp, cols), loss_state(vm, cols)
            if not np.array_equal(sp, sm):
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dp[vtx, a]) <= 1e-4 * max(abs(fd), 1e-3), (vtx, a, fd, dp[vtx, a])
            checked += 1
    assert checked >= 30
    for vtx in rng.choice(used, 6, replace=False):  # colours: the loss is quadratic in them
        cp, cm = cols.copy(), cols.copy()
        cp[vtx, 1] += 1e-3
        cm[vtx, 1] -= 1e-3
        fd = (loss_state(verts, cp)[0] - loss_state(verts, cm)[0]) / 2e-3
        assert abs(fd - dc[vtx, 1]) <= 1e-8 * max(1.0, abs(fd))
