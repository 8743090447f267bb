"""Differentiable Lambertian shading on the GPU vs the FP64 oracle: forward image,
adjoint gradient, recompute mode, the autograd.Function, a scene where visibility matters
(a sphere shadowing the ground), and the full 1920x1080 check
against FP64 central differences (h = 1e-4) on 1,000 parameters."""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import Geometry, device_tensor, hits_to_numpy, new_hits
from paper_2603_00292_gb300.shading import LambertRenderer, lambert_shade

pytestmark = pytest.mark.gpu


def _problem(gpu, W, H):
    P = scenegen.shading_problem(W, H)
    rays = oracle.camera_rays(P.camera.packed(), W, H)
    verts64 = P.mesh.vertices.astype(np.float64)
    target = oracle.lambert_forward(verts64, P.mesh.indices, P.target_colours.astype(np.float64),
                                    P.target_light.astype(np.float64), rays).image
    d = dict(pos=device_tensor(P.mesh.vertices), idx=device_tensor(P.mesh.indices), col=device_tensor(P.colours),
             light=device_tensor(P.light), rays=device_tensor(rays))
    g = Geometry(gpu, vertices=d["pos"], indices=d["idx"]).build()
    return P, rays, verts64, target, d, g


def _gpu_forward(gpu, d, g, n):
    hits = new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, g.handle, d["rays"], n, hits)
    img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    vis = torch.empty(n, dtype=torch.uint8, device="cuda")
    grt.grtShadeLambert(gpu.handle, g.handle, d["rays"], hits, n, d["idx"], d["pos"], d["col"], d["light"], img, vis)
    torch.cuda.synchronize()
    return hits, img, vis


def _gpu_backward(gpu, d, g, n, hits, vis, gimg):
    gc = torch.zeros_like(d["col"])
    gl = torch.zeros_like(d["light"])
    gp = torch.zeros_like(d["pos"])
    grt.grtShadeLambertBackward(gpu.handle, g.handle, d["rays"], hits, vis, n, d["idx"], d["pos"], d["col"],
                                d["light"], gimg, gc, gl, gp)
    torch.cuda.synchronize()
    return gc.cpu().numpy().astype(np.float64), gl.cpu().numpy().astype(np.float64), gp.cpu().numpy().astype(np.float64)


U32 = 2.0 ** -24  # unit roundoff of float32


def _rel_ok(g, ref, rel=1e-3, l1=None):
    """|g - ref| <= 1e-3 max(|ref|, 1e-6 max|ref|), or, where the gradient's per-pixel terms
    cancel, <= 32 u S1 with S1 the sum of |terms| (oracle.lambert_gradient_l1): the GPU
    evaluates each term in float32 (a dozen rounded operations, <= 16u of the term
    relative) and sums them in float32 (warp shuffles, then atomics; <= 16u of S1 for the
    few hundred terms of a vertex). Where S1 / |ref| > 1e-3 / (32u), about 520, no float32
    evaluation can reach 1e-3 of ref."""
    scale = np.abs(ref).max()
    tol = rel * np.maximum(np.abs(ref), 1e-6 * scale) + 1e-12
    if l1 is not None:
        tol = np.maximum(tol, 32 * U32 * l1)
    return np.abs(g - ref) <= tol


def test_forward_matches_oracle(gpu):
    W, H = 320, 180
    P, rays, verts64, target, d, g = _problem(gpu, W, H)
    n = W * H
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    R = oracle.lambert_forward(verts64, P.mesh.indices, P.colours.astype(np.float64), P.light.astype(np.float64), rays)
    gprim = hits_to_numpy(hits)[1].astype(np.int64)
    oprim = np.where(R.prim < 0, 0xFFFFFFFF, R.prim.astype(np.int64))
    same = gprim == oprim
    assert (~same).sum() <= max(3, 1e-4 * n)
    gi = img.cpu().numpy()
    assert np.abs(gi[same] - R.image[same]).max() < 2e-5
    lit = same & (R.prim >= 0) & (R.sign > 0)
    assert np.array_equal(vis.cpu().numpy()[lit], R.vis[lit].astype(np.uint8))
    assert lit.sum() > 1000


def _mismatched(hits, vis, R):
    """Pixels where the GPU and the oracle disagree on the primary hit's triangle, or, on
    a lit hit, on the shadow ray's visibility (edge-grazing and shadow-edge rays)."""
    gprim = hits_to_numpy(hits)[1].astype(np.int64)
    oprim = np.where(R.prim < 0, 0xFFFFFFFF, R.prim.astype(np.int64))
    bad = gprim != oprim
    lit = ~bad & (R.prim >= 0) & (R.sign > 0)
    bad |= lit & (vis.cpu().numpy() != R.vis.astype(np.uint8))
    return bad


@pytest.mark.parametrize("recompute", [False, True])
def test_backward_matches_oracle_gradient(gpu, recompute):
    """Every colour, light and position gradient within 1e-3 relative of the oracle's
    FP64 analytic gradient. Pixels whose primary hit (or visibility) differs between
    the GPU and the oracle, at most 1e-4 of them, get dL/dI = 0 on the GPU side and are
    left out of the oracle's loss."""
    W, H = 320, 180
    P, rays, verts64, target, d, g = _problem(gpu, W, H)
    n = W * H
    cols64, l64 = P.colours.astype(np.float64), P.light.astype(np.float64)
    R = oracle.lambert_forward(verts64, P.mesh.indices, cols64, l64, rays)
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    exclude = _mismatched(hits, vis, R)
    assert exclude.sum() <= max(3, 1e-4 * n)
    _, dc, dl, dp = oracle.lambert_gradient(verts64, P.mesh.indices, cols64, l64, rays[~exclude], target[~exclude])
    l1 = oracle.lambert_gradient_l1(verts64, P.mesh.indices, cols64, l64, rays[~exclude], target[~exclude])
    gimg = 2.0 * (R.image - target)
    gimg[exclude] = 0.0
    gc, gl, gp = _gpu_backward(gpu, d, g, n, None if recompute else hits, None if recompute else vis,
                               device_tensor(gimg.astype(np.float32)))
    _check_every_gradient((gc, gl, gp), (dc, dl, dp), l1)


def _check_every_gradient(got, ref, l1):
    """Every element of the colour, light and position gradients within _rel_ok's bound
    (the float32 floor can decide an element only where its terms cancel by more than
    ~520x)."""
    for name, a, b, s1 in zip(("colour", "light", "position"), got, ref, l1):
        ok = _rel_ok(a, b, l1=s1)
        assert ok.all(), (name, np.nonzero(~ok), a[~ok][:5], b[~ok][:5], s1[~ok][:5])


@pytest.mark.parametrize("layout", ["global", "mixed"])
def test_backward_accumulation_paths_agree(gpu, layout):
    """The adjoint sums vertex gradients in a block-private shared-memory copy when the
    geometry's vertex count fits it, else in global memory; a vertex index at or beyond
    the declared count goes to global memory. All three give the same gradients."""
    W, H = 320, 180
    P, rays, verts64, target, d, g = _problem(gpu, W, H)
    n = W * H
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    gimg = 2.0 * (img - device_tensor(target.astype(np.float32)))
    ref = _gpu_backward(gpu, d, g, n, hits, vis, gimg)
    nv = P.mesh.vertices.shape[0]
    if layout == "global":  # 5,000 unused vertices appended: above the shared-memory budget
        extra = np.zeros((5000, 3), np.float32)
        d2 = dict(d, pos=device_tensor(np.concatenate([P.mesh.vertices, extra])),
                  col=device_tensor(np.concatenate([P.colours, extra])))
        g2 = Geometry(gpu, vertices=d2["pos"], indices=d2["idx"]).build()
    else:  # declared vertex count 100: indices 100..641 take the global path
        d2 = d
        g2 = Geometry(gpu, vertices=d["pos"], indices=d["idx"], vertex_count=100).build()
    got = _gpu_backward(gpu, d2, g2, n, hits, vis, gimg)
    for a, b in zip(got, ref):
        a = a.reshape(-1, 3)[:nv] if a.size > 3 else a
        assert np.allclose(a, b, rtol=1e-4, atol=1e-4 * np.abs(b).max())
    if layout == "global":
        assert not got[0][nv:].any() and not got[2][nv:].any()


def test_autograd_function(gpu):
    W, H = 160, 90
    P, rays, verts64, target, d, g = _problem(gpu, W, H)
    n = W * H
    tgt = device_tensor(target.astype(np.float32))
    out = {}
    for store in (True, False):
        col = d["col"].clone().requires_grad_(True)
        light = d["light"].clone().requires_grad_(True)
        pos = d["pos"].clone().requires_grad_(True)
        R = LambertRenderer(gpu, g, d["idx"], d["rays"], store=store)
        img = lambert_shade(col, light, pos, R)
        loss = ((img - tgt) ** 2).sum()
        loss.backward()
        out[store] = (loss.item(), col.grad.clone(), light.grad.clone(), pos.grad.clone())
    # direct calls give the same gradient (up to the order of float atomics)
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    gimg = 2.0 * (img - tgt)
    gc, gl, gp = _gpu_backward(gpu, d, g, n, hits, vis, gimg)
    for store in (True, False):
        l, c_, l_, p_ = out[store]
        assert np.allclose(c_.cpu().numpy(), gc, rtol=1e-4, atol=1e-5)
        assert np.allclose(l_.cpu().numpy(), gl, rtol=1e-4, atol=1e-4)
        assert np.allclose(p_.cpu().numpy(), gp, rtol=1e-3, atol=1e-4)


def _central_differences(args, params, exclude, h0=1e-4, agree=2.5e-4, halvings=4):
    """FP64 central differences the gradient is held to, one per parameter.

    Each value is the difference quotient of the loss over the pixels whose (hit
    triangle, visibility, sign of n.l) is the same at theta-h, theta, theta+h, plus the
    oracle's analytic term of the few pixels where it is not (there the loss jumps and
    the quotient does not approximate the interior derivative). Returns (ref, plain):
    plain marks the parameters whose h0 quotient agrees with the h0/2 quotient within
    `agree` relative, i.e. whose h0 quotient is in its O(h^2) regime, and ref is that
    h0 quotient. At grazing hits (|n.d| of a few 1e-2 near the silhouette) the hit point
    moves like 1/|n.d| with the vertices and the h0 quotient is still far from its limit;
    there h is halved `halvings` times and ref is the Richardson value (4 q(h) - q(2h)) / 3
    of the two finest quotients."""
    def quotient(q, h):
        fd, masked, _ = oracle.lambert_fd(*args, q, h, exclude=exclude)
        return fd + masked

    q0, q1 = quotient(params, h0), quotient(params, h0 / 2)
    plain = np.abs(q0 - q1) <= agree * np.abs(q0)
    ref = q0.copy()
    late = np.nonzero(~plain)[0]
    if late.size:
        coarse, h = q1[late], h0 / 2
        for _ in range(halvings - 1):
            h /= 2
            fine = quotient(params[late], h)
            coarse, last = fine, coarse
        ref[late] = (4.0 * coarse - last) / 3.0
    return ref, plain


def test_full_size_gradient_against_central_differences(gpu):
    """1920x1080, 1,000 parameters drawn (seeded) among those with a nonzero gradient,
    checked three ways at 1e-3 relative: against the FP64 CPU reference gradient (all
    of them), against the plain h = 1e-4 central difference wherever that quotient has
    converged, and against the extrapolated central difference elsewhere. Pixels where
    the GPU and the oracle hit different triangles (edge-grazing) get dL/dI = 0 on the
    GPU side and are left out of the oracle's loss."""
    W, H = 1920, 1080
    P, rays, verts64, target, d, g = _problem(gpu, W, H)
    n = W * H
    cols64, l64 = P.colours.astype(np.float64), P.light.astype(np.float64)
    R = oracle.lambert_forward(verts64, P.mesh.indices, cols64, l64, rays)
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    gprim = hits_to_numpy(hits)[1].astype(np.int64)
    oprim = np.where(R.prim < 0, 0xFFFFFFFF, R.prim.astype(np.int64))
    exclude = gprim != oprim
    assert exclude.sum() <= max(3, 1e-4 * n)
    gimg = 2.0 * (R.image - target)
    gimg[exclude] = 0.0
    gc, gl, gp = _gpu_backward(gpu, d, g, n, hits, vis, device_tensor(gimg.astype(np.float32)))
    nv = verts64.shape[0]
    grad = np.concatenate([gc.ravel(), gl, gp.ravel()])
    cand = np.nonzero(grad != 0)[0]
    rng = np.random.default_rng(20260301)
    params = np.sort(rng.choice(cand, size=min(1000, cand.size), replace=False))
    grad = grad[params]
    kinds = np.where(params < 3 * nv, "colour", np.where(params < 3 * nv + 3, "light", "position"))
    assert (kinds == "colour").sum() > 100 and (kinds == "position").sum() > 100

    def failures(ok, ref):
        return [(int(p), k, a, b) for p, k, a, b in zip(params[~ok], kinds[~ok], grad[~ok], ref[~ok])][:8]

    _, dc, dl, dp = oracle.lambert_gradient(verts64, P.mesh.indices, cols64, l64, rays[~exclude], target[~exclude])
    ac, al, ap = oracle.lambert_gradient_l1(verts64, P.mesh.indices, cols64, l64, rays[~exclude], target[~exclude])
    analytic = np.concatenate([dc.ravel(), dl, dp.ravel()])[params]
    s1 = np.concatenate([ac.ravel(), al, ap.ravel()])[params]
    ok = _rel_ok(grad, analytic, l1=s1)
    assert ok.all(), failures(ok, analytic)

    args = (verts64, P.mesh.indices, cols64, l64, rays, target)
    ref, plain = _central_differences(args, params, exclude)
    assert plain.mean() >= 0.9, plain.mean()
    ok = _rel_ok(grad, ref)
    assert ok[plain].all(), failures(ok | ~plain, ref)
    assert ok[~plain].all(), failures(ok | plain, ref)


def test_shadowed_scene_forward_and_gradient(gpu):
    """The icosphere above a ground quad, lit from above and in front, so the sphere casts a
    shadow the camera sees: visibility decides thousands of lit pixels (V = 0, I = 0).
    Forward image and visibility, and the adjoint gradients, against the FP64 oracle."""
    W, H = 320, 180
    ico = scenegen.icosphere(3)
    ground = np.array([[-4, -1.2, -4], [4, -1.2, -4], [4, -1.2, 4], [-4, -1.2, 4]], np.float32)
    verts = np.concatenate([ico.vertices, ground]).astype(np.float32)
    nv = ico.vertices.shape[0]
    idx = np.concatenate([ico.indices, np.array([[0, 2, 1], [0, 3, 2]], np.uint32) + nv]).astype(np.uint32)
    rng = np.random.default_rng(11)
    cols = rng.uniform(0.2, 1.0, verts.shape).astype(np.float32)
    tcols = (cols + rng.uniform(-0.05, 0.05, cols.shape)).astype(np.float32)
    light = np.array([0.2, 1.0, -0.6], np.float64)  # toward the light: the shadow falls toward the camera
    light = (light / np.linalg.norm(light)).astype(np.float32)
    cam = scenegen.look_down_z_camera([0, 0.4, 3.5], W, H)
    rays = oracle.camera_rays(cam.packed(), W, H)
    v64 = verts.astype(np.float64)
    target = oracle.lambert_forward(v64, idx, tcols.astype(np.float64), light.astype(np.float64), rays).image
    R = oracle.lambert_forward(v64, idx, cols.astype(np.float64), light.astype(np.float64), rays)
    n = W * H
    d = dict(pos=device_tensor(verts), idx=device_tensor(idx), col=device_tensor(cols), light=device_tensor(light),
             rays=device_tensor(rays))
    g = Geometry(gpu, vertices=d["pos"], indices=d["idx"]).build()
    hits, img, vis = _gpu_forward(gpu, d, g, n)
    gprim = hits_to_numpy(hits)[1].astype(np.int64)
    oprim = np.where(R.prim < 0, 0xFFFFFFFF, R.prim.astype(np.int64))
    lit = (gprim == oprim) & (R.prim >= 0) & (R.sign > 0)
    gv = vis.cpu().numpy()
    shadowed = lit & (R.vis == 0)
    assert shadowed.sum() > 1500, shadowed.sum()  # the sphere's shadow on the ground (2,145 pixels)
    agree = gv[lit] == R.vis[lit].astype(np.uint8)
    assert (~agree).sum() <= max(3, 1e-3 * lit.sum())  # shadow-edge rays only
    same = lit & (gv == R.vis.astype(np.uint8))
    gi = img.cpu().numpy()
    assert np.all(gi[shadowed & same] == 0)
    assert np.abs(gi[same] - R.image[same]).max() < 2e-5
    # adjoint against the oracle's analytic gradient of the same loss, over the pixels
    # where the GPU and the oracle agree on the hit and the visibility: every gradient
    # within 1e-3 relative
    exclude = _mismatched(hits, vis, R)
    assert exclude.sum() <= max(3, 1e-3 * lit.sum())
    _, dc, dl, dp = oracle.lambert_gradient(v64, idx, cols.astype(np.float64), light.astype(np.float64),
                                            rays[~exclude], target[~exclude])
    l1 = oracle.lambert_gradient_l1(v64, idx, cols.astype(np.float64), light.astype(np.float64), rays[~exclude],
                                    target[~exclude])
    gimg = 2.0 * (R.image - target)
    gimg[exclude] = 0.0
    gc, gl, gp = _gpu_backward(gpu, d, g, n, hits, vis, device_tensor(gimg.astype(np.float32)))
    _check_every_gradient((gc, gl, gp), (dc, dl, dp), l1)
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    g.close()


def test_two_forwards_through_one_renderer(gpu):
    """Two forwards through one LambertRenderer under two lights, then the first one's
    backward: it uses its own visibility, not the second forward's. The scene is the
    icosphere over a ground quad, so the two lights shadow different pixels."""
    W, H = 160, 90
    ico = scenegen.icosphere(3)
    ground = np.array([[-4, -1.2, -4], [4, -1.2, -4], [4, -1.2, 4], [-4, -1.2, 4]], np.float32)
    verts = np.concatenate([ico.vertices, ground]).astype(np.float32)
    nv = ico.vertices.shape[0]
    idx = np.concatenate([ico.indices, np.array([[0, 2, 1], [0, 3, 2]], np.uint32) + nv]).astype(np.uint32)
    cols = np.random.default_rng(12).uniform(0.2, 1.0, verts.shape).astype(np.float32)
    lights = [np.array(l, np.float64) / np.linalg.norm(l) for l in ([0.2, 1.0, -0.6], [-0.7, 1.0, 0.3])]
    cam = scenegen.look_down_z_camera([0, 0.4, 3.5], W, H)
    rays = device_tensor(oracle.camera_rays(cam.packed(), W, H))
    pos, ind, col = device_tensor(verts), device_tensor(idx), device_tensor(cols)
    g = Geometry(gpu, vertices=pos, indices=ind).build()
    R = LambertRenderer(gpu, g, ind, rays, store=True)
    tgt = torch.zeros((W * H, 3), dtype=torch.float32, device="cuda")
    params, imgs = [], []
    for l in lights:
        p = (col.clone().requires_grad_(True), device_tensor(l.astype(np.float32)).requires_grad_(True),
             pos.clone().requires_grad_(True))
        params.append(p)
        imgs.append(lambert_shade(*p, R))
    ((imgs[0] - tgt) ** 2).sum().backward()
    # the same gradient from direct calls with the first light
    d = dict(pos=pos, idx=ind, col=col, light=device_tensor(lights[0].astype(np.float32)), rays=rays)
    hits, img, vis = _gpu_forward(gpu, d, g, W * H)
    hits2, img2, vis2 = _gpu_forward(gpu, dict(d, light=device_tensor(lights[1].astype(np.float32))), g, W * H)
    assert (vis.cpu() != vis2.cpu()).sum() > 100  # the lights shadow different pixels
    gc, gl, gp = _gpu_backward(gpu, d, g, W * H, hits, vis, 2.0 * (img - tgt))
    c_, l_, p_ = (t.grad.cpu().numpy() for t in params[0])
    assert np.allclose(c_, gc, rtol=1e-4, atol=1e-5)
    assert np.allclose(l_, gl, rtol=1e-4, atol=1e-4)
    assert np.allclose(p_, gp, rtol=1e-3, atol=1e-4)
    g.close()


def test_two_level_scene_shading_and_adjoint(gpu):
    """grtShadeLambertScene / grtShadeLambertSceneBackward on a two-level scene: an
    icosphere instance (scaled, rotated) above a ground-quad instance, and a second
    instance of the same icosphere mesh, light from above so the spheres shadow the
    ground (shadow rays through the whole scene). Forward image and visibility against
    the oracle's world-space composition (oracle.LambertScene); the adjoint, stored and
    recomputed, against its gradient in object space (colours summed over the instances
    sharing a vertex, positions through each frame's M^T): every gradient within the
    bound of _rel_ok, pixels whose hit or visibility differ excluded."""
    from paper_2603_00292_gb300.objects import Scene

    W, H = 320, 180
    ico = scenegen.icosphere(3)
    ground = np.array([[-4, 0, -4], [4, 0, -4], [4, 0, 4], [-4, 0, 4]], np.float32)
    nv_ico, nt = ico.vertices.shape[0], ico.indices.shape[0]
    gidx = np.array([[0, 2, 1], [0, 3, 2]], np.uint32)
    verts = np.concatenate([ico.vertices, ground]).astype(np.float32)
    idx = np.concatenate([ico.indices, gidx + nv_ico]).astype(np.uint32)
    frames = np.array([[0.1, 0.2, 0.0, 0.97, 0.7, 0.7, 0.7, 0.0, 0.2, 0.0], [0, 0, 0, 1, 1, 1, 1, 0, -1.2, 0],
                       [0.0, 0.6, 0.3, 0.74, 0.5, 0.4, 0.45, 1.6, -0.3, 0.8]], np.float32)
    offs, cnts = [0, nt, 0], [nt, 2, nt]
    rng = np.random.default_rng(21)
    cols = rng.uniform(0.2, 1.0, verts.shape).astype(np.float32)
    tcols = (cols + rng.uniform(-0.05, 0.05, cols.shape)).astype(np.float32)
    light = np.array([0.3, 1.0, 0.4], np.float64)
    light = (light / np.linalg.norm(light)).astype(np.float32)
    cam = scenegen.look_at_camera([0, 1.0, 5.0], [0, -0.4, 0], W, H)
    rays = oracle.camera_rays(cam.packed(), W, H)
    n = W * H
    L = oracle.LambertScene(verts, idx, offs, cnts, frames)
    l64, c64 = light.astype(np.float64), cols.astype(np.float64)
    R = L.forward(c64, l64, rays)
    target = L.forward(tcols.astype(np.float64), l64, rays).image

    g_ico = Geometry(gpu, vertices=device_tensor(ico.vertices), indices=device_tensor(ico.indices)).build()
    g_gnd = Geometry(gpu, vertices=device_tensor(ground), indices=device_tensor(gidx)).build()
    sc = Scene(gpu, [g_ico.handle, g_gnd.handle, g_ico.handle], device_tensor(frames)).build()
    d = dict(pos=device_tensor(verts), idx=device_tensor(idx), col=device_tensor(cols), light=device_tensor(light),
             rays=device_tensor(rays), off=device_tensor(np.array(offs, np.uint32)))
    hits = new_hits(n)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, d["rays"], n, hits)
    img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    vis = torch.empty(n, dtype=torch.uint8, device="cuda")
    grt.grtShadeLambertScene(gpu.handle, sc.handle, d["rays"], hits, n, d["off"], d["idx"], d["pos"], d["col"],
                             d["light"], img, vis)
    torch.cuda.synchronize()
    gi_, gp_ = hits_to_numpy(hits)[0:2]
    same = (gp_.astype(np.int64) == np.where(R.iprim < 0, 0xFFFFFFFF, R.iprim)) & \
           (np.where(gp_ == 0xFFFFFFFF, -1, gi_.astype(np.int64)) == np.where(R.iprim < 0, -1, R.inst))
    assert (~same).sum() <= max(3, 1e-4 * n)
    lit = same & (R.prim >= 0) & (R.sign > 0)
    gv = vis.cpu().numpy()
    shadowed = lit & (R.vis == 0)
    assert shadowed.sum() > 300, shadowed.sum()  # the spheres' shadows on the ground
    assert ((gv != R.vis.astype(np.uint8)) & lit).sum() <= max(3, 1e-3 * lit.sum())
    ok_px = same & ~(lit & (gv != R.vis.astype(np.uint8)))
    gimg_h = img.cpu().numpy()
    assert np.abs(gimg_h[ok_px] - R.image[ok_px]).max() < 2e-5
    assert np.all(gimg_h[shadowed & ok_px] == 0)

    exclude = ~ok_px
    _, dc, dl, dp = L.gradient(c64, l64, rays[~exclude], target[~exclude])
    l1 = L.gradient_l1(c64, l64, rays[~exclude], target[~exclude])
    gimg = 2.0 * (R.image - target)
    gimg[exclude] = 0.0
    gimg_d = device_tensor(gimg.astype(np.float32))
    results = []
    for stored in (True, False):
        gc, gl, gp = torch.zeros_like(d["col"]), torch.zeros_like(d["light"]), torch.zeros_like(d["pos"])
        grt.grtShadeLambertSceneBackward(gpu.handle, sc.handle, d["rays"], hits if stored else None,
                                         vis if stored else None, n, d["off"], d["idx"], d["pos"], verts.shape[0],
                                         d["col"], d["light"], gimg_d, gc, gl, gp)
        torch.cuda.synchronize()
        got = tuple(t.cpu().numpy().astype(np.float64) for t in (gc, gl, gp))
        _check_every_gradient(got, (dc, dl, dp), l1)
        results.append(got)
    for a, b in zip(*results):  # recomputed hits are the stored ones: equal up to the order of float atomics
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    for obj in (sc, g_gnd, g_ico):
        obj.close()
