"""Ray queries from a user's own CUDA kernel through include/grt_device.cuh.

tests/device_api_kernel.cu is compiled here, as a user would compile it, against the
public header; its hit records must equal the library's grtTraceClosest / grtTraceAnyHit
on a geometry, a two-level scene and custom spheres: identical primitives except at
equal-t ties, where both hits are then valid, and identical t, u, v (the same FP64
refinement) wherever the primitives agree; any-hit occlusion identical.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import oracle
import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import FuncTable, Geometry, Scene, device_tensor, hits_to_numpy, new_hits
from parity import NONE

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def user_lib(gpu, tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("devapi") / "libdevapi.so")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
           "-shared", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2603_00292_gb300", "csrc"),
           os.path.join(ROOT, "tests", "device_api_kernel.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.userTraceLaunch.argtypes = [ctypes.POINTER(grt.grtDeviceTarget), ctypes.c_void_p, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.userTraceLaunch.restype = ctypes.c_int
    L.userTraceMaskedLaunch.argtypes = [ctypes.POINTER(grt.grtDeviceTarget), ctypes.c_void_p, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p]
    L.userTraceMaskedLaunch.restype = ctypes.c_int
    L.userAllHitsLaunch.argtypes = [ctypes.POINTER(grt.grtDeviceTarget), ctypes.c_void_p, ctypes.c_uint32,
                                    ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    L.userAllHitsLaunch.restype = ctypes.c_int
    return L


def _user(L, target, rays, any_hit):
    n = rays.shape[0]
    h = new_hits(n)
    assert L.userTraceLaunch(ctypes.byref(target), rays.data_ptr(), n, h.data_ptr(), int(any_hit),
                             torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    return hits_to_numpy(h)


def _library(gpu, rays, any_hit, scene=None, geom=None, table=None):
    n = rays.shape[0]
    h = new_hits(n)
    fn = grt.grtTraceAnyHit if any_hit else grt.grtTraceClosest
    fn(gpu.handle, scene, geom, rays, n, h, table)
    torch.cuda.synchronize()
    return hits_to_numpy(h)


def _same_closest(a, b, S, rays):
    same = (a[0] == b[0]) & (a[1] == b[1])
    for k in (2, 3, 4):
        assert np.array_equal(a[k][same].view(np.uint32), b[k][same].view(np.uint32))
    for i in np.nonzero(~same)[0]:  # equal-t ties: both hits valid at the same t
        assert a[1][i] != NONE and b[1][i] != NONE
        ok, t, _, _ = S.intersect_prim(rays[i], int(a[0][i]), int(a[1][i]))
        assert ok and abs(t - float(b[2][i])) <= 1e-5 * abs(float(b[2][i]))
    assert (~same).sum() <= max(3, 1e-4 * len(same))


def test_user_kernel_on_a_geometry(gpu, user_lib):
    m = scenegen.terrain(cells=64, amplitude=0.2)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    rays_np = scenegen.random_rays(50_000, [-1.0, -0.3, -1.0], [1.0, 0.3, 1.0], config=71)
    rays = device_tensor(rays_np)
    T = grt.grtGetDeviceTarget(gpu.handle, geom=g.handle)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(m.vertices, m.indices))
    S.build()
    _same_closest(_user(user_lib, T, rays, False), _library(gpu, rays, False, geom=g.handle), S, rays_np)
    assert np.array_equal(_user(user_lib, T, rays, True)[1] != NONE,
                          _library(gpu, rays, True, geom=g.handle)[1] != NONE)
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


def test_user_kernel_on_a_two_level_scene(gpu, user_lib):
    m = scenegen.terrain(cells=48, amplitude=0.2)
    fr = scenegen.random_frames(12, seed=5)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    sc = Scene(gpu, [g.handle] * 12, device_tensor(fr.packed())).build()
    lo, hi = scenegen.world_bounds([m], np.zeros(12, np.int32), fr)
    rays_np = scenegen.random_rays(60_000, lo, hi, config=72)
    rays = device_tensor(rays_np)
    T = grt.grtGetDeviceTarget(gpu.handle, scene=sc.handle)
    S = oracle.Scene()
    gi = S.add_mesh(m.vertices, m.indices)
    for f in fr.packed():
        S.add_instance(gi, f)
    S.build()
    _same_closest(_user(user_lib, T, rays, False), _library(gpu, rays, False, scene=sc.handle), S, rays_np)
    assert np.array_equal(_user(user_lib, T, rays, True)[1] != NONE,
                          _library(gpu, rays, True, scene=sc.handle)[1] != NONE)


def test_user_kernel_with_custom_spheres(gpu, user_lib):
    s = scenegen.spheres(20_000, half=10.0, rmin=0.01, rmax=0.5, config=73)
    g = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s))).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    rays_np = scenegen.random_rays(40_000, [-10.0] * 3, [10.0] * 3, config=74)
    rays_np[1::2, 7] = 2.5
    rays = device_tensor(rays_np)
    T = grt.grtGetDeviceTarget(gpu.handle, geom=g.handle, table=table.handle)
    S = oracle.Scene()
    S.add_instance(S.add_spheres(s))
    S.build()
    a = _user(user_lib, T, rays, False)
    _same_closest(a, _library(gpu, rays, False, geom=g.handle, table=table.handle), S, rays_np)
    assert (a[1] != NONE).sum() > 1000
    assert np.array_equal(_user(user_lib, T, rays, True)[1] != NONE,
                          _library(gpu, rays, True, geom=g.handle, table=table.handle)[1] != NONE)


def test_user_kernel_with_a_ray_mask(gpu, user_lib):
    m = scenegen.terrain(cells=32, amplitude=0.2)
    fr = scenegen.random_frames(10, seed=6)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    masks = [1 << (k % 4) for k in range(10)]
    sc = Scene(gpu, [g.handle] * 10, device_tensor(fr.packed()), masks=masks).build()
    lo, hi = scenegen.world_bounds([m], np.zeros(10, np.int32), fr)
    rays_np = scenegen.random_rays(40_000, lo, hi, config=75)
    rays = device_tensor(rays_np)
    T = grt.grtGetDeviceTarget(gpu.handle, scene=sc.handle)
    for ray_mask in (0x1, 0x6):
        for any_hit in (False, True):
            h = new_hits(rays.shape[0])
            assert user_lib.userTraceMaskedLaunch(ctypes.byref(T), rays.data_ptr(), rays.shape[0], h.data_ptr(),
                                                  int(any_hit), ray_mask,
                                                  torch.cuda.current_stream().cuda_stream) == 0
            torch.cuda.synchronize()
            a = hits_to_numpy(h)
            hl = new_hits(rays.shape[0])
            fn = grt.grtTraceAnyHit if any_hit else grt.grtTraceClosest
            fn(gpu.handle, sc.handle, None, rays, rays.shape[0], hl, None, grt.trace_options(ray_mask=ray_mask))
            torch.cuda.synchronize()
            b = hits_to_numpy(hl)
            assert np.array_equal(a[1] != NONE, b[1] != NONE)
            hit = a[1] != NONE
            assert all(masks[k] & ray_mask for k in np.unique(a[0][hit]).tolist())
            assert hit.sum() > 500


def test_user_kernel_all_hits(gpu, user_lib):
    """grt_device::AllHits in a user kernel returns exactly what grtTraceAllHits stores
    (the same walk), and reports the walk as done after its last hit."""
    m = scenegen.terrain(cells=32, amplitude=0.3)
    fr = scenegen.random_frames(8, seed=7)
    g = Geometry(gpu, vertices=device_tensor(m.vertices), indices=device_tensor(m.indices)).build()
    sc = Scene(gpu, [g.handle] * 8, device_tensor(fr.packed())).build()
    lo, hi = scenegen.world_bounds([m], np.zeros(8, np.int32), fr)
    rays_np = scenegen.random_rays(30_000, lo, hi, config=76)
    rays = device_tensor(rays_np)
    n, k = rays.shape[0], 8
    T = grt.grtGetDeviceTarget(gpu.handle, scene=sc.handle)
    hu, cu = new_hits(n * k), torch.empty(n, dtype=torch.int32, device="cuda")
    assert user_lib.userAllHitsLaunch(ctypes.byref(T), rays.data_ptr(), n, hu.data_ptr(), k, cu.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream) == 0
    hl, cl = new_hits(n * k), torch.empty(n, dtype=torch.int32, device="cuda")
    grt.grtTraceAllHits(gpu.handle, sc.handle, None, rays, n, hl, k, cl)
    torch.cuda.synchronize()
    assert torch.equal(cu, cl) and torch.equal(hu, hl)
    assert (cl >= 2).sum().item() > 100
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS


# ---------------------------------------------------------------- user intersection code (Sec. 7.4, 7.6)
DISC_GRAZE = 1e-4  # float32 user code: |rho^2 / r^2 - 1| of a rim crossing within this is exempt


def _disc_data(m, seed):
    rng = np.random.default_rng(seed)
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    c = rng.uniform(-3, 3, (m, 3))
    r = rng.uniform(0.05, 0.6, m)
    d = np.zeros((m, 8), np.float32)
    d[:, 0:3], d[:, 3], d[:, 4:7] = c, r, n
    # AABB-list input: c +- r sqrt(1 - n_a^2), widened by 1e-6 relative and rounded outward
    e = d[:, 3:4].astype(np.float64) * np.sqrt(np.maximum(0.0, 1.0 - d[:, 4:7].astype(np.float64) ** 2))
    lo = d[:, 0:3].astype(np.float64) - e
    hi = d[:, 0:3].astype(np.float64) + e
    pad = 1e-6 * (np.abs(lo) + np.abs(hi)) + 1e-7
    boxes = np.concatenate([np.nextafter((lo - pad).astype(np.float32), -np.inf),
                            np.nextafter((hi + pad).astype(np.float32), np.inf)], axis=1).astype(np.float32)
    return d, boxes


def _exempt_disc(report, S, rays, got=None, discs=None, disc_instances=()):
    """Failures of compare_closest / compare_any that graze a disc's rim move to the
    grazing exemptions (the user's float32 disc test decides them). A disc hit's t is
    the user's float32 ((c - o).n) / (d.n) on the object-space ray: its error is about
    13u t / |cos| (cos of the angle between that ray and the disc's normal) plus, from
    the rounded plane distance and origin, u (|c| + |o|) / (|d| |cos|), which dominates
    for rays born next to a disc (t of 1e-6). Disc hits are held to (1e-5 + 32u / |cos|) t
    + 16u (|c| + |o|) / (|d| |cos|); library primitives keep the plain 1e-5 relative
    (their t is refined in FP64)."""
    keep = []
    for i in report.failures:
        if S.min_disc_margin(rays[i]) <= DISC_GRAZE:
            report.exempt_graze.append(i)
        else:
            keep.append(i)
    report.failures = keep
    if got is not None:
        gi, gp, gt, _, _ = got
        bad = []
        for i in report.t_bad:
            inst = int(gi[i])
            if inst not in disc_instances:
                bad.append(i)
                continue
            _, inv = S.instance_frames(inst)
            d = inv[:, :3] @ rays[i, 4:7].astype(np.float64)
            o = inv[:, :3] @ rays[i, 0:3].astype(np.float64) + inv[:, 3]
            nrm = discs[int(gp[i]), 4:7].astype(np.float64)
            cos = max(abs(d @ nrm) / (np.linalg.norm(d) * np.linalg.norm(nrm)), 1e-30)
            u = 2.0 ** -24
            ok, t_ref, _, _ = S.intersect_prim(rays[i], inst, int(gp[i]))
            tol = (1e-5 + 32 * u / cos) * abs(t_ref) + 16 * u * (np.linalg.norm(discs[int(gp[i]), 0:3]) +
                                                                 np.linalg.norm(o)) / (np.linalg.norm(d) * cos)
            if not (ok and abs(float(gt[i]) - t_ref) <= tol):
                bad.append(i)
        report.t_bad = bad
    return report


def test_user_disc_intersector_and_filter(gpu, user_lib):
    """A user kernel traces a two-level scene of two disc instances (an AABB-list geometry
    whose function-table entry names a user intersector, GRT_INTERSECT_USER) and a
    terrain instance, with the intersection code passed as a functor to
    grt_device::traceClosest / traceAnyHit / AllHits. Closest and any hit against the
    oracle's FP64 discs; ray type 1 adds a user filter (even primitive IDs stand) against
    the oracle with those primitives filtered; the payload counts intersector calls; the
    library's own traces reject a table that names user functions."""
    from parity import compare_any, compare_closest

    L = user_lib
    L.userTraceDiscsLaunch.argtypes = [ctypes.POINTER(grt.grtDeviceTarget), ctypes.c_void_p, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.userTraceDiscsLaunch.restype = ctypes.c_int
    L.userAllHitsDiscsLaunch.argtypes = [ctypes.POINTER(grt.grtDeviceTarget), ctypes.c_void_p, ctypes.c_uint32,
                                         ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    L.userAllHitsDiscsLaunch.restype = ctypes.c_int
    discs, boxes = _disc_data(1500, 31)
    dd = device_tensor(discs)
    gd = Geometry(gpu, boxes=device_tensor(boxes)).build()
    mesh = scenegen.terrain(cells=24, amplitude=0.2)
    gm = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices), geom_type=1).build()
    frames = np.array([[0, 0, 0, 1, 1, 1, 1, 0, 0, 0], [0.3, -0.2, 0.1, 0.93, 0.8, 1.4, 1.1, 5, 1, -2],
                       [0.1, 0.7, 0.0, 0.7, 2, 2, 2, -4, -1, 2]], np.float32)
    sc = Scene(gpu, [gd.handle, gd.handle, gm.handle], device_tensor(frames)).build()
    table = FuncTable(gpu, num_geom_types=2, num_ray_types=2)
    table.set(0, 0, grt.GRT_INTERSECT_USER, dd)
    table.set(0, 1, grt.GRT_INTERSECT_USER, dd, grt.GRT_FILTER_USER, None)
    S = oracle.Scene()
    og = S.add_discs(discs)
    om = S.add_mesh(mesh.vertices, mesh.indices)
    for g, f in zip((og, og, om), frames):
        S.add_instance(g, f)
    S.build()
    F = oracle.Scene()  # ray type 1: only the even discs stand
    fg = F.add_discs(discs)
    even = np.arange(0, discs.shape[0], 2)
    words = np.zeros((discs.shape[0] + 31) // 32, np.uint32)
    np.bitwise_or.at(words, even >> 5, (np.uint32(1) << (even & 31).astype(np.uint32)))
    F.set_prim_filter(fg, words)
    fm = F.add_mesh(mesh.vertices, mesh.indices)
    for g, f in zip((fg, fg, fm), frames):
        F.add_instance(g, f)
    F.build()
    rays_np = scenegen.random_rays(40_000, [-7] * 3, [7] * 3, config=99)
    rays_np[::4, 7] = 2.0
    rays = device_tensor(rays_np)
    n = rays_np.shape[0]
    for ray_type, ref_scene in ((0, S), (1, F)):
        target = grt.grtGetDeviceTarget(gpu.handle, scene=sc.handle, table=table.handle, ray_type=ray_type)
        ref = ref_scene.trace(rays_np)
        got = {}
        for any_hit in (0, 1):
            h, calls = new_hits(n), torch.zeros(n, dtype=torch.int32, device="cuda")
            assert L.userTraceDiscsLaunch(ctypes.byref(target), rays.data_ptr(), n, h.data_ptr(), any_hit,
                                          calls.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
            torch.cuda.synchronize()
            got[any_hit] = (hits_to_numpy(h), calls.cpu().numpy())
        rep = _exempt_disc(compare_closest(got[0][0], ref, ref_scene, rays_np, extent=14.0), ref_scene, rays_np,
                           got[0][0], discs, (0, 1))
        rep.check()
        disc_hits = (got[0][0][1] != NONE) & (got[0][0][0] < 2)
        assert disc_hits.sum() > 2000, rep.summary()
        assert np.all(got[0][1][disc_hits] >= 1) and got[0][1].sum() > disc_hits.sum()
        _exempt_disc(compare_any(got[1][0][1], ref, ref_scene, rays_np, extent=14.0), ref_scene, rays_np).check()
        if ray_type == 1:
            assert np.all(got[0][0][1][disc_hits] % 2 == 0)
    # every hit through AllHits with the functor, ray type 0
    target = grt.grtGetDeviceTarget(gpu.handle, scene=sc.handle, table=table.handle, ray_type=0)
    m, k = 4000, 6
    sub = rays_np[:m]
    hits_all, counts = new_hits(m * k), torch.empty(m, dtype=torch.int32, device="cuda")
    assert L.userAllHitsDiscsLaunch(ctypes.byref(target), device_tensor(sub).data_ptr(), m, hits_all.data_ptr(), k,
                                    counts.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    gi, gp, _, _, _ = hits_to_numpy(hits_all)
    cnt = counts.cpu().numpy()
    ri, rp, _, _, _, rc = S.all_hits(sub, k)
    checked = 0
    for i in range(m):
        if S.min_disc_margin(sub[i]) <= DISC_GRAZE or S.min_edge_margin(sub[i]) <= 1e-6:
            continue
        assert cnt[i] == rc[i], i
        if cnt[i] <= k:  # the same set of (instance, primitive) pairs
            j = int(cnt[i])
            assert set(zip(gi[i * k:i * k + j].tolist(), gp[i * k:i * k + j].tolist())) == \
                set(zip(ri[i, :j].tolist(), rp[i, :j].tolist())), i
        checked += 1
    assert checked > 0.99 * m and cnt.sum() > 1000
    # libgrt.so's own queries cannot run user code: they reject the table
    for fn in (grt.grtTraceClosest, grt.grtTraceAnyHit):
        with pytest.raises(grt.GrtError) as e:
            fn(gpu.handle, sc.handle, None, rays, n, new_hits(n), table.handle)
        assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    # a table whose user entries were replaced by built-in ones is accepted again
    plain = FuncTable(gpu, num_geom_types=2, num_ray_types=1)
    plain.set(0, 0, grt.GRT_INTERSECT_USER, dd)
    plain.set(0, 0, grt.GRT_INTERSECT_NONE, None)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, rays, n, new_hits(n), plain.handle)
    torch.cuda.synchronize()
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS
    for obj in (plain, table, sc, gm, gd):
        obj.close()
