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
