"""grtTraceClosestNoAlloc: the closest-hit entry point for callers that cannot allocate
device memory (stream capture, externally owned memory, no device-wide sync allowed).

It must return exactly what grtTraceClosest returns, call after call, using only the
library's static scratch array. This file is named to be collected last, so that a
run stopping at its first failure has run every other test already."""
import numpy as np
import pytest
import torch

import paper_2603_00292_gb300 as grt
import scenegen
from paper_2603_00292_gb300.objects import (FuncTable, Geometry, Scene, device_tensor, hits_to_numpy, new_hits)

pytestmark = pytest.mark.gpu


def _rays(n, targets, seed):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-12, 12, (n, 3))
    t = targets[rng.integers(0, len(targets), n)] + rng.normal(0, 0.8, (n, 3))
    d = t - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = d
    r[:, 7] = np.inf
    r[::4, 7] = 5.0
    return r


def test_no_alloc_closest_hit_matches_the_allocating_entry_point(gpu):
    mesh = scenegen.terrain(cells=48, amplitude=0.2)
    fr = scenegen.random_frames(10, config=70)
    g = Geometry(gpu, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    s = scenegen.spheres(4000, half=1.0, rmin=0.01, rmax=0.2, config=71)
    gs = Geometry(gpu, boxes=device_tensor(scenegen.sphere_aabbs(s))).build()
    table = FuncTable(gpu)
    table.set(0, 0, grt.GRT_INTERSECT_SPHERE, device_tensor(s))
    frames = np.concatenate([fr.packed(), np.array([[0, 0, 0, 1, 1.5, 1.5, 1.5, 2, -1, 3]], np.float32)])
    sc = Scene(gpu, [g.handle] * 10 + [gs.handle], device_tensor(frames)).build()
    targets = np.concatenate([fr.translation.astype(np.float64), [[2, -1, 3]]])
    n = 150_000
    rays = device_tensor(_rays(n, targets, 72))

    ref = new_hits(n)
    grt.grtTraceClosest(gpu.handle, sc.handle, None, rays, n, ref, table.handle)
    torch.cuda.synchronize()
    want = hits_to_numpy(ref)
    assert (want[1] != grt.GRT_INVALID_ID).sum() > 10_000

    for call in range(2):  # two calls in a row share the static scratch
        got_t = new_hits(n)
        got_t.fill_(7)
        grt.grtTraceClosestNoAlloc(gpu.handle, sc.handle, None, rays, n, got_t, table.handle)
        torch.cuda.synchronize()
        got = hits_to_numpy(got_t)
        for a, b in zip(want, got):
            assert np.array_equal(a, b), f"call {call} differs"
    assert grt.grtGetLastDeviceError(gpu.handle) == grt.GRT_SUCCESS

    # a geometry traced directly, with a small shared stack that spills often
    opts = grt.trace_options(shared_depth=2, global_depth=64)
    ref2 = new_hits(n)
    grt.grtTraceClosest(gpu.handle, None, gs.handle, rays, n, ref2, table.handle, opts)
    got2 = new_hits(n)
    grt.grtTraceClosestNoAlloc(gpu.handle, None, gs.handle, rays, n, got2, table.handle, opts)
    torch.cuda.synchronize()
    assert torch.equal(ref2, got2)

    # a stack that cannot fit even one block is rejected, not truncated
    with pytest.raises(grt.GrtError) as err:
        grt.grtTraceClosestNoAlloc(gpu.handle, sc.handle, None, rays, n, got2, table.handle,
                                   grt.trace_options(block_size=256, global_depth=4096))
    assert err.value.code == grt.GRT_ERROR_INVALID_PARAMETER


def test_no_alloc_on_a_fresh_context_allocates_nothing(gpu):
    """On a context that has never run an allocating trace, the entry point leaves the
    device's free memory unchanged (one earlier call caches the scratch array's address
    and loads the kernels), while grtTraceClosest on the same context then grows the
    context's global-stack area by cudaMalloc: the measurement sees that allocation. A
    call with no rays succeeds and leaves the hit buffer as it was; a call with another
    device current is rejected (on machines with more than one device)."""
    from paper_2603_00292_gb300.objects import Context

    ctx = Context(0)
    mesh = scenegen.terrain(cells=64, amplitude=0.2)
    g = Geometry(ctx, vertices=device_tensor(mesh.vertices), indices=device_tensor(mesh.indices)).build()
    n = 400_000
    rng = np.random.default_rng(73)
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = np.stack([rng.uniform(-1, 1, n), np.full(n, 1.5), rng.uniform(-1, 1, n)], axis=1)
    d = np.stack([rng.normal(0, 0.3, n), -np.ones(n), rng.normal(0, 0.3, n)], axis=1)
    r[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    r[:, 7] = np.inf
    rays = device_tensor(r)
    got = [new_hits(n) for _ in range(3)]
    ref = new_hits(n)
    grt.grtTraceClosestNoAlloc(ctx.handle, None, g.handle, rays, n, got[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for h in got[1:]:
        grt.grtTraceClosestNoAlloc(ctx.handle, None, g.handle, rays, n, h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"the allocation-free entry point changed free device memory by {free0 - free1} bytes"
    grt.grtTraceClosest(ctx.handle, None, g.handle, rays, n, ref)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 < free1, "the allocating entry point's global stack should show up as less free memory"
    for h in got:
        assert torch.equal(h, ref)
    assert (hits_to_numpy(ref)[1] != grt.GRT_INVALID_ID).sum() > n // 2
    # no rays: success, hit buffer untouched
    untouched = new_hits(4)
    untouched.fill_(-5)
    grt.grtTraceClosestNoAlloc(ctx.handle, None, g.handle, rays, 0, untouched)
    torch.cuda.synchronize()
    assert bool((untouched == -5).all())
    if torch.cuda.device_count() > 1:
        with torch.cuda.device(1):
            with pytest.raises(grt.GrtError) as err:
                grt.grtTraceClosestNoAlloc(ctx.handle, None, g.handle, rays, n, got[1])
        assert err.value.code == grt.GRT_ERROR_INVALID_PARAMETER
    assert grt.grtGetLastDeviceError(ctx.handle) == grt.GRT_SUCCESS
    g.close()
    ctx.close()
