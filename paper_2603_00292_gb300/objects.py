"""Object-style helpers over the C-ABI binding: they own the torch device buffers that
the C calls need (temporary build buffers, instance arrays) and forward to the
functions of the same names. No computation happens here."""
from __future__ import annotations

import numpy as np
import torch

from . import (GRT_BUILD_OPERATION_BUILD, GRT_INSTANCE_GEOMETRY, aabb_list_input, batch_scene, build_options,
               grtBatchBuildTrace, grtBuildGeometry, grtBuildScene, grtCreateBatch, grtCreateContext,
               grtCreateFuncTable, grtCreateGeometry, grtCreateScene, grtDestroyBatch, grtDestroyContext,
               grtDestroyFuncTable, grtDestroyGeometry, grtDestroyScene, grtGetBatchInfo, grtGetBvhInfo,
               grtGetGeometryBuildTemporaryBufferSize, grtGetSceneBuildTemporaryBufferSize, grtSetFuncTable,
               scene_input, triangle_mesh_input)


def device_tensor(a: np.ndarray, device="cuda") -> torch.Tensor:
    """Copy a numpy array to the device (unsigned integer arrays travel as the signed
    type of the same width: the bits are what the C calls read)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(device)


def empty_bytes(nbytes: int, device="cuda") -> torch.Tensor:
    """A 256-byte aligned device buffer of at least nbytes."""
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


class Context:
    def __init__(self, device: int = 0):
        self.device = device
        self.handle = grtCreateContext(device)

    def close(self):
        if self.handle:
            grtDestroyContext(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Geometry:
    """A bottom-level BVH over an indexed triangle mesh or an AABB list. build_flags:
    GRT_BUILD_PREFER_FAST (linear BVH), _BALANCED or _HIGH_QUALITY (PLOC clustering) or
    GRT_BUILD_CLUSTER_SUBTREES, optionally ORed with GRT_BUILD_QUANTIZED_NODES or
    GRT_BUILD_WIDE8_NODES (the node format traversal reads) and GRT_BUILD_SPLIT_TRIANGLES
    (spatial splits; split_factor = extra references per triangle, 0 = 0.5)."""

    def __init__(self, ctx: Context, *, vertices=None, indices=None, boxes=None, geom_type: int = 0,
                 morton_bits: int = 0, temp: torch.Tensor | None = None, vertex_count: int | None = None,
                 build_flags: int = 0, split_factor: float = 0.0):
        self.ctx = ctx
        if boxes is not None:
            self.boxes = boxes
            self.input = aabb_list_input(boxes, geom_type=geom_type)
        else:
            self.vertices, self.indices = vertices, indices
            self.input = triangle_mesh_input(indices, vertices, vertex_count=vertex_count, geom_type=geom_type)
        self.options = build_options(morton_bits, build_flags, split_factor)
        self.temp_bytes = grtGetGeometryBuildTemporaryBufferSize(ctx.handle, self.input, self.options)
        self.temp = temp if temp is not None and temp.numel() >= self.temp_bytes else empty_bytes(self.temp_bytes)
        self.handle = grtCreateGeometry(ctx.handle, self.input, self.options)

    def build(self, stream=None, op: int = GRT_BUILD_OPERATION_BUILD):
        grtBuildGeometry(self.ctx.handle, op, self.input, self.options, self.temp, stream, self.handle)
        return self

    def info(self):
        return grtGetBvhInfo(self.ctx.handle, geom=self.handle)

    def close(self):
        if self.handle:
            grtDestroyGeometry(self.ctx.handle, self.handle)
            self.handle = None


def instance_records(geometry_handles, masks=None) -> np.ndarray:
    """16-byte grtInstance records {type, mask, geometry} as raw bytes (masks: one 32-bit
    visibility mask per instance, 0 = all bits; default all bits)."""
    n = len(geometry_handles)
    rec = np.zeros(n, dtype=np.dtype([("type", "<u4"), ("mask", "<u4"), ("geometry", "<u8")]))
    rec["type"] = GRT_INSTANCE_GEOMETRY
    if masks is not None:
        rec["mask"] = np.asarray(masks, dtype=np.uint32)
    rec["geometry"] = np.asarray(geometry_handles, dtype=np.uint64)
    return rec.view(np.uint8)


class Scene:
    """A top-level BVH over instances of geometries with SRT frames (float32 (I,10):
    quaternion xyzw, scale xyz, translation xyz). build_flags: GRT_BUILD_WIDE8_NODES gives
    the top level 8-wide nodes (other bits are ignored for scenes)."""

    def __init__(self, ctx: Context, geometry_handles, frames: torch.Tensor, morton_bits: int = 0, masks=None,
                 build_flags: int = 0):
        self.ctx = ctx
        self.instances = device_tensor(instance_records(geometry_handles, masks))
        self.frames = frames
        self.input = scene_input(self.instances, self.frames, count=len(geometry_handles))
        self.options = build_options(morton_bits, build_flags)
        self.temp_bytes = grtGetSceneBuildTemporaryBufferSize(ctx.handle, self.input, self.options)
        self.temp = empty_bytes(self.temp_bytes)
        self.handle = grtCreateScene(ctx.handle, self.input, self.options)

    def build(self, stream=None, op: int = GRT_BUILD_OPERATION_BUILD):
        grtBuildScene(self.ctx.handle, op, self.input, self.options, self.temp, stream, self.handle)
        return self

    def info(self):
        return grtGetBvhInfo(self.ctx.handle, scene=self.handle)

    def close(self):
        if self.handle:
            grtDestroyScene(self.ctx.handle, self.handle)
            self.handle = None


class Batch:
    """Many triangle geometries, each with its own rays, built and traced (closest hit)
    in one persistent launch. `scenes` is a list of (Geometry, rays (R,8), hits (R,5));
    the tensors are kept alive with the batch."""

    def __init__(self, ctx: Context, scenes, options=None):
        self.ctx = ctx
        self.scenes = list(scenes)
        recs = [batch_scene(g.handle, g.input, rays, int(rays.shape[0]), hits) for g, rays, hits in self.scenes]
        self.options = options
        self.handle = grtCreateBatch(ctx.handle, recs, options)

    def run(self, stream=None):
        grtBatchBuildTrace(self.ctx.handle, self.handle, stream)
        return self

    def info(self):
        return grtGetBatchInfo(self.ctx.handle, self.handle)

    def close(self):
        if self.handle:
            grtDestroyBatch(self.ctx.handle, self.handle)
            self.handle = None


class FuncTable:
    def __init__(self, ctx: Context, num_geom_types: int = 1, num_ray_types: int = 1):
        self.ctx = ctx
        self.handle = grtCreateFuncTable(ctx.handle, num_geom_types, num_ray_types)
        self._keep = []

    def set(self, geom_type: int, ray_type: int, func: int, data, filter_func: int = 0, filter_data=None):
        self._keep += [data, filter_data]
        grtSetFuncTable(self.ctx.handle, self.handle, geom_type, ray_type, func, data, filter_func, filter_data)

    def close(self):
        if self.handle:
            grtDestroyFuncTable(self.ctx.handle, self.handle)
            self.handle = None


def hits_to_numpy(hits: torch.Tensor):
    """Split a (n,5) 32-bit hit tensor into (inst, prim, t, u, v) numpy arrays."""
    h = hits.detach().cpu().contiguous().view(torch.int32).numpy().view(np.uint32).reshape(-1, 5)
    f = h.view(np.float32)
    return h[:, 0].copy(), h[:, 1].copy(), f[:, 2].copy(), f[:, 3].copy(), f[:, 4].copy()


def new_hits(n: int, device="cuda") -> torch.Tensor:
    return torch.empty((n, 5), dtype=torch.int32, device=device)


def new_rays(n: int, device="cuda") -> torch.Tensor:
    return torch.empty((n, 8), dtype=torch.float32, device=device)


class _DeviceArray:
    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, nbytes: int) -> torch.Tensor:
    """A uint8 torch view of nbytes of device memory at `ptr` (no copy)."""
    return torch.as_tensor(_DeviceArray(ptr, nbytes), device="cuda")


def read_device(ptr: int, nbytes: int, dtype) -> np.ndarray:
    """Host copy of device memory at `ptr` viewed as `dtype`."""
    if nbytes == 0:
        return np.zeros(0, dtype)
    torch.cuda.synchronize()
    return device_view(ptr, nbytes).cpu().numpy().view(dtype).copy()
