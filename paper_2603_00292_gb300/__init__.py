"""Python binding of libgrt (include/grt.h): GPU BVH build and ray traversal on sm_103a.

Argument marshalling only. Every function below calls the C function of the same
name in libgrt.so, which runs the work in hand-written CUDA kernels; device buffers
are passed as addresses (torch tensors' data_ptr()) and streams as cudaStream_t
handles. There is no CPU fallback: loading fails loudly when the library has not
been built (see build.py) or when no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrt.so")

GRT_API_VERSION = 1
GRT_SUCCESS = 0
GRT_ERROR_INVALID_PARAMETER = 1
GRT_ERROR_OUT_OF_MEMORY = 2
GRT_ERROR_INVALID_API_VERSION = 3
GRT_ERROR_NOT_BUILT = 4
GRT_ERROR_STACK_OVERFLOW = 5
GRT_ERROR_STEP_LIMIT = 6
GRT_ERROR_TIMEOUT = 7
GRT_ERROR_CUDA = 8
GRT_ERROR_INTERNAL = 9
ERROR_NAMES = {0: "SUCCESS", 1: "INVALID_PARAMETER", 2: "OUT_OF_MEMORY", 3: "INVALID_API_VERSION", 4: "NOT_BUILT",
               5: "STACK_OVERFLOW", 6: "STEP_LIMIT", 7: "TIMEOUT", 8: "CUDA", 9: "INTERNAL"}

GRT_PRIMITIVE_TRIANGLE_MESH = 0
GRT_PRIMITIVE_AABB_LIST = 1
GRT_BUILD_OPERATION_BUILD = 0
GRT_BUILD_OPERATION_UPDATE = 1
GRT_BUILD_PREFER_FAST = 0          # linear BVH (Morton order, Karras emission)
GRT_BUILD_PREFER_BALANCED = 1      # PLOC clustering, search radius 8
GRT_BUILD_PREFER_HIGH_QUALITY = 2  # PLOC clustering, search radius 32
GRT_BUILD_CLUSTER_SUBTREES = 3     # clustering inside the linear BVH's subtrees, one bottom-up pass
GRT_BUILD_QUANTIZED_NODES = 0x100  # ORed with a method: traversal reads 64-byte quantised 4-wide nodes
GRT_BUILD_WIDE8_NODES = 0x200      # ORed with a method: traversal reads 256-byte 8-wide nodes
GRT_BUILD_SPLIT_TRIANGLES = 0x400  # ORed with a method: spatial splits of triangles before the build
CLUSTER_CAP = 16                   # clusters a subtree passes up (the library's kClusterCap)
GRT_INSTANCE_GEOMETRY = 0
GRT_INTERSECT_NONE = 0
GRT_INTERSECT_SPHERE = 1
GRT_INTERSECT_USER = 0x100  # and above: user code, run only through grt_device.cuh functors
GRT_FILTER_NONE = 0
GRT_FILTER_PRIMITIVE_MASK = 1
GRT_FILTER_USER = 0x100
GRT_INVALID_ID = 0xFFFFFFFF
GRT_LOG_NONE, GRT_LOG_ERROR, GRT_LOG_WARN, GRT_LOG_INFO = 0, 1, 2, 4

RAY_BYTES = 32
HIT_BYTES = 20


class GrtError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where} failed: GRT_ERROR_{ERROR_NAMES.get(code, code)}")
        self.code = code


# ------------------------------------------------------------------ C structures
class grtContextCreationInput(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32)]


class grtTriangleMeshPrimitive(ctypes.Structure):
    _fields_ = [("triangleCount", ctypes.c_uint32), ("triangleStride", ctypes.c_uint32),
                ("triangleIndices", ctypes.c_void_p), ("vertexCount", ctypes.c_uint32),
                ("vertexStride", ctypes.c_uint32), ("vertices", ctypes.c_void_p)]


class grtAABBListPrimitive(ctypes.Structure):
    _fields_ = [("aabbCount", ctypes.c_uint32), ("aabbStride", ctypes.c_uint32), ("aabbs", ctypes.c_void_p)]


class grtGeometryBuildInput(ctypes.Structure):
    _fields_ = [("type", ctypes.c_uint32), ("geomType", ctypes.c_uint32),
                ("triangleMesh", grtTriangleMeshPrimitive), ("aabbList", grtAABBListPrimitive)]


class grtBuildOptions(ctypes.Structure):
    _fields_ = [("buildFlags", ctypes.c_uint32), ("mortonBits", ctypes.c_uint32), ("splitFactor", ctypes.c_float)]


class grtSceneBuildInput(ctypes.Structure):
    _fields_ = [("instanceCount", ctypes.c_uint32), ("frameCount", ctypes.c_uint32),
                ("instances", ctypes.c_void_p), ("instanceFrames", ctypes.c_void_p)]


class grtFuncDataSet(ctypes.Structure):
    _fields_ = [("intersectFunc", ctypes.c_uint32), ("filterFunc", ctypes.c_uint32),
                ("intersectFuncData", ctypes.c_void_p), ("filterFuncData", ctypes.c_void_p)]


class grtTraceOptions(ctypes.Structure):
    _fields_ = [("rayType", ctypes.c_uint32), ("blockSize", ctypes.c_uint32),
                ("sharedStackDepth", ctypes.c_uint32), ("globalStackDepth", ctypes.c_uint32),
                ("compactThreshold", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("globalStack", ctypes.c_void_p), ("globalStackBytes", ctypes.c_size_t),
                ("rayMask", ctypes.c_uint32)]


class grtCamera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3)]


class grtBvhInfo(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("leaves", ctypes.c_void_p), ("parents", ctypes.c_void_p),
                ("nodeCount", ctypes.c_uint32), ("primCount", ctypes.c_uint32), ("primType", ctypes.c_uint32),
                ("mortonBits", ctypes.c_uint32), ("wideNodes", ctypes.c_void_p), ("quantNodes", ctypes.c_void_p),
                ("wide8Nodes", ctypes.c_void_p), ("leafCount", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class grtPathTraceInput(ctypes.Structure):
    _fields_ = [("albedo", ctypes.c_void_p), ("emission", ctypes.c_void_p), ("materialOffset", ctypes.c_void_p),
                ("lights", ctypes.c_void_p), ("lightCount", ctypes.c_uint32), ("maxDepth", ctypes.c_uint32),
                ("samplesPerPixel", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("sky", ctypes.c_float * 3), ("reserved2", ctypes.c_float)]


class grtDeviceTarget(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("leaves", ctypes.c_void_p), ("primToLeaf", ctypes.c_void_p),
                ("frames64", ctypes.c_void_p), ("frames32", ctypes.c_void_p), ("funcTable", ctypes.c_void_p),
                ("deviceError", ctypes.c_void_p), ("primType", ctypes.c_uint32), ("geomType", ctypes.c_uint32),
                ("primCount", ctypes.c_uint32), ("numGeomTypes", ctypes.c_uint32), ("rayType", ctypes.c_uint32),
                ("nodeFormat", ctypes.c_uint32)]


class grtBatchScene(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_void_p), ("input", grtGeometryBuildInput), ("rays", ctypes.c_void_p),
                ("rayCount", ctypes.c_uint32), ("hits", ctypes.c_void_p)]


class grtBatchOptions(ctypes.Structure):
    _fields_ = [("blockSize", ctypes.c_uint32), ("sharedStackDepth", ctypes.c_uint32),
                ("globalStackDepth", ctypes.c_uint32), ("compactThreshold", ctypes.c_float),
                ("smallScenePrims", ctypes.c_uint32), ("sortChunkTiles", ctypes.c_uint32),
                ("buildChunk", ctypes.c_uint32), ("traceChunk", ctypes.c_uint32), ("sceneGroup", ctypes.c_uint32),
                ("waitLimitMs", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class grtBatchInfo(ctypes.Structure):
    _fields_ = [("sceneCount", ctypes.c_uint32), ("itemCount", ctypes.c_uint32), ("smallScenes", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("blockSize", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("deviceBytes", ctypes.c_size_t)]


GRT_BATCH_FLAG_GRAPH = 1
GRT_BATCH_FLAG_PROFILE = 2
GRT_BATCH_FLAG_TEST_EXPIRE_WAIT = 4


class grtBatchItemRecord(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_uint32), ("phase", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("sm", ctypes.c_uint32), ("startNs", ctypes.c_uint64), ("readyNs", ctypes.c_uint64),
                ("endNs", ctypes.c_uint64)]

# ------------------------------------------------------------------ loading
_lib = None

_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_SIGS = {
    "grtCreateContext": [_U32, ctypes.POINTER(grtContextCreationInput), ctypes.POINTER(_P)],
    "grtDestroyContext": [_P],
    "grtSetLogLevel": [_U32],
    "grtGetLastDeviceError": [_P, _P, ctypes.POINTER(ctypes.c_int)],
    "grtGetGeometryBuildTemporaryBufferSize": [_P, ctypes.POINTER(grtGeometryBuildInput),
                                               ctypes.POINTER(grtBuildOptions), ctypes.POINTER(ctypes.c_size_t)],
    "grtCreateGeometry": [_P, ctypes.POINTER(grtGeometryBuildInput), ctypes.POINTER(grtBuildOptions),
                          ctypes.POINTER(_P)],
    "grtBuildGeometry": [_P, _U32, ctypes.POINTER(grtGeometryBuildInput), ctypes.POINTER(grtBuildOptions), _P, _P,
                         _P],
    "grtDestroyGeometry": [_P, _P],
    "grtGetSceneBuildTemporaryBufferSize": [_P, ctypes.POINTER(grtSceneBuildInput), ctypes.POINTER(grtBuildOptions),
                                            ctypes.POINTER(ctypes.c_size_t)],
    "grtCreateScene": [_P, ctypes.POINTER(grtSceneBuildInput), ctypes.POINTER(grtBuildOptions), ctypes.POINTER(_P)],
    "grtBuildScene": [_P, _U32, ctypes.POINTER(grtSceneBuildInput), ctypes.POINTER(grtBuildOptions), _P, _P, _P],
    "grtDestroyScene": [_P, _P],
    "grtCreateFuncTable": [_P, _U32, _U32, ctypes.POINTER(_P)],
    "grtSetFuncTable": [_P, _P, _U32, _U32, grtFuncDataSet],
    "grtDestroyFuncTable": [_P, _P],
    "grtGetTraceGlobalStackSize": [_P, ctypes.POINTER(grtTraceOptions), ctypes.POINTER(ctypes.c_size_t)],
    "grtTraceClosest": [_P, _P, _P, _P, _U32, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtTraceAnyHit": [_P, _P, _P, _P, _U32, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtTraceClosestNoAlloc": [_P, _P, _P, _P, _U32, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtTraceAllHits": [_P, _P, _P, _P, _U32, _P, _U32, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtGetPathTraceWorkspaceSize": [_U32, ctypes.POINTER(ctypes.c_size_t)],
    "grtPathTrace": [_P, _P, _P, _U32, ctypes.POINTER(grtPathTraceInput), _P, _P, ctypes.POINTER(grtTraceOptions),
                     _P],
    "grtGenerateCameraRays": [_P, ctypes.POINTER(grtCamera), _U32, _U32, _P, _P],
    "grtGenerateUniformRays": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_uint64,
                               _U32, ctypes.c_float, ctypes.c_float, _P, _P],
    "grtGenerateAORays": [_P, _P, _P, _P, _U32, _U32, ctypes.c_uint64, ctypes.c_float, _P, _P],
    "grtTraceAmbientOcclusion": [_P, _P, _P, _P, _U32, _U32, ctypes.c_uint64, ctypes.c_float, _P,
                                 ctypes.POINTER(grtTraceOptions), _P],
    "grtGetBvhInfo": [_P, _P, _P, ctypes.POINTER(grtBvhInfo)],
    "grtGetBuildTemporaryLayout": [_U32, _U32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_size_t)],
    "grtShadeLambert": [_P, _P, _P, _P, _U32, _P, _P, _P, _P, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtShadeLambertBackward": [_P, _P, _P, _P, _P, _U32, _P, _P, _P, _P, _P, _P, _P, _P,
                                ctypes.POINTER(grtTraceOptions), _P],
    "grtShadeLambertScene": [_P, _P, _P, _P, _U32, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(grtTraceOptions), _P],
    "grtShadeLambertSceneBackward": [_P, _P, _P, _P, _P, _U32, _P, _P, _P, _U32, _P, _P, _P, _P, _P, _P,
                                     ctypes.POINTER(grtTraceOptions), _P],
    "grtGetLaunchCount": [ctypes.POINTER(ctypes.c_uint64)],
    "grtGetTraceStatistics": [_P, _P, ctypes.c_void_p],
    "grtSortTemporaryBufferSize": [_U32, _U32, ctypes.POINTER(ctypes.c_size_t)],
    "grtSortPairs": [_P, _P, _P, _U32, _U32, _U32, _P, _P],
    "grtGetDeviceTarget": [_P, _P, _P, _P, _U32, ctypes.POINTER(grtDeviceTarget)],
    "grtCreateBatch": [_P, ctypes.POINTER(grtBatchScene), _U32, ctypes.POINTER(grtBatchOptions), ctypes.POINTER(_P)],
    "grtBatchBuildTrace": [_P, _P, _P],
    "grtGetBatchInfo": [_P, _P, ctypes.POINTER(grtBatchInfo)],
    "grtGetBatchProfile": [_P, _P, ctypes.c_void_p, _U32, ctypes.POINTER(_U32)],
    "grtDestroyBatch": [_P, _P],
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """dlopen libgrt.so and declare every signature (does not touch the GPU)."""
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2603_00292_gb300.build.build()")
    L = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return L


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def check(code: int, where: str = "grt call"):
    if code != GRT_SUCCESS:
        raise GrtError(code, where)


def _ptr(x) -> int | None:
    """Device address of a tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ thin wrappers (C names)
def grtCreateContext(device: int = 0) -> int:
    inp = grtContextCreationInput(device)
    out = _P()
    check(lib().grtCreateContext(GRT_API_VERSION, ctypes.byref(inp), ctypes.byref(out)), "grtCreateContext")
    return out.value


def grtDestroyContext(ctx: int):
    check(lib().grtDestroyContext(ctx), "grtDestroyContext")


def grtSetLogLevel(levels: int):
    check(lib().grtSetLogLevel(levels), "grtSetLogLevel")


def grtGetLastDeviceError(ctx: int, stream=None) -> int:
    err = ctypes.c_int()
    check(lib().grtGetLastDeviceError(ctx, _stream(stream), ctypes.byref(err)), "grtGetLastDeviceError")
    return err.value


def triangle_mesh_input(indices, vertices, triangle_count=None, vertex_count=None, triangle_stride=12,
                        vertex_stride=12, geom_type=0) -> grtGeometryBuildInput:
    """Build input of an indexed mesh from device tensors (uint32 (T,3) / float32 (V,3))."""
    tc = indices.shape[0] if triangle_count is None else triangle_count
    vc = vertices.shape[0] if vertex_count is None else vertex_count
    m = grtTriangleMeshPrimitive(tc, triangle_stride, _ptr(indices), vc, vertex_stride, _ptr(vertices))
    return grtGeometryBuildInput(GRT_PRIMITIVE_TRIANGLE_MESH, geom_type, m, grtAABBListPrimitive())


def aabb_list_input(boxes, count=None, stride=24, geom_type=0) -> grtGeometryBuildInput:
    """Build input of an AABB list from a device tensor float32 (N,6)."""
    n = boxes.shape[0] if count is None else count
    return grtGeometryBuildInput(GRT_PRIMITIVE_AABB_LIST, geom_type, grtTriangleMeshPrimitive(),
                                 grtAABBListPrimitive(n, stride, _ptr(boxes)))


def build_options(morton_bits: int = 0, flags: int = GRT_BUILD_PREFER_FAST, split_factor: float = 0.0) -> grtBuildOptions:
    return grtBuildOptions(flags, morton_bits, split_factor)


def grtGetGeometryBuildTemporaryBufferSize(ctx, inp, opts) -> int:
    sz = ctypes.c_size_t()
    check(lib().grtGetGeometryBuildTemporaryBufferSize(ctx, ctypes.byref(inp), ctypes.byref(opts), ctypes.byref(sz)),
          "grtGetGeometryBuildTemporaryBufferSize")
    return sz.value


def grtCreateGeometry(ctx, inp, opts) -> int:
    out = _P()
    check(lib().grtCreateGeometry(ctx, ctypes.byref(inp), ctypes.byref(opts), ctypes.byref(out)), "grtCreateGeometry")
    return out.value


def grtBuildGeometry(ctx, op, inp, opts, temp, stream, geom):
    check(lib().grtBuildGeometry(ctx, op, ctypes.byref(inp), ctypes.byref(opts), _ptr(temp), _stream(stream), geom),
          "grtBuildGeometry")


def grtDestroyGeometry(ctx, geom):
    check(lib().grtDestroyGeometry(ctx, geom), "grtDestroyGeometry")


def scene_input(instances, frames, count=None) -> grtSceneBuildInput:
    """instances: device tensor of 16-byte grtInstance records; frames: float32 (I,10)."""
    n = frames.shape[0] if count is None else count
    return grtSceneBuildInput(n, n, _ptr(instances), _ptr(frames))


def grtGetSceneBuildTemporaryBufferSize(ctx, inp, opts) -> int:
    sz = ctypes.c_size_t()
    check(lib().grtGetSceneBuildTemporaryBufferSize(ctx, ctypes.byref(inp), ctypes.byref(opts), ctypes.byref(sz)),
          "grtGetSceneBuildTemporaryBufferSize")
    return sz.value


def grtCreateScene(ctx, inp, opts) -> int:
    out = _P()
    check(lib().grtCreateScene(ctx, ctypes.byref(inp), ctypes.byref(opts), ctypes.byref(out)), "grtCreateScene")
    return out.value


def grtBuildScene(ctx, op, inp, opts, temp, stream, scene):
    check(lib().grtBuildScene(ctx, op, ctypes.byref(inp), ctypes.byref(opts), _ptr(temp), _stream(stream), scene),
          "grtBuildScene")


def grtDestroyScene(ctx, scene):
    check(lib().grtDestroyScene(ctx, scene), "grtDestroyScene")


def grtCreateFuncTable(ctx, num_geom_types: int, num_ray_types: int) -> int:
    out = _P()
    check(lib().grtCreateFuncTable(ctx, num_geom_types, num_ray_types, ctypes.byref(out)), "grtCreateFuncTable")
    return out.value


def grtSetFuncTable(ctx, table, geom_type: int, ray_type: int, func: int, data, filter_func: int = 0,
                    filter_data=None):
    check(lib().grtSetFuncTable(ctx, table, geom_type, ray_type,
                                grtFuncDataSet(func, filter_func, _ptr(data), _ptr(filter_data))),
          "grtSetFuncTable")


def grtDestroyFuncTable(ctx, table):
    check(lib().grtDestroyFuncTable(ctx, table), "grtDestroyFuncTable")


def trace_options(ray_type=0, block_size=0, shared_depth=0, global_depth=0, compact=0.0, global_stack=None,
                  global_stack_bytes=0, flags=0, ray_mask=0) -> grtTraceOptions:
    return grtTraceOptions(ray_type, block_size, shared_depth, global_depth, compact, flags, _ptr(global_stack),
                           global_stack_bytes, ray_mask)


def grtGetTraceGlobalStackSize(ctx, opts=None) -> int:
    sz = ctypes.c_size_t()
    check(lib().grtGetTraceGlobalStackSize(ctx, ctypes.byref(opts) if opts else None, ctypes.byref(sz)),
          "grtGetTraceGlobalStackSize")
    return sz.value


def grtTraceClosest(ctx, scene, geom, rays, count, hits, table=None, opts=None, stream=None):
    check(lib().grtTraceClosest(ctx, scene, geom, _ptr(rays), count, _ptr(hits), table,
                                ctypes.byref(opts) if opts else None, _stream(stream)), "grtTraceClosest")


def grtTraceAnyHit(ctx, scene, geom, rays, count, hits, table=None, opts=None, stream=None):
    check(lib().grtTraceAnyHit(ctx, scene, geom, _ptr(rays), count, _ptr(hits), table,
                               ctypes.byref(opts) if opts else None, _stream(stream)), "grtTraceAnyHit")


def grtTraceAllHits(ctx, scene, geom, rays, count, hits, max_hits, counts, table=None, opts=None, stream=None):
    """hits: (count * max_hits, 5) records; counts: uint32 device tensor of count entries."""
    check(lib().grtTraceAllHits(ctx, scene, geom, _ptr(rays), count, _ptr(hits), max_hits, _ptr(counts), table,
                                ctypes.byref(opts) if opts else None, _stream(stream)), "grtTraceAllHits")


def path_trace_input(albedo, emission, material_offset, lights, light_count, max_depth, spp, seed,
                     sky) -> grtPathTraceInput:
    """albedo / emission: device float32 (M, 3); material_offset: device uint32 per instance;
    lights: device uint32 (K, 2) (instance, primitive) pairs."""
    return grtPathTraceInput(_ptr(albedo), _ptr(emission), _ptr(material_offset), _ptr(lights), light_count,
                             max_depth, spp, 0, seed, (ctypes.c_float * 3)(*[float(x) for x in sky]), 0.0)


def grtGetPathTraceWorkspaceSize(count: int) -> int:
    sz = ctypes.c_size_t()
    check(lib().grtGetPathTraceWorkspaceSize(count, ctypes.byref(sz)), "grtGetPathTraceWorkspaceSize")
    return sz.value


def grtPathTrace(ctx, scene, rays, count, inp, workspace, radiance, opts=None, stream=None):
    check(lib().grtPathTrace(ctx, scene, _ptr(rays), count, ctypes.byref(inp), _ptr(workspace), _ptr(radiance),
                             ctypes.byref(opts) if opts else None, _stream(stream)), "grtPathTrace")


def grtTraceClosestNoAlloc(ctx, scene, geom, rays, count, hits, table=None, opts=None, stream=None):
    """Closest hit without any device allocation (scratch in the library's static
    16 MiB device array): for callers that cannot call cudaMalloc, e.g. during CUDA
    graph capture or under an allocator that owns all device memory."""
    check(lib().grtTraceClosestNoAlloc(ctx, scene, geom, _ptr(rays), count, _ptr(hits), table,
                                       ctypes.byref(opts) if opts else None, _stream(stream)),
          "grtTraceClosestNoAlloc")


def camera(origin, right, up) -> grtCamera:
    return grtCamera((ctypes.c_float * 3)(*origin), (ctypes.c_float * 3)(*right), (ctypes.c_float * 3)(*up))


def grtGenerateUniformRays(ctx, lo, hi, seed: int, count: int, rays, min_t: float = 0.0,
                           max_t: float = float("inf"), stream=None):
    f3 = ctypes.c_float * 3
    check(lib().grtGenerateUniformRays(ctx, f3(*[float(x) for x in lo]), f3(*[float(x) for x in hi]),
                                       ctypes.c_uint64(seed), count, ctypes.c_float(min_t), ctypes.c_float(max_t),
                                       _ptr(rays), _stream(stream)), "grtGenerateUniformRays")


def grtGenerateCameraRays(ctx, cam: grtCamera, width: int, height: int, rays, stream=None):
    check(lib().grtGenerateCameraRays(ctx, ctypes.byref(cam), width, height, _ptr(rays), _stream(stream)),
          "grtGenerateCameraRays")


def grtGenerateAORays(ctx, scene, primary_rays, primary_hits, pixels, spp, seed, length, ao_rays, stream=None):
    check(lib().grtGenerateAORays(ctx, scene, _ptr(primary_rays), _ptr(primary_hits), pixels, spp, seed, length,
                                  _ptr(ao_rays), _stream(stream)), "grtGenerateAORays")


def grtTraceAmbientOcclusion(ctx, scene, primary_rays, primary_hits, pixels, spp, seed, length, ao, opts=None,
                             stream=None):
    check(lib().grtTraceAmbientOcclusion(ctx, scene, _ptr(primary_rays), _ptr(primary_hits), pixels, spp, seed, length,
                                         _ptr(ao), ctypes.byref(opts) if opts else None, _stream(stream)),
          "grtTraceAmbientOcclusion")


def grtShadeLambert(ctx, geom, rays, hits, count, indices, positions, colours, light, image, visibility=None,
                    opts=None, stream=None):
    check(lib().grtShadeLambert(ctx, geom, _ptr(rays), _ptr(hits), count, _ptr(indices), _ptr(positions),
                                _ptr(colours), _ptr(light), _ptr(image), _ptr(visibility),
                                ctypes.byref(opts) if opts else None, _stream(stream)), "grtShadeLambert")


def grtShadeLambertBackward(ctx, geom, rays, hits, visibility, count, indices, positions, colours, light, grad_image,
                            grad_colours, grad_light, grad_positions, opts=None, stream=None):
    check(lib().grtShadeLambertBackward(ctx, geom, _ptr(rays), _ptr(hits), _ptr(visibility), count, _ptr(indices),
                                        _ptr(positions), _ptr(colours), _ptr(light), _ptr(grad_image),
                                        _ptr(grad_colours), _ptr(grad_light), _ptr(grad_positions),
                                        ctypes.byref(opts) if opts else None, _stream(stream)),
          "grtShadeLambertBackward")


def grtShadeLambertScene(ctx, scene, rays, hits, count, tri_offset, indices, positions, colours, light, image,
                         visibility=None, opts=None, stream=None):
    """tri_offset: device uint32, the first triangle of each instance ID's geometry in indices."""
    check(lib().grtShadeLambertScene(ctx, scene, _ptr(rays), _ptr(hits), count, _ptr(tri_offset), _ptr(indices),
                                     _ptr(positions), _ptr(colours), _ptr(light), _ptr(image), _ptr(visibility),
                                     ctypes.byref(opts) if opts else None, _stream(stream)), "grtShadeLambertScene")


def grtShadeLambertSceneBackward(ctx, scene, rays, hits, visibility, count, tri_offset, indices, positions,
                                 vertex_count, colours, light, grad_image, grad_colours, grad_light, grad_positions,
                                 opts=None, stream=None):
    check(lib().grtShadeLambertSceneBackward(ctx, scene, _ptr(rays), _ptr(hits), _ptr(visibility), count,
                                             _ptr(tri_offset), _ptr(indices), _ptr(positions), vertex_count,
                                             _ptr(colours), _ptr(light), _ptr(grad_image), _ptr(grad_colours),
                                             _ptr(grad_light), _ptr(grad_positions),
                                             ctypes.byref(opts) if opts else None, _stream(stream)),
          "grtShadeLambertSceneBackward")


def grtGetBvhInfo(ctx, geom=None, scene=None) -> grtBvhInfo:
    info = grtBvhInfo()
    check(lib().grtGetBvhInfo(ctx, geom, scene, ctypes.byref(info)), "grtGetBvhInfo")
    return info


def grtGetBuildTemporaryLayout(count: int, morton_bits: int):
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    check(lib().grtGetBuildTemporaryLayout(count, morton_bits, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "grtGetBuildTemporaryLayout")
    return a.value, b.value, c.value


GRT_TRACE_FLAG_COUNT = 1


class grtTraceStatistics(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_uint64), ("nodesVisited", ctypes.c_uint64), ("trianglesTested", ctypes.c_uint64),
                ("customTested", ctypes.c_uint64), ("instancesEntered", ctypes.c_uint64),
                ("fp64Tests", ctypes.c_uint64)]


def grtGetLaunchCount() -> int:
    v = ctypes.c_uint64()
    check(lib().grtGetLaunchCount(ctypes.byref(v)), "grtGetLaunchCount")
    return v.value


def grtGetTraceStatistics(ctx, stream=None) -> dict:
    st = grtTraceStatistics()
    check(lib().grtGetTraceStatistics(ctx, _stream(stream), ctypes.byref(st)), "grtGetTraceStatistics")
    return {name: getattr(st, name) for name, _ in grtTraceStatistics._fields_}


def grtSortTemporaryBufferSize(count: int, key_bits: int) -> int:
    sz = ctypes.c_size_t()
    check(lib().grtSortTemporaryBufferSize(count, key_bits, ctypes.byref(sz)), "grtSortTemporaryBufferSize")
    return sz.value


def grtSortPairs(ctx, keys, values, count, key_bits, significant_bits, temp, stream=None):
    check(lib().grtSortPairs(ctx, _ptr(keys), _ptr(values), count, key_bits, significant_bits, _ptr(temp),
                             _stream(stream)), "grtSortPairs")


def batch_options(block_size=0, shared_depth=0, global_depth=0, compact=0.0, small_scene_prims=0,
                  sort_chunk_tiles=0, build_chunk=0, trace_chunk=0, scene_group=0, wait_limit_ms=0, graph=False,
                  profile=False, test_expire_wait=False) -> grtBatchOptions:
    flags = ((GRT_BATCH_FLAG_GRAPH if graph else 0) | (GRT_BATCH_FLAG_PROFILE if profile else 0) |
             (GRT_BATCH_FLAG_TEST_EXPIRE_WAIT if test_expire_wait else 0))
    return grtBatchOptions(block_size, shared_depth, global_depth, compact, small_scene_prims, sort_chunk_tiles,
                           build_chunk, trace_chunk, scene_group, wait_limit_ms, flags)


def batch_scene(geometry: int, inp: grtGeometryBuildInput, rays, ray_count: int, hits) -> grtBatchScene:
    return grtBatchScene(geometry, inp, _ptr(rays), ray_count, _ptr(hits))


def grtCreateBatch(ctx, scenes, opts=None) -> int:
    arr = (grtBatchScene * max(1, len(scenes)))(*scenes)
    out = _P()
    check(lib().grtCreateBatch(ctx, arr, len(scenes), ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(out)), "grtCreateBatch")
    return out.value


def grtBatchBuildTrace(ctx, batch, stream=None):
    check(lib().grtBatchBuildTrace(ctx, batch, _stream(stream)), "grtBatchBuildTrace")


def grtGetBatchInfo(ctx, batch) -> grtBatchInfo:
    info = grtBatchInfo()
    check(lib().grtGetBatchInfo(ctx, batch, ctypes.byref(info)), "grtGetBatchInfo")
    return info


def grtDestroyBatch(ctx, batch):
    check(lib().grtDestroyBatch(ctx, batch), "grtDestroyBatch")


def grtGetBatchProfile(ctx, batch):
    """Item records of the batch's last launch as a numpy structured array (empty
    without GRT_BATCH_FLAG_PROFILE)."""
    import numpy as np

    count = _U32()
    check(lib().grtGetBatchProfile(ctx, batch, None, 0, ctypes.byref(count)), "grtGetBatchProfile")
    recs = (grtBatchItemRecord * max(1, count.value))()
    check(lib().grtGetBatchProfile(ctx, batch, recs, count.value, ctypes.byref(count)), "grtGetBatchProfile")
    dt = np.dtype([("scene", "<u4"), ("phase", "<u4"), ("chunk", "<u4"), ("sm", "<u4"), ("startNs", "<u8"),
                   ("readyNs", "<u8"), ("endNs", "<u8")])
    return np.frombuffer(bytes(recs), dtype=dt, count=count.value).copy()


def grtGetDeviceTarget(ctx, scene=None, geom=None, table=None, ray_type: int = 0) -> grtDeviceTarget:
    """The plain-data description of a built scene or geometry that user kernels pass to
    grt_device.cuh's traceClosest / traceAnyHit."""
    out = grtDeviceTarget()
    check(lib().grtGetDeviceTarget(ctx, scene, geom, table, ray_type, ctypes.byref(out)), "grtGetDeviceTarget")
    return out
