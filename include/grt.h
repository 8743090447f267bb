/*
 * grt.h - C ABI of a GB300 (sm_103a) BVH builder and ray tracer.
 *
 * The API follows the problem statement of "Ray Tracing using HIP" (Yoshimura, Eto,
 * Meister, Harada), Sec. 7: a context; bottom-level geometries built from an indexed
 * triangle mesh or from a list of AABBs of custom primitives (Sec. 7.2); a two-level
 * scene built from instances of geometries with SRT frames (Sec. 7.3); a function
 * table that maps (geometry type, ray type) to a custom intersection (Sec. 7.4); and
 * closest-hit / any-hit queries that write hit records (Sec. 7.5).
 *
 * Conventions for every call:
 *  - Every function returns grtError. GRT_SUCCESS is 0.
 *  - "device pointer" = an address in the current CUDA device's global memory owned
 *    by the CALLER (the paper's Sec. 7.1: all input buffers live on the device). The
 *    library never frees caller memory.
 *  - Objects (context, geometry, scene, function table) are owned by the library and
 *    released by the matching grtDestroy* call. A scene refers to its geometries,
 *    which must outlive it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Builds and traces are asynchronous on it; errors detected by device code
 *    (stack overflow, step limit, wait timeout) are latched in the context and
 *    read by grtGetLastDeviceError.
 *  - Sizes are element counts unless the name says bytes.
 *  - The library is single-device: a context binds the device given at creation,
 *    and every call made with it must run with that device current.
 */
#ifndef GRT_H_
#define GRT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRT_API_VERSION 1u

typedef enum grtError {
    GRT_SUCCESS = 0,
    GRT_ERROR_INVALID_PARAMETER = 1, /* null handle/pointer, bad enum, count or stride */
    GRT_ERROR_OUT_OF_MEMORY = 2,     /* a library-owned allocation failed */
    GRT_ERROR_INVALID_API_VERSION = 3,
    GRT_ERROR_NOT_BUILT = 4,         /* trace on a geometry/scene that was never built */
    GRT_ERROR_STACK_OVERFLOW = 5,    /* device: a ray needed more stack than configured */
    GRT_ERROR_STEP_LIMIT = 6,        /* device: a ray exceeded the traversal step bound */
    GRT_ERROR_TIMEOUT = 7,           /* device: a bounded wait expired */
    GRT_ERROR_CUDA = 8,              /* a CUDA runtime call or launch failed */
    GRT_ERROR_INTERNAL = 9
} grtError;

/* Opaque handles. A grtGeometry and a grtScene are device addresses of small
 * library-owned headers, so they may be stored in device memory (grtInstance). */
typedef struct grtContext_* grtContext;
typedef struct grtGeometry_* grtGeometry;
typedef struct grtScene_* grtScene;
typedef struct grtFuncTable_* grtFuncTable;

/* ---------------------------------------------------------------- context (Sec. 7.1) */
typedef struct grtContextCreationInput {
    int32_t device; /* CUDA device ordinal; the paper's vendor/device fields reduce to this */
} grtContextCreationInput;

typedef enum grtLogLevel {
    GRT_LOG_NONE = 0,
    GRT_LOG_ERROR = 1,
    GRT_LOG_WARN = 2,
    GRT_LOG_INFO = 4
} grtLogLevel;

/* Creates a context on input->device. apiVersion must equal GRT_API_VERSION
 * (else GRT_ERROR_INVALID_API_VERSION). Allocates the context's small device
 * workspace (error word, work counters). */
grtError grtCreateContext(uint32_t apiVersion, const grtContextCreationInput* input, grtContext* out);
/* Frees the context and its device workspace (Sec. 7.1). Objects created from it must be
 * destroyed first and no work of it may be in flight. */
grtError grtDestroyContext(grtContext ctx);
/* Bit set of grtLogLevel values printed to stderr (Sec. 7.1's log level). */
grtError grtSetLogLevel(uint32_t levels);

/* Reads and clears the device error latched by builds and traces enqueued on
 * `stream` (synchronises the stream). *err = GRT_SUCCESS when none. */
grtError grtGetLastDeviceError(grtContext ctx, void* stream, grtError* err);

/* ---------------------------------------------------------------- geometry (Sec. 7.2) */
typedef enum grtPrimitiveType {
    GRT_PRIMITIVE_TRIANGLE_MESH = 0,
    GRT_PRIMITIVE_AABB_LIST = 1
} grtPrimitiveType;

/* Indexed triangles: triangle i = three uint32 vertex indices at
 * triangleIndices + i*triangleStride (stride >= 12 bytes, multiple of 4);
 * vertex k = three float32 at vertices + k*vertexStride (stride >= 12, multiple
 * of 4). Both are device pointers. */
typedef struct grtTriangleMeshPrimitive {
    uint32_t triangleCount;
    uint32_t triangleStride;
    const void* triangleIndices;
    uint32_t vertexCount;
    uint32_t vertexStride;
    const void* vertices;
} grtTriangleMeshPrimitive;

/* Custom primitives given by their boxes: box i = float32 lo.xyz, hi.xyz at
 * aabbs + i*aabbStride (stride >= 24, multiple of 4; device pointer). */
typedef struct grtAABBListPrimitive {
    uint32_t aabbCount;
    uint32_t aabbStride;
    const void* aabbs;
} grtAABBListPrimitive;

typedef struct grtGeometryBuildInput {
    uint32_t type;     /* grtPrimitiveType */
    uint32_t geomType; /* column of the function table for AABB lists */
    grtTriangleMeshPrimitive triangleMesh;
    grtAABBListPrimitive aabbList;
} grtGeometryBuildInput;

/* The paper's fast / balanced / high-quality flags (Sec. 7.2) choose the build of a
 * geometry (Sec. 6.2 "BVH Construction": top-down splitting or bottom-up clustering):
 *   FAST         linear BVH: Morton codes, radix sort, Karras emission, bottom-up fit;
 *   BALANCED     bottom-up clustering (PLOC, Meister and Bittner 2018) over the same
 *                Morton order, nearest neighbours searched 8 positions either side;
 *   HIGH_QUALITY the same clustering with a 32-position search (spatial splits, which
 *                the paper names for this option, are the separate bit
 *                GRT_BUILD_SPLIT_TRIANGLES below, combinable with any method);
 *   CLUSTER_SUBTREES clustering inside the linear BVH's subtrees in one bottom-up pass
 *                (the one-pass form of locally-ordered clustering, H-PLOC, that the paper
 *                names for the balanced option, Sec. 8): every LBVH node merges its
 *                children's clusters by mutual nearest neighbours (union surface area)
 *                down to 16 and passes the rest up; the root merges to one. About the
 *                quality of BALANCED at close to the LBVH's build cost.
 * All four give binary nodes, 4-wide nodes and leaves of the same layout, and all
 * support GRT_BUILD_OPERATION_UPDATE (not with GRT_BUILD_SPLIT_TRIANGLES). A geometry's flag is fixed by grtCreateGeometry;
 * grtGetGeometryBuildTemporaryBufferSize and grtBuildGeometry must be given the same
 * flag (the clustering builds need 68 more bytes of temporary memory per primitive).
 * Scene (top-level) builds always use the linear BVH. Other values are rejected with
 * GRT_ERROR_INVALID_PARAMETER; so are clustering builds of 2^30 or more primitives. */
typedef enum grtBuildFlags {
    GRT_BUILD_PREFER_FAST = 0,
    GRT_BUILD_PREFER_BALANCED = 1,
    GRT_BUILD_PREFER_HIGH_QUALITY = 2,
    GRT_BUILD_CLUSTER_SUBTREES = 3,
    GRT_BUILD_QUANTIZED_NODES = 0x100,
    GRT_BUILD_WIDE8_NODES = 0x200,
    GRT_BUILD_SPLIT_TRIANGLES = 0x400
} grtBuildFlags;
/* GRT_BUILD_QUANTIZED_NODES, ORed with any of the four: traversal reads 64-byte
 * quantised 4-wide nodes instead of the 128-byte ones (the paper's wide trees, Sec. 6.2,
 * stored compactly; the encoding of Ylitie, Karras and Laine, HPG 2017). Per node and
 * axis, over the used slots: origin p = the least slot lo, step 2^e with e the least
 * integer in [-126, 127] for which fl(p + 255 * 2^e) reaches the greatest slot hi;
 * each slot's lower plane is the largest byte q with fl(p + q 2^e) <= lo, its upper
 * plane the smallest with fl(p + q 2^e) >= hi (fl = float32 rounding to nearest), so
 * the decoded box contains the exact one and results are those of the 128-byte nodes
 * up to equal-t ties. Node words (16 x 32 bits): p.xyz; biased exponents e + 127 in
 * bytes 0-2; qlo.x, qhi.x, qlo.y, qhi.y, qlo.z, qhi.z with slot j in byte j (an empty
 * slot 255 / 0); the four child words; two zero words. The build writes them after the
 * fit (and after each UPDATE), beside the 128-byte nodes (grtBvhInfo.quantNodes). Like
 * the method, the bit is fixed by grtCreateGeometry; a grtBuildGeometry given options
 * must repeat it. Scene (top-level) builds ignore it: their own nodes stay 128-byte,
 * while instances of quantised geometries are traversed in their format.
 *
 * GRT_BUILD_WIDE8_NODES, ORed with any of the four (not with QUANTIZED_NODES), for
 * geometries and scenes: traversal reads 256-byte 8-wide nodes (the branching factor 8
 * the paper names beside 4, Sec. 6.2), written after the fit (and after each UPDATE)
 * beside the 4-wide ones (grtBvhInfo.wide8Nodes). The 8-wide node of binary node k holds
 * k's descendants three levels down: slots 4s..4s+3 come from child s, a leaf child in
 * slot 4s alone, an internal child's children t in slots 4s+2t and 4s+2t+1 (their own
 * two children, or the leaf itself and an empty slot); a walk from node 0 meets the
 * nodes of binary depth divisible by 3. Layout (16 float4): row 4a + 2 side + half =
 * axis a's lower (side 0) or upper (side 1) planes of slots 4 half .. 4 half + 3; rows
 * 12 and 13 the child words (0xFFFFFFFF = empty, box +inf / -inf); rows 14-15 zero. A
 * scene built with the bit has an 8-wide top level and walks its instances' 8-wide
 * nodes: every instanced geometry must have them (an instance of another geometry is
 * left empty and latches GRT_ERROR_INVALID_PARAMETER for grtGetLastDeviceError). A
 * scene without the bit walks the 4-wide (or quantised) nodes of every geometry,
 * 8-wide ones included. The batched launch builds the 8-wide nodes of such geometries
 * and traces them through their 4-wide nodes.
 *
 * GRT_BUILD_SPLIT_TRIANGLES, ORed with any method and node format, for triangle meshes
 * (other geometries and scenes: GRT_ERROR_INVALID_PARAMETER for geometries, ignored by
 * scene builds): spatial splits, the paper's high-quality option (Sec. 8, SBVH), made
 * before the build as in Karras and Aila (HPG 2013): a triangle may be referenced by
 * several leaves, each bounding the part of it on one side of a set of cutting planes.
 * S = floor(splitFactor * triangleCount) extra references (splitFactor in [0, 1],
 * 0 = 0.5; triangleCount + S must stay below 2^31) are shared out by priority; a
 * grtBuildGeometry given options must repeat the creation's bit and factor (0 and 0.5
 * are the same factor). The build then runs over exactly
 * triangleCount + S leaves (grtBvhInfo.leafCount). In this order, in float32 rounded to
 * nearest (the integer steps exact):
 *   box B_t of triangle t's vertices; G = union of all B_t; per axis a grid of 1024 cells
 *   over G, q(x) = (x - G.lo) * (1024 / (G.hi - G.lo)); a box [lo, hi] spans cells
 *   cl = floor(q(lo + d)) to ch = max(cl, ceil(q(hi - d)) - 1), clamped to [0, 1023],
 *   d = 2^-18 max(|lo|, |hi|) (all 0 on an axis of zero extent); level(B) = the largest
 *   bit length of cl xor ch over the axes;
 *   weight w_t = the integer cube root of 2^53 (max(0, A(B_t) - A_t) / A(G)) 2^level(B_t),
 *   A(B) = (dx dy + dy dz) + dz dx, A_t = ((|c.x| + |c.y|) + |c.z|) / 2, c = (v1-v0) x
 *   (v2-v0); W = sum of w_t; with C_t = w_0 + .. + w_{t-1}, triangle t takes
 *   min(31, floor(S C_{t+1} / W) - floor(S C_t / W)) splits (0 when W = 0), and the
 *   R = S - sum left over go one each to triangles 0 .. R-1;
 *   the box is cut recursively, s splits at a time: the plane is, over the axes with
 *   cl != ch, the grid line j = (ch >> b) << b (b the highest bit of cl xor ch) of the
 *   largest b (ties: longer box extent, then lower axis), at G.lo + j ((G.hi - G.lo) /
 *   1024); with no such axis, (lo + hi) / 2 of the longest axis. Each side's box is the
 *   box of the triangle's vertices on that side (<= / >= the plane), then of its edges'
 *   crossings of the plane (t = (P - a_k) / (e_k - a_k), a_c + (e_c - a_c) t widened by
 *   2^-19 max(|a_c|, |e_c|) + 2^-140, which bounds its rounding error), intersected with
 *   the box being cut; an empty side copies the other side's box and takes no splits.
 *   Of the s - 1 splits left, the left side takes floor((s - 1) wL / (wL + wR) + 0.5)
 *   (w = longest extent; (s - 1) / 2 when both are 0), the right side the rest; the left
 *   side's references come first.
 * References are numbered triangle by triangle; each triangle's first one is the leaf
 * that primToLeaf names. Closest-hit and any-hit queries return each primitive at most
 * once as before (the leaf record is the whole triangle); an all-hits query skips a
 * split geometry (GRT_ERROR_INVALID_PARAMETER: on the host for grtTraceAllHits on the
 * geometry itself, latched for grtGetLastDeviceError for instances of it), and an
 * intersection filter may be called more than once for one primitive. UPDATE of a
 * split geometry is GRT_ERROR_INVALID_PARAMETER; a BUILD from new vertex data re-splits.
 * The batched launch splits such geometries in seven phases of its own before their
 * build (never by one block) and leaves them as grtBuildGeometry does. */

typedef struct grtBuildOptions {
    uint32_t buildFlags; /* grtBuildFlags */
    uint32_t mortonBits; /* 30 or 63; 0 = 30 when the leaf count <= 2^20, else 63 */
    float splitFactor;   /* GRT_BUILD_SPLIT_TRIANGLES: extra references per triangle, in [0, 1]; 0 = 0.5 */
} grtBuildOptions;

typedef enum grtBuildOperation {
    GRT_BUILD_OPERATION_BUILD = 0, /* full rebuild */
    GRT_BUILD_OPERATION_UPDATE = 1 /* refit: same topology, boxes recomputed bottom-up (Sec. 6.2) */
} grtBuildOperation;

/* Size in bytes of the caller-allocated temporary buffer for building `input`
 * (Sec. 7.2); the buffer may be reused for other builds once a build completes. */
grtError grtGetGeometryBuildTemporaryBufferSize(grtContext ctx, const grtGeometryBuildInput* input,
                                                const grtBuildOptions* options, size_t* sizeBytes);
/* Allocates the library-owned node and leaf arrays for `input`'s primitive count. */
grtError grtCreateGeometry(grtContext ctx, const grtGeometryBuildInput* input, const grtBuildOptions* options,
                           grtGeometry* out);
/* Enqueues the build chosen by the geometry's flag (or, for UPDATE, the refit) on
 * `stream`. `temp` is a device buffer of at least the size queried with the same
 * options, 16-byte aligned. The primitive count must equal the one given to
 * grtCreateGeometry. A clustering build is one persistent launch whose blocks wait on
 * one another at grid barriers; each wait is bounded (2 s), and one that runs out (the
 * blocks could not all be resident, e.g. beside other work on the device) latches
 * GRT_ERROR_TIMEOUT for grtGetLastDeviceError and leaves an unusable tree. */
grtError grtBuildGeometry(grtContext ctx, uint32_t op, const grtGeometryBuildInput* input,
                          const grtBuildOptions* options, void* temp, void* stream, grtGeometry geom);
/* Frees the geometry's node, leaf and link arrays and any captured build graph. No scene
 * that instances it may be traced afterwards; no work using it may be in flight.
 * GRT_ERROR_INVALID_PARAMETER for a handle that is not a live geometry. */
grtError grtDestroyGeometry(grtContext ctx, grtGeometry geom);

/* ---------------------------------------------------------------- scene (Sec. 7.3) */
typedef enum grtInstanceType { GRT_INSTANCE_GEOMETRY = 0 } grtInstanceType;

typedef struct grtInstance { /* 16 bytes */
    uint32_t type;           /* grtInstanceType */
    uint32_t mask;           /* visibility mask (Sec. 7.5): a ray sees the instance only when
                                mask & the ray mask != 0; 0 = all bits set */
    grtGeometry geometry;
} grtInstance;

/* Instance transform world = T * R * S * object. rotation is a quaternion x,y,z,w
 * (normalised by the library; the paper leaves the encoding unspecified). 40 bytes. */
typedef struct grtFrameSRT {
    float rotation[4];
    float scale[3];
    float translation[3];
} grtFrameSRT;

typedef struct grtSceneBuildInput {
    uint32_t instanceCount;
    uint32_t frameCount;               /* must equal instanceCount */
    const grtInstance* instances;      /* device pointer, instanceCount entries */
    const grtFrameSRT* instanceFrames; /* device pointer, frameCount entries */
} grtSceneBuildInput;

/* Size in bytes of the caller-allocated temporary buffer for building the top level of
 * `input` (Sec. 7.3); instanceCount must equal frameCount (else GRT_ERROR_INVALID_PARAMETER). */
grtError grtGetSceneBuildTemporaryBufferSize(grtContext ctx, const grtSceneBuildInput* input,
                                             const grtBuildOptions* options, size_t* sizeBytes);
/* Allocates the library-owned top level for `input`'s instance count: nodes, instance
 * records and the FP64 frames. Top levels are linear BVHs whatever the method bits;
 * GRT_BUILD_WIDE8_NODES gives them 8-wide nodes (and then needs 8-wide instances), and
 * grtBuildScene must be given the same bit. */
grtError grtCreateScene(grtContext ctx, const grtSceneBuildInput* input, const grtBuildOptions* options,
                        grtScene* out);
/* Builds the top level over the instances' world boxes. The instances' geometries
 * must have been built earlier on the same stream (or be complete). */
grtError grtBuildScene(grtContext ctx, uint32_t op, const grtSceneBuildInput* input, const grtBuildOptions* options,
                       void* temp, void* stream, grtScene scene);
/* Frees the top level (not the geometries it instances); no work using it may be in flight. */
grtError grtDestroyScene(grtContext ctx, grtScene scene);

/* ---------------------------------------------------------------- custom intersection (Sec. 7.4) */
typedef enum grtIntersectFunc {
    GRT_INTERSECT_NONE = 0,    /* custom primitives of this (geomType, rayType) are never hit */
    GRT_INTERSECT_SPHERE = 1,  /* built-in: data = float4 {centre.xyz, radius} per primitive */
    GRT_INTERSECT_USER = 0x100 /* this and higher IDs: user intersection code (Sec. 7.4), run only by
                                  kernels that trace through grt_device.cuh with a functor, which
                                  gets the ID; traces of libgrt.so reject a table naming one */
} grtIntersectFunc;

/* Intersection filters (Sec. 7.6): called on every hit the intersector (or the
 * built-in triangle test) accepts, for triangles and custom primitives alike; a hit the
 * filter rejects is skipped and traversal goes on, as for alpha masking. */
typedef enum grtFilterFunc {
    GRT_FILTER_NONE = 0,          /* every hit stands */
    GRT_FILTER_PRIMITIVE_MASK = 1, /* built-in: data = uint32 bit array over primitive IDs; a hit on
                                      primitive p stands only when bit p (word p / 32, bit p % 32) is set */
    GRT_FILTER_USER = 0x100        /* this and higher IDs: user filter code (Sec. 7.6), as for
                                      GRT_INTERSECT_USER */
} grtFilterFunc;

typedef struct grtFuncDataSet {
    uint32_t intersectFunc;        /* grtIntersectFunc */
    uint32_t filterFunc;           /* grtFilterFunc */
    const void* intersectFuncData; /* device pointer handed to the intersector */
    const void* filterFuncData;    /* device pointer handed to the filter */
} grtFuncDataSet;

/* A numRayTypes x numGeomTypes table, row-major (row = ray type), as the paper's
 * flattened function layout. */
grtError grtCreateFuncTable(grtContext ctx, uint32_t numGeomTypes, uint32_t numRayTypes, grtFuncTable* out);
/* Sets entry (rayType, geomType) (Sec. 7.4's hiprtSetFuncTable): the intersector and filter
 * IDs and their device data pointers, which stay owned by the caller and must outlive every
 * trace that uses the table. Synchronous copy to the device. GRT_ERROR_INVALID_PARAMETER for
 * an index out of range, an unknown intersector or filter ID, or a filter without data. */
grtError grtSetFuncTable(grtContext ctx, grtFuncTable table, uint32_t geomType, uint32_t rayType,
                         grtFuncDataSet set);
/* Frees the table; no trace using it may be in flight. */
grtError grtDestroyFuncTable(grtContext ctx, grtFuncTable table);

/* ---------------------------------------------------------------- traversal (Sec. 6.2, 7.5, 7.6) */
/* R(t) = origin + t*direction, t in [minT, maxT] (both inclusive). 32 bytes. */
typedef struct grtRay {
    float origin[3];
    float minT;
    float direction[3];
    float maxT;
} grtRay;

/* 20 bytes. A miss has instanceID = primID = 0xFFFFFFFF and t = +inf. Triangle
 * barycentrics: hit point = (1-u-v)*v0 + u*v1 + v*v2; custom primitives: u = v = 0.
 * Tracing a geometry directly reports instanceID 0. */
typedef struct grtHit {
    uint32_t instanceID;
    uint32_t primID;
    float t;
    float u;
    float v;
} grtHit;

#define GRT_INVALID_ID 0xFFFFFFFFu

/* Traversal stack (Sec. 7.5): each thread keeps its first sharedStackDepth entries in
 * shared memory and the next globalStackDepth entries in a global buffer sized for
 * every thread of the persistent grid. A ray that needs more is finished with the
 * entries it has and latches GRT_ERROR_STACK_OVERFLOW. */
typedef struct grtTraceOptions {
    uint32_t rayType;          /* row of the function table */
    uint32_t blockSize;        /* threads per block: 0 = default (128); 64, 128 or 256 */
    uint32_t sharedStackDepth; /* entries per thread in shared memory: 0 = default (16), 1..32 */
    uint32_t globalStackDepth; /* further entries per thread in global memory: 0 = default (64) */
    float compactThreshold;    /* warp refill threshold (fraction of live lanes), 0 = default (0.6 for
                                  grtTraceAmbientOcclusion, else 0.5) */
    uint32_t flags;            /* GRT_TRACE_FLAG_COUNT: accumulate grtTraceStatistics (slower) */
    void* globalStack;         /* optional caller-owned device buffer for the global entries; NULL = the
                                  context's own (then traces on one context must not overlap in time) */
    size_t globalStackBytes;   /* size of globalStack; must be >= grtGetTraceGlobalStackSize */
    uint32_t rayMask;          /* ray mask (Sec. 7.5), ANDed with each instance's mask; 0 = all bits set */
} grtTraceOptions;

/* Bytes of global stack a trace with `options` (NULL = defaults) needs. */
grtError grtGetTraceGlobalStackSize(grtContext ctx, const grtTraceOptions* options, size_t* sizeBytes);

/* Closest hit of each ray against a scene (two levels) or a single geometry (pass
 * exactly one of scene / geom). rays and hits are device pointers of rayCount
 * entries. table may be NULL when no custom primitives are reached. options may be
 * NULL (defaults). */
grtError grtTraceClosest(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                         grtHit* hits, grtFuncTable table, const grtTraceOptions* options, void* stream);
/* Every hit of each ray (Sec. 7.5: all intersections, as repeated getNextHit() calls on
 * the any-hit traversal object return them): each (instance, primitive) whose exact
 * intersection lies in [minT, maxT], once. Ray r's first maxHitsPerRay hits, in
 * traversal order (not sorted by t) with t, u, v recomputed to ~48 bits, go to
 * hits[r * maxHitsPerRay ...]; its remaining slots are set to misses; hitCounts[r]
 * (device, rayCount uint32) gets the number of hits found, which may exceed
 * maxHitsPerRay. Instance masks, the ray mask and intersection filters apply as for
 * the other queries. One thread per ray with a 96-entry local stack (a deeper walk
 * latches GRT_ERROR_STACK_OVERFLOW); maxHitsPerRay = 0 is GRT_ERROR_INVALID_PARAMETER. */
grtError grtTraceAllHits(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                         grtHit* hits, uint32_t maxHitsPerRay, uint32_t* hitCounts, grtFuncTable table,
                         const grtTraceOptions* options, void* stream);
/* ---------------------------------------------------------------- path tracing (Sec. 5) */
/* Materials and lights of a path trace. Primitive p of instance i uses material entry
 * materialOffset[i] + p of albedo and emission (3 floats each, device); an entry with
 * nonzero emission marks an emitting triangle. lights lists the emitting triangles for
 * next event estimation as lightCount (instanceID, primID) pairs (device). The caller
 * keeps every material index within albedo and emission (the device does not know their
 * length). A light entry naming no triangle of the scene is skipped and latches
 * GRT_ERROR_INVALID_PARAMETER (grtGetLastDeviceError). */
typedef struct grtPathTraceInput {
    const float* albedo;
    const float* emission;
    const uint32_t* materialOffset;
    const uint32_t* lights;
    uint32_t lightCount;
    uint32_t maxDepth;        /* path vertices per sample, >= 1 */
    uint32_t samplesPerPixel; /* >= 1 */
    uint32_t reserved;
    uint64_t seed;            /* stream of the splitmix64 random numbers */
    float sky[3];             /* radiance of rays that leave the scene */
    float reserved2;
} grtPathTraceInput;

/* Bytes of device workspace grtPathTrace needs for rayCount rays (path and shadow rays
 * and hits, throughput, radiance, pending light samples: about 152 B per ray). */
grtError grtGetPathTraceWorkspaceSize(uint32_t rayCount, size_t* sizeBytes);

/* Path tracing with next event estimation (Sec. 5) over a two-level scene of triangle
 * meshes, one path per (ray, sample) from the given rays (e.g. camera rays from
 * grtGenerateCameraRays). Per path vertex: a miss adds throughput * sky; a hit on an
 * emitting triangle adds throughput * emission at the first vertex only (later ones
 * count lights through next event estimation) and ends the path; otherwise one light
 * triangle and a uniform point on it are sampled, its contribution
 * T (albedo / pi) cos_s |cos_l| / dist^2 emission_l / pdf (pdf = 1 / (lightCount area_l))
 * counts when an any-hit shadow ray from p + 1e-4 n over (1 - 1e-4) dist finds nothing,
 * and the path continues along a cosine-weighted direction with T *= albedo. n is the
 * face normal turned toward the incoming ray. radiance (device, 3 floats per ray) gets
 * the mean over samplesPerPixel. workspace: device, 256-byte aligned, at least
 * grtGetPathTraceWorkspaceSize bytes. options apply to every trace of the walk
 * (ray mask, stack sizes). Runs as a wavefront of the library's closest-hit and any-hit
 * queries with a shading pass per vertex, all on `stream`. */
grtError grtPathTrace(grtContext ctx, grtScene scene, const grtRay* rays, uint32_t rayCount,
                      const grtPathTraceInput* input, void* workspace, float* radiance,
                      const grtTraceOptions* options, void* stream);

/* The same closest-hit query as grtTraceClosest for callers that must not allocate
 * device memory: code running while a stream is being captured into a CUDA graph
 * (where cudaMalloc is not allowed), code whose memory is fully owned by another
 * allocator or reserved up front, and latency-critical loops that cannot afford the
 * device-wide synchronisation a cudaMalloc or cudaFree implies. grtTraceClosest may
 * grow the context's global-stack area with cudaMalloc; this entry point never
 * allocates or frees anything. (The paper has no counterpart: it is an addition of
 * this library.)
 *
 * Its scratch (work counter and global traversal stack) is a 16 MiB array that the
 * library keeps resident on every device that loads it, until the process exits.
 * The caller still provides rays, hits and the built scene or geometry, as for
 * grtTraceClosest; options->globalStack is ignored. The persistent grid is reduced
 * so that every thread's global stack fits the array, down to one block per SM
 * (or one block per blockSize rays, if that is fewer). A request that cannot fit
 * that minimum grid (blocks * blockSize * globalStackDepth * 4 bytes > 16 MiB - 256;
 * with 152 SMs and 128-thread blocks, globalStackDepth above 215) is rejected with
 * GRT_ERROR_INVALID_PARAMETER and a logged message.
 *
 * The first call on each device looks up the array's device address and caches it;
 * make that first call before any stream capture begins. Every call shares the one
 * array (the work counter is cleared on `stream` at the start of each call): calls
 * that overlap on the GPU race, so serialise them on one stream or order them with
 * events. The device current at the call must be the context's. The cached address
 * belongs to the device's primary context as it is when first looked up: after
 * cudaDeviceReset (or anything else that tears that context down) it no longer names
 * the array, so do not call this entry point again in that process. */
grtError grtTraceClosestNoAlloc(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays,
                                uint32_t rayCount, grtHit* hits, grtFuncTable table, const grtTraceOptions* options,
                                void* stream);

/* Any hit in [minT, maxT]: primID = GRT_INVALID_ID means unoccluded; otherwise the
 * record describes one (not necessarily the closest) valid hit. */
grtError grtTraceAnyHit(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                        grtHit* hits, grtFuncTable table, const grtTraceOptions* options, void* stream);

/* ---------------------------------------------------------------- device-side queries (Sec. 7.5) */
/* Everything a user CUDA kernel needs to trace rays itself through grt_device.cuh (the
 * paper's device traversal object, Sec. 7.5): device pointers of the target's arrays,
 * of a scene's instance frames and of the function table. Plain data: pass it to a
 * kernel by value. Valid while the target, the table and the context live and the
 * target is not rebuilt with a different primitive count. */
typedef struct grtDeviceTarget {
    const void* nodes;            /* the target's 4-wide nodes, in nodeFormat */
    const void* leaves;           /* triangle records / primitive IDs / instance records */
    const uint32_t* primToLeaf;   /* primitive (instance) ID -> sorted leaf position */
    const void* frames64;         /* scenes: FP64 inverse frame per instance ID, else NULL */
    const void* frames32;         /* scenes: float32 frame rows per instance ID, else NULL */
    const void* funcTable;        /* function-table entries (grtSetFuncTable), or NULL */
    uint32_t* deviceError;        /* the context's device error word (grtGetLastDeviceError) */
    uint32_t primType;            /* grtPrimitiveType of a geometry; 2 for a scene */
    uint32_t geomType;
    uint32_t primCount;
    uint32_t numGeomTypes;        /* of the function table */
    uint32_t rayType;             /* function-table row used by the queries */
    uint32_t nodeFormat;          /* bits 0-7: 0 nodes are 128-byte 4-wide nodes, 1 64-byte quantised ones,
                                     2 8-wide; bit 8: a geometry built with GRT_BUILD_SPLIT_TRIANGLES */
} grtDeviceTarget;

/* Fills *out for exactly one of scene / geom (built), with an optional function table
 * and the ray type selecting its row. Errors: GRT_ERROR_INVALID_PARAMETER,
 * GRT_ERROR_NOT_BUILT. */
grtError grtGetDeviceTarget(grtContext ctx, grtScene scene, grtGeometry geom, grtFuncTable table, uint32_t rayType,
                            grtDeviceTarget* out);

/* ---------------------------------------------------------------- ray generation (Sec. 3.2, 4) */
/* Pinhole camera (Sec. 3.2): lens at origin, film at distance 1 along
 * normalize(up x right), spanning +-right and +-up. */
typedef struct grtCamera {
    float origin[3];
    float right[3];
    float up[3];
} grtCamera;

/* width*height primary rays through pixel centres, row-major from the top row:
 * ray y*width + x; minT = 0, maxT = +inf. rays: device pointer. */
grtError grtGenerateCameraRays(grtContext ctx, const grtCamera* camera, uint32_t width, uint32_t height,
                               grtRay* rays, void* stream);

/* count rays with origins uniform in the box [lo, hi] and directions uniform on the
 * unit sphere, t in [minT, maxT]: the incoherent rays of a custom-primitive workload
 * (the paper traces its rays from a generator kernel, Sec. 3.2-3.3; this is the
 * uniform counterpart of its camera). Ray i takes the splitmix64 numbers xi(s, d) of
 * stream `seed` at counter (i << 32) | (s << 1) | d, top 24 bits as a float in [0,1):
 * origin = lo + (hi - lo) * (xi(0,0), xi(0,1), xi(1,0)); z = 1 - 2 xi(1,1), azimuth =
 * 2 pi xi(2,0), direction = (sqrt(1 - z^2) cos, sqrt(1 - z^2) sin, z). lo, hi: host
 * arrays of 3 floats (hi >= lo, finite); rays: device, 16-byte aligned, count entries.
 * Errors: GRT_ERROR_INVALID_PARAMETER for a null or misaligned pointer or a bad box. */
grtError grtGenerateUniformRays(grtContext ctx, const float lo[3], const float hi[3], uint64_t seed, uint32_t count,
                                float minT, float maxT, grtRay* rays, void* stream);

/* Ambient-occlusion rays (Sec. 4): for pixel p with a primary hit, samplesPerPixel
 * cosine-weighted directions about the world face normal turned toward the viewer
 * (tangent = world v1 - v0), origin = hit point + 1e-4 * normal, t in [0, length].
 * Random numbers: splitmix64 of stream `seed` at counter
 * (p << 32) | (sample << 1) | dim, top 24 bits. A pixel without a hit gets empty rays
 * (direction 0, minT 0, maxT -1). primaryRays/primaryHits: pixelCount entries;
 * aoRays: pixelCount*samplesPerPixel entries; all device pointers. The scene must be
 * the one the primary hits came from (triangle geometries only). */
grtError grtGenerateAORays(grtContext ctx, grtScene scene, const grtRay* primaryRays, const grtHit* primaryHits,
                           uint32_t pixelCount, uint32_t samplesPerPixel, uint64_t seed, float length,
                           grtRay* aoRays, void* stream);

/* Fused ambient occlusion: generates the same rays as grtGenerateAORays in
 * registers and traces them as any-hit queries without storing them; writes
 * ao[p] = occluded samples / samplesPerPixel (0 for pixels without a primary hit). */
grtError grtTraceAmbientOcclusion(grtContext ctx, grtScene scene, const grtRay* primaryRays,
                                  const grtHit* primaryHits, uint32_t pixelCount, uint32_t samplesPerPixel,
                                  uint64_t seed, float length, float* ao, const grtTraceOptions* options,
                                  void* stream);

/* ---------------------------------------------------------------- differentiable Lambertian shading */
/* Shading of the primary hits on a triangle geometry (the cosine law of Sec. 4.1 with
 * the Lambert BRDF c/pi of Sec. 5.2, the constant pi folded into the caller's loss
 * scale). For pixel p with hit (prim, t, u, v) from grtTraceClosest on `geom`:
 *   n_f = normalize((v1-v0) x (v2-v0)) turned to face the ray, s = max(0, n_f . l)
 *   with l = light[0..2] used as given (not normalised), V = 0 if the shadow ray from
 *   o + t d + 1e-4 n_f along l (t in [0, inf)) hits `geom` (any hit), else 1,
 *   c(u,v) = (1-u-v) c[i0] + u c[i1] + v c[i2] from per-vertex colours,
 *   image[p] = V s c(u,v) (3 float32); 0 for a miss or an unlit pixel.
 * indices (3 uint32 per triangle), positions and colours (3 float32 per vertex) are the
 * mesh the geometry was built from; light is 3 float32; all device pointers.
 * visibility (pixelCount bytes, may be NULL) receives V for the backward pass. */
grtError grtShadeLambert(grtContext ctx, grtGeometry geom, const grtRay* rays, const grtHit* hits, uint32_t pixelCount,
                         const uint32_t* indices, const float* positions, const float* colours, const float* light,
                         float* image, uint8_t* visibility, const grtTraceOptions* options, void* stream);

/* Adjoint of grtShadeLambert: given gradImage = dL/dimage (3 float32 per pixel), ADDS
 * dL/dcolours (3 per vertex), dL/dlight (3) and dL/dpositions (3 per vertex) into the
 * caller's buffers. Positions are differentiated through the face normal and through
 * the hit's barycentrics on the fixed primary ray (interior hits: visibility and the
 * hit triangle are piecewise constant and contribute nothing). hits and visibility as
 * stored by the forward pass; hits = NULL recomputes the primary hits (refined as grtTraceClosest does)
 * and the visibility by tracing again within the call (the closest-hit query and the
 * forward's visibility pass into context memory held only during the call), trading
 * about one forward pass for the 21 bytes per pixel kept between the passes. */
grtError grtShadeLambertBackward(grtContext ctx, grtGeometry geom, const grtRay* rays, const grtHit* hits,
                                 const uint8_t* visibility, uint32_t pixelCount, const uint32_t* indices,
                                 const float* positions, const float* colours, const float* light,
                                 const float* gradImage, float* gradColours, float* gradLight, float* gradPositions,
                                 const grtTraceOptions* options, void* stream);

/* Shading of a two-level scene (Sec. 6.2's instances under SRT frames), with shadows
 * cast by every instance: grtShadeLambert in world space. hits come from grtTraceClosest
 * on `scene`. The scene's meshes are one object-space mesh: indices (3 uint32 per
 * triangle, vertex numbers into positions and colours, 3 float32 per vertex), and
 * instanceTriangleOffset[i] (device, one uint32 per instance ID) is the first triangle
 * of instance i's geometry in it, so that hit (i, prim) is triangle
 * instanceTriangleOffset[i] + prim; instances of one geometry share its triangles and
 * vertices. A triangle's world vertices are its object-space vertices under instance
 * i's frame (the scene's float32 forward frame); n_f, s, c(u,v) and the image follow
 * grtShadeLambert; the shadow ray from o + t d + 1e-4 n_f along l is an any-hit query
 * through the whole scene (every instance occludes). A hit on an instance of custom
 * primitives is not shaded (image 0). */
grtError grtShadeLambertScene(grtContext ctx, grtScene scene, const grtRay* rays, const grtHit* hits,
                              uint32_t pixelCount, const uint32_t* instanceTriangleOffset, const uint32_t* indices,
                              const float* positions, const float* colours, const float* light, float* image,
                              uint8_t* visibility, const grtTraceOptions* options, void* stream);

/* Adjoint of grtShadeLambertScene, as grtShadeLambertBackward: ADDS dL/dcolours and
 * dL/dpositions (object space, 3 per vertex of the shared mesh; world-space derivatives
 * mapped back through each instance's frame, M^T g) and dL/dlight. vertexCount: the
 * number of vertices in positions / colours (sizes the block-private accumulation).
 * hits = NULL traces the primary hits and visibility again within the call. */
grtError grtShadeLambertSceneBackward(grtContext ctx, grtScene scene, const grtRay* rays, const grtHit* hits,
                                      const uint8_t* visibility, uint32_t pixelCount,
                                      const uint32_t* instanceTriangleOffset, const uint32_t* indices,
                                      const float* positions, uint32_t vertexCount, const float* colours,
                                      const float* light, const float* gradImage, float* gradColours, float* gradLight,
                                      float* gradPositions, const grtTraceOptions* options, void* stream);

/* ---------------------------------------------------------------- batched build + trace */
/* Many independent triangle geometries, each with its own ray batch, built and traced
 * (closest hit) in one persistent launch that takes work items from a device queue.
 * The paper builds and traces one geometry per call (Sec. 7.2-7.5) and has no batched
 * form; each geometry ends up exactly as grtBuildGeometry(BUILD) would leave it and each
 * hit record exactly as grtTraceClosest would write it. */
typedef struct grtBatch_t* grtBatch;

typedef struct grtBatchScene {
    grtGeometry geometry;         /* from grtCreateGeometry on `input` (triangle mesh) */
    grtGeometryBuildInput input;  /* the mesh (device pointers), read during every launch */
    const grtRay* rays;           /* rayCount rays, 16-byte aligned (device) */
    uint32_t rayCount;
    grtHit* hits;                 /* rayCount closest-hit records (device) */
} grtBatchScene;

enum {
    GRT_BATCH_FLAG_GRAPH = 1,  /* capture the launch sequence once into a CUDA graph and replay it */
    GRT_BATCH_FLAG_PROFILE = 2, /* record when each work item started, was ready and ended */
    /* Test of the bounded waits: one work item is planned to wait for one completion more
     * than can ever happen, so its wait expires after waitLimitMs, GRT_ERROR_TIMEOUT is
     * latched and the launch aborts (the other items skip their work and end). */
    GRT_BATCH_FLAG_TEST_EXPIRE_WAIT = 4
};

/* Tuning knobs (0 selects the default in brackets). */
typedef struct grtBatchOptions {
    uint32_t blockSize;         /* threads per block: 64, 128 or 256 [128] */
    uint32_t sharedStackDepth;  /* traversal stack entries in shared memory, <= 32 [16] */
    uint32_t globalStackDepth;  /* spill entries per thread, <= 4096 [64] */
    float compactThreshold;     /* refill a warp when <= this fraction of lanes hold a ray [0.75] */
    uint32_t smallScenePrims;   /* scenes up to this many triangles are built by one block [8192] */
    uint32_t sortChunkTiles;    /* radix tiles (blockSize x 8 keys) per sort work item [8] */
    uint32_t buildChunk;        /* primitives per prep / emission / fit work item [16384] */
    uint32_t traceChunk;        /* rays per trace work item [16384] */
    uint32_t sceneGroup;        /* scenes per scheduling group, largest first: a group's builds, then its
                                   traces [32] */
    uint32_t waitLimitMs;       /* a work item's wait for another expires after this long [2000] */
    uint32_t flags;             /* GRT_BATCH_FLAG_* */
} grtBatchOptions;

typedef struct grtBatchInfo {
    uint32_t sceneCount;
    uint32_t itemCount;   /* work items per launch */
    uint32_t smallScenes; /* scenes built by a single block */
    uint32_t blocks;      /* persistent grid */
    uint32_t blockSize;
    uint32_t pad;
    size_t deviceBytes;   /* library-owned device memory of the batch (scratch, queue, stacks) */
} grtBatchInfo;

/* Plans the work items and allocates the batch's device memory (scratch for every
 * scene's build, the queue and the traversal stacks), so that a launch allocates
 * nothing. Every geometry must be a triangle-mesh geometry created from its input's
 * triangle count; the scenes' buffers must stay valid while the batch is used. A
 * geometry created with GRT_BUILD_CLUSTER_SUBTREES is built by that method (whatever its
 * size, never by the single-block path), every other one as a linear BVH; either way
 * the result equals grtBuildGeometry's for the subtree clustering and the linear BVH.
 * A geometry created with GRT_BUILD_SPLIT_TRIANGLES is split first, in seven phases of
 * its own (never by the single-block path), into the references grtBuildGeometry makes.
 * Errors: GRT_ERROR_INVALID_PARAMETER (bad option, input, geometry or buffer),
 * GRT_ERROR_OUT_OF_MEMORY. */
grtError grtCreateBatch(grtContext ctx, const grtBatchScene* scenes, uint32_t sceneCount,
                        const grtBatchOptions* options, grtBatch* batch);

/* Builds every geometry and traces every scene's rays on `stream`: a small reset kernel
 * and the persistent kernel, or their CUDA graph with GRT_BATCH_FLAG_GRAPH (captured on
 * the first call). Work items wait for the items they depend on with bounded waits; an
 * expired wait latches GRT_ERROR_TIMEOUT (read with grtGetLastDeviceError). Launches of
 * one batch must not overlap. */
grtError grtBatchBuildTrace(grtContext ctx, grtBatch batch, void* stream);

/* The batch's plan (host memory out): scene and item counts, the persistent grid and the
 * library-owned device bytes. */
grtError grtGetBatchInfo(grtContext ctx, grtBatch batch, grtBatchInfo* info);

/* One work item of the last launch of a batch created with GRT_BATCH_FLAG_PROFILE:
 * scene, phase and chunk, the SM that ran it, and the device clock (ns) when its block
 * took it, when its dependencies were met, and when it finished. */
typedef struct grtBatchItemRecord {
    uint32_t scene;
    uint32_t phase;
    uint32_t chunk;
    uint32_t sm;
    uint64_t startNs;
    uint64_t readyNs;
    uint64_t endNs;
} grtBatchItemRecord;

/* Copies up to `capacity` item records of the last launch (queue order) into `records`
 * (host memory) and sets *count to the batch's item count (0 without profiling).
 * Synchronous: call after the launch has finished. */
grtError grtGetBatchProfile(grtContext ctx, grtBatch batch, grtBatchItemRecord* records, uint32_t capacity,
                            uint32_t* count);
/* Frees the batch's device memory and captured graph (not the geometries, rays or hit
 * buffers, which the caller owns); no launch of it may be in flight. */
grtError grtDestroyBatch(grtContext ctx, grtBatch batch);

/* ---------------------------------------------------------------- introspection and building blocks */
/* Device-side layout of a built geometry or scene, for tests and tools. */
typedef struct grtBvhInfo {
    const void* nodes;   /* nodeCount x 64-byte binary nodes (layout below) */
    const void* leaves;  /* triangles: primCount x 48 bytes; AABB lists: primCount x uint32 primitive IDs;
                            scenes: primCount x 128-byte instance records */
    const void* parents; /* (2*primCount - 1) int32: parent of internal node k at [k], of leaf k at [primCount-1+k] */
    uint32_t nodeCount;
    uint32_t primCount;
    uint32_t primType;   /* grtPrimitiveType; 2 for a scene */
    uint32_t mortonBits; /* key width used by the last build */
    const void* wideNodes; /* nodeCount x 128-byte 4-wide nodes (layout below), read by traversal unless quantised */
    const void* quantNodes; /* nodeCount x 64-byte quantised 4-wide nodes (GRT_BUILD_QUANTIZED_NODES), read by
                               traversal instead of wideNodes; NULL for other geometries and for scenes */
    const void* wide8Nodes; /* nodeCount x 256-byte 8-wide nodes (GRT_BUILD_WIDE8_NODES), read by traversal
                               instead of wideNodes; NULL otherwise */
    uint32_t leafCount;     /* leaves: primCount, or primCount + S with GRT_BUILD_SPLIT_TRIANGLES (the
                               leaf, parent and node arrays above are sized by it instead of primCount) */
    uint32_t reserved;
} grtBvhInfo;
/*
 * Node (64 bytes, 4 x float4): children c0 and c1 of internal node k
 *   [0] = c0.lo.x, c0.hi.x, c1.lo.x, c1.hi.x
 *   [1] = c0.lo.y, c0.hi.y, c1.lo.y, c1.hi.y
 *   [2] = c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z
 *   [3] = (uint32) c0 index, c1 index, 0, 0 ; bit 31 set = leaf, low bits = sorted position
 * Node 0 is the root. Triangle leaf k (48 bytes): {v0.xyz, primID}, {v1.xyz, 0}, {v2.xyz, 0}.
 * A single-primitive geometry has one node whose second child is empty.
 *
 * Wide node k (128 bytes, 8 x float4): binary node k with each internal child replaced
 * by that child's two children, so up to four slots j = 0..3; slots 2s and 2s+1 come
 * from child s (its two children, or the leaf itself and an empty slot):
 *   [0] = lo.x of slots 0-3   [1] = hi.x   [2] = lo.y   [3] = hi.y   [4] = lo.z   [5] = hi.z
 *   [6] = (uint32) slot indices as in binary nodes; 0xFFFFFFFF = empty (box lo = +inf, hi = -inf)
 *   [7] = unused
 * Traversal starts at wide node 0 and follows slot indices, so it visits the wide nodes
 * of binary nodes at even depth; the rest are written but not read.
 */
grtError grtGetBvhInfo(grtContext ctx, grtGeometry geom, grtScene scene, grtBvhInfo* info);

/* Offsets (bytes) inside the build temporary buffer where, after a geometry build
 * of `count` primitives, the sorted Morton keys (uint32 for 30-bit, uint64 for
 * 63-bit) and the sorted primitive indices (uint32) are left. For a build with split
 * triangles, count is the leaf count (grtBvhInfo.leafCount) and the indices are those of
 * the references (numbered triangle by triangle). */
grtError grtGetBuildTemporaryLayout(uint32_t count, uint32_t mortonBits, size_t* sortedKeysOffset,
                                    size_t* sortedValuesOffset, size_t* centroidBoundsOffset);

/* Number of kernels the library has launched in this process, all contexts. */
grtError grtGetLaunchCount(uint64_t* count);

/* Traversal work counted by traces launched with GRT_TRACE_FLAG_COUNT, summed since
 * the last read (the read synchronises `stream` and resets the sums). */
#define GRT_TRACE_FLAG_COUNT 1u
typedef struct grtTraceStatistics {
    uint64_t rays;            /* rays traced */
    uint64_t nodesVisited;    /* 4-wide nodes fetched (112 bytes each: boxes and children) */
    uint64_t trianglesTested; /* 48-byte triangle records tested */
    uint64_t customTested;    /* custom primitives tested */
    uint64_t instancesEntered;/* 128-byte instance records read on entry */
    uint64_t fp64Tests;       /* primitive tests decided again in FP64 */
} grtTraceStatistics;
grtError grtGetTraceStatistics(grtContext ctx, void* stream, grtTraceStatistics* stats);

/* Stable LSD radix sort of (key, value) pairs in place (device pointers). keyBits =
 * 32 (uint32 keys) or 64 (uint64 keys); only the low `significantBits` bits are
 * sorted (<= keyBits). temp: device buffer of grtSortTemporaryBufferSize bytes. */
grtError grtSortTemporaryBufferSize(uint32_t count, uint32_t keyBits, size_t* sizeBytes);
grtError grtSortPairs(grtContext ctx, void* keys, uint32_t* values, uint32_t count, uint32_t keyBits,
                      uint32_t significantBits, void* temp, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRT_H_ */
