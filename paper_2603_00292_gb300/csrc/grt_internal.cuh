// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "../../include/grt.h"

namespace grt {

constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kInvalid = 0xFFFFFFFFu;
constexpr uint32_t kPrimScene = 2;  // primType of a scene header
constexpr int kWideWords = 8;       // float4 per 4-wide node (128 B)
constexpr int kQuantWords = 4;      // float4 per quantised 4-wide node (64 B)
constexpr int kWide8Words = 16;     // float4 per 8-wide node (256 B)

// Device-resident header that a grtGeometry / grtScene handle points to (128 B).
struct alignas(16) BvhHeader {
    float rootLo[3];      // box of everything below the root (written by the build)
    uint32_t primCount;
    float rootHi[3];
    uint16_t primType;    // grtPrimitiveType, or kPrimScene
    uint16_t nodeFormat;  // of `nodes`: 0 4-wide nodes (kWideWords float4), 1 quantised (kQuantWords)
    const float4* nodes;  // nodeCount nodes in nodeFormat: what a 4-wide walk reads
    const void* leaves;   // triangle records / prim IDs / instance records
    uint32_t nodeCount;
    uint32_t geomType;
    const uint32_t* primToLeaf;  // primitive (or instance) ID -> sorted leaf position
    const float4* nodes8;        // nodeCount 8-wide nodes (kWide8Words float4), or null: what an 8-wide walk reads
    uint32_t flags;              // kHeaderSplit
    uint32_t pad[13];
};
constexpr uint32_t kHeaderSplit = 1u;  // triangles split over several leaves (GRT_BUILD_SPLIT_TRIANGLES)
static_assert(sizeof(BvhHeader) == 128, "header size");

// Instance record of a scene leaf (128 B): the float32 inverse frame and the bottom
// level's arrays (read when a ray enters the instance), the instance's world box
// (bounds the parameter range inside it), and the geometry header.
struct alignas(16) InstanceRecord {
    float4 inv[3];          // object = inv * world (rows; w = translation), rounded from FP64
    const float4* nodes;    // bottom-level nodes (4-wide, or quantised with kInstQuant)
    const void* leaves;     // bottom-level leaves
    uint32_t instanceID;
    uint32_t typeBits;      // geomType (bits 0-23) | primType << 24 | kInstSplit | kInstWide8 | kInstQuant | kInstEmpty
    const BvhHeader* geometry;
    float4 worldLo;         // xyz: world box (rounded outward)
    float4 worldHi;
    uint32_t mask;          // visibility mask, ANDed with the ray mask
    uint32_t pad[3];
};

// Per-instance frames of a scene, indexed by instance ID.
struct InstanceFrames64 {
    double inv[3][4];  // object = inv * world, FP64 from the SRT frame
};
constexpr uint32_t kInstEmpty = 0x80000000u;
constexpr uint32_t kInstQuant = 0x40000000u;  // the instance's geometry has quantised nodes
constexpr uint32_t kInstWide8 = 0x20000000u;  // the instance's geometry has 8-wide nodes
constexpr uint32_t kInstSplit = 0x10000000u;  // the instance's geometry has split triangles (several leaves each)
constexpr int kFrameRows = 6;  // float4 rows per instance in BvhObject::fwd32
__host__ __device__ inline uint32_t instGeomType(uint32_t bits) { return bits & 0xFFFFFFu; }
__host__ __device__ inline uint32_t instPrimType(uint32_t bits) { return (bits >> 24) & 0x0Fu; }
static_assert(sizeof(InstanceRecord) == 128, "instance record size");

// Device error word values are grtError codes; the first nonzero one latched wins
// by atomicCAS from 0.
constexpr int kCounterSlots = 256;
struct DeviceWorkspace {
    uint32_t error;
    uint32_t pad[31];
    unsigned long long stats[16];  // traversal statistics (grtTraceStatistics order)
    unsigned long long counters[kCounterSlots];  // per-launch work counters (round robin)
};

// ------------------------------------------------------------------ host helpers
int logLevel();
void noteLaunches(unsigned n);  // adds to the process-wide kernel launch count
void logf(int level, const char* fmt, ...);

#define GRT_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::grt::logf(GRT_LOG_ERROR, "%s:%d %s: %s", __FILE__, __LINE__, #call,       \
                        cudaGetErrorString(e_));                                       \
            return e_ == cudaErrorMemoryAllocation ? GRT_ERROR_OUT_OF_MEMORY : GRT_ERROR_CUDA; \
        }                                                                              \
    } while (0)

#define GRT_LAUNCH_CHECK()                                                             \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            ::grt::logf(GRT_LOG_ERROR, "%s:%d launch: %s", __FILE__, __LINE__,           \
                        cudaGetErrorString(e_));                                       \
            return GRT_ERROR_CUDA;                                                     \
        }                                                                              \
    } while (0)

inline size_t alignUp(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline unsigned ceilDiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Context internals used across files.
struct Context;
Context* asContext(grtContext c);
DeviceWorkspace* workspace(Context* c);
unsigned long long* nextCounter(Context* c);  // a zeroed-on-use work counter slot
// Caller-or-context global stack memory for traversal spills (grown on demand).
grtError contextScratch(Context* c, size_t bytes, void** ptr);
// Context memory for buffers one call passes between its own launches (grown on demand;
// calls on one context must not overlap in time, as for the global stack).
grtError contextAux(Context* c, size_t bytes, void** ptr);
int smCount(Context* c);
int deviceOf(Context* c);

// Host-side records of library-owned objects, looked up by handle.
struct BvhObject {
    BvhHeader* dHeader;  // == handle
    void* nodes;  // binary nodes (64 B each)
    void* wide;   // 4-wide nodes (128 B each), one per binary node
    void* qnodes; // quantised 4-wide nodes (64 B each), one per binary node, or null
    void* w8nodes; // 8-wide nodes (256 B each), one per binary node, or null
    void* leaves;
    int32_t* parents;
    uint32_t* primToLeaf;  // primitive (instance) ID -> sorted position (triangles, scenes)
    InstanceFrames64* inv64;  // scenes: FP64 inverse frame per instance ID
    float4* fwd32;            // scenes: per instance ID kFrameRows float4: forward frame rows 0-2, then
                              // the low parts of the inverse frame (FP64 minus the record's float32 rows)
    uint32_t primCount;
    uint32_t leafCount;  // primCount, or primCount + splitBudget with split triangles
    uint32_t nodeCount;  // max(leafCount - 1, 1) (0 when empty)
    uint32_t primType;
    uint32_t geomType;
    uint32_t mortonBits;
    uint32_t vertexCount;  // triangle meshes: the vertex count of the last build input
    bool built;
    bool quant;  // built with GRT_BUILD_QUANTIZED_NODES (qnodes allocated when primCount > 0)
    bool wide8;  // built with GRT_BUILD_WIDE8_NODES (w8nodes allocated when primCount > 0)
    bool split;  // built with GRT_BUILD_SPLIT_TRIANGLES
    float splitFactor;     // the creation's factor (0 resolved to 0.5)
    uint32_t splitBudget;  // extra references: floor(factor * primCount)
};
BvhObject* findBvh(const void* handle);
bool anyQuantGeometry();  // whether a geometry with quantised nodes exists in the process
grtError registerBvh(BvhObject* obj);
void unregisterBvh(const void* handle);

// Function-table record in device memory: one per (rayType, geomType).
struct FuncEntry {
    uint32_t func;
    uint32_t filter;
    const void* data;
    const void* filterData;
};
struct FuncTableObject {
    FuncEntry* dEntries;
    uint32_t numGeomTypes;
    uint32_t numRayTypes;
    std::vector<uint8_t> userEntry;  // per entry: names a user intersector or filter
    uint32_t userEntries = 0;        // how many do (libgrt.so's own traces reject such a table)
};
FuncTableObject* findFuncTable(grtFuncTable t);
// Whether geometry o was created with GRT_BUILD_CLUSTER_SUBTREES (build.cu).
bool buildsBySubtreeClustering(const BvhObject* o);

// Build-time temporary layout.
struct BuildLayout {
    size_t bounds;       // 8 x uint32 ordered-float centroid bounds
    size_t centroids;    // float4 per prim
    size_t keys[2];      // ping-pong keys
    size_t vals[2];      // ping-pong values
    size_t hist;         // sort histogram / offsets
    size_t flags;        // fit visit counters
    size_t extra;        // scene: instance world boxes and records
    size_t total;
    int passes;          // radix passes
    int finalBuf;        // which ping-pong buffer holds the sorted result
    int keyBytes;
};
BuildLayout buildLayout(uint32_t count, uint32_t mortonBits, bool scene);
uint32_t resolveMortonBits(uint32_t count, const grtBuildOptions* opt);

// Radix sort (build.cu).
size_t sortScratchBytes(uint32_t count);
grtError radixSort(Context* ctx, void* keys0, void* keys1, uint32_t* vals0, uint32_t* vals1, uint32_t count,
                   int keyBytes, int significantBits, uint32_t* hist, cudaStream_t stream, int* finalBuf);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ uint32_t floatToOrdered(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float orderedToFloat(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ void latchError(uint32_t* err, uint32_t code) { atomicCAS(err, 0u, code); }

}  // namespace grt
