// Batched build and trace: many independent triangle geometries, each with its own
// ray batch, built (LBVH) and traced (closest hit) in one persistent launch that takes
// work items from a device queue.
//
// The paper builds and traces one geometry or scene per call (Sec. 7.2-7.5); this
// scheduler has no counterpart there. Every item runs the same per-element work as the
// per-geometry path (lbvh.cuh, traverse.cuh), so each geometry ends up bit-identical to
// a grtBuildGeometry of the same input and each hit record identical to grtTraceClosest.
//
// Items. A scene of more than smallScenePrims primitives is split into phases, each a
// set of chunk items:
//   0            prep: centroids, centroid bounds (atomics), zeroed fit counters
//   1 + 3p       radix pass p, digit histograms per chunk (pass 0 also writes the
//                Morton codes)
//   2 + 3p       radix pass p, exclusive scan of the histograms (one item)
//   3 + 3p       radix pass p, stable scatter per chunk
//   1 + 3P       Karras emission over internal-node chunks
//   2 + 3P       bottom-up fit over leaf chunks
//   3 + 3P       closest-hit trace over ray chunks (refill loop), then the hits' refinement
// A smaller scene is built entirely by one block (phase 0) and traced in phase 1.
// A scene whose geometry was created with GRT_BUILD_CLUSTER_SUBTREES (any size) has its
// emission write the LBVH topology to scratch, then one more phase, the bottom-up
// clustering walk over leaf chunks (cluster.cuh), before the fit; its trace is 4 + 3P.
// A scene whose geometry has split triangles (GRT_BUILD_SPLIT_TRIANGLES) first runs
// kSplitPhases splitting phases (split.cuh): the scene box, the weights, their scan (one
// item), the shares, their scan (one item), the slots, then the references over chunks
// of references; its prep and every later phase then run over the references, numbered
// from kSplitPhases on. Such a scene is never built by one block.
// A scene whose geometry has quantised or 8-wide nodes (GRT_BUILD_QUANTIZED_NODES,
// GRT_BUILD_WIDE8_NODES) has one more phase after the fit, writing them over node
// chunks, before its trace; a scene built by one block writes them at the end of that
// block's build. Traces read the quantised nodes, or the 4-wide ones of 8-wide
// geometries (the persistent kernel keeps one 4-slot traversal to stay within its
// register budget).
// An item of phase k waits until every item of phase k-1 of its scene has finished
// (per-scene completion counters). The host orders the queue so that an item only
// ever waits for items taken from the queue before it, so a waiting block never
// blocks the progress it waits for; every wait is bounded in time all the same
// (waitLimitMs) and latches GRT_ERROR_TIMEOUT if it expires. Scenes are queued in groups, largest
// first, each group's builds followed by its traces (see grtCreateBatch).
//
// Memory. Data written earlier in the launch by another block (centroids, keys,
// histograms, parents, boxes) is read with L1-bypassing loads. Node and leaf records,
// which traversal reads through the read-only path, are never read through L1 before
// their scene's fit has finished.
#include <algorithm>
#include <mutex>
#include <vector>

#include "cluster.cuh"
#include "lbvh_block.cuh"
#include "split.cuh"
#include "traverse.cuh"

namespace grt {

constexpr uint32_t kBatchPhases = 40;
constexpr uint32_t kSplitPhases = 7;  // phases before prep of a scene with split triangles
constexpr uint32_t kBatchWaitSpins = 1u << 25;  // a wait polls at most this many times

// A scene of the batch: its build (BlockBuild) plus its rays and the trace phase.
struct BatchSceneDev : BlockBuild {
    uint32_t rays;
    uint32_t small;       // built by one item
    uint32_t tracePhase;
    uint32_t cluster;     // built by subtree clustering
    uint32_t quant;       // quantised 4-wide nodes written after the fit (one more phase)
    uint32_t wide8;       // 8-wide nodes written after the fit (the same added phase)
    uint32_t splitPhases; // kSplitPhases for a geometry with split triangles, else 0
    uint32_t splitChunks; // chunks of its triangles in the splitting phases
    SplitParams split;    // its splitting (split.cuh): triangles, budget, scratch
    const float4* rayBuf;
    uint32_t* hitBuf;
    // subtree clustering scratch (cluster.cuh)
    uint2* topoChild;
    uint32_t* topoParent;
    uint4* topoRecord;
    float4* clusters;
    uint32_t* freeIds;
    uint32_t* clusterFlags;
};

// Leaves per thread of a clustering-walk item. A walk item is much smaller than the
// other build items: its per-leaf work is the merging of up to 32 clusters at every
// node of more than 16 leaves that the leaf's thread reaches last, done by a whole
// warp, and a large item would keep one block busy long after the rest of its scene's
// walk has finished, holding up the scene's fit and trace items.
constexpr uint32_t kWalkLeavesPerThread = 4;

__device__ __forceinline__ ClusterParams clusterParamsOf(const BatchSceneDev& S) {
    ClusterParams C{};
    C.src = S.src;
    C.n = S.n;
    C.sortedPrims = S.vals[S.passes & 1u];
    C.topoChild = S.topoChild;
    C.topoParent = S.topoParent;
    C.record = S.topoRecord;
    C.clusters = S.clusters;
    C.freeIds = S.freeIds;
    C.flags = S.clusterFlags;
    C.nodes = S.nodes;
    C.parents = S.parents;
    C.error = S.error;
    return C;
}

// Emission of a clustered scene: the leaf clusters of sorted positions [begin, end) and
// the LBVH topology of those internal nodes into the scratch (keys and order written by
// other blocks: L2 loads).
template <typename K>
__device__ __noinline__ void clusterTopologyRange(const BatchSceneDev& S, uint32_t begin, uint32_t end) {
    const ClusterParams C = clusterParamsOf(S);
    const K* keys = static_cast<const K*>(S.keys[S.passes & 1u]);
    for (uint32_t i = begin + threadIdx.x; i < end; i += blockDim.x) karrasTopology<true>(keys, (int)i, C);
}

struct BatchItemDev {
    uint32_t scene;
    uint32_t phase;
    uint32_t chunk;
    uint32_t waitCount;  // items of phase-1 of the scene
};

struct BatchParams {
    const BatchSceneDev* scenes;
    const BatchItemDev* items;
    uint32_t itemCount;
    uint32_t sceneCount;
    uint32_t* done;  // sceneCount x kBatchPhases completion counters
    unsigned long long* head;
    unsigned long long* traceCounters;  // per item
    uint32_t* error;
    uint32_t* abort;  // set when a wait expired: later items skip their work
    unsigned long long* profile;  // with GRT_BATCH_FLAG_PROFILE: 4 words per item, else null
    uint32_t* globalStack;
    uint32_t globalDepth;
    uint32_t globalStride;
    uint32_t sharedDepth;
    uint32_t refillBelow;
    uint32_t buildChunk;
    uint32_t sortChunkKeys;
    uint32_t traceChunk;
    unsigned long long waitNs;  // time limit of one wait
};

__device__ __forceinline__ unsigned long long globalTimerNs() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 only: returns once `need` items of (scene, phase) are done or the launch is
// aborted. A wait that runs out latches GRT_ERROR_TIMEOUT and aborts the launch.
__device__ void waitPhase(const BatchParams& B, uint32_t scene, uint32_t phase, uint32_t need) {
    volatile uint32_t* d = B.done + (size_t)scene * kBatchPhases + phase;
    volatile uint32_t* abort = B.abort;
    if (*d < need) {
        const unsigned long long t0 = globalTimerNs();
        for (uint32_t k = 0; *d < need; ++k) {
            if (*abort != 0u) break;
            if (k >= kBatchWaitSpins || ((k & 63u) == 0u && globalTimerNs() - t0 > B.waitNs)) {
                latchError(B.error, GRT_ERROR_TIMEOUT);
                atomicExch(B.abort, 1u);
                break;
            }
            __nanosleep(200);
        }
    }
    __threadfence();
}

// ------------------------------------------------------------------ trace phase
// Items = the rays of one chunk of a scene's ray batch.
struct ChunkRaySource {
    const TraceParams* P;
    uint32_t base, n;
    __device__ unsigned long long count() const { return n; }
    __device__ bool begin(uint32_t i, const TraceParams& Q, Stack& st, RayState& s) const {
        const size_t r = (size_t)base + i;
        const float4 a = Q.rays[2 * r], b = Q.rays[2 * r + 1];
        beginRay<false>(Q, st, s, f3(a), f3(b), a.w, b.w);
        return true;
    }
    __device__ void finish(uint32_t i, const RayState& s) const { storeHit(P->hits, base + i, s.best); }
};

__device__ __noinline__ void traceChunk(const BatchParams& B, const BatchSceneDev& S, uint32_t chunk, unsigned long long item,
                           uint32_t* smem) {
    TraceParams P{};
    P.target.nodes = S.qnodes ? S.qnodes : S.wide;  // 8-wide geometries are traced through their 4-wide nodes
    P.target.fmt = S.qnodes ? 1u : 0u;
    P.target.leaves = S.leaves;
    P.target.primType = GRT_PRIMITIVE_TRIANGLE_MESH;
    P.target.geomType = 0;
    P.target.empty = S.n == 0;
    P.rays = S.rayBuf;
    P.hits = S.hitBuf;
    P.count = S.rays;
    P.sharedDepth = B.sharedDepth;
    P.globalDepth = B.globalDepth;
    P.globalStack = B.globalStack;
    P.globalStride = B.globalStride;
    P.counter = B.traceCounters + item;
    P.error = B.error;
    P.maxSteps = 1u << 26;
    P.refillBelow = B.refillBelow;
    P.rayMask = 0xFFFFFFFFu;
    P.targetPrimToLeaf = S.primToLeaf;
    const uint32_t base = chunk * B.traceChunk;
    const uint32_t n = min(B.traceChunk, S.rays - base);
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{smem + threadIdx.x, B.globalStack + gtid, B.sharedDepth, B.globalDepth, B.globalStride, 0};
    ChunkRaySource src{&P, base, n};
    refillLoop<false, false, false, kFmQuant>(P, st, src);
    __syncthreads();  // hit records of the chunk complete
    for (uint32_t r = base + threadIdx.x; r < base + n; r += blockDim.x) refineHit(P, r);
}

// ------------------------------------------------------------------ splitting phases
// Phase `phase` (< kSplitPhases) of a scene with split triangles, over chunk `chunk` of
// its triangles (of its references in the last phase); the two scans are one item each.
__device__ __noinline__ void splitPhase(const BatchParams& B, const BatchSceneDev& S, uint32_t phase, uint32_t chunk) {
    const SplitParams& P = S.split;
    const uint32_t b0 = chunk * B.buildChunk, b1 = min(P.n, b0 + B.buildChunk);
    switch (phase) {
        case 0: splitBoundsRange(P, b0, b1); break;
        case 1: splitWeightRange(P, chunk, b0, b1); break;
        case 2: splitScanWeights(P, S.splitChunks); break;
        case 3: splitCountRange(P, chunk, b0, b1); break;
        case 4: scanBlockSums<uint32_t>(P.blockSums, S.splitChunks, nullptr); break;
        case 5: splitSlotsRange(P, chunk, b0, b1); break;
        default: {
            const uint32_t m = P.n + P.budget;
            splitEmitRange<false>(P, b0, min(m, b0 + B.buildChunk));  // the prep phase takes the centroids
        }
    }
}

// ------------------------------------------------------------------ the persistent kernel
__global__ void batchInitKernel(BatchParams B) {
    const size_t doneWords = (size_t)B.sceneCount * kBatchPhases;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < max(doneWords, (size_t)B.itemCount);
         i += (size_t)gridDim.x * blockDim.x) {
        if (i < doneWords) B.done[i] = 0u;
        if (i < B.itemCount) B.traceCounters[i] = 0ull;
        if (i < B.sceneCount) {
            uint32_t* b = B.scenes[i].bounds;
            b[0] = b[1] = b[2] = 0xFFFFFFFFu;  // running minima start at the top
            b[3] = b[4] = b[5] = 0u;           // running maxima at the bottom
            if (B.scenes[i].splitPhases) {     // the splitting's scene box and totals
                const SplitParams& q = B.scenes[i].split;
                q.sceneBounds[0] = q.sceneBounds[1] = q.sceneBounds[2] = 0xFFFFFFFFu;
                q.sceneBounds[3] = q.sceneBounds[4] = q.sceneBounds[5] = 0u;
                q.totals[0] = q.totals[1] = 0ull;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.head = 0ull, *B.abort = 0u;
}

__global__ void __launch_bounds__(256, 2) batchKernel(BatchParams B) {
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long itemS;
    __shared__ uint32_t skipS;
    for (;;) {
        if (threadIdx.x == 0) itemS = atomicAdd(B.head, 1ull);
        __syncthreads();
        const unsigned long long item = itemS;
        if (item >= B.itemCount) break;
        const BatchItemDev it = B.items[item];
        const BatchSceneDev& S = B.scenes[it.scene];
        unsigned long long t0 = 0, t1 = 0;
        if (threadIdx.x == 0) {
            if (B.profile) t0 = globalTimerNs();
            if (it.phase > 0) waitPhase(B, it.scene, it.phase - 1, it.waitCount);
            skipS = *(volatile uint32_t*)B.abort;
            if (B.profile) t1 = globalTimerNs();
        }
        __syncthreads();
        const bool wide = S.bits != 30;
        const uint32_t ph = it.phase - S.splitPhases;  // the phase among the build's own (after the splitting)
        if (skipS) {
            // aborted launch: the item only counts as done
        } else if (S.small) {
            if (it.phase == 0) {
                if (wide)
                    buildWhole<unsigned long long, 21>(S, B.sortChunkKeys, smem);
                else
                    buildWhole<uint32_t, 10>(S, B.sortChunkKeys, smem);
            } else {
                traceChunk(B, S, it.chunk, item, smem);
            }
        } else if (it.phase < S.splitPhases) {
            splitPhase(B, S, it.phase, it.chunk);
        } else if (ph == 0) {
            const uint32_t b0 = it.chunk * B.buildChunk;
            prepRange(S, b0, min(S.n, b0 + B.buildChunk));
        } else if (ph <= 3 * S.passes) {
            const uint32_t p = (ph - 1) / 3, step = (ph - 1) % 3;
            if (step == 0) {
                if (wide)
                    sortUpsweepChunk<unsigned long long, 21>(S, it.chunk, p, B.sortChunkKeys, smem);
                else
                    sortUpsweepChunk<uint32_t, 10>(S, it.chunk, p, B.sortChunkKeys, smem);
            } else if (step == 1) {
                sortScanScene(S, smem);
            } else if (wide) {
                sortDownsweepChunk<unsigned long long>(S, it.chunk, p, B.sortChunkKeys, smem);
            } else {
                sortDownsweepChunk<uint32_t>(S, it.chunk, p, B.sortChunkKeys, smem);
            }
        } else if (ph == 3 * S.passes + 1) {
            const uint32_t b0 = it.chunk * B.buildChunk, b1 = min(S.n - 1 + S.cluster, b0 + B.buildChunk);
            if (S.cluster) {
                if (wide)
                    clusterTopologyRange<unsigned long long>(S, b0, b1);
                else
                    clusterTopologyRange<uint32_t>(S, b0, b1);
            } else if (wide) {
                karrasRange<unsigned long long>(S, b0, b1);
            } else {
                karrasRange<uint32_t>(S, b0, b1);
            }
        } else if (S.cluster && ph == 3 * S.passes + 2) {
            const uint32_t w = kWalkLeavesPerThread * blockDim.x, b0 = it.chunk * w;
            clusterRange(clusterParamsOf(S), b0, min(S.n, b0 + w), reinterpret_cast<ClusterWarpList*>(smem));
        } else if (ph == 3 * S.passes + 2 + S.cluster) {
            const uint32_t b0 = it.chunk * B.buildChunk;
            fitRange(S, b0, min(S.n, b0 + B.buildChunk));
        } else if ((S.quant | S.wide8) && ph == 3 * S.passes + 3 + S.cluster) {
            const uint32_t m = S.n > 1 ? S.n - 1 : 1u, b1 = min(m, (it.chunk + 1) * B.buildChunk);
            for (uint32_t k = it.chunk * B.buildChunk + threadIdx.x; k < b1; k += blockDim.x) {
                if (S.quant) quantizeWideNode(S.wide + kWideWords * (size_t)k, S.qnodes + kQuantWords * (size_t)k);
                if (S.wide8) wide8Node(S.nodes, S.n, k, S.w8nodes);
            }
        } else {
            traceChunk(B, S, it.chunk, item, smem);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(B.done + (size_t)it.scene * kBatchPhases + it.phase, 1u);
            if (B.profile) {
                unsigned smid;
                asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
                unsigned long long* pr = B.profile + 4 * item;
                pr[0] = t0, pr[1] = t1, pr[2] = globalTimerNs(), pr[3] = ((unsigned long long)smid << 32) | blockIdx.x;
            }
        }
    }
}

// ------------------------------------------------------------------ host side
struct BatchObject {
    int device = 0;
    uint32_t sceneCount = 0, itemCount = 0;
    uint32_t blockSize = 128, blocks = 0;
    size_t smem = 0;
    std::vector<grtGeometry> geometries;
    std::vector<uint32_t> vertexCounts;
    void* deviceMem = nullptr;  // descriptors, items, counters, scratch, global stack
    size_t deviceBytes = 0;
    BatchParams params{};
    grtBatchInfo info{};
    bool useGraph = false;
    cudaGraphExec_t graph = nullptr;
};

static std::mutex g_batchMutex;
static std::vector<BatchObject*> g_batches;

static BatchObject* findBatch(grtBatch b) {
    std::lock_guard<std::mutex> g(g_batchMutex);
    for (BatchObject* o : g_batches)
        if (reinterpret_cast<grtBatch>(o) == b) return o;
    return nullptr;
}

static grtError resolveBatchOptions(const grtBatchOptions* o, grtBatchOptions* r) {
    grtBatchOptions d{};
    if (o) d = *o;
    if (!d.blockSize) d.blockSize = 128;
    if (!d.sharedStackDepth) d.sharedStackDepth = 16;
    if (!d.globalStackDepth) d.globalStackDepth = 64;
    if (!(d.compactThreshold > 0.f)) d.compactThreshold = 0.75f;
    if (!d.smallScenePrims) d.smallScenePrims = 8192;
    if (!d.sortChunkTiles) d.sortChunkTiles = 8;
    if (!d.buildChunk) d.buildChunk = 16384;
    if (!d.traceChunk) d.traceChunk = 16384;
    if (!d.sceneGroup) d.sceneGroup = 32;
    if (!d.waitLimitMs) d.waitLimitMs = 2000;
    if (d.blockSize != 64 && d.blockSize != 128 && d.blockSize != 256) return GRT_ERROR_INVALID_PARAMETER;
    if (d.sharedStackDepth > 32 || d.globalStackDepth > 4096) return GRT_ERROR_INVALID_PARAMETER;
    if (d.compactThreshold > 1.f || d.sortChunkTiles > 4096) return GRT_ERROR_INVALID_PARAMETER;
    if (d.buildChunk > (1u << 24) || d.traceChunk > (1u << 24)) return GRT_ERROR_INVALID_PARAMETER;
    if (d.flags & ~(uint32_t)(GRT_BATCH_FLAG_GRAPH | GRT_BATCH_FLAG_PROFILE | GRT_BATCH_FLAG_TEST_EXPIRE_WAIT))
        return GRT_ERROR_INVALID_PARAMETER;
    if (d.waitLimitMs > 600000) return GRT_ERROR_INVALID_PARAMETER;
    *r = d;
    return GRT_SUCCESS;
}

static void destroyBatchObject(BatchObject* o) {
    if (o->graph) cudaGraphExecDestroy(o->graph);
    if (o->deviceMem) cudaFree(o->deviceMem);
    delete o;
}

}  // namespace grt

using namespace grt;

extern "C" {

grtError grtCreateBatch(grtContext ctx, const grtBatchScene* scenes, uint32_t sceneCount,
                        const grtBatchOptions* options, grtBatch* out) {
    if (!ctx || !out || (sceneCount && !scenes)) return GRT_ERROR_INVALID_PARAMETER;
    grtBatchOptions opt;
    grtError e = resolveBatchOptions(options, &opt);
    if (e != GRT_SUCCESS) return e;
    Context* c = asContext(ctx);
    const uint32_t bs = opt.blockSize;
    const uint32_t warps = bs / 32;
    const uint32_t chunkKeys = opt.sortChunkTiles * bs * kBlockSortItems;

    // scene descriptors (pointers into the scratch region are filled in below)
    std::vector<BatchSceneDev> S(sceneCount);
    std::vector<size_t> scratchOff(sceneCount);
    size_t scratch = 0;
    for (uint32_t i = 0; i < sceneCount; ++i) {
        const grtBatchScene& in = scenes[i];
        uint32_t n = 0;
        e = validateGeometryInput(&in.input, &n);
        if (e != GRT_SUCCESS) return e;
        BvhObject* o = findBvh(in.geometry);
        if (!o || o->primType != GRT_PRIMITIVE_TRIANGLE_MESH || in.input.type != GRT_PRIMITIVE_TRIANGLE_MESH ||
            o->primCount != n)
            return GRT_ERROR_INVALID_PARAMETER;
        if (in.rayCount && (!in.rays || !in.hits || ((uintptr_t)in.rays & 15) || ((uintptr_t)in.hits & 3)))
            return GRT_ERROR_INVALID_PARAMETER;
        BatchSceneDev& d = S[i];
        const bool split = o->split && n > 0;
        const uint32_t m = n == 0 ? 0u : o->leafCount;  // leaves: the triangles, or their references
        d.src = primSource(&in.input, n);
        d.kind = 0;  // triangles
        d.n = m;
        d.rays = in.rayCount;
        d.bits = o->mortonBits;
        d.cluster = (buildsBySubtreeClustering(o) && m >= 2) ? 1u : 0u;
        d.small = n <= opt.smallScenePrims && !d.cluster && !split;
        d.sortChunks = std::max(1u, ceilDiv(m, chunkKeys));
        d.passes = (d.bits + 7) / 8;
        d.quant = (o->quant && n > 0) ? 1u : 0u;
        d.wide8 = (o->wide8 && n > 0) ? 1u : 0u;
        d.splitPhases = split ? kSplitPhases : 0u;
        d.splitChunks = split ? ceilDiv(n, opt.buildChunk) : 0u;
        d.split = SplitParams{};
        if (split) {
            d.split.src = d.src;  // the triangles (kind 0)
            d.split.n = n;
            d.split.budget = o->splitBudget;
            d.split.blocks = d.splitChunks;
            d.split.error = &workspace(c)->error;
            d.src.kind = 2;  // the build reads the references (pointer set below)
            d.src.count = m;
        }
        d.tracePhase = d.small ? 1u : d.splitPhases + 3u * d.passes + 3u + d.cluster + (d.quant | d.wide8);
        d.rayBuf = (const float4*)in.rays;
        d.hitBuf = (uint32_t*)in.hits;
        d.nodes = (float4*)o->nodes;
        d.wide = (float4*)o->wide;
        d.qnodes = (float4*)o->qnodes;
        d.w8nodes = (float4*)o->w8nodes;
        d.leaves = o->leaves;
        d.parents = (uint32_t*)o->parents;
        d.primToLeaf = o->primToLeaf;
        d.header = o->dHeader;
        d.error = &workspace(c)->error;
        const size_t kb = d.bits == 30 ? 4 : 8, nn = std::max(m, 1u);  // per leaf (reference)
        scratchOff[i] = scratch;
        scratch += 256 + alignUp(16 * nn, 256) + 2 * alignUp(kb * nn, 256) + 2 * alignUp(4 * nn, 256) +
                   alignUp(4 * (size_t)kBlockRadix * d.sortChunks, 256) + alignUp(4 * nn, 256);
        if (d.cluster)  // LBVH child words, parent entries, range starts; clusters, numbers, counts, flags
            scratch += 2 * alignUp(8 * nn, 256) + alignUp(16 * nn, 256) + alignUp(32 * nn, 256) + 2 * alignUp(4 * nn, 256);
        if (split)  // scene box and totals; weights / shares, first slots; chunk sums; slot triangles; references
            scratch += 256 + 2 * alignUp(4 * (size_t)n, 256) + alignUp(8 * (size_t)d.splitChunks, 256) +
                       alignUp(4 * (size_t)d.splitChunks, 256) + alignUp(4 * nn, 256) + alignUp(32 * nn, 256);
    }

    // work items. Scenes go in groups of opt.sceneGroup, largest first: a group's build
    // phases in rounds (every scene's phase r before any scene's phase r+1), then the
    // group's trace items, largest scene first. The largest scenes, whose rays are the
    // longest, are thus built first and their traces overlap the later groups' builds.
    // Every wait points to a phase of the same scene placed earlier in the queue.
    std::vector<BatchItemDev> items;
    std::vector<uint32_t> order(sceneCount);
    for (uint32_t i = 0; i < sceneCount; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return S[a].n > S[b].n; });
    auto phaseItems = [&](const BatchSceneDev& d, uint32_t ph) -> uint32_t {
        if (ph == d.tracePhase) return ceilDiv(d.rays, opt.traceChunk);
        if (d.small) return ph == 0 ? 1u : 0u;
        if (ph < d.splitPhases)  // the two scans are one item; the references have chunks of their own
            return (ph == 2 || ph == 4) ? 1u : ph == kSplitPhases - 1 ? ceilDiv(d.n, opt.buildChunk) : d.splitChunks;
        ph -= d.splitPhases;
        if (ph == 0) return ceilDiv(d.n, opt.buildChunk);
        if (ph <= 3 * d.passes) return (ph - 1) % 3 == 1 ? 1u : d.sortChunks;
        if (ph == 3 * d.passes + 1) return ceilDiv(d.n - 1 + d.cluster, opt.buildChunk);  // clustered: every leaf too
        if (d.cluster && ph == 3 * d.passes + 2) return ceilDiv(d.n, kWalkLeavesPerThread * opt.blockSize);
        if (ph == 3 * d.passes + 2) return ceilDiv(d.n, opt.buildChunk);  // the fit
        if (d.cluster && ph == 3 * d.passes + 3) return ceilDiv(d.n, opt.buildChunk);  // the fit after clustering
        if ((d.quant | d.wide8) && ph == 3 * d.passes + 3 + d.cluster)
            return ceilDiv(std::max(d.n - 1, 1u), opt.buildChunk);
        return 0u;
    };
    for (uint32_t g0 = 0; g0 < sceneCount; g0 += opt.sceneGroup) {
        const uint32_t g1 = std::min(sceneCount, g0 + opt.sceneGroup);
        for (uint32_t r = 0; r < kBatchPhases; ++r)
            for (uint32_t k = g0; k < g1; ++k) {
                const uint32_t i = order[k];
                const BatchSceneDev& d = S[i];
                if (r >= d.tracePhase) continue;
                const uint32_t cnt = phaseItems(d, r), wait = r ? phaseItems(d, r - 1) : 0u;
                for (uint32_t c = 0; c < cnt; ++c) items.push_back(BatchItemDev{i, r, c, wait});
            }
        for (uint32_t k = g0; k < g1; ++k) {
            const uint32_t i = order[k];
            const BatchSceneDev& d = S[i];
            const uint32_t cnt = phaseItems(d, d.tracePhase), wait = phaseItems(d, d.tracePhase - 1);
            for (uint32_t c = 0; c < cnt; ++c) items.push_back(BatchItemDev{i, d.tracePhase, c, wait});
        }
    }

    if (opt.flags & GRT_BATCH_FLAG_TEST_EXPIRE_WAIT) {
        for (BatchItemDev& it : items)
            if (it.phase > 0) {  // one completion more than the phase before it has items
                ++it.waitCount;
                break;
            }
    }

    // launch shape and the device allocation
    BatchObject* b = new BatchObject();
    b->device = deviceOf(c);
    b->sceneCount = sceneCount;
    b->itemCount = (uint32_t)items.size();
    b->blockSize = bs;
    const size_t stackSmem = (size_t)bs * traceSmemWords(opt.sharedStackDepth) * 4;
    const size_t sortSmem = ((size_t)warps * kBlockRadix + 2 * kBlockRadix) * 4;
    const size_t clusterSmem = (size_t)warps * sizeof(ClusterWarpList);
    b->smem = std::max<size_t>(std::max(std::max(stackSmem, sortSmem), clusterSmem), 33 * 4);
    int perSm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSm, batchKernel, (int)bs, b->smem) != cudaSuccess ||
        perSm < 1)
        perSm = 1;
    b->blocks = (uint32_t)perSm * (uint32_t)smCount(c);
    const size_t threads = (size_t)b->blocks * bs;
    const size_t offScenes = 0;
    const size_t offItems = alignUp(sizeof(BatchSceneDev) * std::max(sceneCount, 1u), 256);
    const size_t offDone = offItems + alignUp(sizeof(BatchItemDev) * std::max<size_t>(items.size(), 1), 256);
    const size_t offHead = offDone + alignUp(4 * (size_t)std::max(sceneCount, 1u) * kBatchPhases, 256);
    const size_t offTrace = offHead + 256;  // head (8 bytes) and abort flag (4 bytes at +64)
    const size_t offStack = offTrace + alignUp(8 * std::max<size_t>(items.size(), 1), 256);
    const size_t offProfile = offStack + alignUp(threads * opt.globalStackDepth * 4, 256);
    const bool profile = (opt.flags & GRT_BATCH_FLAG_PROFILE) != 0;
    const size_t offScratch = offProfile + (profile ? alignUp(32 * std::max<size_t>(items.size(), 1), 256) : 0);
    b->deviceBytes = offScratch + scratch;
    if (cudaMalloc(&b->deviceMem, b->deviceBytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return GRT_ERROR_OUT_OF_MEMORY;
    }
    char* base = static_cast<char*>(b->deviceMem);
    for (uint32_t i = 0; i < sceneCount; ++i) {
        BatchSceneDev& d = S[i];
        const size_t kb = d.bits == 30 ? 4 : 8, nn = std::max(d.n, 1u);
        char* p = base + offScratch + scratchOff[i];
        d.bounds = (uint32_t*)p, p += 256;
        d.centroids = (float4*)p, p += alignUp(16 * nn, 256);
        d.keys[0] = p, p += alignUp(kb * nn, 256);
        d.keys[1] = p, p += alignUp(kb * nn, 256);
        d.vals[0] = (uint32_t*)p, p += alignUp(4 * nn, 256);
        d.vals[1] = (uint32_t*)p, p += alignUp(4 * nn, 256);
        d.counts = (uint32_t*)p, p += alignUp(4 * (size_t)kBlockRadix * d.sortChunks, 256);
        d.flags = (uint32_t*)p, p += alignUp(4 * nn, 256);
        if (d.cluster) {
            d.topoChild = (uint2*)p, p += alignUp(8 * nn, 256);
            d.topoParent = (uint32_t*)p, p += alignUp(8 * nn, 256);
            d.topoRecord = (uint4*)p, p += alignUp(16 * nn, 256);
            d.clusters = (float4*)p, p += alignUp(32 * nn, 256);
            d.freeIds = (uint32_t*)p, p += alignUp(4 * nn, 256);
            d.clusterFlags = (uint32_t*)p, p += alignUp(4 * nn, 256);
        }
        if (d.splitPhases) {
            SplitParams& q = d.split;
            const size_t nt = q.n;
            q.sceneBounds = (uint32_t*)p;
            q.totals = (unsigned long long*)(p + 32), p += 256;
            q.counts = (uint32_t*)p, p += alignUp(4 * nt, 256);
            q.firstSlot = (uint32_t*)p, p += alignUp(4 * nt, 256);
            q.weightSums = (unsigned long long*)p, p += alignUp(8 * (size_t)d.splitChunks, 256);
            q.blockSums = (uint32_t*)p, p += alignUp(4 * (size_t)d.splitChunks, 256);
            q.slotTriangle = (uint32_t*)p, p += alignUp(4 * nn, 256);
            q.refs = (float4*)p;
            d.src.refs = q.refs;
        }
    }
    cudaError_t ce = cudaSuccess;
    if (sceneCount)
        ce = cudaMemcpy(base + offScenes, S.data(), sizeof(BatchSceneDev) * sceneCount, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !items.empty())
        ce = cudaMemcpy(base + offItems, items.data(), sizeof(BatchItemDev) * items.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        destroyBatchObject(b);
        return GRT_ERROR_CUDA;
    }
    BatchParams& P = b->params;
    P.scenes = (const BatchSceneDev*)(base + offScenes);
    P.items = (const BatchItemDev*)(base + offItems);
    P.itemCount = (uint32_t)items.size();
    P.sceneCount = sceneCount;
    P.done = (uint32_t*)(base + offDone);
    P.head = (unsigned long long*)(base + offHead);
    P.abort = (uint32_t*)(base + offHead + 64);
    P.profile = profile ? (unsigned long long*)(base + offProfile) : nullptr;
    P.traceCounters = (unsigned long long*)(base + offTrace);
    P.error = &workspace(c)->error;
    P.globalStack = (uint32_t*)(base + offStack);
    P.globalDepth = opt.globalStackDepth;
    P.globalStride = (uint32_t)threads;
    P.sharedDepth = opt.sharedStackDepth;
    P.refillBelow = (uint32_t)(opt.compactThreshold * 32.f);
    P.buildChunk = opt.buildChunk;
    P.sortChunkKeys = chunkKeys;
    P.traceChunk = opt.traceChunk;
    P.waitNs = (unsigned long long)opt.waitLimitMs * 1000000ull;
    b->useGraph = (opt.flags & GRT_BATCH_FLAG_GRAPH) != 0;
    for (uint32_t i = 0; i < sceneCount; ++i) {
        b->geometries.push_back(scenes[i].geometry);
        b->vertexCounts.push_back(scenes[i].input.triangleMesh.vertexCount);
    }
    grtBatchInfo& I = b->info;
    I.sceneCount = sceneCount;
    I.itemCount = (uint32_t)items.size();
    I.blocks = b->blocks;
    I.blockSize = bs;
    I.deviceBytes = b->deviceBytes;
    I.smallScenes = 0;
    for (const BatchSceneDev& d : S) I.smallScenes += d.small;
    {
        std::lock_guard<std::mutex> g(g_batchMutex);
        g_batches.push_back(b);
    }
    *out = reinterpret_cast<grtBatch>(b);
    return GRT_SUCCESS;
}

static grtError enqueueBatch(BatchObject* b, cudaStream_t s) {
    batchInitKernel<<<64, 256, 0, s>>>(b->params);
    if (b->params.itemCount) batchKernel<<<b->blocks, b->blockSize, b->smem, s>>>(b->params);
    GRT_LAUNCH_CHECK();
    return GRT_SUCCESS;
}

grtError grtBatchBuildTrace(grtContext ctx, grtBatch batch, void* stream) {
    BatchObject* b = findBatch(batch);
    if (!ctx || !b) return GRT_ERROR_INVALID_PARAMETER;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->useGraph) {
        if (!b->graph) {
            // capture once on a private stream, then replay on the caller's
            cudaStream_t cap;
            GRT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            grtError e = GRT_SUCCESS;
            if (ce == cudaSuccess) {
                e = enqueueBatch(b, cap);
                ce = cudaStreamEndCapture(cap, &g);
            }
            if (ce == cudaSuccess && e == GRT_SUCCESS) ce = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (e != GRT_SUCCESS) return e;
            GRT_CUDA(ce);
        }
        GRT_CUDA(cudaGraphLaunch(b->graph, s));
    } else {
        grtError e = enqueueBatch(b, s);
        if (e != GRT_SUCCESS) return e;
    }
    noteLaunches(b->params.itemCount ? 2 : 1);
    for (size_t i = 0; i < b->geometries.size(); ++i) {
        BvhObject* o = findBvh(b->geometries[i]);
        if (o) {
            o->built = true;
            o->vertexCount = b->vertexCounts[i];
        }
    }
    return GRT_SUCCESS;
}

grtError grtGetBatchProfile(grtContext ctx, grtBatch batch, grtBatchItemRecord* records, uint32_t capacity,
                            uint32_t* count) {
    BatchObject* b = findBatch(batch);
    if (!ctx || !b || !count || (capacity && !records)) return GRT_ERROR_INVALID_PARAMETER;
    *count = b->params.profile ? b->itemCount : 0u;
    if (!b->params.profile || capacity == 0) return GRT_SUCCESS;
    const uint32_t n = std::min(capacity, b->itemCount);
    std::vector<unsigned long long> raw(4 * (size_t)n);
    std::vector<BatchItemDev> items(n);
    GRT_CUDA(cudaMemcpy(raw.data(), b->params.profile, raw.size() * 8, cudaMemcpyDeviceToHost));
    GRT_CUDA(cudaMemcpy(items.data(), b->params.items, items.size() * sizeof(BatchItemDev), cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < n; ++i) {
        grtBatchItemRecord& r = records[i];
        r.scene = items[i].scene;
        r.phase = items[i].phase;
        r.chunk = items[i].chunk;
        r.sm = (uint32_t)(raw[4 * i + 3] >> 32);
        r.startNs = raw[4 * i];
        r.readyNs = raw[4 * i + 1];
        r.endNs = raw[4 * i + 2];
    }
    return GRT_SUCCESS;
}

grtError grtGetBatchInfo(grtContext ctx, grtBatch batch, grtBatchInfo* info) {
    BatchObject* b = findBatch(batch);
    if (!ctx || !b || !info) return GRT_ERROR_INVALID_PARAMETER;
    *info = b->info;
    return GRT_SUCCESS;
}

grtError grtDestroyBatch(grtContext ctx, grtBatch batch) {
    BatchObject* b = findBatch(batch);
    if (!ctx || !b) return GRT_ERROR_INVALID_PARAMETER;
    {
        std::lock_guard<std::mutex> g(g_batchMutex);
        g_batches.erase(std::find(g_batches.begin(), g_batches.end(), b));
    }
    destroyBatchObject(b);
    return GRT_SUCCESS;
}

}  // extern "C"
