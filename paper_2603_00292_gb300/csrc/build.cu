// LBVH construction on the GPU: primitive boxes and centroid bounds, Morton codes,
// a stable LSD radix sort, Karras hierarchy emission and a bottom-up fit with
// atomic visit counters, plus the top-level (instance) build.
//
// Method: the paper describes BVH construction, its surface-area cost and refitting
// from child boxes (Sec. 6.2) and the geometry / scene build API (Sec. 7.2-7.3). The
// linear build follows Karras, "Maximizing Parallelism in the Construction of BVHs,
// Octrees, and k-d Trees" (HPG 2012): node i of the n-1 internal nodes finds its
// range and split from the sorted codes alone, and leaves walk up to the root,
// the second child to arrive at a node computing its box.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "cluster.cuh"
#include "lbvh_block.cuh"
#include "ploc.cuh"
#include "split.cuh"

namespace grt {

// ======================================================================= radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;
constexpr int kMaxSortBlocks = 1024;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;

size_t sortScratchBytes(uint32_t) { return (size_t)kRadix * kMaxSortBlocks * sizeof(uint32_t); }

struct SortGrid {
    unsigned tiles, tilesPerBlock, blocks;
};

static SortGrid sortGrid(uint32_t n, int sms) {
    SortGrid g;
    g.tiles = std::max(1u, ceilDiv(n, kSortTile));
    unsigned want = std::min<unsigned>(g.tiles, std::min<unsigned>(kMaxSortBlocks, (unsigned)std::max(1, sms) * 2));
    g.tilesPerBlock = ceilDiv(g.tiles, want);
    g.blocks = ceilDiv(g.tiles, g.tilesPerBlock);
    return g;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) sortUpsweep(const K* __restrict__ keys, uint32_t n, int shift,
                                                            uint32_t tilesPerBlock, uint32_t* __restrict__ counts,
                                                            uint32_t blocks) {
    __shared__ uint32_t h[kSortWarps][kRadix];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int d = tid; d < kSortWarps * kRadix; d += kSortThreads) (&h[0][0])[d] = 0;
    __syncthreads();
    const size_t begin = (size_t)blockIdx.x * tilesPerBlock * kSortTile;
    const size_t end = min((size_t)n, begin + (size_t)tilesPerBlock * kSortTile);
    for (size_t i = begin + tid; i < end; i += kSortThreads) {
        const uint32_t d = (uint32_t)(keys[i] >> shift) & (kRadix - 1);
        atomicAdd(&h[warp][d], 1u);
    }
    __syncthreads();
    for (int d = tid; d < kRadix; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
        counts[(size_t)d * blocks + blockIdx.x] = s;
    }
}

// Exclusive prefix sum in place over `total` counters (one block).
__global__ void __launch_bounds__(kScanThreads) sortScan(uint32_t* __restrict__ counts, uint32_t total) {
    __shared__ uint32_t warpSums[kScanThreads / 32];
    __shared__ uint32_t carryS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carryS = 0;
    __syncthreads();
    for (uint32_t base = 0; base < total; base += kScanThreads * kScanItems) {
        uint32_t v[kScanItems];
        uint32_t sum = 0;
        const uint32_t my = base + (uint32_t)tid * kScanItems;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (my + i < total) ? counts[my + i] : 0u;
            sum += v[i];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warpSums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warpSums[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warpSums[lane] = wi - w;  // exclusive
        }
        __syncthreads();
        uint32_t run = carryS + warpSums[warp] + (incl - sum);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (my + i < total) counts[my + i] = run;
            run += v[i];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) carryS = run;
        __syncthreads();
    }
}

// Up to kFusedScanBlocks blocks the downsweep derives its digit offsets from the raw
// per-block counts itself (every block reads all kRadix x blocks counts from L2), so a
// radix pass is two launches instead of three; the offsets are those sortScan gives.
constexpr uint32_t kFusedScanBlocks = 64;

template <typename K, bool FUSED = false>
__global__ void __launch_bounds__(kSortThreads) sortDownsweep(const K* __restrict__ keysIn,
                                                              const uint32_t* __restrict__ valsIn,
                                                              K* __restrict__ keysOut, uint32_t* __restrict__ valsOut,
                                                              uint32_t n, int shift, uint32_t tilesPerBlock,
                                                              uint32_t tiles, const uint32_t* __restrict__ offsets,
                                                              uint32_t blocks) {
    __shared__ uint32_t warpHist[kSortWarps][kRadix];
    __shared__ uint32_t digitBase[kRadix];
    __shared__ uint32_t tileTotal[kRadix];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ltMask = (1u << lane) - 1u;
    if constexpr (FUSED) {
        static_assert(kSortThreads == kRadix, "one thread per digit");
        // offsets[d * blocks + b] are the raw counts: this block's base for digit d is the
        // sum of all counts of smaller digits plus those of earlier blocks in digit d
        uint32_t total = 0, before = 0;
        for (uint32_t b = 0; b < blocks; ++b) {
            const uint32_t c = offsets[(size_t)tid * blocks + b];
            total += c;
            before += b < blockIdx.x ? c : 0u;
        }
        uint32_t incl = total;  // exclusive scan of the digit totals over the block
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) tileTotal[warp] = incl;
        __syncthreads();
        uint32_t warpBase = 0;
        for (int w = 0; w < warp; ++w) warpBase += tileTotal[w];
        __syncthreads();
        digitBase[tid] = warpBase + incl - total + before;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) warpHist[w][tid] = 0;
    } else {
        for (int d = tid; d < kRadix; d += kSortThreads) {
            digitBase[d] = offsets[(size_t)d * blocks + blockIdx.x];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) warpHist[w][d] = 0;
        }
    }
    __syncthreads();
    const unsigned t0 = blockIdx.x * tilesPerBlock;
    const unsigned t1 = min(tiles, t0 + tilesPerBlock);
    for (unsigned tile = t0; tile < t1; ++tile) {
        const size_t base = (size_t)tile * kSortTile + (size_t)warp * 32 * kSortItems;
        K k[kSortItems];
        uint32_t v[kSortItems], dg[kSortItems], rank[kSortItems];
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const size_t idx = base + (size_t)i * 32 + lane;
            const bool ok = idx < n;
            k[i] = ok ? keysIn[idx] : (K)0;
            v[i] = ok ? valsIn[idx] : 0u;
            dg[i] = ok ? ((uint32_t)(k[i] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        }
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t peers = __match_any_sync(0xffffffffu, dg[i]);
            const int leader = __ffs(peers) - 1;
            const bool ok = dg[i] < kRadix;
            const uint32_t b = ok ? warpHist[warp][dg[i]] : 0u;
            __syncwarp();
            if (ok && lane == leader) warpHist[warp][dg[i]] = b + __popc(peers);
            __syncwarp();
            rank[i] = b + __popc(peers & ltMask);
        }
        __syncthreads();
        for (int d = tid; d < kRadix; d += kSortThreads) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t t = warpHist[w][d];
                warpHist[w][d] = run;
                run += t;
            }
            tileTotal[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            if (dg[i] < kRadix) {
                const uint32_t pos = digitBase[dg[i]] + warpHist[warp][dg[i]] + rank[i];
                keysOut[pos] = k[i];
                valsOut[pos] = v[i];
            }
        }
        __syncthreads();
        for (int d = tid; d < kRadix; d += kSortThreads) {
            digitBase[d] += tileTotal[d];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) warpHist[w][d] = 0;
        }
        __syncthreads();
    }
}

template <typename K>
static grtError radixSortT(Context* ctx, K* keys0, K* keys1, uint32_t* vals0, uint32_t* vals1, uint32_t n,
                           int significantBits, uint32_t* hist, cudaStream_t s, int* finalBuf) {
    const SortGrid g = sortGrid(n, smCount(ctx));
    const int passes = (significantBits + 7) / 8;
    K* kin = keys0;
    K* kout = keys1;
    uint32_t* vin = vals0;
    uint32_t* vout = vals1;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        sortUpsweep<K><<<g.blocks, kSortThreads, 0, s>>>(kin, n, shift, g.tilesPerBlock, hist, g.blocks);
        if (g.blocks <= kFusedScanBlocks) {
            sortDownsweep<K, true><<<g.blocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, g.tilesPerBlock,
                                                                      g.tiles, hist, g.blocks);
            noteLaunches(2);
        } else {
            sortScan<<<1, kScanThreads, 0, s>>>(hist, kRadix * g.blocks);
            sortDownsweep<K><<<g.blocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, g.tilesPerBlock,
                                                                g.tiles, hist, g.blocks);
            noteLaunches(3);
        }
        GRT_LAUNCH_CHECK();
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    *finalBuf = passes & 1;
    return GRT_SUCCESS;
}

grtError radixSort(Context* ctx, void* keys0, void* keys1, uint32_t* vals0, uint32_t* vals1, uint32_t n, int keyBytes,
                   int significantBits, uint32_t* hist, cudaStream_t s, int* finalBuf) {
    if (n == 0) {
        *finalBuf = 0;
        return GRT_SUCCESS;
    }
    if (keyBytes == 4)
        return radixSortT<uint32_t>(ctx, (uint32_t*)keys0, (uint32_t*)keys1, vals0, vals1, n, significantBits, hist, s,
                                    finalBuf);
    return radixSortT<unsigned long long>(ctx, (unsigned long long*)keys0, (unsigned long long*)keys1, vals0, vals1, n,
                                          significantBits, hist, s, finalBuf);
}

// ======================================================================= element kernels (A1-A7)
__global__ void __launch_bounds__(256) primCentroidKernel(PrimSource S, float4* __restrict__ centroids,
                                                          uint32_t* __restrict__ bounds) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < S.count;
    float3 c = make_float3(0.f, 0.f, 0.f);
    if (valid) {
        float3 v[3];
        c = boxCentroid(primBox(S, i, v));
        centroids[i] = make_float4(c.x, c.y, c.z, 0.f);
    }
    reduceBounds(c, valid, bounds);
}

template <typename K, int BITS>
__global__ void __launch_bounds__(256) mortonKernel(const float4* __restrict__ centroids, uint32_t n,
                                                    const uint32_t* __restrict__ bounds, K* __restrict__ keys,
                                                    uint32_t* __restrict__ vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = mortonCode<K, BITS>(centroids[i], bounds);
    vals[i] = i;
}

// One thread per internal node i in [0, n-2].
template <typename K>
__global__ void __launch_bounds__(256) karrasKernel(const K* __restrict__ keys, int n, float4* __restrict__ nodes,
                                                    uint32_t* __restrict__ parents) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) karrasNode<false>(keys, n, i, nodes, parents);
}

template <int KIND>  // 0 triangles, 1 AABB list, 2 instances
__global__ void __launch_bounds__(256) fitKernel(FitParams P) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) fitLeaf<KIND>(P, k);
}

// Quantised form of each of the m 4-wide nodes (the GRT_BUILD_QUANTIZED_NODES layout).
__global__ void __launch_bounds__(256) quantizeKernel(const float4* wide, uint32_t m, float4* qnodes) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) quantizeWideNode(wide + kWideWords * (size_t)k, qnodes + kQuantWords * (size_t)k);
}

// The 8-wide node of each of the m binary nodes of an n-primitive tree (the
// GRT_BUILD_WIDE8_NODES layout).
__global__ void __launch_bounds__(256) wide8Kernel(const float4* nodes, uint32_t n, uint32_t m, float4* w8) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) wide8Node(nodes, n, k, w8);
}

// The extra node formats of object o, after its fit.
static grtError launchNodeFormats(const BvhObject* o, cudaStream_t s) {
    if (o->qnodes) {
        quantizeKernel<<<ceilDiv(o->nodeCount, 256), 256, 0, s>>>((const float4*)o->wide, o->nodeCount,
                                                                  (float4*)o->qnodes);
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
    }
    if (o->w8nodes) {
        wide8Kernel<<<ceilDiv(o->nodeCount, 256), 256, 0, s>>>((const float4*)o->nodes, o->leafCount, o->nodeCount,
                                                               (float4*)o->w8nodes);
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
    }
    return GRT_SUCCESS;
}

// ======================================================================= small builds
// Up to kSmallBuild primitives (kSmallScene instances) a build runs in one block of
// kSmallBuildThreads threads, as one launch, instead of a dozen grid-wide launches whose
// cost is their own latency at this size. The thresholds are where the measured times
// cross (one block against the graph of grid launches, 30-bit codes): a 1,280-triangle
// icosphere 0.070 vs 0.080 ms, 2,048 triangles 0.093 vs 0.083 ms, 4,050 triangles 0.19
// vs 0.095 ms; a top level of 4,000 instances 0.61 vs 0.15 ms (its FP64 instance setup
// runs on one SM). Up to kSharedFitMax primitives the block keeps the whole build on
// chip (bitonicSortShared, fitLeafShared).
#ifndef GRT_SMALL_BUILD
#define GRT_SMALL_BUILD 2048
#endif
constexpr uint32_t kSmallBuild = GRT_SMALL_BUILD;
constexpr uint32_t kSmallScene = 1024;
#ifndef GRT_SMALL_BUILD_THREADS
#define GRT_SMALL_BUILD_THREADS 1024
#endif
constexpr int kSmallBuildThreads = GRT_SMALL_BUILD_THREADS;
constexpr int kSmallSceneThreads = 512;  // its FP64 instance setup needs more than 64 registers

// Dynamic shared memory of a single-block build: the radix routines' histograms, or
// the on-chip path's sort pairs, boxes and counters for kSmallBuild primitives.
template <typename K>
constexpr size_t smallBuildSmemBytes() {
    return std::max(blockBuildSmemWords(kSmallBuildThreads) * sizeof(uint32_t),
                    std::max(sharedBuildBytes<K>(kSmallBuild), sharedBuildBytes<K>(kSmallScene)));
}

template <typename K, int BITS>
__global__ void __launch_bounds__(kSmallBuildThreads) smallBuildKernel(BlockBuild B) {
    extern __shared__ uint32_t smem[];
    buildWhole<K, BITS>(B, B.n > 0 ? B.n : 1u, smem, smallBuildSmemBytes<K>());  // one sort chunk
}

// Opts the single-block kernels in to their dynamic shared memory (above the default
// 48 KB for 63-bit codes), once per process and device.
template <class Kern>
static grtError allowSmem(Kern kernel, size_t bytes) {
    int dev = 0;
    GRT_CUDA(cudaGetDevice(&dev));
    static std::mutex m;
    static std::unordered_map<size_t, bool> done;
    const size_t key = (size_t)(void*)kernel ^ ((size_t)dev << 56);
    std::lock_guard<std::mutex> g(m);
    if (done.count(key)) return GRT_SUCCESS;
    GRT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done[key] = true;
    return GRT_SUCCESS;
}

// The device pointers of a build of object o in temporary buffer t.
static BlockBuild blockBuildOf(Context* c, BvhObject* o, const BuildLayout& L, char* t, uint32_t kind) {
    BlockBuild B{};
    B.n = o->leafCount;
    B.bits = o->mortonBits;
    B.sortChunks = 1;
    B.passes = (o->mortonBits + 7) / 8;
    B.kind = kind;
    B.nodes = (float4*)o->nodes;
    B.wide = (float4*)o->wide;
    B.qnodes = (float4*)o->qnodes;
    B.w8nodes = (float4*)o->w8nodes;
    B.leaves = o->leaves;
    B.parents = (uint32_t*)o->parents;
    B.primToLeaf = o->primToLeaf;
    B.header = o->dHeader;
    B.bounds = (uint32_t*)(t + L.bounds);
    B.centroids = (float4*)(t + L.centroids);
    B.keys[0] = t + L.keys[0];
    B.keys[1] = t + L.keys[1];
    B.vals[0] = (uint32_t*)(t + L.vals[0]);
    B.vals[1] = (uint32_t*)(t + L.vals[1]);
    B.counts = (uint32_t*)(t + L.hist);
    B.flags = (uint32_t*)(t + L.flags);
    B.error = &workspace(c)->error;
    return B;
}

static grtError launchSmallBuild(const BlockBuild& B, cudaStream_t s) {
    if (B.bits == 30) {
        const size_t smem = smallBuildSmemBytes<uint32_t>();
        grtError e = allowSmem(smallBuildKernel<uint32_t, 10>, smem);
        if (e != GRT_SUCCESS) return e;
        smallBuildKernel<uint32_t, 10><<<1, kSmallBuildThreads, smem, s>>>(B);
    } else {
        const size_t smem = smallBuildSmemBytes<unsigned long long>();
        grtError e = allowSmem(smallBuildKernel<unsigned long long, 21>, smem);
        if (e != GRT_SUCCESS) return e;
        smallBuildKernel<unsigned long long, 21><<<1, kSmallBuildThreads, smem, s>>>(B);
    }
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

// ======================================================================= instances (A8)
struct InstanceInput {
    const grtInstance* instances;
    const grtFrameSRT* frames;
    uint32_t count;
    float4* boxes;             // 2 float4 per instance: world lo, hi
    InstanceRecord* records;   // unsorted
    InstanceFrames64* inv64;   // per instance ID
    float4* fwd32;             // kFrameRows rows per instance ID
    float4* centroids;
    uint32_t* bounds;
    uint32_t wide8;            // the scene has 8-wide nodes: so must every instanced geometry
    uint32_t* error;           // the context's device error word
};

// Per instance: frame M = T R S and its inverse S^-1 R^T (x - T) in FP64 (rounded to
// float32), the world box of the bottom level's root box (8 corners through M,
// rounded outward), and the centroid of that box.
__device__ __forceinline__ float3 setupInstance(const InstanceInput& I, uint32_t i) {
    float3 c;
    const grtInstance in = I.instances[i];
    const grtFrameSRT f = I.frames[i];
    const BvhHeader* g = reinterpret_cast<const BvhHeader*>(in.geometry);
    double qx = f.rotation[0], qy = f.rotation[1], qz = f.rotation[2], qw = f.rotation[3];
    const double qn = sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
    qx /= qn, qy /= qn, qz /= qn, qw /= qn;
    const double R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)},
                            {2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)},
                            {2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)}};
    const double S[3] = {f.scale[0], f.scale[1], f.scale[2]};
    const double T[3] = {f.translation[0], f.translation[1], f.translation[2]};
    double F[3][4], G[3][4];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) {
            F[r][q] = R[r][q] * S[q];
            G[r][q] = R[q][r] / S[r];
        }
        F[r][3] = T[r];
        G[r][3] = -(G[r][0] * T[0] + G[r][1] * T[1] + G[r][2] * T[2]);
    }
    InstanceRecord rec;
    for (int r = 0; r < 3; ++r) {
        rec.inv[r] = make_float4(__double2float_rn(G[r][0]), __double2float_rn(G[r][1]),
                                 __double2float_rn(G[r][2]), __double2float_rn(G[r][3]));
        I.fwd32[kFrameRows * (size_t)i + 3 + r] =
            make_float4(__double2float_rn(G[r][0] - (double)rec.inv[r].x),
                        __double2float_rn(G[r][1] - (double)rec.inv[r].y),
                        __double2float_rn(G[r][2] - (double)rec.inv[r].z),
                        __double2float_rn(G[r][3] - (double)rec.inv[r].w));
        I.fwd32[kFrameRows * (size_t)i + r] = make_float4(__double2float_rn(F[r][0]), __double2float_rn(F[r][1]),
                                                 __double2float_rn(F[r][2]), __double2float_rn(F[r][3]));
        for (int q = 0; q < 4; ++q) I.inv64[i].inv[r][q] = G[r][q];
    }
    // an 8-wide top level walks 8-wide bottom levels; a 4-wide one the geometry's 4-wide
    // (or quantised) nodes. An 8-wide scene instancing a geometry without 8-wide nodes
    // latches GRT_ERROR_INVALID_PARAMETER and leaves that instance empty.
    const bool missing8 = I.wide8 && g->primCount > 0 && g->nodes8 == nullptr;
    if (missing8) latchError(I.error, GRT_ERROR_INVALID_PARAMETER);
    rec.nodes = I.wide8 ? g->nodes8 : g->nodes;
    rec.leaves = g->leaves;
    rec.instanceID = i;
    rec.typeBits = (g->geomType & 0xFFFFFFu) | ((uint32_t)g->primType << 24) |
                   (I.wide8 ? kInstWide8 : g->nodeFormat == 1 ? kInstQuant : 0u) |
                   ((g->flags & kHeaderSplit) ? kInstSplit : 0u) |
                   ((g->primCount == 0 || missing8) ? kInstEmpty : 0u);
    rec.geometry = g;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (g->primCount > 0) {
        for (int cnr = 0; cnr < 8; ++cnr) {
            const double p[3] = {(cnr & 1) ? g->rootHi[0] : g->rootLo[0], (cnr & 2) ? g->rootHi[1] : g->rootLo[1],
                                 (cnr & 4) ? g->rootHi[2] : g->rootLo[2]};
            for (int r = 0; r < 3; ++r) {
                const double w = F[r][0] * p[0] + F[r][1] * p[1] + F[r][2] * p[2] + F[r][3];
                lo[r] = fmin(lo[r], w);
                hi[r] = fmax(hi[r], w);
            }
        }
    } else {
        for (int r = 0; r < 3; ++r) lo[r] = hi[r] = T[r];  // empty: a point box, skipped by traversal
    }
    Box3 b;
    b.lo = make_float3(__double2float_rd(lo[0]), __double2float_rd(lo[1]), __double2float_rd(lo[2]));
    b.hi = make_float3(__double2float_ru(hi[0]), __double2float_ru(hi[1]), __double2float_ru(hi[2]));
    I.boxes[2 * (size_t)i] = make_float4(b.lo.x, b.lo.y, b.lo.z, 0.f);
    I.boxes[2 * (size_t)i + 1] = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.f);
    rec.worldLo = make_float4(b.lo.x, b.lo.y, b.lo.z, 0.f);
    rec.worldHi = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.f);
    rec.mask = in.mask ? in.mask : 0xFFFFFFFFu;
    rec.pad[0] = rec.pad[1] = rec.pad[2] = 0u;
    I.records[i] = rec;
    c = boxCentroid(b);
    I.centroids[i] = make_float4(c.x, c.y, c.z, 0.f);
    return c;
}

__global__ void __launch_bounds__(128) instanceSetupKernel(InstanceInput I) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < I.count;
    const float3 c = valid ? setupInstance(I, i) : make_float3(0.f, 0.f, 0.f);
    reduceBounds(c, valid, I.bounds);
}

// A top level of at most kSmallScene instances in one block and one launch: the bounds
// and fit counters initialised, the instance setup, then every LBVH step.
template <typename K, int BITS>
__global__ void __launch_bounds__(kSmallSceneThreads) smallSceneKernel(BlockBuild B, InstanceInput I) {
    extern __shared__ uint32_t smem[];
    if (threadIdx.x == 0) {
        B.bounds[0] = B.bounds[1] = B.bounds[2] = 0xFFFFFFFFu;
        B.bounds[3] = B.bounds[4] = B.bounds[5] = 0u;
    }
    for (uint32_t i = threadIdx.x; i + 1 < B.n; i += blockDim.x) B.flags[i] = 0u;
    __syncthreads();
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = threadIdx.x; i < I.count; i += blockDim.x) {
        const float3 c = setupInstance(I, i);
        mn[0] = fminf(mn[0], c.x), mn[1] = fminf(mn[1], c.y), mn[2] = fminf(mn[2], c.z);
        mx[0] = fmaxf(mx[0], c.x), mx[1] = fmaxf(mx[1], c.y), mx[2] = fmaxf(mx[2], c.z);
    }
    reduceBoxBounds(mn, mx, B.bounds);
    __syncthreads();
    buildWhole<K, BITS>(B, B.n, smem, smallBuildSmemBytes<K>());
}

// ======================================================================= host drivers
grtError validateGeometryInput(const grtGeometryBuildInput* in, uint32_t* count) {
    if (!in) return GRT_ERROR_INVALID_PARAMETER;
    if (in->type == GRT_PRIMITIVE_TRIANGLE_MESH) {
        const grtTriangleMeshPrimitive& m = in->triangleMesh;
        if (m.triangleCount && (!m.triangleIndices || !m.vertices || m.triangleStride < 12 || m.vertexStride < 12 ||
                                (m.triangleStride & 3) || (m.vertexStride & 3)))
            return GRT_ERROR_INVALID_PARAMETER;
        if (m.triangleCount >= 0x7FFFFFFFu) return GRT_ERROR_INVALID_PARAMETER;
        *count = m.triangleCount;
        return GRT_SUCCESS;
    }
    if (in->type == GRT_PRIMITIVE_AABB_LIST) {
        const grtAABBListPrimitive& a = in->aabbList;
        if (a.aabbCount && (!a.aabbs || a.aabbStride < 24 || (a.aabbStride & 3))) return GRT_ERROR_INVALID_PARAMETER;
        if (a.aabbCount >= 0x7FFFFFFFu) return GRT_ERROR_INVALID_PARAMETER;
        *count = a.aabbCount;
        return GRT_SUCCESS;
    }
    return GRT_ERROR_INVALID_PARAMETER;
}

PrimSource primSource(const grtGeometryBuildInput* in, uint32_t count) {
    PrimSource S{};
    S.count = count;
    if (in->type == GRT_PRIMITIVE_TRIANGLE_MESH) {
        S.kind = 0;
        S.idx = (const char*)in->triangleMesh.triangleIndices;
        S.idxStride = in->triangleMesh.triangleStride;
        S.verts = (const char*)in->triangleMesh.vertices;
        S.vertStride = in->triangleMesh.vertexStride;
    } else {
        S.kind = 1;
        S.boxes = (const char*)in->aabbList.aabbs;
        S.boxStride = in->aabbList.aabbStride;
    }
    return S;
}

// Live geometries created with GRT_BUILD_QUANTIZED_NODES. While there are none, no
// 4-wide walk can meet quantised nodes, and traces run kernels without that form.
static std::atomic<int> g_quantGeometries{0};
bool anyQuantGeometry() { return g_quantGeometries.load(std::memory_order_relaxed) > 0; }

// count primitives over leafCount leaves (more than count only with split triangles).
static grtError createBvhObject(uint32_t count, uint32_t primType, uint32_t geomType, uint32_t mortonBits,
                                BvhObject** out, bool quant = false, bool wide8 = false, uint32_t leafCount = 0) {
    BvhObject* o = new BvhObject();
    o->primCount = count;
    o->leafCount = count == 0 ? 0 : std::max(leafCount, count);
    o->nodeCount = count == 0 ? 0 : std::max(o->leafCount - 1, 1u);
    o->primType = primType;
    o->geomType = geomType;
    o->mortonBits = mortonBits;
    o->built = false;
    o->quant = quant;
    o->wide8 = wide8;
    size_t leafBytes = primType == GRT_PRIMITIVE_TRIANGLE_MESH ? 48 : (primType == kPrimScene ? 128 : 4);
    cudaError_t e = cudaMalloc(&o->dHeader, sizeof(BvhHeader));
    if (e == cudaSuccess && count) e = cudaMalloc(&o->nodes, (size_t)o->nodeCount * 64);
    if (e == cudaSuccess && count) e = cudaMalloc(&o->wide, (size_t)o->nodeCount * kWideWords * sizeof(float4));
    if (e == cudaSuccess && count && quant)
        e = cudaMalloc(&o->qnodes, (size_t)o->nodeCount * kQuantWords * sizeof(float4));
    if (e == cudaSuccess && count && wide8)
        e = cudaMalloc(&o->w8nodes, (size_t)o->nodeCount * kWide8Words * sizeof(float4));
    if (e == cudaSuccess && count) e = cudaMalloc(&o->leaves, (size_t)o->leafCount * leafBytes);
    if (e == cudaSuccess && count) e = cudaMalloc(&o->parents, (size_t)(2 * (size_t)o->leafCount - 1) * 4);
    if (e == cudaSuccess && count && primType != GRT_PRIMITIVE_AABB_LIST) e = cudaMalloc(&o->primToLeaf, (size_t)count * 4);
    if (e == cudaSuccess && count && primType == kPrimScene) e = cudaMalloc(&o->inv64, (size_t)count * sizeof(InstanceFrames64));
    if (e == cudaSuccess && count && primType == kPrimScene) e = cudaMalloc(&o->fwd32, (size_t)count * kFrameRows * sizeof(float4));
    BvhHeader h{};
    for (int a = 0; a < 3; ++a) h.rootLo[a] = INFINITY, h.rootHi[a] = -INFINITY;
    h.primCount = count;
    h.primType = (uint16_t)primType;
    h.nodeFormat = quant ? 1 : 0;
    h.nodes = (const float4*)(quant ? o->qnodes : o->wide);
    h.nodes8 = (const float4*)o->w8nodes;
    h.leaves = o->leaves;
    h.nodeCount = o->nodeCount;
    h.geomType = geomType;
    h.primToLeaf = o->primToLeaf;
    h.flags = o->leafCount > count ? kHeaderSplit : 0u;
    if (e == cudaSuccess) e = cudaMemcpy(o->dHeader, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(o->dHeader);
        cudaFree(o->nodes);
        cudaFree(o->wide);
        cudaFree(o->qnodes);
        cudaFree(o->w8nodes);
        cudaFree(o->leaves);
        cudaFree(o->parents);
        cudaFree(o->primToLeaf);
        cudaFree(o->inv64);
        cudaFree(o->fwd32);
        delete o;
        logf(GRT_LOG_ERROR, "allocation of a BVH with %u primitives failed: %s", count, cudaGetErrorString(e));
        return GRT_ERROR_OUT_OF_MEMORY;
    }
    registerBvh(o);
    if (quant) g_quantGeometries.fetch_add(1, std::memory_order_relaxed);
    *out = o;
    return GRT_SUCCESS;
}

static void destroyBvhObject(BvhObject* o) {
    if (o->quant) g_quantGeometries.fetch_sub(1, std::memory_order_relaxed);
    unregisterBvh(o->dHeader);
    cudaFree(o->dHeader);
    cudaFree(o->nodes);
    cudaFree(o->wide);
    cudaFree(o->qnodes);
    cudaFree(o->w8nodes);
    cudaFree(o->leaves);
    cudaFree(o->parents);
    cudaFree(o->primToLeaf);
    cudaFree(o->inv64);
    cudaFree(o->fwd32);
    delete o;
}

// Morton + sort + Karras over the centroids already in temp (count >= 1).
static grtError sortAndEmit(Context* ctx, BvhObject* o, const BuildLayout& L, char* temp, cudaStream_t s,
                            const uint32_t** sortedOut, bool emit = true, const void** sortedKeysOut = nullptr) {
    const uint32_t n = o->leafCount;
    const float4* cen = (const float4*)(temp + L.centroids);
    const uint32_t* bounds = (const uint32_t*)(temp + L.bounds);
    void* k0 = temp + L.keys[0];
    uint32_t* v0 = (uint32_t*)(temp + L.vals[0]);
    if (o->mortonBits == 30)
        mortonKernel<uint32_t, 10><<<ceilDiv(n, 256), 256, 0, s>>>(cen, n, bounds, (uint32_t*)k0, v0);
    else
        mortonKernel<unsigned long long, 21><<<ceilDiv(n, 256), 256, 0, s>>>(cen, n, bounds, (unsigned long long*)k0,
                                                                            v0);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    int fb = 0;
    grtError err = radixSort(ctx, temp + L.keys[0], temp + L.keys[1], (uint32_t*)(temp + L.vals[0]),
                             (uint32_t*)(temp + L.vals[1]), n, L.keyBytes, (int)o->mortonBits, (uint32_t*)(temp + L.hist),
                             s, &fb);
    if (err != GRT_SUCCESS) return err;
    const void* sk = temp + L.keys[fb];
    if (n >= 2 && emit) {
        if (o->mortonBits == 30)
            karrasKernel<uint32_t><<<ceilDiv(n - 1, 256), 256, 0, s>>>((const uint32_t*)sk, (int)n,
                                                                        (float4*)o->nodes, (uint32_t*)o->parents);
        else
            karrasKernel<unsigned long long><<<ceilDiv(n - 1, 256), 256, 0, s>>>(
                (const unsigned long long*)sk, (int)n, (float4*)o->nodes, (uint32_t*)o->parents);
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
    }
    *sortedOut = (const uint32_t*)(temp + L.vals[fb]);
    if (sortedKeysOut) *sortedKeysOut = sk;
    return GRT_SUCCESS;
}

static grtError resetBuildScratch(const BuildLayout& L, char* temp, uint32_t n, cudaStream_t s) {
    GRT_CUDA(cudaMemsetAsync(temp + L.bounds, 0xFF, 12, s));       // running minima start at the top
    GRT_CUDA(cudaMemsetAsync(temp + L.bounds + 12, 0x00, 12, s));  // running maxima start at the bottom
    GRT_CUDA(cudaMemsetAsync(temp + L.flags, 0, 4 * (size_t)std::max(n, 1u), s));
    return GRT_SUCCESS;
}

// ======================================================================= clustering builds
// A geometry's build method is fixed when it is created: 0 = LBVH (GRT_BUILD_PREFER_FAST),
// kSubtreeMethod = clustering inside the LBVH's subtrees (cluster.cuh), else PLOC with
// this search radius (ploc.cuh).
constexpr uint32_t kSubtreeMethod = 0xFFFFu;
static uint32_t buildMethod(const grtBuildOptions* opt) {
    return opt ? opt->buildFlags &
                     ~(uint32_t)(GRT_BUILD_QUANTIZED_NODES | GRT_BUILD_WIDE8_NODES | GRT_BUILD_SPLIT_TRIANGLES)
               : 0u;
}
static bool quantFlag(const grtBuildOptions* opt) { return opt && (opt->buildFlags & GRT_BUILD_QUANTIZED_NODES); }
static bool wide8Flag(const grtBuildOptions* opt) { return opt && (opt->buildFlags & GRT_BUILD_WIDE8_NODES); }
static uint32_t clusterRadius(const grtBuildOptions* opt) {
    const uint32_t m = buildMethod(opt);
    if (m == GRT_BUILD_PREFER_FAST) return 0;
    if (m == GRT_BUILD_CLUSTER_SUBTREES) return kSubtreeMethod;
    return m == GRT_BUILD_PREFER_BALANCED ? 8u : 32u;
}
static bool validBuildFlags(const grtBuildOptions* opt) {
    return !opt || (buildMethod(opt) <= 3u && !(quantFlag(opt) && wide8Flag(opt)));
}
static bool splitFlag(const grtBuildOptions* opt) { return opt && (opt->buildFlags & GRT_BUILD_SPLIT_TRIANGLES); }
// The split bit is for triangle meshes, with a factor in [0, 1] (0 = 0.5).
static bool validSplit(const grtBuildOptions* opt, uint32_t primType) {
    if (!splitFlag(opt)) return true;
    return primType == GRT_PRIMITIVE_TRIANGLE_MESH && opt->splitFactor >= 0.f && opt->splitFactor <= 1.f;
}
// The split factor of a split build (0 selects 0.5), and its extra references for n
// triangles: floor(factor * n).
static double splitFactorOf(const grtBuildOptions* opt) {
    return opt->splitFactor == 0.f ? 0.5 : (double)opt->splitFactor;
}
static uint32_t splitBudgetOf(uint32_t n, const grtBuildOptions* opt) {
    if (!splitFlag(opt)) return 0;
    return (uint32_t)std::floor(splitFactorOf(opt) * (double)n);
}
// Leaf count of a build: the primitives plus the split references; false past 2^31 - 2.
static bool leafCountOf(uint32_t n, const grtBuildOptions* opt, uint32_t* m) {
    const uint64_t total = (uint64_t)n + splitBudgetOf(n, opt);
    if (total >= 0x7FFFFFFFull) return false;
    *m = (uint32_t)total;
    return true;
}

static std::mutex g_methodLock;
static std::unordered_map<const BvhObject*, uint32_t> g_clusterRadius;  // objects with a PLOC build

static uint32_t radiusOf(const BvhObject* o) {
    std::lock_guard<std::mutex> g(g_methodLock);
    auto it = g_clusterRadius.find(o);
    return it == g_clusterRadius.end() ? 0u : it->second;
}

bool buildsBySubtreeClustering(const BvhObject* o) { return radiusOf(o) == kSubtreeMethod; }

// PLOC scratch after the LBVH layout: two cluster arrays (32 B per cluster), the
// per-position neighbour words, per-block counts and the barrier words.
struct PlocLayout {
    size_t clusters, pick, counts, sync, total;
};
static PlocLayout plocLayout(const BuildLayout& L, uint32_t n) {
    PlocLayout P{};
    const size_t m = n ? n : 1;
    P.clusters = alignUp(L.total, 256);
    P.pick = P.clusters + alignUp(2 * 32 * m, 256);
    P.counts = P.pick + alignUp(4 * m, 256);
    P.sync = P.counts + alignUp(8 * (size_t)ceilDiv(m, kPlocThreads), 256);
    P.total = P.sync + 256;
    return P;
}

// Per-geometry build: the LBVH topology into the temporary arrays (one thread per
// internal node), the arrival counters zeroed.
template <typename K>
__global__ void clusterTopologyKernel(ClusterParams C, const K* __restrict__ sortedKeys) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.n) karrasTopology<false>(sortedKeys, (int)i, C);
}

constexpr int kClusterThreads = 256;

__global__ void __launch_bounds__(kClusterThreads) clusterWalkKernel(ClusterParams C) {
    __shared__ ClusterWarpList lists[kClusterThreads / 32];
    const uint32_t begin = blockIdx.x * blockDim.x;
    clusterRange(C, begin, min(C.n, begin + blockDim.x), lists);
}

// Subtree-clustering scratch after the LBVH layout: the LBVH's child words, parent
// entries, per-node records (leaf range, clusters passed up), the per-position cluster
// and number arrays and arrival counters (72 B per primitive).
struct SubtreeLayout {
    size_t child, parent, record, clusters, freeIds, flags, total;
};
static SubtreeLayout subtreeLayout(const BuildLayout& L, uint32_t n) {
    SubtreeLayout Q{};
    const size_t m = n ? n : 1;
    Q.child = alignUp(L.total, 256);
    Q.parent = Q.child + alignUp(8 * m, 256);
    Q.record = Q.parent + alignUp(4 * 2 * m, 256);
    Q.clusters = Q.record + alignUp(16 * m, 256);
    Q.freeIds = Q.clusters + alignUp(32 * m, 256);
    Q.flags = Q.freeIds + alignUp(4 * m, 256);
    Q.total = Q.flags + alignUp(4 * m, 256);
    return Q;
}

// The subtree clustering over the sorted leaves (n >= 2): the LBVH topology into the
// scratch, then the bottom-up walk, which writes the final child words and parent links.
static grtError launchSubtreeCluster(Context* c, BvhObject* o, const BuildLayout& L, char* t, const PrimSource& S,
                                     const uint32_t* sorted, const void* sortedKeys, cudaStream_t s) {
    const uint32_t n = o->leafCount;
    const SubtreeLayout Q = subtreeLayout(L, n);
    ClusterParams C{};
    C.src = S;
    C.n = n;
    C.sortedPrims = sorted;
    C.topoChild = (uint2*)(t + Q.child);
    C.topoParent = (uint32_t*)(t + Q.parent);
    C.record = (uint4*)(t + Q.record);
    C.clusters = (float4*)(t + Q.clusters);
    C.freeIds = (uint32_t*)(t + Q.freeIds);
    C.flags = (uint32_t*)(t + Q.flags);
    C.nodes = (float4*)o->nodes;
    C.parents = (uint32_t*)o->parents;
    C.error = &workspace(c)->error;
    if (o->mortonBits == 30)
        clusterTopologyKernel<uint32_t><<<ceilDiv(n, 256), 256, 0, s>>>(C, (const uint32_t*)sortedKeys);
    else
        clusterTopologyKernel<unsigned long long><<<ceilDiv(n, 256), 256, 0, s>>>(
            C, (const unsigned long long*)sortedKeys);
    GRT_LAUNCH_CHECK();
    clusterWalkKernel<<<ceilDiv(n, kClusterThreads), kClusterThreads, 0, s>>>(C);
    GRT_LAUNCH_CHECK();
    noteLaunches(2);
    return GRT_SUCCESS;
}

// The clustering kernel over the sorted leaves: writes child words and parent links.
static grtError launchPloc(Context* c, BvhObject* o, const BuildLayout& L, char* t, const PrimSource& S,
                           const uint32_t* sorted, uint32_t radius, cudaStream_t s) {
    const uint32_t n = o->leafCount;
    const PlocLayout Q = plocLayout(L, n);
    PlocParams P{};
    P.src = S;
    P.n = n;
    P.radius = radius;
    P.sortedPrims = sorted;
    P.clusters[0] = (float4*)(t + Q.clusters);
    P.clusters[1] = P.clusters[0] + 2 * (size_t)n;
    P.pick = (uint32_t*)(t + Q.pick);
    P.blockCounts = (uint2*)(t + Q.counts);
    P.sync = (uint32_t*)(t + Q.sync);
    P.nodes = (float4*)o->nodes;
    P.parents = (uint32_t*)o->parents;
    P.error = &workspace(c)->error;
    P.waitNs = 2000000000ull;
    // below this many clusters one block is faster than the grid: a grid iteration costs
    // about 12 us (r = 8) to 24 us (r = 32) of round trips and barriers, the block's
    // neighbour search about 2r area tests per cluster on one SM
    P.finishAt = std::min<uint32_t>(kPlocFinishMax, 49152u / radius);
    const uint32_t blocks = std::min<uint32_t>(ceilDiv(n, kPlocThreads), 2u * (uint32_t)std::max(smCount(c), 1));
    GRT_CUDA(cudaMemsetAsync(P.sync, 0, 32, s));
    plocKernel<<<blocks, kPlocThreads, plocSmemBytes(radius), s>>>(P);
    GRT_LAUNCH_CHECK();
    plocFinishKernel<<<1, kPlocFinishThreads, plocFinishSmemBytes(), s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(2);
    return GRT_SUCCESS;
}

// Bytes of the method's temporary layout for leaf count n (the LBVH layout L plus the
// clustering scratch).
static size_t methodTempBytes(const BuildLayout& L, uint32_t n, uint32_t radius) {
    return radius == kSubtreeMethod ? subtreeLayout(L, n).total : radius ? plocLayout(L, n).total : L.total;
}

// Triangle-splitting scratch after the method's: the scene bounds and the two totals,
// per-triangle counts, per-block sums and the references (32 B each).
struct SplitLayout {
    size_t misc, counts, firstSlot, weightSums, blockSums, slotTriangle, refs, total;
};
static SplitLayout splitLayout(size_t base, uint32_t n, uint32_t m) {
    SplitLayout Q{};
    const size_t blocks = ceilDiv(std::max(n, 1u), kSplitThreads);
    Q.misc = alignUp(base, 256);
    Q.counts = Q.misc + 256;
    Q.firstSlot = Q.counts + alignUp(4 * (size_t)std::max(n, 1u), 256);
    Q.weightSums = Q.firstSlot + alignUp(4 * (size_t)std::max(n, 1u), 256);
    Q.blockSums = Q.weightSums + alignUp(8 * blocks, 256);
    Q.slotTriangle = Q.blockSums + alignUp(4 * blocks, 256);
    Q.refs = Q.slotTriangle + alignUp(4 * (size_t)std::max(m, 1u), 256);
    Q.total = Q.refs + alignUp(32 * (size_t)std::max(m, 1u), 256);
    return Q;
}
static SplitLayout splitLayoutOf(const BvhObject* o, const BuildLayout& L, uint32_t radius) {
    return splitLayout(methodTempBytes(L, o->leafCount, radius), o->primCount, o->leafCount);
}

// Splitting kernels of per-geometry builds (split.cuh): a chunk of kSplitThreads
// triangles (references) per block.
__device__ __forceinline__ void chunkOf(uint32_t count, uint32_t* b0, uint32_t* b1) {
    *b0 = blockIdx.x * blockDim.x;
    *b1 = min(count, *b0 + blockDim.x);
}

__global__ void __launch_bounds__(kSplitThreads) splitBoundsKernel(SplitParams P) {
    uint32_t b0, b1;
    chunkOf(P.n, &b0, &b1);
    splitBoundsRange(P, b0, b1);
}

__global__ void __launch_bounds__(kSplitThreads) splitWeightKernel(SplitParams P) {
    uint32_t b0, b1;
    chunkOf(P.n, &b0, &b1);
    splitWeightRange(P, blockIdx.x, b0, b1);
}

__global__ void __launch_bounds__(kSplitScanThreads) splitScanWeightsKernel(SplitParams P) {
    splitScanWeights(P, P.blocks);
}

__global__ void __launch_bounds__(kSplitThreads) splitCountKernel(SplitParams P) {
    uint32_t b0, b1;
    chunkOf(P.n, &b0, &b1);
    splitCountRange(P, blockIdx.x, b0, b1);
}

__global__ void __launch_bounds__(kSplitScanThreads) splitScanKernel(SplitParams P) {
    scanBlockSums<uint32_t>(P.blockSums, P.blocks, nullptr);
}

__global__ void __launch_bounds__(kSplitThreads) splitSlotsKernel(SplitParams P) {
    uint32_t b0, b1;
    chunkOf(P.n, &b0, &b1);
    splitSlotsRange(P, blockIdx.x, b0, b1);
}

__global__ void __launch_bounds__(kSplitThreads) splitEmitKernel(SplitParams P) {
    uint32_t r0, r1;
    chunkOf(P.n + P.budget, &r0, &r1);
    splitEmitRange<true>(P, r0, r1);
}

// The splitting launches of a split build (o->primCount >= 1 triangles): references,
// their centroids and the centroid bounds, in the scratch the rest of the build reads.
static grtError launchSplit(Context* c, BvhObject* o, const BuildLayout& L, char* t, const PrimSource& S,
                            uint32_t radius, cudaStream_t s) {
    const SplitLayout Q = splitLayoutOf(o, L, radius);
    SplitParams P{};
    P.src = S;
    P.n = o->primCount;
    P.budget = o->splitBudget;
    P.sceneBounds = (uint32_t*)(t + Q.misc);
    P.totals = (unsigned long long*)(t + Q.misc + 32);
    P.counts = (uint32_t*)(t + Q.counts);
    P.weightSums = (unsigned long long*)(t + Q.weightSums);
    P.blockSums = (uint32_t*)(t + Q.blockSums);
    P.firstSlot = (uint32_t*)(t + Q.firstSlot);
    P.slotTriangle = (uint32_t*)(t + Q.slotTriangle);
    P.blocks = ceilDiv(P.n, kSplitThreads);
    P.refs = (float4*)(t + Q.refs);
    P.centroids = (float4*)(t + L.centroids);
    P.centroidBounds = (uint32_t*)(t + L.bounds);
    P.error = &workspace(c)->error;
    GRT_CUDA(cudaMemsetAsync(t + Q.misc, 0xFF, 12, s));       // running minima start at the top
    GRT_CUDA(cudaMemsetAsync(t + Q.misc + 12, 0x00, 36, s));  // maxima at the bottom, totals at 0
    splitBoundsKernel<<<P.blocks, kSplitThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitWeightKernel<<<P.blocks, kSplitThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitScanWeightsKernel<<<1, kSplitScanThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitCountKernel<<<P.blocks, kSplitThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitScanKernel<<<1, kSplitScanThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitSlotsKernel<<<P.blocks, kSplitThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    splitEmitKernel<<<ceilDiv((size_t)P.n + P.budget, kSplitThreads), kSplitThreads, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(7);
    return GRT_SUCCESS;
}

// The launch sequence of a geometry BUILD (above kSmallBuild) or UPDATE on stream s:
// scratch reset, centroids and bounds, Morton codes, the radix passes, the hierarchy
// (Karras emission, or PLOC clustering when radius > 0), the fit.
static grtError issueGeometryBuild(Context* c, BvhObject* o, uint32_t op, const grtGeometryBuildInput* input,
                                   const BuildLayout& L, char* t, const PrimSource& S, cudaStream_t s,
                                   uint32_t radius = 0) {
    const uint32_t n = o->leafCount;
    grtError e = resetBuildScratch(L, t, n, s);
    if (e != GRT_SUCCESS) return e;
    const uint32_t* sorted = nullptr;
    if (op == GRT_BUILD_OPERATION_BUILD) {
        if (o->split) {
            e = launchSplit(c, o, L, t, S, radius, s);
            if (e != GRT_SUCCESS) return e;
        } else {
            primCentroidKernel<<<ceilDiv(n, 256), 256, 0, s>>>(S, (float4*)(t + L.centroids),
                                                               (uint32_t*)(t + L.bounds));
            GRT_LAUNCH_CHECK();
            noteLaunches(1);
        }
        const void* sortedKeys = nullptr;
        e = sortAndEmit(c, o, L, t, s, &sorted, radius == 0, &sortedKeys);
        if (e != GRT_SUCCESS) return e;
        if (radius == kSubtreeMethod && n >= 2) {
            e = launchSubtreeCluster(c, o, L, t, S, sorted, sortedKeys, s);
            if (e != GRT_SUCCESS) return e;
        } else if (radius != 0 && n >= 2) {
            e = launchPloc(c, o, L, t, S, sorted, radius, s);
            if (e != GRT_SUCCESS) return e;
        }
    }
    FitParams P{};
    P.src = S;
    P.n = n;
    P.sortedPrims = sorted;  // null for UPDATE: IDs come from the leaves
    P.nodes = (float4*)o->nodes;
    P.wide = (float4*)o->wide;
    P.leaves = o->leaves;
    P.primToLeaf = o->primToLeaf;
    P.parents = (const uint32_t*)o->parents;
    P.flags = (uint32_t*)(t + L.flags);
    P.header = o->dHeader;
    if (input->type == GRT_PRIMITIVE_TRIANGLE_MESH)
        fitKernel<0><<<ceilDiv(n, 256), 256, 0, s>>>(P);
    else
        fitKernel<1><<<ceilDiv(n, 256), 256, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return launchNodeFormats(o, s);
}

// Repeated BUILDs of a geometry from the same buffers replay a CUDA graph of the launch
// sequence. Every kernel argument is a function of the build input (addresses, strides,
// counts), the temporary buffer, the object's own arrays and the device, so a graph
// captured once serves every later build with the same description: new vertex data in
// the same buffers is read by the replay. The graph is captured on a private stream and
// launched on the caller's; a different description captures again, and a caller's
// stream that is itself being captured gets the launches directly.
struct BuildKey {
    grtGeometryBuildInput input;
    const void* temp;
    int device;
    uint32_t radius;
    bool operator==(const BuildKey& k) const { return std::memcmp(this, &k, sizeof(*this)) == 0; }
};
struct BuildGraph {
    BuildKey key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;
};
static std::mutex g_buildGraphLock;
static std::unordered_map<const BvhObject*, BuildGraph> g_buildGraphs;
unsigned long long launchCountNow();  // context.cu

static void dropBuildGraph(const BvhObject* o) {
    std::lock_guard<std::mutex> g(g_buildGraphLock);
    auto it = g_buildGraphs.find(o);
    if (it == g_buildGraphs.end()) return;
    cudaGraphExecDestroy(it->second.exec);
    g_buildGraphs.erase(it);
}

static grtError replayOrCaptureBuild(Context* c, BvhObject* o, const grtGeometryBuildInput* input,
                                     const BuildLayout& L, char* t, const PrimSource& S, cudaStream_t s,
                                     uint32_t radius) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (s && cudaStreamIsCapturing(s, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    if (cap != cudaStreamCaptureStatusNone) {  // the caller is capturing: issue directly
        grtError e = issueGeometryBuild(c, o, GRT_BUILD_OPERATION_BUILD, input, L, t, S, s, radius);
        if (e == GRT_SUCCESS) o->built = true;
        return e;
    }
    BuildKey key;
    std::memset(&key, 0, sizeof(key));
    key.input.type = input->type;  // only the fields the launches read
    if (input->type == GRT_PRIMITIVE_TRIANGLE_MESH)
        key.input.triangleMesh = input->triangleMesh;
    else
        key.input.aabbList = input->aabbList;
    key.temp = t;
    key.device = deviceOf(c);
    key.radius = radius;
    std::lock_guard<std::mutex> g(g_buildGraphLock);
    auto it = g_buildGraphs.find(o);
    if (it != g_buildGraphs.end() && !(it->second.key == key)) {
        cudaGraphExecDestroy(it->second.exec);
        g_buildGraphs.erase(it);
        it = g_buildGraphs.end();
    }
    if (it == g_buildGraphs.end()) {
        cudaStream_t cs = nullptr;
        GRT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const unsigned long long before = launchCountNow();
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        grtError e = ce == cudaSuccess
                         ? issueGeometryBuild(c, o, GRT_BUILD_OPERATION_BUILD, input, L, t, S, cs, radius)
                         : GRT_ERROR_CUDA;
        if (ce == cudaSuccess) ce = cudaStreamEndCapture(cs, &graph);
        cudaGraphExec_t exec = nullptr;
        if (e == GRT_SUCCESS && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != GRT_SUCCESS || ce != cudaSuccess) {  // no graph: the launches go straight to s
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            e = issueGeometryBuild(c, o, GRT_BUILD_OPERATION_BUILD, input, L, t, S, s, radius);
            if (e == GRT_SUCCESS) o->built = true;
            return e;
        }
        BuildGraph bg;
        bg.key = key;
        bg.exec = exec;
        bg.launches = launchCountNow() - before;  // counted once at capture, for this first replay
        it = g_buildGraphs.emplace(o, bg).first;
    } else {
        noteLaunches((unsigned)it->second.launches);
    }
    GRT_CUDA(cudaGraphLaunch(it->second.exec, s));
    o->built = true;
    return GRT_SUCCESS;
}

}  // namespace grt

using namespace grt;

extern "C" {

grtError grtGetGeometryBuildTemporaryBufferSize(grtContext ctx, const grtGeometryBuildInput* input,
                                                const grtBuildOptions* options, size_t* sizeBytes) {
    uint32_t n = 0;
    if (!ctx || !sizeBytes) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateGeometryInput(input, &n);
    if (e != GRT_SUCCESS) return e;
    uint32_t m = 0;
    if (!validBuildFlags(options) || !validSplit(options, input->type) || !leafCountOf(n, options, &m))
        return GRT_ERROR_INVALID_PARAMETER;
    const BuildLayout L = buildLayout(m, resolveMortonBits(m, options), false);
    const size_t bytes = methodTempBytes(L, m, clusterRadius(options));
    *sizeBytes = splitFlag(options) ? splitLayout(bytes, n, m).total : bytes;
    return GRT_SUCCESS;
}

grtError grtCreateGeometry(grtContext ctx, const grtGeometryBuildInput* input, const grtBuildOptions* options,
                           grtGeometry* out) {
    uint32_t n = 0;
    if (!ctx || !out) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateGeometryInput(input, &n);
    if (e != GRT_SUCCESS) return e;
    uint32_t m = 0;
    if (!validBuildFlags(options) || !validSplit(options, input->type) || !leafCountOf(n, options, &m))
        return GRT_ERROR_INVALID_PARAMETER;
    if (clusterRadius(options) && m > kPlocIndex) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = nullptr;
    e = createBvhObject(n, input->type, input->geomType, resolveMortonBits(m, options), &o, quantFlag(options),
                        wide8Flag(options), m);
    if (e != GRT_SUCCESS) return e;
    o->split = splitFlag(options);
    o->splitFactor = o->split ? (float)splitFactorOf(options) : 0.f;
    o->splitBudget = m - n;
    if (clusterRadius(options)) {
        // the finishing block's shared memory is above the default limit
        cudaError_t ce = cudaFuncSetAttribute(plocFinishKernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)plocFinishSmemBytes());
        if (ce != cudaSuccess) {
            cudaGetLastError();
            destroyBvhObject(o);
            logf(GRT_LOG_ERROR, "clustering build: %s", cudaGetErrorString(ce));
            return GRT_ERROR_CUDA;
        }
        std::lock_guard<std::mutex> g(g_methodLock);
        g_clusterRadius[o] = clusterRadius(options);
    }
    *out = reinterpret_cast<grtGeometry>(o->dHeader);
    return GRT_SUCCESS;
}

grtError grtBuildGeometry(grtContext ctx, uint32_t op, const grtGeometryBuildInput* input,
                          const grtBuildOptions* options, void* temp, void* stream, grtGeometry geom) {
    uint32_t n = 0;
    if (!ctx || !geom) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateGeometryInput(input, &n);
    if (e != GRT_SUCCESS) return e;
    BvhObject* o = findBvh(geom);
    if (!o || o->primType == kPrimScene || o->primType != input->type || o->primCount != n)
        return GRT_ERROR_INVALID_PARAMETER;
    if (op != GRT_BUILD_OPERATION_BUILD && op != GRT_BUILD_OPERATION_UPDATE) return GRT_ERROR_INVALID_PARAMETER;
    if (op == GRT_BUILD_OPERATION_UPDATE && !o->built) return GRT_ERROR_NOT_BUILT;
    if (op == GRT_BUILD_OPERATION_UPDATE && o->split) return GRT_ERROR_INVALID_PARAMETER;
    if (n > 0 && (!temp || ((uintptr_t)temp & 15))) return GRT_ERROR_INVALID_PARAMETER;
    if (options && options->mortonBits && resolveMortonBits(o->leafCount, options) != o->mortonBits)
        return GRT_ERROR_INVALID_PARAMETER;
    if (options && (splitFlag(options) != o->split || (o->split && (float)splitFactorOf(options) != o->splitFactor)))
        return GRT_ERROR_INVALID_PARAMETER;
    const uint32_t radius = radiusOf(o);
    if (!validBuildFlags(options) || (options && clusterRadius(options) != radius)) return GRT_ERROR_INVALID_PARAMETER;
    if (options && (quantFlag(options) != o->quant || wide8Flag(options) != o->wide8))
        return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    o->geomType = input->geomType;
    if (input->type == GRT_PRIMITIVE_TRIANGLE_MESH) o->vertexCount = input->triangleMesh.vertexCount;
    if (n == 0) {
        o->built = true;
        return GRT_SUCCESS;
    }
    const BuildLayout L = buildLayout(o->leafCount, o->mortonBits, false);
    char* t = (char*)temp;
    PrimSource S = primSource(input, n);
    if (o->split) {  // the build reads the references the splitting writes
        S.kind = 2;
        S.count = o->leafCount;
        S.refs = (const float4*)(t + splitLayoutOf(o, L, radius).refs);
    }
    if (op == GRT_BUILD_OPERATION_BUILD && n <= kSmallBuild && radius == 0 && !o->split) {  // initialises its own scratch
        BlockBuild B = blockBuildOf(c, o, L, t, input->type == GRT_PRIMITIVE_TRIANGLE_MESH ? 0u : 1u);
        B.src = S;
        e = launchSmallBuild(B, s);
        if (e != GRT_SUCCESS) return e;
        o->built = true;
        return GRT_SUCCESS;
    }
    if (op == GRT_BUILD_OPERATION_BUILD) return replayOrCaptureBuild(c, o, input, L, t, S, s, radius);
    e = issueGeometryBuild(c, o, op, input, L, t, S, s);
    if (e != GRT_SUCCESS) return e;
    o->built = true;
    return GRT_SUCCESS;
}

grtError grtDestroyGeometry(grtContext ctx, grtGeometry geom) {
    BvhObject* o = findBvh(geom);
    if (!ctx || !o || o->primType == kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    dropBuildGraph(o);
    {
        std::lock_guard<std::mutex> g(g_methodLock);
        g_clusterRadius.erase(o);
    }
    destroyBvhObject(o);
    return GRT_SUCCESS;
}

static grtError validateSceneInput(const grtSceneBuildInput* in) {
    if (!in) return GRT_ERROR_INVALID_PARAMETER;
    if (in->instanceCount != in->frameCount) return GRT_ERROR_INVALID_PARAMETER;
    if (in->instanceCount && (!in->instances || !in->instanceFrames)) return GRT_ERROR_INVALID_PARAMETER;
    if (in->instanceCount >= 0x7FFFFFFFu) return GRT_ERROR_INVALID_PARAMETER;
    return GRT_SUCCESS;
}

grtError grtGetSceneBuildTemporaryBufferSize(grtContext ctx, const grtSceneBuildInput* input,
                                             const grtBuildOptions* options, size_t* sizeBytes) {
    if (!ctx || !sizeBytes) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateSceneInput(input);
    if (e != GRT_SUCCESS) return e;
    *sizeBytes = buildLayout(input->instanceCount, resolveMortonBits(input->instanceCount, options), true).total;
    return GRT_SUCCESS;
}

grtError grtCreateScene(grtContext ctx, const grtSceneBuildInput* input, const grtBuildOptions* options,
                        grtScene* out) {
    if (!ctx || !out) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateSceneInput(input);
    if (e != GRT_SUCCESS) return e;
    BvhObject* o = nullptr;
    if (!validBuildFlags(options)) return GRT_ERROR_INVALID_PARAMETER;
    e = createBvhObject(input->instanceCount, kPrimScene, 0, resolveMortonBits(input->instanceCount, options), &o,
                        false, wide8Flag(options));
    if (e != GRT_SUCCESS) return e;
    *out = reinterpret_cast<grtScene>(o->dHeader);
    return GRT_SUCCESS;
}

grtError grtBuildScene(grtContext ctx, uint32_t op, const grtSceneBuildInput* input, const grtBuildOptions* options,
                       void* temp, void* stream, grtScene scene) {
    if (!ctx || !scene) return GRT_ERROR_INVALID_PARAMETER;
    grtError e = validateSceneInput(input);
    if (e != GRT_SUCCESS) return e;
    BvhObject* o = findBvh(scene);
    if (!o || o->primType != kPrimScene || o->primCount != input->instanceCount) return GRT_ERROR_INVALID_PARAMETER;
    if (op != GRT_BUILD_OPERATION_BUILD && op != GRT_BUILD_OPERATION_UPDATE) return GRT_ERROR_INVALID_PARAMETER;
    const uint32_t n = o->primCount;
    if (n > 0 && (!temp || ((uintptr_t)temp & 15))) return GRT_ERROR_INVALID_PARAMETER;
    if (options && (!validBuildFlags(options) || wide8Flag(options) != o->wide8)) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        o->built = true;
        return GRT_SUCCESS;
    }
    // An update of a scene rebuilds its (small) top level: instance frames may move freely.
    const BuildLayout L = buildLayout(n, o->mortonBits, true);
    char* t = (char*)temp;
    InstanceInput I{};
    I.instances = input->instances;
    I.frames = input->instanceFrames;
    I.count = n;
    I.boxes = (float4*)(t + L.extra);
    I.records = (InstanceRecord*)(t + L.extra + alignUp(32 * (size_t)n, 256));
    I.centroids = (float4*)(t + L.centroids);
    I.bounds = (uint32_t*)(t + L.bounds);
    I.inv64 = o->inv64;
    I.fwd32 = o->fwd32;
    I.wide8 = o->wide8 ? 1u : 0u;
    I.error = &workspace(c)->error;
    if (n <= kSmallScene) {
        BlockBuild B = blockBuildOf(c, o, L, t, 2u);
        B.instBoxes = I.boxes;
        B.instRecords = I.records;
        if (B.bits == 30) {
            const size_t smem = smallBuildSmemBytes<uint32_t>();
            e = allowSmem(smallSceneKernel<uint32_t, 10>, smem);
            if (e != GRT_SUCCESS) return e;
            smallSceneKernel<uint32_t, 10><<<1, kSmallSceneThreads, smem, s>>>(B, I);
        } else {
            const size_t smem = smallBuildSmemBytes<unsigned long long>();
            e = allowSmem(smallSceneKernel<unsigned long long, 21>, smem);
            if (e != GRT_SUCCESS) return e;
            smallSceneKernel<unsigned long long, 21><<<1, kSmallSceneThreads, smem, s>>>(B, I);
        }
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
        o->built = true;
        return GRT_SUCCESS;
    }
    e = resetBuildScratch(L, t, n, s);
    if (e != GRT_SUCCESS) return e;
    instanceSetupKernel<<<ceilDiv(n, 128), 128, 0, s>>>(I);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    const uint32_t* sorted = nullptr;
    e = sortAndEmit(c, o, L, t, s, &sorted);
    if (e != GRT_SUCCESS) return e;
    FitParams P{};
    P.n = n;
    P.sortedPrims = sorted;
    P.nodes = (float4*)o->nodes;
    P.wide = (float4*)o->wide;
    P.leaves = o->leaves;
    P.parents = (const uint32_t*)o->parents;
    P.flags = (uint32_t*)(t + L.flags);
    P.header = o->dHeader;
    P.primToLeaf = o->primToLeaf;
    P.instBoxes = I.boxes;
    P.instRecords = I.records;
    fitKernel<2><<<ceilDiv(n, 256), 256, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    e = launchNodeFormats(o, s);
    if (e != GRT_SUCCESS) return e;
    o->built = true;
    return GRT_SUCCESS;
}

grtError grtDestroyScene(grtContext ctx, grtScene scene) {
    BvhObject* o = findBvh(scene);
    if (!ctx || !o || o->primType != kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    destroyBvhObject(o);
    return GRT_SUCCESS;
}

grtError grtSortTemporaryBufferSize(uint32_t count, uint32_t keyBits, size_t* sizeBytes) {
    if (!sizeBytes || (keyBits != 32 && keyBits != 64)) return GRT_ERROR_INVALID_PARAMETER;
    const size_t kb = keyBits / 8;
    *sizeBytes = alignUp(kb * std::max(count, 1u), 256) + alignUp(4 * (size_t)std::max(count, 1u), 256) +
                 sortScratchBytes(count);
    return GRT_SUCCESS;
}

grtError grtSortPairs(grtContext ctx, void* keys, uint32_t* values, uint32_t count, uint32_t keyBits,
                      uint32_t significantBits, void* temp, void* stream) {
    if (!ctx || (keyBits != 32 && keyBits != 64) || significantBits == 0 || significantBits > keyBits)
        return GRT_ERROR_INVALID_PARAMETER;
    if (count == 0) return GRT_SUCCESS;
    if (!keys || !values || !temp || ((uintptr_t)temp & 15)) return GRT_ERROR_INVALID_PARAMETER;
    const size_t kb = keyBits / 8;
    char* t = (char*)temp;
    void* k1 = t;
    uint32_t* v1 = (uint32_t*)(t + alignUp(kb * count, 256));
    uint32_t* hist = (uint32_t*)(t + alignUp(kb * count, 256) + alignUp(4 * (size_t)count, 256));
    cudaStream_t s = (cudaStream_t)stream;
    int fb = 0;
    grtError e = radixSort(asContext(ctx), keys, k1, values, v1, count, (int)kb, (int)significantBits, hist, s, &fb);
    if (e != GRT_SUCCESS) return e;
    if (fb == 1) {
        GRT_CUDA(cudaMemcpyAsync(keys, k1, kb * count, cudaMemcpyDeviceToDevice, s));
        GRT_CUDA(cudaMemcpyAsync(values, v1, 4 * (size_t)count, cudaMemcpyDeviceToDevice, s));
    }
    return GRT_SUCCESS;
}

}  // extern "C"
