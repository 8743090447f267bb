// LBVH build routines run by one thread block over a range of primitives, keys or
// nodes: centroids and bounds, the passes of a stable LSD radix sort (digit histograms,
// their scan, stable scatter), Karras emission and the bottom-up fit. The batched
// persistent kernel runs them as work items over chunks of many scenes; a small
// geometry or scene is built by one block running all of them in a row. Data written
// by other blocks earlier in the same launch is read with L1-bypassing loads.
#pragma once

#include "lbvh.cuh"

namespace grt {

constexpr int kBlockRadix = 256;
constexpr int kBlockSortItems = 8;  // keys per thread in a sort tile
constexpr int kBlockScanItems = 8;

// One LBVH build in device memory.
struct BlockBuild {
    PrimSource src;
    uint32_t n;
    uint32_t bits;        // Morton bits (30 or 63)
    uint32_t sortChunks;  // chunks of a radix pass
    uint32_t passes;      // radix passes
    uint32_t kind;        // 0 triangles, 1 AABB list, 2 instances
    uint32_t pad0;
    float4* nodes;
    float4* wide;
    void* leaves;
    uint32_t* parents;
    uint32_t* primToLeaf;
    BvhHeader* header;
    uint32_t* bounds;  // 6 ordered-int words
    float4* centroids;
    void* keys[2];
    uint32_t* vals[2];
    uint32_t* counts;  // kBlockRadix x sortChunks
    uint32_t* flags;   // fit visit counters
    uint32_t* error;   // the context's device error word
    const float4* instBoxes;            // instances: world boxes (2 float4 each)
    const InstanceRecord* instRecords;  // instances: unsorted records
};

// Shared memory a block needs for these routines, in 32-bit words.
__host__ __device__ constexpr size_t blockBuildSmemWords(uint32_t blockSize) {
    return (size_t)(blockSize / 32) * kBlockRadix + 2 * kBlockRadix;
}

__device__ __forceinline__ void loadBounds(const BlockBuild& S, uint32_t b[6]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) b[a] = __ldcg(S.bounds + a);
}

// Centroids of primitives [begin, end) (triangles or boxes), their bounds, and zeroed
// fit counters.
static __device__ __noinline__ void prepRange(const BlockBuild& S, uint32_t begin, uint32_t end) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        float3 v[3];
        const float3 c = boxCentroid(primBox(S.src, i, v));
        S.centroids[i] = make_float4(c.x, c.y, c.z, 0.f);
        mn[0] = fminf(mn[0], c.x), mn[1] = fminf(mn[1], c.y), mn[2] = fminf(mn[2], c.z);
        mx[0] = fmaxf(mx[0], c.x), mx[1] = fmaxf(mx[1], c.y), mx[2] = fmaxf(mx[2], c.z);
        if (i + 1 < S.n) S.flags[i] = 0u;
    }
    reduceBoxBounds(mn, mx, S.bounds);
}

// Digit histogram of chunk `chunk` of radix pass `pass` into counts[d * chunks + chunk].
// Pass 0 computes the Morton codes (and identity values) from the centroids first.
template <typename K, int BITS>
__device__ __noinline__ void sortUpsweepChunk(const BlockBuild& S, uint32_t chunk, uint32_t pass, uint32_t chunkKeys,
                                 uint32_t* smem) {
    const uint32_t warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    for (uint32_t d = threadIdx.x; d < warps * kBlockRadix; d += blockDim.x) smem[d] = 0u;
    __syncthreads();
    const int shift = 8 * (int)pass;
    const size_t begin = (size_t)chunk * chunkKeys;
    const size_t end = min((size_t)S.n, begin + chunkKeys);
    const K* kin = static_cast<const K*>(S.keys[pass & 1u]);
    uint32_t b[6];
    if (pass == 0) loadBounds(S, b);
    for (size_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        K k;
        if (pass == 0) {
            k = mortonCode<K, BITS>(__ldcg(S.centroids + i), b);
            static_cast<K*>(S.keys[0])[i] = k;
            S.vals[0][i] = (uint32_t)i;
        } else {
            k = __ldcg(kin + i);
        }
        atomicAdd(&smem[warp * kBlockRadix + ((uint32_t)(k >> shift) & (kBlockRadix - 1))], 1u);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < kBlockRadix; d += blockDim.x) {
        uint32_t sum = 0;
        for (uint32_t w = 0; w < warps; ++w) sum += smem[w * kBlockRadix + d];
        S.counts[(size_t)d * S.sortChunks + chunk] = sum;
    }
}

// Exclusive prefix sum in place over the scene's kBlockRadix x sortChunks histogram
// (digit-major, so each (digit, chunk) gets its first output position).
static __device__ __noinline__ void sortScanScene(const BlockBuild& S, uint32_t* smem) {
    uint32_t* warpSums = smem;        // 32
    uint32_t* carry = smem + 32;      // 1
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const uint32_t total = kBlockRadix * S.sortChunks;
    if (threadIdx.x == 0) *carry = 0u;
    __syncthreads();
    for (uint32_t base = 0; base < total; base += blockDim.x * kBlockScanItems) {
        uint32_t v[kBlockScanItems];
        uint32_t sum = 0;
        const uint32_t my = base + threadIdx.x * kBlockScanItems;
#pragma unroll
        for (int i = 0; i < kBlockScanItems; ++i) {
            v[i] = (my + i < total) ? __ldcg(S.counts + my + i) : 0u;
            sum += v[i];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        if (lane == 31u) warpSums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < warps ? warpSums[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= (uint32_t)o) wi += t;
            }
            if (lane < warps) warpSums[lane] = wi - w;
        }
        __syncthreads();
        uint32_t run = *carry + warpSums[warp] + (incl - sum);
#pragma unroll
        for (int i = 0; i < kBlockScanItems; ++i) {
            if (my + i < total) S.counts[my + i] = run;
            run += v[i];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) *carry = run;
        __syncthreads();
    }
}

// Stable scatter of chunk `chunk` of radix pass `pass`: tiles of blockDim x 16 keys in
// order; within a tile each warp ranks its 512 keys (match_any per digit) after the
// warps before it.
template <typename K>
__device__ __noinline__ void sortDownsweepChunk(const BlockBuild& S, uint32_t chunk, uint32_t pass, uint32_t chunkKeys,
                                   uint32_t* smem) {
    const uint32_t warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint32_t* warpHist = smem;                        // warps x kBlockRadix
    uint32_t* digitBase = smem + warps * kBlockRadix;  // kBlockRadix
    uint32_t* tileTotal = digitBase + kBlockRadix;     // kBlockRadix
    const uint32_t ltMask = (1u << lane) - 1u;
    const int shift = 8 * (int)pass;
    const K* kin = static_cast<const K*>(S.keys[pass & 1u]);
    const uint32_t* vin = S.vals[pass & 1u];
    K* kout = static_cast<K*>(S.keys[(pass + 1) & 1u]);
    uint32_t* vout = S.vals[(pass + 1) & 1u];
    for (uint32_t d = threadIdx.x; d < kBlockRadix; d += blockDim.x) {
        digitBase[d] = __ldcg(S.counts + (size_t)d * S.sortChunks + chunk);
        for (uint32_t w = 0; w < warps; ++w) warpHist[w * kBlockRadix + d] = 0u;
    }
    __syncthreads();
    const size_t begin = (size_t)chunk * chunkKeys;
    const size_t end = min((size_t)S.n, begin + chunkKeys);
    const size_t tileKeys = (size_t)blockDim.x * kBlockSortItems;
    for (size_t tile = begin; tile < end; tile += tileKeys) {
        const size_t base = tile + (size_t)warp * 32 * kBlockSortItems;
        K k[kBlockSortItems];
        uint32_t v[kBlockSortItems], dg[kBlockSortItems], rank[kBlockSortItems];
#pragma unroll
        for (int i = 0; i < kBlockSortItems; ++i) {
            const size_t idx = base + (size_t)i * 32 + lane;
            const bool ok = idx < end;
            k[i] = ok ? __ldcg(kin + idx) : (K)0;
            v[i] = ok ? __ldcg(vin + idx) : 0u;
            dg[i] = ok ? ((uint32_t)(k[i] >> shift) & (kBlockRadix - 1)) : (uint32_t)kBlockRadix;
        }
#pragma unroll
        for (int i = 0; i < kBlockSortItems; ++i) {
            const uint32_t peers = __match_any_sync(0xffffffffu, dg[i]);
            const int leader = __ffs(peers) - 1;
            const bool ok = dg[i] < (uint32_t)kBlockRadix;
            const uint32_t b = ok ? warpHist[warp * kBlockRadix + dg[i]] : 0u;
            __syncwarp();
            if (ok && lane == (uint32_t)leader) warpHist[warp * kBlockRadix + dg[i]] = b + __popc(peers);
            __syncwarp();
            rank[i] = b + __popc(peers & ltMask);
        }
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < kBlockRadix; d += blockDim.x) {
            uint32_t run = 0;
            for (uint32_t w = 0; w < warps; ++w) {
                const uint32_t t = warpHist[w * kBlockRadix + d];
                warpHist[w * kBlockRadix + d] = run;
                run += t;
            }
            tileTotal[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kBlockSortItems; ++i) {
            if (dg[i] < (uint32_t)kBlockRadix) {
                const uint32_t pos = digitBase[dg[i]] + warpHist[warp * kBlockRadix + dg[i]] + rank[i];
                if (pos < S.n) {  // always, given consistent histograms
                    kout[pos] = k[i];
                    vout[pos] = v[i];
                } else {
                    latchError(S.error, GRT_ERROR_INTERNAL);
                }
            }
        }
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < kBlockRadix; d += blockDim.x) {
            digitBase[d] += tileTotal[d];
            for (uint32_t w = 0; w < warps; ++w) warpHist[w * kBlockRadix + d] = 0u;
        }
        __syncthreads();
    }
}

template <typename K>
__device__ __noinline__ void karrasRange(const BlockBuild& S, uint32_t begin, uint32_t end) {
    const K* keys = static_cast<const K*>(S.keys[S.passes & 1u]);
    for (uint32_t i = begin + threadIdx.x; i < end; i += blockDim.x)
        karrasNode<true>(keys, (int)S.n, (int)i, S.nodes, S.parents);
}

static __device__ __noinline__ void fitRange(const BlockBuild& S, uint32_t begin, uint32_t end) {
    FitParams P{};
    P.src = S.src;
    P.n = S.n;
    P.sortedPrims = S.vals[S.passes & 1u];
    P.nodes = S.nodes;
    P.wide = S.wide;
    P.leaves = S.leaves;
    P.primToLeaf = S.primToLeaf;
    P.parents = S.parents;
    P.flags = S.flags;
    P.header = S.header;
    P.instBoxes = S.instBoxes;
    P.instRecords = S.instRecords;
    for (uint32_t k = begin + threadIdx.x; k < end; k += blockDim.x) {
        if (S.kind == 0)
            fitLeaf<0>(P, k);
        else if (S.kind == 1)
            fitLeaf<1>(P, k);
        else
            fitLeaf<2>(P, k);
    }
}

// Up to this many primitives, a single-block build sorts by rank in shared memory.
constexpr uint32_t kRankSortMax = 512;

// Stable sort of a small build's Morton codes in shared memory: key i goes to position
// #{j : k_j < k_i, or k_j = k_i and j < i}. A stable sort's output is unique, so this is
// the permutation the radix passes produce. The sorted keys and values go to the final
// ping-pong buffers (keys[passes & 1], vals[passes & 1]) as after the radix passes, and
// the sorted keys stay in shared memory (the first n keys of smem) for emission. Needs
// n * (sizeof(K) + 4) bytes of smem: codes, then ranks.
template <typename K, int BITS>
__device__ __noinline__ void rankSortShared(const BlockBuild& S, uint32_t* smem) {
    const uint32_t n = S.n;
    K* keys = reinterpret_cast<K*>(smem);
    uint32_t* rank = reinterpret_cast<uint32_t*>(keys + n);
    uint32_t b[6];
    loadBounds(S, b);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) keys[i] = mortonCode<K, BITS>(__ldcg(S.centroids + i), b);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const K k = keys[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < n; ++j) {
            const K kj = keys[j];
            r += (kj < k || (kj == k && j < i)) ? 1u : 0u;
        }
        rank[i] = r;
    }
    __syncthreads();
    K* kout = static_cast<K*>(S.keys[S.passes & 1u]);
    uint32_t* vout = S.vals[S.passes & 1u];
    K k[kRankSortMax / 64];  // this thread's keys, read before any is overwritten
    uint32_t c = 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) k[c++] = keys[i];
    __syncthreads();
    c = 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x, ++c) {
        const uint32_t r = rank[i];
        keys[r] = k[c];
        kout[r] = k[c];
        vout[r] = i;
    }
}

// The whole build of a small scene by one block, phase after phase.
template <typename K, int BITS>
// Every step's global writes are read by other threads of the same block after a
// block barrier, which orders them at block scope; no wider fence is needed here. Triangle
// and box builds start from uninitialised bounds and fit counters; an instance build
// expects both prepared with the centroids (its setup runs first).
__device__ __noinline__ void buildWhole(const BlockBuild& S, uint32_t chunkKeys, uint32_t* smem) {
    if (S.n == 0) return;
    if (S.kind != 2) {
        if (threadIdx.x == 0) {
            S.bounds[0] = S.bounds[1] = S.bounds[2] = 0xFFFFFFFFu;  // running minima start at the top
            S.bounds[3] = S.bounds[4] = S.bounds[5] = 0u;           // running maxima at the bottom
        }
        __syncthreads();
        prepRange(S, 0, S.n);
    }
    __syncthreads();
    const bool ranked = S.n <= kRankSortMax && blockDim.x >= 64 &&
                        (size_t)S.n * (sizeof(K) + 4) <= blockBuildSmemWords(blockDim.x) * sizeof(uint32_t);
    if (ranked) {
        rankSortShared<K, BITS>(S, smem);
        __syncthreads();
        const K* sorted = reinterpret_cast<const K*>(smem);
        for (uint32_t i = threadIdx.x; i + 1 < S.n; i += blockDim.x)
            karrasNode<false>(sorted, (int)S.n, (int)i, S.nodes, S.parents);
    } else {
        for (uint32_t p = 0; p < S.passes; ++p) {
            for (uint32_t c = 0; c < S.sortChunks; ++c) {
                sortUpsweepChunk<K, BITS>(S, c, p, chunkKeys, smem);
                __syncthreads();
            }
            sortScanScene(S, smem);
            __syncthreads();
            for (uint32_t c = 0; c < S.sortChunks; ++c) {
                sortDownsweepChunk<K>(S, c, p, chunkKeys, smem);
                __syncthreads();
            }
        }
        if (S.n >= 2) karrasRange<K>(S, 0, S.n - 1);
    }
    __syncthreads();
    fitRange(S, 0, S.n);
}

}  // namespace grt
