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
    float4* qnodes;    // quantised 4-wide nodes, written after the fit when not null
    float4* w8nodes;   // 8-wide nodes, written after the fit when not null
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

// Smallest power of two >= n (n >= 1).
__host__ __device__ constexpr uint32_t pow2Ceil(uint32_t n) {
    uint32_t m = 1;
    while (m < n) m <<= 1;
    return m;
}

// Up to this many primitives the on-chip path of a single-block build also keeps the
// fit's boxes, parent entries and child words in shared memory (fitLeafShared).
constexpr uint32_t kSharedFitMax = 2048;

// Shared memory of a single-block build's sort: m = pow2Ceil(n) elements of 8 bytes
// ((code << 32) | index for 30-bit codes) or 12 bytes (64-bit code, then index).
// Elements of the bitonic sort of n codes: a power of two, at least 64 (one chunk of
// two elements per lane of a warp).
__host__ __device__ constexpr uint32_t sortElems(uint32_t n) { return pow2Ceil(n) < 64u ? 64u : pow2Ceil(n); }

template <typename K>
__host__ __device__ constexpr size_t sharedSortBytes(uint32_t n) {
    return (size_t)sortElems(n) * (sizeof(K) == 4 ? 8 : 12);
}

// Shared memory of the on-chip path of a single-block build of n primitives, in bytes.
// n <= kSharedFitMax: [sort pairs, later the six box arrays of 2n-1 floats] [parent
// entries, 2n-1] [child words, n-1 pairs] [visit counters, n-1]. Larger n: [sort pairs]
// [visit counters, n].
__host__ __device__ constexpr size_t alignSmem(size_t b) { return (b + 15) & ~(size_t)15; }
template <typename K>
__host__ __device__ constexpr size_t sharedBuildBytes(uint32_t n) {
    return n <= kSharedFitMax
               ? alignSmem(sharedSortBytes<K>(n) > 24 * (2 * (size_t)n - 1) ? sharedSortBytes<K>(n)
                                                                           : 24 * (2 * (size_t)n - 1)) +
                     alignSmem(4 * (2 * (size_t)n - 1)) + alignSmem(8 * (size_t)n) + 4 * (size_t)n
               : alignSmem(sharedSortBytes<K>(n)) + 4 * (size_t)n;
}

// Stable sort of a small build's Morton codes in shared memory by Batcher's bitonic
// network (Batcher, "Sorting networks and their applications", 1968) over (code,
// index) pairs: the index breaks ties between equal codes, so the order is the stable
// order the radix passes produce. The pairs are padded to a power of two m with
// all-ones elements, which sort last. Each step compares m/2 disjoint pairs, one per
// thread. Afterwards the sorted codes are the first n entries of smem (as K) for
// emission, and codes and indices also go to the final ping-pong buffers
// (keys[passes & 1], vals[passes & 1]) as after the radix passes.
template <typename K, int BITS>
__device__ __noinline__ void bitonicSortShared(const BlockBuild& S, uint32_t* smem, uint32_t m) {
    const uint32_t n = S.n;
    uint32_t b[6];
    loadBounds(S, b);
    K* kout = static_cast<K*>(S.keys[S.passes & 1u]);
    uint32_t* vout = S.vals[S.passes & 1u];
    if constexpr (sizeof(K) == 4) {
        // Elements (code << 32) | index. Chunk q holds elements [64q, 64q + 64): lane l of
        // the warp that owns it keeps elements 64q + l and 64q + 32 + l in registers, so
        // the steps with j <= 32 run in registers (j = 32 within a lane, j < 32 between
        // lanes by shuffles) and only those with j >= 64 go through shared memory.
        unsigned long long* e = reinterpret_cast<unsigned long long*>(smem);
        const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
        const uint32_t chunks = m >> 6, owned = (chunks + warps - 1 - warp) / warps;  // chunks of this warp
        constexpr uint32_t kChunks = 4;  // m <= 8 blockDim.x
        unsigned long long x[kChunks][2];
#pragma unroll
        for (uint32_t c = 0; c < kChunks; ++c)
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t i = 64u * (warp + c * warps) + 32u * h + lane;
                x[c][h] = (c < owned && i < n)
                              ? ((unsigned long long)mortonCode<K, BITS>(__ldcg(S.centroids + i), b) << 32) | i
                              : ~0ull;
            }
        for (uint32_t k = 2; k <= m; k <<= 1) {
            if (k > 64) {
                __syncthreads();  // every thread has read the previous shared step's results
#pragma unroll
                for (uint32_t c = 0; c < kChunks; ++c)
                    if (c < owned) e[64u * (warp + c * warps) + lane] = x[c][0], e[64u * (warp + c * warps) + 32u + lane] = x[c][1];
                __syncthreads();
                for (uint32_t j = k >> 1; j >= 64; j >>= 1) {
                    for (uint32_t t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                        const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = i | j;
                        const unsigned long long a = e[i], c = e[l];
                        if ((a > c) == ((i & k) == 0)) e[i] = c, e[l] = a;  // ascending where bit k of i is clear
                    }
                    __syncthreads();
                }
#pragma unroll
                for (uint32_t c = 0; c < kChunks; ++c)
                    if (c < owned) x[c][0] = e[64u * (warp + c * warps) + lane], x[c][1] = e[64u * (warp + c * warps) + 32u + lane];
            }
            for (uint32_t j = (k >> 1) < 32u ? (k >> 1) : 32u; j > 0; j >>= 1) {
#pragma unroll
                for (uint32_t c = 0; c < kChunks; ++c) {
                    if (c >= owned) continue;  // warp-uniform
                    const uint32_t i0 = 64u * (warp + c * warps) + lane;
                    if (j == 32) {  // elements i0 and i0 + 32 of this lane (same bit k: k >= 64)
                        const unsigned long long lo = min(x[c][0], x[c][1]), hi = max(x[c][0], x[c][1]);
                        const bool asc = (i0 & k) == 0;
                        x[c][0] = asc ? lo : hi;
                        x[c][1] = asc ? hi : lo;
                    } else {
                        const bool lower = (lane & j) == 0;
#pragma unroll
                        for (uint32_t h = 0; h < 2; ++h) {
                            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[c][h], j);
                            const bool asc = ((i0 + 32u * h) & k) == 0;
                            x[c][h] = (lower == asc) ? min(x[c][h], y) : max(x[c][h], y);
                        }
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (uint32_t c = 0; c < kChunks; ++c)
            if (c < owned) e[64u * (warp + c * warps) + lane] = x[c][0], e[64u * (warp + c * warps) + 32u + lane] = x[c][1];
        __syncthreads();
        // unpack: the codes to the front of smem as K (through registers: the packed
        // elements are read before any code is written over them)
        constexpr uint32_t kMaxPer = 8;  // m / blockDim.x <= 4096 / 512
        unsigned long long mine[kMaxPer];
        uint32_t c = 0;
        for (uint32_t i = threadIdx.x; i < n && c < kMaxPer; i += blockDim.x) mine[c++] = e[i];
        __syncthreads();
        K* keys = reinterpret_cast<K*>(smem);
        c = 0;
        for (uint32_t i = threadIdx.x; i < n && c < kMaxPer; i += blockDim.x, ++c) {
            const K code = (K)(mine[c] >> 32);
            keys[i] = code;
            kout[i] = code;
            vout[i] = (uint32_t)mine[c];
        }
    } else {
        K* keys = reinterpret_cast<K*>(smem);
        uint32_t* idx = reinterpret_cast<uint32_t*>(keys + m);
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
            keys[i] = i < n ? mortonCode<K, BITS>(__ldcg(S.centroids + i), b) : ~(K)0;
            idx[i] = i < n ? i : kInvalid;
        }
        __syncthreads();
        for (uint32_t k = 2; k <= m; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                    const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = i | j;
                    const K ki = keys[i], kl = keys[l];
                    const uint32_t ii = idx[i], il = idx[l];
                    const bool greater = ki > kl || (ki == kl && ii > il);
                    if (greater == ((i & k) == 0)) {
                        keys[i] = kl, keys[l] = ki;
                        idx[i] = il, idx[l] = ii;
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            kout[i] = keys[i];
            vout[i] = idx[i];
        }
    }
}

// The bottom-up fit of a single-block build, counters in shared memory (flags, n - 1
// words, zeroed).
static __device__ __noinline__ void fitRangeBlock(const BlockBuild& S, uint32_t* flags) {
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
    for (uint32_t k = threadIdx.x; k < S.n; k += blockDim.x) {
        if (S.kind == 0)
            fitLeaf<0, true>(P, k, flags);
        else if (S.kind == 1)
            fitLeaf<1, true>(P, k, flags);
        else
            fitLeaf<2, true>(P, k, flags);
    }
}

// The fit of a single-block build of at most kSharedFitMax primitives, all in shared
// memory (fitLeafShared).
static __device__ __noinline__ void fitRangeShared(const BlockBuild& S, const SharedFit& F) {
    FitParams P{};
    P.src = S.src;
    P.n = S.n;
    P.sortedPrims = S.vals[S.passes & 1u];
    P.nodes = S.nodes;
    P.wide = S.wide;
    P.leaves = S.leaves;
    P.primToLeaf = S.primToLeaf;
    P.header = S.header;
    P.instBoxes = S.instBoxes;
    P.instRecords = S.instRecords;
    for (uint32_t k = threadIdx.x; k < S.n; k += blockDim.x) {
        if (S.kind == 0)
            fitLeafShared<0>(P, k, F);
        else if (S.kind == 1)
            fitLeafShared<1>(P, k, F);
        else
            fitLeafShared<2>(P, k, F);
    }
    __syncthreads();  // every box is in shared memory
    // the node arrays, one float4 row per thread and step, so that a warp's stores are
    // contiguous (binary nodes: 4 rows each; 4-wide nodes: 8 rows each)
    const uint32_t n = S.n;
    for (uint32_t q = threadIdx.x; q < 4 * (n - 1); q += blockDim.x) S.nodes[q] = binaryRowShared(F, n, q >> 2, q & 3u);
    for (uint32_t q = threadIdx.x; q < kWideWords * (n - 1); q += blockDim.x)
        S.wide[q] = wideRowShared(F, n, q / kWideWords, q % kWideWords);
}

// The whole build of a small scene by one block, phase after phase.
template <typename K, int BITS>
// Every step's global writes are read by other threads of the same block after a
// block barrier, which orders them at block scope; no wider fence is needed here. Triangle
// and box builds start from uninitialised bounds and fit counters; an instance build
// expects both prepared with the centroids (its setup runs first).
// With smemBytes >= sharedBuildBytes<K>(n) the sort, emission and fit run on chip
// (bitonicSortShared, emission from the shared codes, fitRangeBlock); otherwise the
// codes are ranked in shared memory (n <= kRankSortMax) or radix-sorted through the
// build temporary, and the fit uses the global counters.
__device__ __noinline__ void buildWholeTree(const BlockBuild& S, uint32_t chunkKeys, uint32_t* smem,
                                            size_t smemBytes) {
    if (S.kind != 2) {
        if (threadIdx.x == 0) {
            S.bounds[0] = S.bounds[1] = S.bounds[2] = 0xFFFFFFFFu;  // running minima start at the top
            S.bounds[3] = S.bounds[4] = S.bounds[5] = 0u;           // running maxima at the bottom
        }
        __syncthreads();
        prepRange(S, 0, S.n);
    }
    __syncthreads();
    if (S.n >= 2 && sharedBuildBytes<K>(S.n) <= smemBytes && sortElems(S.n) <= blockDim.x * 8u) {
        const uint32_t n = S.n, m = sortElems(n);
        bitonicSortShared<K, BITS>(S, smem, m);
        __syncthreads();
        const K* sorted = reinterpret_cast<const K*>(smem);
        char* base = reinterpret_cast<char*>(smem);
        if (n <= kSharedFitMax) {
            const size_t boxBytes = alignSmem(sharedSortBytes<K>(n) > 24 * (2 * (size_t)n - 1)
                                                  ? sharedSortBytes<K>(n)
                                                  : 24 * (2 * (size_t)n - 1));
            SharedFit F;
            F.sBox = reinterpret_cast<float*>(base);  // over the sort pairs, once emission is done
            F.sParent = reinterpret_cast<uint32_t*>(base + boxBytes);
            uint2* child = reinterpret_cast<uint2*>(base + boxBytes + alignSmem(4 * (2 * (size_t)n - 1)));
            F.sChild = child;
            F.sFlag = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(child) + alignSmem(8 * (size_t)n));
            for (uint32_t i = threadIdx.x; i + 1 < n; i += blockDim.x) {
                karrasNode<false>(sorted, (int)n, (int)i, S.nodes, S.parents, child, F.sParent);
                F.sFlag[i] = 0u;
            }
            __syncthreads();
            fitRangeShared(S, F);
            return;
        }
        uint32_t* flags = reinterpret_cast<uint32_t*>(base + alignSmem(sharedSortBytes<K>(n)));
        for (uint32_t i = threadIdx.x; i + 1 < n; i += blockDim.x) {
            karrasNode<false>(sorted, (int)n, (int)i, S.nodes, S.parents);
            flags[i] = 0u;
        }
        __syncthreads();
        fitRangeBlock(S, flags);
        return;
    }
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

// buildWholeTree, then (with S.qnodes) the quantised form of every 4-wide node, (with
// S.w8nodes) every 8-wide node.
template <typename K, int BITS>
__device__ __noinline__ void buildWhole(const BlockBuild& S, uint32_t chunkKeys, uint32_t* smem,
                                        size_t smemBytes = 0) {
    if (S.n == 0) return;
    buildWholeTree<K, BITS>(S, chunkKeys, smem, smemBytes);
    if (!S.qnodes && !S.w8nodes) return;
    __threadfence();  // the wide and binary nodes are read back through L2
    __syncthreads();
    const uint32_t m = S.n > 1 ? S.n - 1 : 1u;
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
        if (S.qnodes) quantizeWideNode(S.wide + kWideWords * (size_t)k, S.qnodes + kQuantWords * (size_t)k);
        if (S.w8nodes) wide8Node(S.nodes, S.n, k, S.w8nodes);
    }
}

}  // namespace grt
