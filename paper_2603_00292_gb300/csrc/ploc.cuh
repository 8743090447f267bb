// Bottom-up clustering build: Parallel Locally-Ordered Clustering (PLOC; Meister and
// Bittner, "Parallel Locally-Ordered Clustering for Bounding Volume Hierarchy
// Construction", IEEE TVCG 2018), the clustering family behind the paper's "balanced"
// build (Sec. 6.2 "BVH Construction" describes bottom-up clustering; Sec. 8 names
// H-PLOC as that option).
//
// The clusters start as the leaves in Morton order. Each iteration:
//   1. every cluster i finds its nearest neighbour among the clusters i-r..i+r: the one
//      whose union with i has the smallest surface area (ties: see below);
//   2. every mutual pair (i, j), i < j, merges into a new internal node left = i,
//      right = j, which takes position i; position j is dropped;
//   3. the survivors are compacted in order.
// until one cluster is left. The surface area is the float32 sum dx*dy + dy*dz + dz*dx
// of the union box, each operation rounded to nearest, with a +0 added so that a zero
// area has one sign. Candidates are ordered by (area, pair hash, position): the pair
// hash is MurmurHash3's 32-bit finaliser (fmix32) applied to fmix32(lo) + hi of the
// pair's two positions lo < hi, so equal areas (a regular grid, stacked copies) are
// split pseudo-randomly instead of all in favour of the leftmost candidate, which would
// let a run of equal boxes merge one pair per iteration. The order is the same from
// either end of a pair, so the smallest pair overall is always mutual and every
// iteration merges at least once.
//
// Node numbering: the m-th merge of the whole build (merges counted in iteration order,
// then by position) creates internal node n-2-m, so the last merge is the root, node 0,
// and every internal child has a larger index than its parent. Leaves keep their sorted
// positions. The kernel writes what Karras emission writes (the child words of each
// internal node, word 3 of the binary node, and the parent links); the bottom-up fit
// then computes boxes, leaf records and 4-wide nodes exactly as for an LBVH.
//
// Execution: one persistent launch of at most 2 blocks per SM runs the iterations while
// many clusters are left. A block owns a contiguous range of whole 256-cluster tiles;
// phase A (nearest neighbours, with the r-wide halo recomputed on both sides so the
// mutual test needs no other block) and phase B (offsets from the per-block counts,
// scatter of survivors and merges) are separated by grid barriers. Blocks whose range has
// become empty leave for good. Every barrier wait is bounded in time; one that runs out
// latches GRT_ERROR_TIMEOUT and every block leaves. Once at most finishAt clusters are
// left, a second launch of one block finishes in shared memory, where an iteration costs
// a few block barriers instead of two grid barriers and a dozen round trips to L2.
// Indices read from memory are range-checked before use, so a launch that is cut short
// leaves a wrong tree (and an error) but touches nothing outside its buffers.
#pragma once

#include "lbvh.cuh"
#include "ploc_common.cuh"

namespace grt {

constexpr int kPlocThreads = 256;           // threads per block = clusters per tile
constexpr uint32_t kPlocMaxRadius = 64;
constexpr uint32_t kPlocWaitSpins = 1u << 25;
constexpr uint32_t kPlocKeep = 1u << 30, kPlocMerge = 1u << 31, kPlocIndex = (1u << 30) - 1u;

struct PlocParams {
    PrimSource src;
    uint32_t n;
    uint32_t radius;
    const uint32_t* sortedPrims;  // primitive at each sorted position
    float4* clusters[2];          // ping-pong, 2 float4 per cluster: {lo.xyz, id}, {hi.xyz, 0}
    uint32_t* pick;               // per position: neighbour | kPlocKeep | kPlocMerge
    uint2* blockCounts;           // per block: (survivors, merges) of the current iteration
    uint32_t* sync;               // [0] arrivals, [1] generation, [2] abort, [3..5] hand-over state
                                  // (clusters left, merges so far, current array); zeroed before the launch
    float4* nodes;                // binary nodes: word 3 = child words
    uint32_t* parents;            // parent << 1 | side; internal node k at [k], leaf k at [n-1+k]
    uint32_t* error;
    unsigned long long waitNs;    // time limit of one barrier wait
    uint32_t finishAt;            // the grid launch hands over to one block at this many clusters
};

__device__ __forceinline__ unsigned long long plocTimerNs() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier among `participants` blocks (every thread of each calls it). Returns false
// once the launch has been aborted (a wait ran out here or elsewhere).
__device__ bool plocBarrier(const PlocParams& P, uint32_t participants, uint32_t& gen) {
    __shared__ uint32_t ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* vsync = P.sync;
        uint32_t good = 1u;
        const uint32_t target = gen + 1u;
        __threadfence();
        const uint32_t prev = atomicAdd(P.sync + 0, 1u);
        if (prev == participants - 1u) {
            atomicExch(P.sync + 0, 0u);
            __threadfence();
            atomicExch(P.sync + 1, target);
        } else {
            const unsigned long long t0 = plocTimerNs();
            for (uint32_t k = 0; vsync[1] != target; ++k) {
                if (vsync[2] != 0u) break;
                if (k >= kPlocWaitSpins || ((k & 63u) == 0u && plocTimerNs() - t0 > P.waitNs)) {
                    latchError(P.error, GRT_ERROR_TIMEOUT);
                    atomicExch(P.sync + 2, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (vsync[2] != 0u) good = 0u;
        ok = good;
    }
    __syncthreads();
    gen += 1u;
    return ok != 0u;
}

// Block-wide exclusive ranks of two flags and their block totals (kPlocThreads threads).
__device__ __forceinline__ void plocRanks(bool a, bool b, uint32_t& ra, uint32_t& rb, uint32_t& ta, uint32_t& tb) {
    __shared__ uint32_t wa[kPlocThreads / 32], wb[kPlocThreads / 32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ma = __ballot_sync(0xffffffffu, a), mb = __ballot_sync(0xffffffffu, b);
    const uint32_t below = (1u << lane) - 1u;
    if (lane == 0) wa[warp] = __popc(ma), wb[warp] = __popc(mb);
    __syncthreads();
    uint32_t pa = 0, pb = 0;
    ta = tb = 0;
    for (uint32_t w = 0; w < kPlocThreads / 32; ++w) {
        if (w < warp) pa += wa[w], pb += wb[w];
        ta += wa[w], tb += wb[w];
    }
    ra = pa + __popc(ma & below);
    rb = pb + __popc(mb & below);
    __syncthreads();
}

// Block-wide sums of (x, y) pairs over blockCounts[0..count), and over [0..upTo).
__device__ __forceinline__ void plocCountSums(const uint2* counts, uint32_t count, uint32_t upTo, uint2& below,
                                              uint2& total) {
    __shared__ uint32_t part[4][kPlocThreads / 32];
    uint32_t bx = 0, by = 0, tx = 0, ty = 0;
    for (uint32_t t = threadIdx.x; t < count; t += kPlocThreads) {
        const uint2 v = __ldcg(counts + t);
        tx += v.x, ty += v.y;
        if (t < upTo) bx += v.x, by += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (lane == 0) part[0][warp] = bx, part[1][warp] = by, part[2][warp] = tx, part[3][warp] = ty;
    __syncthreads();
    below = make_uint2(0, 0);
    total = make_uint2(0, 0);
    for (uint32_t w = 0; w < kPlocThreads / 32; ++w) {
        below.x += part[0][w], below.y += part[1][w];
        total.x += part[2][w], total.y += part[3][w];
    }
    __syncthreads();
}

// Nearest neighbour of cluster i among the positions [lo, hi] (i excluded), boxes in
// shared memory at box[2 * (position - base)] (two float4: lo.xyz, hi.xyz).
__device__ __forceinline__ uint32_t plocNearest(const float4* box, int base, int i, int lo, int hi) {
    const float4 alo = box[2 * (i - base)], ahi = box[2 * (i - base) + 1];
    PlocBest b{0u, 0u, kInvalid, false};
    for (int j = lo; j <= hi; ++j) {
        if (j == i) continue;
        const float area = plocUnionArea(alo, ahi, box[2 * (j - base)], box[2 * (j - base) + 1]);
        plocConsider(b, (uint32_t)i, (uint32_t)j, __float_as_uint(area));
    }
    return b.j;
}

// Dynamic shared memory: (kPlocThreads + 4r) cluster boxes (2 float4 each), then
// (kPlocThreads + 2r) neighbour words.
__host__ __device__ inline size_t plocSmemBytes(uint32_t radius) {
    return (size_t)(kPlocThreads + 4 * radius) * 2 * sizeof(float4) + (size_t)(kPlocThreads + 2 * radius) * 4;
}

__global__ void __launch_bounds__(kPlocThreads) plocKernel(PlocParams P) {
    extern __shared__ float4 plocSmem[];
    const int r = (int)P.radius;
    float4* box = plocSmem;                                                  // window of cluster boxes
    uint32_t* nbr = reinterpret_cast<uint32_t*>(plocSmem + 2 * (kPlocThreads + 4 * r));  // neighbours
    const uint32_t n = P.n;
    const uint32_t G = gridDim.x;
    uint32_t gen = 0;

    // the leaves in sorted order
    for (uint32_t k = blockIdx.x * kPlocThreads + threadIdx.x; k < n; k += G * kPlocThreads) {
        const uint32_t prim = __ldcg(P.sortedPrims + k);
        float3 v[3];
        const Box3 b = primBox(P.src, prim < P.src.count ? prim : 0u, v);
        P.clusters[0][2 * (size_t)k] = make_float4(b.lo.x, b.lo.y, b.lo.z, __uint_as_float(kLeafBit | k));
        P.clusters[0][2 * (size_t)k + 1] = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.f);
    }
    if (!plocBarrier(P, G, gen)) return;

    uint32_t c = n, created = 0, src = 0;
    for (uint32_t iter = 0; c > 1u; ++iter) {
        if (c <= P.finishAt) {  // the rest in one block's shared memory (plocFinishKernel)
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                P.sync[3] = c;
                P.sync[4] = created;
                P.sync[5] = src;
            }
            return;
        }
        const uint32_t tiles = (c + kPlocThreads - 1) / kPlocThreads;
        const uint32_t A = min(G, tiles);
        if (blockIdx.x >= A) return;  // no range from now on: the count only shrinks
        const uint32_t per = (tiles + A - 1) / A;
        const uint32_t begin = min(blockIdx.x * per * kPlocThreads, c);
        const uint32_t end = min(begin + per * kPlocThreads, c);
        const float4* cur = P.clusters[src];
        float4* nxt = P.clusters[src ^ 1u];

        // ---- phase A: nearest neighbours of [begin - r, end + r), mutual test on [begin, end)
        uint32_t keepCount = 0, mergeCount = 0;
        for (uint32_t s = begin; s < end; s += kPlocThreads) {
            const int w0 = (int)s - 2 * r;
            for (int t = threadIdx.x; t < kPlocThreads + 4 * r; t += kPlocThreads) {
                const int g = w0 + t;
                if (g >= 0 && g < (int)c) {
                    box[2 * t] = __ldcg(cur + 2 * (size_t)g);
                    box[2 * t + 1] = __ldcg(cur + 2 * (size_t)g + 1);
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kPlocThreads + 2 * r; e += kPlocThreads) {
                const int i = (int)s - r + e;
                uint32_t best = kInvalid;
                if (i >= 0 && i < (int)c) best = plocNearest(box, w0, i, max(i - r, 0), min(i + r, (int)c - 1));
                nbr[e] = best;
            }
            __syncthreads();
            const uint32_t i = s + threadIdx.x;
            if (i < end) {
                const uint32_t j = nbr[threadIdx.x + r];  // in [i - r, i + r]
                const int ej = (int)j - ((int)s - r);
                const bool mutual = ej >= 0 && ej < kPlocThreads + 2 * r && nbr[ej] == i;
                const bool keep = !mutual || i < j, merge = mutual && i < j;
                keepCount += keep, mergeCount += merge;
                P.pick[i] = (j & kPlocIndex) | (keep ? kPlocKeep : 0u) | (merge ? kPlocMerge : 0u);
            }
            __syncthreads();
        }
        {
            __shared__ uint32_t red[2][kPlocThreads / 32];
            for (int o = 16; o > 0; o >>= 1) {
                keepCount += __shfl_xor_sync(0xffffffffu, keepCount, o);
                mergeCount += __shfl_xor_sync(0xffffffffu, mergeCount, o);
            }
            if ((threadIdx.x & 31u) == 0) red[0][threadIdx.x >> 5] = keepCount, red[1][threadIdx.x >> 5] = mergeCount;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint2 v = make_uint2(0, 0);
                for (int w = 0; w < kPlocThreads / 32; ++w) v.x += red[0][w], v.y += red[1][w];
                P.blockCounts[blockIdx.x] = v;
            }
        }
        if (!plocBarrier(P, A, gen)) return;

        // ---- phase B: offsets, then survivors and new nodes written in order
        uint2 below, total;
        plocCountSums(P.blockCounts, A, blockIdx.x, below, total);
        uint32_t keepBase = below.x, mergeBase = below.y;
        for (uint32_t s = begin; s < end; s += kPlocThreads) {
            const uint32_t i = s + threadIdx.x;
            const uint32_t pk = i < end ? P.pick[i] : 0u;
            const bool keep = (pk & kPlocKeep) != 0u, merge = (pk & kPlocMerge) != 0u;
            uint32_t rk, rm, tk, tm;
            plocRanks(keep, merge, rk, rm, tk, tm);
            if (keep) {
                const uint32_t pos = keepBase + rk;
                float4 lo = __ldcg(cur + 2 * (size_t)i), hi = __ldcg(cur + 2 * (size_t)i + 1);
                if (merge) {
                    const uint32_t j = pk & kPlocIndex;
                    const uint32_t m = created + mergeBase + rm;
                    if (j < c && m + 2u <= n) {
                        const uint32_t q = n - 2u - m;
                        const float4 jlo = __ldcg(cur + 2 * (size_t)j), jhi = __ldcg(cur + 2 * (size_t)j + 1);
                        const uint32_t a = __float_as_uint(lo.w), b = __float_as_uint(jlo.w);
                        const uint32_t sa = plocSlot(a, n), sb = plocSlot(b, n);
                        P.nodes[4 * (size_t)q + 3] = make_float4(__uint_as_float(a), __uint_as_float(b), 0.f, 0.f);
                        if (sa < 2u * n - 1u) P.parents[sa] = q << 1;
                        if (sb < 2u * n - 1u) P.parents[sb] = (q << 1) | 1u;
                        lo = make_float4(fminf(lo.x, jlo.x), fminf(lo.y, jlo.y), fminf(lo.z, jlo.z),
                                         __uint_as_float(q));
                        hi = make_float4(fmaxf(hi.x, jhi.x), fmaxf(hi.y, jhi.y), fmaxf(hi.z, jhi.z), 0.f);
                    } else {
                        latchError(P.error, GRT_ERROR_INTERNAL);
                    }
                }
                if (pos < n) {
                    nxt[2 * (size_t)pos] = lo;
                    nxt[2 * (size_t)pos + 1] = hi;
                }
            }
            keepBase += tk, mergeBase += tm;
        }
        if (total.y == 0u || total.x >= c) {  // no merge: cannot happen with consistent keys
            if (threadIdx.x == 0) latchError(P.error, GRT_ERROR_INTERNAL);
            return;
        }
        created += total.y;
        c = total.x;
        src ^= 1u;
        if (!plocBarrier(P, A, gen)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // n <= 1 never gets here; finishAt >= 1
        P.sync[3] = c;
        P.sync[4] = created;
        P.sync[5] = src;
    }
}

// ======================================================================= the last iterations
// One block of kPlocFinishThreads threads takes the clusters left by plocKernel (at most
// finishAt <= kPlocFinishMax) into shared memory and runs the same iterations there.
// Neighbour searches are spread one cluster per thread (the loop is latency-bound: each
// thread runs a chain of 2r area tests, so more threads beat fewer, longer chains); for
// the numbering, thread t owns a contiguous run of positions, so one block-wide scan of
// its survivor and merge counts numbers the survivors and the new nodes in position order.
constexpr int kPlocFinishThreads = 1024;
constexpr uint32_t kPlocFinishMax = 3072;

__host__ __device__ inline size_t plocFinishSmemBytes() {
    return (size_t)kPlocFinishMax * (4 * sizeof(float4) + sizeof(uint32_t));
}

// Block-wide exclusive scan of one word per thread (kPlocFinishThreads threads); the
// block total in *total.
__device__ __forceinline__ uint32_t plocBlockScan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warpSum[kPlocFinishThreads / 32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) warpSum[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (uint32_t w = 0; w < kPlocFinishThreads / 32; ++w) {
        if (w < warp) before += warpSum[w];
        all += warpSum[w];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kPlocFinishThreads) plocFinishKernel(PlocParams P) {
    extern __shared__ float4 finSmem[];
    float4* A = finSmem;                       // clusters, 2 float4 each: {lo.xyz, id}, {hi.xyz, 0}
    float4* B = finSmem + 2 * kPlocFinishMax;  // the next iteration's
    uint32_t* nb = reinterpret_cast<uint32_t*>(finSmem + 4 * kPlocFinishMax);
    const uint32_t n = P.n;
    const int r = (int)P.radius;
    uint32_t c = __ldcg(P.sync + 3), created = __ldcg(P.sync + 4);
    const uint32_t src = __ldcg(P.sync + 5) & 1u;
    if (n < 2 || __ldcg(P.sync + 2) != 0u) return;  // nothing to do, or the grid launch gave up
    if (c == 0u || c > kPlocFinishMax || c > n || created + c != n) {
        if (threadIdx.x == 0) latchError(P.error, GRT_ERROR_INTERNAL);
        return;
    }
    for (uint32_t k = threadIdx.x; k < 2 * c; k += kPlocFinishThreads) A[k] = __ldcg(P.clusters[src] + k);
    __syncthreads();
    while (c > 1u) {
        for (uint32_t i = threadIdx.x; i < c; i += kPlocFinishThreads)
            nb[i] = plocNearest(A, 0, (int)i, max((int)i - r, 0), min((int)i + r, (int)c - 1));
        __syncthreads();
        const uint32_t per = (c + kPlocFinishThreads - 1) / kPlocFinishThreads;
        const uint32_t b0 = min(threadIdx.x * per, c), b1 = min(b0 + per, c);
        uint32_t keeps = 0, merges = 0;
        for (uint32_t i = b0; i < b1; ++i) {
            const uint32_t j = nb[i];
            const bool mutual = j < c && nb[j] == i;
            keeps += !mutual || i < j;
            merges += mutual && i < j;
        }
        uint32_t total;
        const uint32_t off = plocBlockScan(keeps | (merges << 16), &total);
        uint32_t pos = off & 0xFFFFu, m = created + (off >> 16);
        for (uint32_t i = b0; i < b1; ++i) {
            const uint32_t j = nb[i];
            const bool mutual = j < c && nb[j] == i;
            if (mutual && j < i) continue;
            float4 lo = A[2 * i], hi = A[2 * i + 1];
            if (mutual) {
                if (m + 2u <= n) {
                    const uint32_t q = n - 2u - m;
                    const float4 jlo = A[2 * j], jhi = A[2 * j + 1];
                    const uint32_t a = __float_as_uint(lo.w), b = __float_as_uint(jlo.w);
                    const uint32_t sa = plocSlot(a, n), sb = plocSlot(b, n);
                    P.nodes[4 * (size_t)q + 3] = make_float4(__uint_as_float(a), __uint_as_float(b), 0.f, 0.f);
                    if (sa < 2u * n - 1u) P.parents[sa] = q << 1;
                    if (sb < 2u * n - 1u) P.parents[sb] = (q << 1) | 1u;
                    lo = make_float4(fminf(lo.x, jlo.x), fminf(lo.y, jlo.y), fminf(lo.z, jlo.z),
                                     __uint_as_float(q));
                    hi = make_float4(fmaxf(hi.x, jhi.x), fmaxf(hi.y, jhi.y), fmaxf(hi.z, jhi.z), 0.f);
                } else {
                    latchError(P.error, GRT_ERROR_INTERNAL);
                }
                ++m;
            }
            if (pos < kPlocFinishMax) B[2 * pos] = lo, B[2 * pos + 1] = hi;
            ++pos;
        }
        __syncthreads();
        const uint32_t kept = total & 0xFFFFu, merged = total >> 16;
        if (merged == 0u || kept >= c) {
            if (threadIdx.x == 0) latchError(P.error, GRT_ERROR_INTERNAL);
            return;
        }
        created += merged;
        c = kept;
        float4* t = A;
        A = B;
        B = t;
    }
    if (threadIdx.x == 0) P.parents[0] = kInvalid;
}

}  // namespace grt
