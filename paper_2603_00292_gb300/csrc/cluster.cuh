// Clustering inside the linear BVH's subtrees, in one bottom-up pass: the build behind
// GRT_BUILD_CLUSTER_SUBTREES and the batched launch's clustered scenes. The paper names
// locally-ordered clustering (H-PLOC) as HIPRT's balanced build (Sec. 8) and describes
// bottom-up clustering by surface area (Sec. 6.2); this is a one-pass form of it that
// needs no grid-wide barrier.
//
// The linear BVH's topology (Karras emission) goes to temporary arrays. Every LBVH node
// p, once both its children are done, holds a list of clusters: its left child's, then
// its right child's (a leaf is one cluster). While the list has more than kClusterCap
// clusters (more than one at the root), mutual nearest neighbours by union surface area
// merge (the clustering build's distance and tie order, ploc_common.cuh); the rest go to p's
// parent. So clusters from both sides of a Morton split can pair up, which the LBVH's
// fixed split cannot do.
//
// Numbering. Every LBVH node owns one internal-node number (its own). A node passes up,
// with its list of m clusters, the m - 1 numbers its subtree did not use; its merges
// take numbers from its children's unused ones and its own, largest first, so the
// root's final merge takes 0. The tree is therefore a function of the input alone, and
// equals oracle_subtree_cluster's.
//
// Walk. One thread per leaf walks up the LBVH; the second to arrive at a node (an
// acquire-release atomic at GPU scope, as in the fit) hands it to its warp, which holds
// the node's list, one cluster per lane (at most 2 kClusterCap = 32), and merges. A
// node's list is stored in its own leaf range (32 B per position: {lo.xyz, word},
// {hi.xyz, 0}), its unused numbers likewise, so siblings never overlap. Merges write the
// final child words (row 3 of the binary node) and parent links; the fit computes the
// boxes and 4-wide nodes afterwards.
//
// Small subtrees are not processed. A node of at most kClusterCap leaves never merges,
// so its list is its leaves in order, and its unused numbers are all its subtree's: in
// Karras's numbering a subtree over leaves [f, l] holds the internal nodes [f, l] minus
// one end, l when its root is numbered f (a right child, or the root) and f when it is
// numbered l (a left child). The first node above such a subtree reads both directly.
#pragma once

#include "lbvh.cuh"
#include "ploc_common.cuh"

namespace grt {

constexpr uint32_t kClusterCap = 16;

struct ClusterParams {
    PrimSource src;
    uint32_t n;
    const uint32_t* sortedPrims;  // sorted position -> primitive ID
    uint2* topoChild;             // LBVH child words per internal node
    uint32_t* topoParent;         // LBVH parent entry per node, internal then leaves: parent << 2, bit 1
                                  // set when the parent has more than kClusterCap leaves, bit 0 the side
    uint4* record;                // per internal node: leaf range first, last; clusters passed up
    float4* clusters;             // 2 float4 per leaf position
    uint32_t* freeIds;            // per leaf position
    uint32_t* flags;              // arrival counters per internal node (zeroed)
    float4* nodes;                // output: child words in row 3 of each binary node
    uint32_t* parents;            // output: parent links
    uint32_t* error;              // the context's device error word
};

// Position i (0..n-1) of the sorted leaves: its cluster (box and leaf word), and for
// i < n-1 internal node i of the LBVH into the temporary topology arrays, its arrival
// counter zeroed.
template <bool CG, typename K>
__device__ __forceinline__ void karrasTopology(const K* __restrict__ keys, int i, const ClusterParams& C) {
    float3 v[3];
    const Box3 b = primBox(C.src, CG ? __ldcg(C.sortedPrims + i) : C.sortedPrims[i], v);
    C.clusters[2 * (size_t)i] = make_float4(b.lo.x, b.lo.y, b.lo.z, __uint_as_float(kLeafBit | (uint32_t)i));
    C.clusters[2 * (size_t)i + 1] = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.f);
    if ((uint32_t)i + 1 >= C.n) return;
    uint32_t left, right;
    int first, last;
    karrasSplit<CG>(keys, (int)C.n, i, left, right, first, &last);
    C.topoChild[i] = make_uint2(left, right);
    C.record[i] = make_uint4((uint32_t)first, (uint32_t)last, 0u, 0u);
    const uint32_t big = (i == 0 || (uint32_t)(last - first) + 1u > kClusterCap) ? 2u : 0u;
    C.topoParent[plocSlot(left, C.n)] = ((uint32_t)i << 2) | big | 0u;
    C.topoParent[plocSlot(right, C.n)] = ((uint32_t)i << 2) | big | 1u;
    if (i == 0) C.topoParent[0] = kInvalid;
    C.flags[i] = 0u;
}

// A warp's working list in shared memory: boxes of up to 32 clusters, the node's unused
// numbers in descending order, and the union-area bits of every pair of slots (rows
// padded to 36 words: the lanes' row loads, row writes and mirrored writes are free of
// bank conflicts).
struct ClusterWarpList {
    float4 lo[32], hi[32];
    uint32_t freeIds[32];
    uint32_t dist[32][36];
};

// The warp (all 32 lanes) turns LBVH node p's children's lists into p's, merging as
// described above, and stores it (or, at the root, finishes the tree).
static __device__ __noinline__ void clusterNode(const ClusterParams& C, uint32_t p, ClusterWarpList& W) {
    const uint32_t lane = threadIdx.x & 31u, below = (1u << lane) - 1u, n = C.n;
    const uint2 ch = __ldcg(C.topoChild + p);
    // each child: its leaf range, whether it was processed (more than kClusterCap
    // leaves), its cluster count and the number of the unprocessed subtree's end that
    // is not one of its internal nodes
    uint32_t f[2], cnt[2], skip[2];
    bool small[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint32_t w = c ? ch.y : ch.x;
        const uint4 r = (w & kLeafBit) ? make_uint4(w & ~kLeafBit, w & ~kLeafBit, 0u, 0u) : __ldcg(C.record + w);
        f[c] = r.x;
        small[c] = r.y - r.x + 1u <= kClusterCap;
        cnt[c] = small[c] ? r.y - r.x + 1u : r.z;
        skip[c] = w == r.x ? r.y : r.x;
    }
    const uint32_t na = cnt[0], nb = cnt[1];
    if (na - 1u >= kClusterCap || nb - 1u >= kClusterCap) {  // never, given complete child lists
        if (lane == 0) latchError(C.error, GRT_ERROR_INTERNAL);
        return;
    }
    uint32_t m = na + nb;
    // this lane's cluster (lanes below m)
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    uint32_t word = kInvalid;
    if (lane < m) {  // a small subtree's positions still hold its leaves' clusters
        const uint32_t pos = lane < na ? f[0] + lane : f[1] + (lane - na);
        lo = __ldcg(C.clusters + 2 * (size_t)pos), hi = __ldcg(C.clusters + 2 * (size_t)pos + 1);
        word = __float_as_uint(lo.w);
    }
    // unused numbers: the children's, then p; ranked descending (all distinct)
    const uint32_t nfree = m - 1;
    uint32_t fid = 0;
    if (lane < nfree) {
        const int c = lane < na - 1 ? 0 : (lane < na - 1 + nb - 1 ? 1 : 2);
        if (c == 2) {
            fid = p;
        } else {
            const uint32_t j = c ? lane - (na - 1) : lane;
            if (small[c])  // the subtree's range without its non-internal end
                fid = f[c] + j + (f[c] + j >= skip[c] ? 1u : 0u);
            else
                fid = __ldcg(C.freeIds + f[c] + j);
        }
    }
    uint32_t rank = 0;
    for (uint32_t j = 0; j < 32; ++j) {
        const uint32_t o = __shfl_sync(0xffffffffu, fid, j);
        if (j < nfree && lane < nfree && o > fid) ++rank;
    }
    if (lane < nfree) W.freeIds[rank] = fid;
    W.lo[lane] = lo, W.hi[lane] = hi;
    __syncwarp();
    // Distances. The list keeps its slots: a merged cluster stays in its lower slot, the
    // other slot is retired, so the slots' order is the list's order and a cluster's
    // position is the number of live slots below it. The warp holds the union-area bits
    // of every pair of live slots (retired slots and the diagonal at the largest key).
    // The area is symmetric bit for bit, so each lane computes half its row and writes
    // both entries; after a round only the merged clusters' rows are recomputed.
    uint32_t alive = m == 32 ? ~0u : (1u << m) - 1u;
    for (uint32_t k = 1; k <= 16; ++k) {
        const uint32_t t = (lane + k) & 31u;
        const float4 blo = W.lo[t], bhi = W.hi[t];
        const uint32_t bits = lane < m && t < m ? __float_as_uint(plocUnionArea(lo, hi, blo, bhi)) : ~0u;
        W.dist[lane][t] = bits;
        W.dist[t][lane] = bits;
    }
    W.dist[lane][lane] = ~0u;
    __syncwarp();
    // nearest neighbour of this lane's cluster: the lowest slot of the smallest bits,
    // and whether another slot has the same bits (then the pair hash decides, below)
    uint32_t nn = 0, nnBits = ~0u;
    bool tie = false;
    auto consider = [&](uint32_t bits, uint32_t t) {
        tie = bits == nnBits ? true : (bits < nnBits ? false : tie);
        nn = bits < nnBits ? t : nn;
        nnBits = min(bits, nnBits);
    };
    auto scanRow = [&]() {
        nn = 0, nnBits = ~0u, tie = false;
        const uint32_t chunks = (35u - __clz(alive)) >> 2;  // slots below the highest live one
        for (uint32_t c = 0; c < chunks; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(&W.dist[lane][4 * c]);
            consider(v.x, 4 * c), consider(v.y, 4 * c + 1), consider(v.z, 4 * c + 2), consider(v.w, 4 * c + 3);
        }
    };
    // equal smallest bits (frequent where one cluster's box holds others): among the
    // slots of those bits, in list order, the clustering order decides (pair hash of the
    // positions, then the lower position)
    auto breakTies = [&]() {
        const bool mine = tie && ((alive >> lane) & 1u);
        if (!__any_sync(0xffffffffu, mine) || !mine) return;
        const uint32_t ps = __popc(alive & below), chunks = (35u - __clz(alive)) >> 2;
        uint32_t bestHash = ~0u, bestT = kInvalid;
        for (uint32_t c = 0; c < chunks; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(&W.dist[lane][4 * c]);
            const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (uint32_t i = 0; i < 4; ++i) {
                if (e[i] != nnBits) continue;
                const uint32_t t = 4 * c + i, pt = __popc(alive & ((1u << t) - 1u));
                const uint32_t h = pt < ps ? plocPairHash(pt, ps) : plocPairHash(ps, pt);
                if (bestT == kInvalid || h < bestHash) bestHash = h, bestT = t;
            }
        }
        nn = bestT;
    };
    if (lane < m) scanRow();
    breakTies();
    uint32_t nextFree = 0;
    const uint32_t target = p == 0 ? 1u : kClusterCap;
    while (m > target) {
        const bool live = (alive >> lane) & 1u;
        const uint32_t back = __shfl_sync(0xffffffffu, nn, nn & 31u);
        const bool mutual = live && back == lane;
        const bool lead = mutual && lane < nn;
        const uint32_t leads = __ballot_sync(0xffffffffu, lead);
        const uint32_t gone = __ballot_sync(0xffffffffu, mutual && nn < lane);
        const uint32_t otherWord = __shfl_sync(0xffffffffu, word, nn & 31u);
        if (lead) {  // reads only retiring slots' boxes, writes only leading slots'
            const float4 olo = W.lo[nn], ohi = W.hi[nn];
            const uint32_t q = W.freeIds[nextFree + __popc(leads & below)];
            C.nodes[4 * (size_t)q + 3] = make_float4(__uint_as_float(word), __uint_as_float(otherWord), 0.f, 0.f);
            C.parents[plocSlot(word, n)] = (q << 1) | 0u;
            C.parents[plocSlot(otherWord, n)] = (q << 1) | 1u;
            lo = make_float4(fminf(lo.x, olo.x), fminf(lo.y, olo.y), fminf(lo.z, olo.z), 0.f);
            hi = make_float4(fmaxf(hi.x, ohi.x), fmaxf(hi.y, ohi.y), fmaxf(hi.z, ohi.z), 0.f);
            word = q;
            W.lo[lane] = lo, W.hi[lane] = hi;
        }
        nextFree += __popc(leads);
        alive &= ~gone;
        m -= __popc(leads);
        if (m <= target) break;
        __syncwarp();  // the merged boxes
        // a lane whose neighbour merged looks again; the others compare the merged rows
        const bool now = (alive >> lane) & 1u;
        const bool rescan = lead || (now && (((leads | gone) >> nn) & 1u));
        for (uint32_t g = gone; g; g &= g - 1u) W.dist[lane][__ffs(g) - 1] = ~0u;
        for (uint32_t l = leads; l; l &= l - 1u) {
            const uint32_t q = (uint32_t)__ffs(l) - 1u;
            const float4 blo = W.lo[q], bhi = W.hi[q];
            const uint32_t bits = now && lane != q ? __float_as_uint(plocUnionArea(lo, hi, blo, bhi)) : ~0u;
            W.dist[q][lane] = bits;
            if (lane != q) W.dist[lane][q] = bits;
            if (now && !rescan) consider(bits, q);
        }
        __syncwarp();  // the merged rows
        if (__any_sync(0xffffffffu, rescan) && rescan) scanRow();
        breakTies();
    }
    if (p == 0) {
        if (lane == 0) C.parents[0] = kInvalid;
        return;
    }
    const uint32_t fp = __ldcg(C.record + p).x;
    if ((alive >> lane) & 1u) {
        const size_t at = fp + __popc(alive & below);
        C.clusters[2 * at] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
        C.clusters[2 * at + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
    }
    if (lane + 1 < m) C.freeIds[fp + lane] = W.freeIds[nextFree + lane];
    if (lane == 0) C.record[p].z = m;
}

// Leaves [begin, end) of the build: one thread per leaf walks up the LBVH. A thread that
// arrives second at a node (its sibling's list is complete) queues the node; the warp
// then processes its queued nodes one after another (clusterNode) and those threads walk
// on. Every thread of the block calls this (the warp-wide steps need whole warps).
// lists: one ClusterWarpList per warp of the block.
static __device__ __noinline__ void clusterRange(const ClusterParams& C, uint32_t begin, uint32_t end,
                                          ClusterWarpList* lists) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    ClusterWarpList& W = lists[warp];
    for (uint32_t base = begin + (threadIdx.x & ~31u); base < end; base += blockDim.x) {
        const uint32_t k = base + lane;
        uint32_t cur = C.n - 1 + k;  // the last node this thread finished (first its leaf)
        bool walking = k < end;
        for (;;) {
            uint32_t pending = kInvalid;
            while (walking) {
                const uint32_t pe = __ldcg(C.topoParent + cur);
                if (pe == kInvalid) {
                    walking = false;  // cur was the root
                    break;
                }
                // acquire-release at GPU scope: releases this warp's list of cur (the
                // warp's stores come before it through the warp barrier after
                // clusterNode), acquires the sibling's when this thread arrives second
                const uint32_t p = pe >> 2;
                uint32_t prev;
                asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(C.flags + p) : "memory");
                if (prev == 0) {
                    walking = false;  // the sibling's thread will take the node
                    break;
                }
                if (pe & 2u) {
                    pending = p;  // the warp processes it
                    break;
                }
                cur = p;  // a small subtree: nothing to do, walk on
            }
            if (!__any_sync(0xffffffffu, walking)) break;
            for (uint32_t ready = __ballot_sync(0xffffffffu, pending != kInvalid); ready; ready &= ready - 1) {
                const uint32_t leader = (uint32_t)__ffs(ready) - 1u;
                const uint32_t p = __shfl_sync(0xffffffffu, pending, (int)leader);
                __syncwarp();  // the leader's acquire orders the other lanes' loads too
                clusterNode(C, p, W);
                __syncwarp();  // every lane's stores of p's list before the leader's next arrival
                if (lane == leader) cur = p;
            }
        }
    }
}

}  // namespace grt
