// Pieces of the clustering builds shared by PLOC (ploc.cuh) and the subtree clustering
// (cluster.cuh): the union-area distance, its tie-break hash and the order of
// candidates, and the parent-link slot of a child word.
#pragma once

#include "grt_internal.cuh"

namespace grt {

// Surface area (halved) of the union of two cluster boxes, float32 in a fixed order.
__device__ __forceinline__ float plocUnionArea(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    const float dx = __fsub_rn(fmaxf(ahi.x, bhi.x), fminf(alo.x, blo.x));
    const float dy = __fsub_rn(fmaxf(ahi.y, bhi.y), fminf(alo.y, blo.y));
    const float dz = __fsub_rn(fmaxf(ahi.z, bhi.z), fminf(alo.z, blo.z));
    const float a = __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
    return __fadd_rn(a, 0.0f);
}

// fmix32, the 32-bit finaliser of MurmurHash3 (Appleby).
__device__ __forceinline__ uint32_t plocMix(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Tie-break of the pair of positions a < b.
__device__ __forceinline__ uint32_t plocPairHash(uint32_t a, uint32_t b) { return plocMix(plocMix(a) + b); }

// Parent-link slot of a child word: internal node k at k, leaf k at n-1+k.
__device__ __forceinline__ uint32_t plocSlot(uint32_t id, uint32_t n) {
    return (id & kLeafBit) ? n - 1u + (id & ~kLeafBit) : id;
}

// Running choice of cluster i's nearest neighbour; candidates j must come in ascending
// order. Order: smallest (area bits, pair hash), equal keys to the lower position; the
// hash is only evaluated between candidates of equal area.
struct PlocBest {
    uint32_t bits, hash, j;
    bool hashed;
};
__device__ __forceinline__ void plocConsider(PlocBest& b, uint32_t i, uint32_t j, uint32_t bits) {
    if (b.j == kInvalid || bits < b.bits) {
        b.bits = bits, b.j = j, b.hashed = false;
    } else if (bits == b.bits) {
        if (!b.hashed) {
            b.hash = b.j < i ? plocPairHash(b.j, i) : plocPairHash(i, b.j);
            b.hashed = true;
        }
        const uint32_t h = j < i ? plocPairHash(j, i) : plocPairHash(i, j);
        if (h < b.hash) b.hash = h, b.j = j;
    }
}

}  // namespace grt
